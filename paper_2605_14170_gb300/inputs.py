"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds no arithmetic of the decoder.  It only builds the workloads
the decoder is run on:

* CSS check matrices of the codes the paper evaluates (Section IV): bivariate
  bicycle (BB) codes from two bivariate polynomials, and a two-block
  generalized bicycle (GB) code from two univariate polynomials drawn from a
  seed (a stand-in for the paper's B1 code, whose polynomials are not given
  in the paper);
* seeded random error patterns and channel LLR vectors for tests.

Every function is deterministic in its arguments.  GF(2) rank here exists
only to pick a GB code with k > 0 and to report k; it is not used by the
decoder.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSSCode",
    "bb_code",
    "gb_code",
    "gb_code_from_seed",
    "named_code",
    "gf2_rank_np",
    "random_errors",
    "channel_llr",
]


@dataclass
class CSSCode:
    """A CSS code: H_X H_Z^T = 0 (Section II-A).

    X errors are decoded with H_Z and Z errors with H_X.
    """

    name: str
    HX: np.ndarray  # (mx, n) uint8 0/1
    HZ: np.ndarray  # (mz, n) uint8 0/1
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.HX.shape[1])

    @property
    def k(self) -> int:
        return self.n - gf2_rank_np(self.HX) - gf2_rank_np(self.HZ)


def _shift(size: int) -> np.ndarray:
    """size x size cyclic shift matrix S with S[i, (i+1) % size] = 1."""
    S = np.zeros((size, size), dtype=np.uint8)
    S[np.arange(size), (np.arange(size) + 1) % size] = 1
    return S


def _matpow(M: np.ndarray, e: int) -> np.ndarray:
    R = np.eye(M.shape[0], dtype=np.int64)
    for _ in range(e):
        R = (R @ M) % 2
    return R.astype(np.uint8)


def bb_code(l: int, m: int, A_terms, B_terms, name: str | None = None) -> CSSCode:
    """Bivariate bicycle code of Bravyi et al. (the BB codes of Section IV).

    x = S_l (x) I_m and y = I_l (x) S_m.  ``A_terms``/``B_terms`` are lists of
    monomials ("x", e) or ("y", e).  H_X = [A | B], H_Z = [B^T | A^T].
    """
    x = np.kron(_shift(l), np.eye(m, dtype=np.uint8)).astype(np.uint8)
    y = np.kron(np.eye(l, dtype=np.uint8), _shift(m)).astype(np.uint8)

    def poly(terms):
        P = np.zeros((l * m, l * m), dtype=np.int64)
        for var, e in terms:
            P += _matpow(x if var == "x" else y, e)
        return (P % 2).astype(np.uint8)

    A, B = poly(A_terms), poly(B_terms)
    HX = np.concatenate([A, B], axis=1)
    HZ = np.concatenate([B.T, A.T], axis=1)
    return CSSCode(name or f"bb_{l}x{m}", HX.copy(), HZ.copy(),
                   {"l": l, "m": m, "A": list(A_terms), "B": list(B_terms)})


def gb_code(L: int, a_exps, b_exps, name: str | None = None) -> CSSCode:
    """Two-block generalized bicycle code: A = a(P), B = b(P), P the L x L shift."""
    P = _shift(L)

    def circ(exps):
        C = np.zeros((L, L), dtype=np.int64)
        for e in exps:
            C += np.roll(np.eye(L, dtype=np.int64), e, axis=1)
        return (C % 2).astype(np.uint8)

    del P
    A, B = circ(a_exps), circ(b_exps)
    HX = np.concatenate([A, B], axis=1)
    HZ = np.concatenate([B.T, A.T], axis=1)
    return CSSCode(name or f"gb_{2 * L}", HX.copy(), HZ.copy(),
                   {"L": L, "a": list(a_exps), "b": list(b_exps)})


def gb_code_from_seed(L: int = 441, seed: int = 20260518, weight: int = 3,
                      max_tries: int = 1000) -> CSSCode:
    """First GB code with k > 0 among seeded draws of two ``weight``-term
    polynomials (distinct exponents in [0, L)).  Draw j uses
    ``numpy.random.default_rng([seed, j])``."""
    for j in range(max_tries):
        rng = np.random.default_rng([seed, j])
        a = sorted(int(v) for v in rng.choice(L, weight, replace=False))
        b = sorted(int(v) for v in rng.choice(L, weight, replace=False))
        code = gb_code(L, a, b, name=f"gb_{2 * L}")
        k = code.k
        if k > 0:
            code.params.update({"seed": seed, "draw": j, "k": k})
            return code
    raise RuntimeError("no GB code with k > 0 found")


def named_code(name: str) -> CSSCode:
    """The codes of the benchmark configurations, by [[n,k,d]] name."""
    if name == "bb72":
        return bb_code(6, 6, [("x", 3), ("y", 1), ("y", 2)],
                       [("y", 3), ("x", 1), ("x", 2)], "[[72,12,6]]")
    if name == "bb144":
        return bb_code(12, 6, [("x", 3), ("y", 1), ("y", 2)],
                       [("y", 3), ("x", 1), ("x", 2)], "[[144,12,12]]")
    if name == "bb288":
        return bb_code(12, 12, [("x", 3), ("y", 2), ("y", 7)],
                       [("y", 3), ("x", 1), ("x", 2)], "[[288,12,18]]")
    if name == "gb882":
        return gb_code_from_seed(441)
    raise KeyError(name)


def gf2_rank_np(A: np.ndarray) -> int:
    """Rank over GF(2) of a 0/1 matrix (bit-packed row elimination)."""
    A = np.asarray(A, dtype=np.uint8) & 1
    rows, cols = A.shape
    if rows == 0 or cols == 0:
        return 0
    W = np.packbits(A, axis=1, bitorder="little")
    pad = (-W.shape[1]) % 8
    if pad:
        W = np.concatenate([W, np.zeros((rows, pad), np.uint8)], axis=1)
    W = W.view(np.uint64).copy()
    rank = 0
    for c in range(cols):
        w, b = divmod(c, 64)
        bit = np.uint64(1) << np.uint64(b)
        col = (W[rank:, w] & bit) != 0
        nz = np.nonzero(col)[0]
        if nz.size == 0:
            continue
        piv = rank + nz[0]
        if piv != rank:
            W[[rank, piv]] = W[[piv, rank]]
        below = rank + 1 + np.nonzero((W[rank + 1:, w] & bit) != 0)[0]
        W[below] ^= W[rank]
        rank += 1
        if rank == rows:
            break
    return rank


def random_errors(batch: int, n: int, p: float, seed: int) -> np.ndarray:
    """(batch, n) uint8 i.i.d. Bernoulli(p) error bits from numpy's PCG64."""
    rng = np.random.default_rng(seed)
    return (rng.random((batch, n)) < p).astype(np.uint8)


def channel_llr(n: int, p: float) -> np.ndarray:
    """Channel LLR mu_i = log((1-p)/p) for every variable (Section II-B)."""
    return np.full(n, np.log((1.0 - p) / p), dtype=np.float64)
