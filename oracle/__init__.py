"""CPU oracle for MBBP-LD (test infrastructure only).

A plain, slow, step-by-step restatement of the paper's method in C
(``mbbp_oracle.c`` + ``bp_body.inc``), loaded with ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import this package.  It shares no code with the CUDA library: it neither
imports the package ``paper_2605_14170_gb300`` nor includes its headers.

Functions and the passages they follow:

=========================  ====================================================
``splitmix64_at``          counter-based generator (splitmix64)
``sample``                 BSC / depolarizing error sampler (Section IV)
``gf2_rank``, ``syndrome``  GF(2) rank, s = H e (Section II-A)
``subtrees``               Algorithm 2, maximal subtrees
``permutation``            root orders pi_j (Section III-A)
``collect_subtrees``       the collection T over several orders (Section III-A)
``bp``                     syndrome BP on one representation (Section II-B),
                           flooding or serial schedule
``fws``                    Frequency-Weighted Scoring (Section III-B)
``lms``                    least-metric selection of classical MBBP (III-A)
``random_sets``            random augmentation of Table II
``mbbp_decode``            Algorithm 1 over a batch of syndromes
``judge``                  logical-error test by GF(2) rank
``wms_forward``            weighted min-sum, FP64 (a reading of Section II-B)
``wms_backward``           its hand-written adjoint
=========================  ====================================================

Every function takes and returns numpy arrays.  ``precision`` is ``"f64"``
(default; the FP64 oracle) or ``"f32"`` (the FP32 oracle, for comparing
decisions that floating point makes: hard decisions, convergence, selection).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "mbbp_oracle.c"), os.path.join(_HERE, "bp_body.inc")]
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lib_path = None  # set by use_library() to load another build (tests only)
_lock = threading.Lock()

RULE_NMS = 0
RULE_SP = 1
LMAX = 1.0e4
SPMAX = 16.635532333438686  # 2 atanh(1 - 2^-23)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) and return the path."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC[0], "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(_lib_path or build())
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
            vp = C.c_void_p
            lib.or_splitmix64_at.restype = C.c_uint64
            lib.or_splitmix64_at.argtypes = [C.c_uint64, C.c_uint64]
            lib.or_sample.restype = None
            lib.or_sample.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_int,
                                      C.c_double, C.c_int, u8p, vp]
            lib.or_gf2_rank.restype = C.c_int
            lib.or_gf2_rank.argtypes = [u8p, C.c_int, C.c_int]
            lib.or_syndrome.restype = None
            lib.or_syndrome.argtypes = [u8p, C.c_int, C.c_int, C.c_int, u8p, u8p]
            lib.or_subtrees.restype = C.c_int
            lib.or_subtrees.argtypes = [u8p, C.c_int, C.c_int, i32p, i32p, i32p]
            lib.or_permutation.restype = None
            lib.or_permutation.argtypes = [C.c_uint64, C.c_int, C.c_int, i32p]
            lib.or_collect_subtrees.restype = C.c_int
            lib.or_collect_subtrees.argtypes = [u8p, C.c_int, C.c_int, C.c_int,
                                                C.c_uint64, C.c_int, i32p, i32p]
            lib.or_fws.restype = C.c_int
            lib.or_fws.argtypes = [u8p, u8p, C.c_int, C.c_int, u8p, C.POINTER(C.c_int)]
            for name, fp, real in (("or_bp_one_f64", f64p, C.c_double),
                                   ("or_bp_one_f32", f32p, C.c_float)):
                fn = getattr(lib, name)
                fn.restype = None
                fn.argtypes = [u8p, C.c_int, C.c_int, u8p, fp, C.c_int, real,
                               C.c_int, C.c_int, u8p, C.POINTER(C.c_int),
                               C.POINTER(C.c_int), vp, vp]
            for name, fp, real in (("or_bp_serial_one_f64", f64p, C.c_double),
                                   ("or_bp_serial_one_f32", f32p, C.c_float)):
                fn = getattr(lib, name)
                fn.restype = None
                fn.argtypes = [u8p, C.c_int, C.c_int, u8p, fp, C.c_int, real, C.c_int, C.c_int,
                               u8p, C.POINTER(C.c_int), C.POINTER(C.c_int), vp]
            for name, fp, real in (("or_mbbp_decode_f64", f64p, C.c_double),
                                   ("or_mbbp_decode_f32", f32p, C.c_float)):
                fn = getattr(lib, name)
                fn.restype = None
                fn.argtypes = [u8p, C.c_int, C.c_int, C.c_int, i32p, i32p,
                               C.c_int, u8p, fp, C.c_int, C.c_int, real, C.c_int, C.c_int, C.c_int,
                               u8p, u8p, vp, u8p, vp, vp, vp]
            for name in ("or_wms_forward", "or_wms_backward"):
                fn = getattr(lib, name)
                fn.restype = C.c_double
            lib.or_wms_forward.argtypes = [u8p, C.c_int, C.c_int, u8p, f64p, C.c_int, f64p, f64p,
                                           vp, C.c_double, C.c_int, vp]
            lib.or_wms_backward.argtypes = [u8p, C.c_int, C.c_int, u8p, f64p, C.c_int, f64p, f64p,
                                            u8p, C.c_double, C.c_int, f64p, f64p]
            lib.or_lms.restype = C.c_int
            lib.or_lms.argtypes = [u8p, u8p, C.c_int, C.c_int, f32p, u8p, C.POINTER(C.c_int)]
            lib.or_random_sets.restype = None
            lib.or_random_sets.argtypes = [C.c_int, C.c_int, i32p, C.c_uint64, i32p, i32p]
            lib.or_clamp_reset.restype = None
            lib.or_clamp_reset.argtypes = []
            lib.or_clamp_stats.restype = None
            lib.or_clamp_stats.argtypes = [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
            lib.or_judge.restype = None
            lib.or_judge.argtypes = [u8p, C.c_int, u8p, C.c_int, C.c_int, C.c_int,
                                     u8p, u8p, u8p]
            _lib = lib
    return _lib


def use_library(path):
    """Load the oracle from another shared object (``None``: the default
    build).  Used by the mutation tests, which compile deliberately broken
    copies of the oracle to show that the pins catch them."""
    global _lib, _lib_path
    with _lock:
        _lib, _lib_path = None, path


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.uint8)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def splitmix64_at(state: int, i: int) -> int:
    """i-th output (i >= 1) of splitmix64 started at ``state``."""
    return int(_load().or_splitmix64_at(C.c_uint64(state), C.c_uint64(i)))


def sample(seed: int, first_shot: int, batch: int, n: int, p: float, noise: str):
    """Errors of shots first_shot .. first_shot+batch-1 as (batch, n) uint8.

    ``noise`` is ``"bsc"`` (X errors only) or ``"depolarizing"``.  Returns
    (ex, ez): the X part (decoded with H_Z) and the Z part (decoded with H_X).
    """
    lib = _load()
    ex = np.zeros((batch, n), np.uint8)
    ez = np.zeros((batch, n), np.uint8)
    lib.or_sample(seed, first_shot, batch, n, float(p),
                  0 if noise == "bsc" else 1, ex, _ptr(ez))
    return ex, ez


def gf2_rank(A) -> int:
    A = _u8(A)
    if A.ndim != 2 or A.size == 0:
        return 0
    return int(_load().or_gf2_rank(A, A.shape[0], A.shape[1]))


def syndrome(H, e) -> np.ndarray:
    """(batch, m) syndromes s = H e over GF(2) for (batch, n) errors."""
    H, e = _u8(H), _u8(e)
    e2 = e.reshape(-1, H.shape[1])
    s = np.zeros((e2.shape[0], H.shape[0]), np.uint8)
    _load().or_syndrome(H, H.shape[0], H.shape[1], e2.shape[0], e2, s)
    return s.reshape(e.shape[:-1] + (H.shape[0],))


def subtrees(H, perm):
    """Algorithm 2.  Returns (check_sets (1-based), acceptance order, count)."""
    H = _u8(H)
    m, n = H.shape
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    cs = np.zeros(m, np.int32)
    order = np.zeros(m, np.int32)
    ns = _load().or_subtrees(H, m, n, perm, cs, order)
    return cs, order, int(ns)


def permutation(seed: int, j: int, m: int) -> np.ndarray:
    perm = np.zeros(m, np.int32)
    _load().or_permutation(seed, j, m, perm)
    return perm


def collect_subtrees(H, R: int, seed: int, max_perms: int = 1024):
    """The R subtrees used as representations: list of int32 row arrays."""
    H = _u8(H)
    m, n = H.shape
    set_ptr = np.zeros(R + 1, np.int32)
    set_rows = np.zeros(max(R * m, 1), np.int32)
    found = _load().or_collect_subtrees(H, m, n, R, seed, max_perms, set_ptr, set_rows)
    return [set_rows[set_ptr[t]:set_ptr[t + 1]].copy() for t in range(found)]


def _sets_arrays(sets):
    set_ptr = np.zeros(len(sets) + 1, np.int32)
    for t, s in enumerate(sets):
        set_ptr[t + 1] = set_ptr[t] + len(s)
    rows = np.concatenate([np.asarray(s, np.int32) for s in sets]) if sets else np.zeros(0, np.int32)
    return set_ptr, np.ascontiguousarray(rows if rows.size else np.zeros(1, np.int32), dtype=np.int32)


def bp(Ht, st, mu, iters: int, alpha: float, rule: int = RULE_NMS,
       early_stop: bool = True, precision: str = "f64", want_c2v: bool = False,
       schedule: int = 0):
    """BP on one representation.  Returns dict(ehat, conv, K, post[, c2v]).
    schedule 0: flooding; 1: serial (layer-major check order, no c2v
    output)."""
    Ht, st = _u8(Ht), _u8(st)
    M, n = Ht.shape
    dt = np.float64 if precision == "f64" else np.float32
    mu = np.ascontiguousarray(mu, dtype=dt)
    ehat = np.zeros(n, np.uint8)
    post = np.zeros(n, dt)
    conv, K = C.c_int(0), C.c_int(0)
    if schedule == 1:
        if want_c2v:
            raise ValueError("serial schedule: no c2v output")
        fn = _load().or_bp_serial_one_f64 if precision == "f64" else _load().or_bp_serial_one_f32
        fn(Ht, M, n, st, mu, iters, alpha, rule, int(early_stop), ehat, C.byref(conv), C.byref(K),
           _ptr(post))
        return {"ehat": ehat, "conv": bool(conv.value), "K": int(K.value), "post": post}
    c2v = np.zeros((M, n), dt) if want_c2v else None
    fn = _load().or_bp_one_f64 if precision == "f64" else _load().or_bp_one_f32
    fn(Ht, M, n, st, mu, iters, alpha, rule, int(early_stop), ehat,
       C.byref(conv), C.byref(K), _ptr(post), _ptr(c2v))
    out = {"ehat": ehat, "conv": bool(conv.value), "K": int(K.value), "post": post}
    if want_c2v:
        out["c2v"] = c2v
    return out


def clamp_reset() -> None:
    """Zero this thread's clamp counters (see clamp_stats)."""
    _load().or_clamp_reset()


def clamp_stats():
    """(v->c messages computed, messages clamped to +-LMAX) by this thread's
    BP calls (flooding and serial, both precisions) since clamp_reset."""
    total, clamped = C.c_longlong(0), C.c_longlong(0)
    _load().or_clamp_stats(C.byref(total), C.byref(clamped))
    return int(total.value), int(clamped.value)


def fws(cand, conv):
    """FWS over (R, n) candidates with (R,) convergence flags.

    Returns (ehat, success, selected index or -1)."""
    cand, conv = _u8(cand), _u8(conv)
    R, n = cand.shape
    ehat = np.zeros(n, np.uint8)
    sel = C.c_int(-1)
    ok = _load().or_fws(cand, conv, R, n, ehat, C.byref(sel))
    return ehat, bool(ok), int(sel.value)


def lms(cand, conv, mu):
    """Least-metric selection over (R, n) candidates: (ehat, success, index)."""
    cand, conv = _u8(cand), _u8(conv)
    R, n = cand.shape
    ehat = np.zeros(n, np.uint8)
    sel = C.c_int(-1)
    ok = _load().or_lms(cand, conv, R, n, np.ascontiguousarray(mu, dtype=np.float32), ehat, C.byref(sel))
    return ehat, bool(ok), int(sel.value)


def random_sets(m: int, sizes, seed: int):
    """Random augmentation of Table II: len(sizes) sets of distinct random rows."""
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    R = len(sizes)
    ptr = np.zeros(R + 1, np.int32)
    rows = np.zeros(max(int(sizes.sum()), 1), np.int32)
    _load().or_random_sets(m, R, sizes, seed, ptr, rows)
    return [rows[ptr[t]:ptr[t + 1]].copy() for t in range(R)]


SCHEDULE_FLOODING = 0
SCHEDULE_SERIAL = 1
DECISION_FWS = 0
DECISION_LMS = 1


def mbbp_decode(H, sets, synd, llr, iters: int, alpha: float,
                rule: int = RULE_NMS, precision: str = "f64", want_post: bool = False,
                schedule: int = SCHEDULE_FLOODING, decision: int = DECISION_FWS):
    """Algorithm 1 for a batch: H (m, n); sets = list of R row arrays (H_t);
    synd (batch, m); llr (n,) shared or (batch, n) per shot.

    Returns dict with ehat (batch, n), conv (batch, R), iters (batch, R),
    success (batch,), selected (batch,), cand (batch, R, n)[, post]."""
    H = _u8(H)
    m, n = H.shape
    synd = _u8(synd).reshape(-1, m)
    batch = synd.shape[0]
    R = len(sets)
    dt = np.float64 if precision == "f64" else np.float32
    llr = np.ascontiguousarray(llr, dtype=dt)
    stride = 0 if llr.ndim == 1 else n
    set_ptr, set_rows = _sets_arrays(sets)
    out = {
        "ehat": np.zeros((batch, n), np.uint8),
        "conv": np.zeros((batch, R), np.uint8),
        "iters": np.zeros((batch, R), np.uint16),
        "success": np.zeros(batch, np.uint8),
        "selected": np.zeros(batch, np.int16),
        "cand": np.zeros((batch, R, n), np.uint8),
    }
    post = np.zeros((batch, R, n), dt) if want_post else None
    fn = _load().or_mbbp_decode_f64 if precision == "f64" else _load().or_mbbp_decode_f32
    fn(H, m, n, R, set_ptr, set_rows, batch, synd if synd.size else np.zeros(1, np.uint8),
       llr, stride, iters, alpha, rule, schedule, decision, out["ehat"] if batch else np.zeros(1, np.uint8),
       out["conv"] if out["conv"].size else np.zeros(1, np.uint8), _ptr(out["iters"]),
       out["success"] if batch else np.zeros(1, np.uint8), _ptr(out["selected"]),
       _ptr(out["cand"]), _ptr(post))
    if want_post:
        out["post"] = post
    return out


def wms_forward(Ht, st, mu, w, g, etrue=None, scale: float = 1.0, all_iters: bool = False):
    """Weighted min-sum on one representation, FP64 (see mbbp_oracle.c).
    w, g: [T, E] (edges row by row, columns ascending).  Returns
    (loss, posterior) with loss = scale * sum_v BCE(sigmoid(-post_v), e_v)
    of the last iteration, or its mean over all iterations (all_iters)."""
    Ht, st = _u8(Ht), _u8(st)
    M, n = Ht.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    post = np.zeros(n)
    et = None if etrue is None else _u8(etrue)
    L = _load().or_wms_forward(Ht, M, n, st, mu, w.shape[0], w, g, _ptr(et), scale, int(all_iters), _ptr(post))
    return float(L), post


def wms_backward(Ht, st, mu, w, g, etrue, scale: float = 1.0, all_iters: bool = False):
    """Adjoint of wms_forward: (loss, dL/dw [T, E], dL/dg [T, E])."""
    Ht, st, et = _u8(Ht), _u8(st), _u8(etrue)
    M, n = Ht.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    gw = np.zeros_like(w)
    gg = np.zeros_like(g)
    L = _load().or_wms_backward(Ht, M, n, st, mu, w.shape[0], w, g, et, scale, int(all_iters), gw, gg)
    return float(L), gw, gg


def judge(Hc, Ho, e, ehat) -> np.ndarray:
    """Per-shot failure codes: 0 ok, 1 syndrome not reproduced, 2 logical error."""
    Hc, Ho, e, ehat = _u8(Hc), _u8(Ho), _u8(e), _u8(ehat)
    n = Hc.shape[1]
    e = e.reshape(-1, n)
    ehat = ehat.reshape(-1, n)
    fail = np.zeros(e.shape[0], np.uint8)
    _load().or_judge(Hc, Hc.shape[0], Ho, Ho.shape[0], n, e.shape[0], e, ehat, fail)
    return fail
