"""Learned weights for MBBP-LD: weighted min-sum (WMS) trained on the GPU.

Every step of training runs in the library's kernels, called through the C
ABI: the counter-based sampler draws fresh code-capacity errors, the syndrome
kernel computes s = H e, the WMS forward kernel unrolls T flooding iterations
over all R representations (checkpointing every `ckpt` iterations), the
hand-written adjoint kernel accumulates dL/dw and dL/dg, and the Adam kernel
updates the weights.  Python only sequences the launches.

`compare_ler` decodes the same fresh shots with plain MBBP-LD (normalized
min-sum, mbbp_decode) and with the learned weights (mbbp_wms_decode) and
judges both with the logical-error kernel, so the learned form is measured
against the method without it on identical inputs.
"""
from __future__ import annotations

import math

import numpy as np

from . import mbbp


def _llr(n, p, device):
    import torch
    pm = 2.0 * p / 3.0  # X (or Z) marginal of the depolarizing channel
    return torch.full((n,), float(np.log((1 - pm) / pm)), dtype=torch.float32, device=device)


def _failures(B, L, w, g, syn, e, llr, iters, device):
    import torch
    out = mbbp.wms_decode(B, syn, llr, iters, w, g)
    cnt = torch.zeros(3, dtype=torch.int64, device=device)
    mbbp.mbbp_judge(L, e, out["e_hat"], None, cnt)
    c = cnt.cpu().numpy()
    return int(c[1] + c[2])


def train_wms(B: "mbbp.Bases", p: float, T: int = 25, ckpt: int = 5, batch: int = 4096, steps: int = 200,
              lr: float = 1e-3, seed: int = 20260516, alpha: float = 0.625, which: str = "X",
              w_bounds=(0.0, 2.0), g_bounds=(0.0, 0.9), all_iters: bool = True, log_every: int = 10,
              L: "mbbp.Logicals | None" = None, val_shots: int = 20000, val_every: int = 25,
              val_iters: int = 100, val_p: float | None = None, keep_initial: bool = True, device="cuda"):
    """Train per-edge, per-iteration weights w and damping g of WMS on the
    representations B (built from H_Z for X errors, H_X for Z errors).
    The loss is the BCE of every iteration's posterior (all_iters, which
    rewards early convergence under the halting rule) or of the last one.
    With logical operators L, the weights are scored every `val_every` steps
    by their logical failures on `val_shots` held-out shots (decoded with the
    halting rule, up to `val_iters` iterations) and the best weights seen are
    returned, the initial (plain min-sum) weights included unless
    keep_initial is False (then the best trained weights are returned).  The
    held-out shots are drawn at `val_p` (default: p), e.g. a higher error
    rate where a strong code still fails often enough to tell weights apart.
    Returns (w, g, history) with history = [(step, mean BCE, validation
    failures or None)]."""
    import torch
    n, W = B.n, B.words
    w, g = mbbp.wms_params(B, T, alpha=alpha, device=device)
    mw, vw = torch.zeros_like(w), torch.zeros_like(w)
    mg, vg = torch.zeros_like(g), torch.zeros_like(g)
    gw, gg = torch.zeros_like(w), torch.zeros_like(g)
    ex = torch.empty((batch, W), dtype=torch.int32, device=device)
    ez = torch.empty_like(ex)
    syn = torch.empty((batch, B.m), dtype=torch.uint8, device=device)
    post = torch.empty((batch, B.R, n), dtype=torch.float32, device=device)
    loss = torch.empty((batch, B.R), dtype=torch.float32, device=device)
    ws = torch.empty(mbbp.mbbp_wms_workspace_size(B, batch, T, ckpt), dtype=torch.uint8, device=device)
    llr = _llr(n, p, device)
    scale = 1.0 / (batch * B.R * n)
    history = []
    best = None
    if L is not None:
        vx = torch.empty((val_shots, W), dtype=torch.int32, device=device)
        vz = torch.empty_like(vx)
        vp = p if val_p is None else val_p
        vllr = _llr(n, vp, device)
        mbbp.mbbp_sample_errors(n, val_shots, 5_000_000_000, seed + 1, vp, mbbp.NOISE_DEPOLARIZING, vx, vz)
        ve = vx if which == "X" else vz
        vsyn = torch.empty((val_shots, B.m), dtype=torch.uint8, device=device)
        mbbp.mbbp_syndrome(B, ve, vsyn)
        f0 = _failures(B, L, w, g, vsyn, ve, vllr, val_iters, device)
        best = (f0 if keep_initial else 1 << 62, 0, w.clone(), g.clone())
        history.append((0, None, f0))
    for k in range(steps):
        mbbp.mbbp_sample_errors(n, batch, k * batch, seed, p, mbbp.NOISE_DEPOLARIZING, ex, ez)
        e = ex if which == "X" else ez
        mbbp.mbbp_syndrome(B, e, syn)
        mbbp.mbbp_wms_forward(B, syn, llr, T, w, g, ckpt, e, scale, post, loss, ws, all_iters=all_iters)
        gw.zero_()
        gg.zero_()
        mbbp.mbbp_wms_backward(B, syn, llr, T, w, g, ckpt, e, scale, post, gw, gg, ws, all_iters=all_iters)
        mbbp.mbbp_adam_step(w, gw, mw, vw, lr, 0.9, 0.999, 1e-8, k + 1, *w_bounds)
        mbbp.mbbp_adam_step(g, gg, mg, vg, lr, 0.9, 0.999, 1e-8, k + 1, *g_bounds)
        val = None
        if L is not None and ((k + 1) % val_every == 0 or k == steps - 1):
            val = _failures(B, L, w, g, vsyn, ve, vllr, val_iters, device)
            if val < best[0]:
                best = (val, k + 1, w.clone(), g.clone())
        if val is not None or (log_every and (k % log_every == 0 or k == steps - 1)):
            history.append((k + 1, float(loss.sum().item()), val))
    if best is not None:
        return best[2], best[3], history
    return w, g, history


def two_proportion_z(k1: int, k2: int, n: int) -> float:
    """One-sided two-proportion z statistic for k1 / n > k2 / n (pooled
    variance; conservative for the paired shots of compare_ler, whose two
    failure counts are positively correlated)."""
    pp = (k1 + k2) / (2.0 * n)
    if pp <= 0.0 or pp >= 1.0:
        return 0.0
    return (k1 - k2) / n / math.sqrt(2.0 * pp * (1.0 - pp) / n)


def wilson(k: int, n: int, z: float = 1.96):
    """Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return (0.0, 1.0)
    ph = k / n
    d = 1 + z * z / n
    c = (ph + z * z / (2 * n)) / d
    h = z * math.sqrt(ph * (1 - ph) / n + z * z / (4 * n * n)) / d
    # the ends are exactly 0 and 1 at k = 0 and k = n (c - h, c + h round there)
    lo = 0.0 if k == 0 else max(0.0, c - h)
    hi = 1.0 if k == n else min(1.0, c + h)
    return (lo, hi)


def compare_ler(B: "mbbp.Bases", L: "mbbp.Logicals", w, g, p: float, shots: int, iters: int,
                alpha: float = 0.625, seed: int = 20260517, which: str = "X", chunk: int = 200000,
                device="cuda") -> dict:
    """LER of plain MBBP-LD and of learned-weight MBBP-LD on the same fresh
    shots (failures: syndrome not reproduced or logical error)."""
    import torch
    n, W = B.n, B.words
    llr = _llr(n, p, device)
    fails = {"plain": torch.zeros(3, dtype=torch.int64, device=device),
             "learned": torch.zeros(3, dtype=torch.int64, device=device)}
    done = 0
    while done < shots:
        b = min(chunk, shots - done)
        ex = torch.empty((b, W), dtype=torch.int32, device=device)
        ez = torch.empty_like(ex)
        mbbp.mbbp_sample_errors(n, b, 10_000_000_000 + done, seed, p, mbbp.NOISE_DEPOLARIZING, ex, ez)
        e = ex if which == "X" else ez
        syn = torch.empty((b, B.m), dtype=torch.uint8, device=device)
        mbbp.mbbp_syndrome(B, e, syn)
        plain = mbbp.decode(B, syn, llr, iters, alpha)
        learned = mbbp.wms_decode(B, syn, llr, iters, w, g)
        mbbp.mbbp_judge(L, e, plain["e_hat"], None, fails["plain"])
        mbbp.mbbp_judge(L, e, learned["e_hat"], None, fails["learned"])
        done += b
    out = {"shots": shots, "p": p, "iters": iters}
    for key, f in fails.items():
        c = f.cpu().numpy()
        k = int(c[1] + c[2])
        out[key] = {"failures": k, "ler": k / shots, "ci95": wilson(k, shots)}
    return out
