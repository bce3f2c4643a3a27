"""Differentiable weighted min-sum (WMS) on the GPU against the oracle.

* w == alpha, g == 0: mbbp_wms_decode equals mbbp_decode bit for bit;
* with a weight and damping of its own on every edge and iteration,
  mbbp_wms_decode's halting iterations, flags and candidates equal those of
  the FP64 oracle's posteriors;
* forward posteriors within 1e-4 relative of the FP64 oracle;
* the hand-written adjoint (mbbp_wms_backward) within 1e-3 relative of the
  oracle's FP64 adjoint and of FP64 central finite differences, on a regular
  and an irregular code;
* the checkpoint interval does not change the gradients;
* the torch.autograd.Function returns the kernel's gradients;
* the Adam step matches its definition.
"""
import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import channel_llr, named_code

pytestmark = pytest.mark.gpu


def _setup(code="bb72", R=2, shots=12, T=8, seed=1, p=0.07):
    import torch
    from paper_2605_14170_gb300 import mbbp
    H = _irregular_H(11) if code == "irregular" else named_code(code).HZ
    n = H.shape[1]
    ex, _ = oracle.sample(seed, 0, shots, n, p, "depolarizing")
    s = oracle.syndrome(H, ex)
    B = mbbp.mbbp_build_bases(H, R, seed)
    rng = np.random.default_rng(seed)
    mu = rng.uniform(1.5, 3.5, n)  # distinct magnitudes: no exact ties in the mins
    E = int(B.edges.max())
    w = rng.uniform(0.5, 1.0, (R, T, E))
    g = rng.uniform(0.0, 0.4, (R, T, E))
    dev = torch.device("cuda:0")
    t = {"s": torch.from_numpy(s).to(dev), "mu": torch.from_numpy(mu.astype(np.float32)).to(dev),
         "w": torch.from_numpy(w.astype(np.float32)).to(dev), "g": torch.from_numpy(g.astype(np.float32)).to(dev),
         "e": torch.from_numpy(mbbp.pack_bits(ex)).to(dev)}
    return H, B, s, ex, mu, w, g, t


def _same_sums(a, b, rel=1e-4):
    """Two launches' weight / damping gradients.  The backward kernel adds
    each (shot, representation) item's terms with float atomics, so the
    summation order, and with it the last bits, varies from launch to
    launch: two orders of the same N terms differ by at most 2 N u sum|terms|
    (u = 2^-24), which bounds their difference in norm, not elementwise
    (an element whose terms cancel can differ by more than its own size
    times 1e-5).  An error in what is summed changes the norm by O(1)."""
    a = np.asarray(a.cpu().numpy() if hasattr(a, "cpu") else a, np.float64)
    b = np.asarray(b.cpu().numpy() if hasattr(b, "cpu") else b, np.float64)
    assert np.linalg.norm(a - b) <= rel * np.linalg.norm(b) + 1e-12, (np.linalg.norm(a - b), np.linalg.norm(b))


def _oracle_item(H, B, s, mu, w, g, e, shot, b, scale):
    rows = B.sets[b]
    Ht = np.concatenate([H, H[rows]])
    st = np.concatenate([s[shot], s[shot][rows]])
    Eb = int(Ht.sum())
    return Ht, st, w[b][:, :Eb], g[b][:, :Eb], Eb


def test_wms_with_alpha_weights_is_normalized_min_sum():
    import torch
    from paper_2605_14170_gb300 import mbbp
    c = named_code("bb144")
    H = c.HZ
    ex, _ = oracle.sample(3, 0, 300, 144, 0.06, "depolarizing")
    s = torch.from_numpy(oracle.syndrome(H, ex)).cuda()
    llr = torch.from_numpy(channel_llr(144, 0.04).astype(np.float32)).cuda()
    B = mbbp.mbbp_build_bases(H, 8, 3)
    w, g = mbbp.wms_params(B, 10, alpha=0.625)
    got = mbbp.wms_decode(B, s, llr, 60, w, g)
    ref = mbbp.decode(B, s, llr, 60, 0.625)
    for key in ("e_hat", "conv", "iters", "success", "selected"):
        assert torch.equal(got[key], ref[key]), key


def _irregular_H(seed, m=30, n=60):
    """Rows of weight 3..6, columns of weight 1..4: H^(t) rows of several
    degrees (the kernels' non-regular paths)."""
    rng = np.random.default_rng(seed)
    H = np.zeros((m, n), np.uint8)
    H[np.arange(n) % m, np.arange(n)] = 1
    for r in range(m):
        want = int(rng.integers(3, 7))
        free = [v for v in rng.permutation(n) if H[r, v] == 0 and H[:, v].sum() < 4]
        for v in free[:max(0, want - int(H[r].sum()))]:
            H[r, v] = 1
    return H


@pytest.mark.parametrize("code,R,shots", [("bb72", 4, 16), ("irregular", 4, 16), ("bb288", 8, 6), ("gb882", 64, 3)])
def test_wms_decode_with_learned_weights_matches_oracle(code, R, shots):
    """mbbp_wms_decode with a different weight and damping on every edge and
    iteration (T = 6, 10 iterations: the last four reuse the weights of
    iteration 6) against the oracle: for every (shot, representation) the
    FP64 weighted min-sum posteriors after t = 0, 1, ... iterations give the
    halting iteration, the flag and the candidate.  Items whose posteriors
    come within 3e-4 of 0 (where FP32 rounding may decide differently; the
    forward test bounds the FP32 posteriors' error by 1e-4) are not
    compared: a few percent of them on the length-882 code.  The codes'
    message areas lead the launcher to different numbers of warps per item
    (one on [[72]], four on the length-882 code)."""
    import torch
    from paper_2605_14170_gb300 import mbbp
    T, iters = 6, 10
    H = _irregular_H(11) if code == "irregular" else named_code(code).HZ
    m, n = H.shape
    ex, _ = oracle.sample(7, 0, shots, n, 0.06, "depolarizing")
    s = oracle.syndrome(H, ex)
    B = mbbp.mbbp_build_bases(H, R, 7)
    rng = np.random.default_rng(7)
    mu = rng.uniform(1.0, 3.0, n).astype(np.float32)
    E = int(B.edges.max())
    w = rng.uniform(0.4, 1.0, (R, T, E)).astype(np.float32)
    g = rng.uniform(0.0, 0.5, (R, T, E)).astype(np.float32)
    dev = torch.device("cuda:0")
    W = (n + 31) // 32
    s_t, mu_t = torch.from_numpy(s).to(dev), torch.from_numpy(mu).to(dev)
    w_t, g_t = torch.from_numpy(w).to(dev), torch.from_numpy(g).to(dev)
    out = {"e_hat": torch.empty((shots, n), dtype=torch.uint8, device=dev),
           "conv": torch.empty((shots, R), dtype=torch.uint8, device=dev),
           "iters": torch.empty((shots, R), dtype=torch.int16, device=dev),
           "success": torch.empty((shots,), dtype=torch.uint8, device=dev),
           "selected": torch.empty((shots,), dtype=torch.int16, device=dev)}
    ws = torch.empty(mbbp.mbbp_wms_decode_workspace_size(B, shots, T), dtype=torch.uint8, device=dev)
    assert ws.numel() >= mbbp.mbbp_decode_workspace_size(B, shots) + 8 * R * T * E
    with pytest.raises(mbbp.MBBPError):
        mbbp.mbbp_wms_decode(B, s_t, mu_t, iters, T, w_t, g_t, out["e_hat"], out["conv"], out["success"],
                             ws[:mbbp.mbbp_decode_workspace_size(B, shots)])
    mbbp.mbbp_wms_decode(B, s_t, mu_t, iters, T, w_t, g_t, out["e_hat"], out["conv"], out["success"], ws,
                         iters_run=out["iters"], selected=out["selected"])
    torch.cuda.synchronize()
    cand = ws[:shots * R * W * 4].view(torch.int32).cpu().numpy().reshape(shots, R, W).view(np.uint32)
    conv, its = out["conv"].cpu().numpy(), out["iters"].cpu().numpy()
    mu64 = mu.astype(np.float64)
    compared = 0
    for shot in range(shots):
        for b in range(R):
            Ht, st, wb, gb, _ = _oracle_item(H, B, s, mu64, w.astype(np.float64), g.astype(np.float64), ex, shot, b, 1.0)
            wext = np.concatenate([wb, np.repeat(wb[-1:], iters - T, axis=0)])
            gext = np.concatenate([gb, np.repeat(gb[-1:], iters - T, axis=0)])
            e, margin, K, cv = (mu64 < 0).astype(np.uint8), float(np.abs(mu64).min()), iters, 0
            for t in range(iters + 1):
                if t > 0:
                    _, post = oracle.wms_forward(Ht, st, mu64, wext[:t], gext[:t])
                    e, margin = (post < 0).astype(np.uint8), min(margin, float(np.abs(post).min()))
                if np.array_equal(H.astype(np.int64) @ e % 2, s[shot]):
                    K, cv = t, 1
                    break
            if margin < 3e-4:
                continue
            compared += 1
            assert (int(conv[shot, b]), int(its[shot, b])) == (cv, K), (shot, b)
            bits = (cand[shot, b][np.arange(n) >> 5] >> (np.arange(n) & 31)) & 1
            assert np.array_equal(bits.astype(np.uint8), e), (shot, b)
    assert compared >= 0.9 * shots * R, compared


def test_wms_forward_matches_fp64_oracle():
    import torch
    from paper_2605_14170_gb300 import mbbp
    H, B, s, ex, mu, w, g, t = _setup(shots=20, T=8)
    scale = 1.0 / 72
    post = torch.empty((20, B.R, 72), dtype=torch.float32, device="cuda")
    loss = torch.empty((20, B.R), dtype=torch.float32, device="cuda")
    ws = torch.empty(mbbp.mbbp_wms_workspace_size(B, 20, 8, 3), dtype=torch.uint8, device="cuda")
    mbbp.mbbp_wms_forward(B, t["s"], t["mu"], 8, t["w"], t["g"], 3, t["e"], scale, post, loss, ws, all_iters=True)
    torch.cuda.synchronize()
    post, loss = post.cpu().numpy(), loss.cpu().numpy()
    mu32 = mu.astype(np.float32).astype(np.float64)
    for shot in range(20):
        for b in range(B.R):
            Ht, st, wb, gb, _ = _oracle_item(H, B, s, mu32, w.astype(np.float32), g.astype(np.float32), ex, shot, b, scale)
            L, p64 = oracle.wms_forward(Ht, st, mu32, wb, gb, ex[shot], scale, all_iters=True)
            err = np.abs(post[shot, b] - p64) / np.maximum(np.abs(p64), 1.0)
            assert err.max() <= 1e-4, (shot, b, err.max())
            assert loss[shot, b] == pytest.approx(L, rel=1e-4)


@pytest.mark.parametrize("all_iters", [False, True])
def test_wms_gradients_match_oracle_adjoint_and_finite_differences(all_iters):
    import torch
    from paper_2605_14170_gb300 import mbbp
    shots, T = 12, 8
    H, B, s, ex, mu, w, g, t = _setup(shots=shots, T=T)
    scale = 1.0 / (shots * B.R * 72)
    w32, g32, mu32 = (x.astype(np.float32).astype(np.float64) for x in (w, g, mu))
    gw_ref, gg_ref = np.zeros_like(w32), np.zeros_like(g32)
    items = []
    for shot in range(shots):
        for b in range(B.R):
            Ht, st, wb, gb, Eb = _oracle_item(H, B, s, mu32, w32, g32, ex, shot, b, scale)
            _, gwb, ggb = oracle.wms_backward(Ht, st, mu32, wb, gb, ex[shot], scale, all_iters=all_iters)
            gw_ref[b][:, :Eb] += gwb
            gg_ref[b][:, :Eb] += ggb
            items.append((shot, b, Ht, st, Eb))
    post = torch.empty((shots, B.R, 72), dtype=torch.float32, device="cuda")
    ws = torch.empty(mbbp.mbbp_wms_workspace_size(B, shots, T, 3), dtype=torch.uint8, device="cuda")
    mbbp.mbbp_wms_forward(B, t["s"], t["mu"], T, t["w"], t["g"], 3, t["e"], scale, post, None, ws,
                          all_iters=all_iters)
    gw = torch.zeros_like(t["w"])
    gg = torch.zeros_like(t["g"])
    mbbp.mbbp_wms_backward(B, t["s"], t["mu"], T, t["w"], t["g"], 3, t["e"], scale, post, gw, gg, ws,
                           all_iters=all_iters)
    torch.cuda.synchronize()
    gw, gg = gw.cpu().numpy().astype(np.float64), gg.cpu().numpy().astype(np.float64)
    for got, ref in ((gw, gw_ref), (gg, gg_ref)):
        assert np.linalg.norm(got - ref) <= 1e-3 * np.linalg.norm(ref)
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        assert (np.abs(got - ref)[big] <= 1e-3 * np.abs(ref)[big] + 1e-7).mean() >= 0.99
    # FP64 central finite differences of the summed oracle loss
    rng = np.random.default_rng(0)
    h, checked = 1e-6, 0

    def total(wx, gx):
        tot = 0.0
        for shot, b, Ht, st, Eb in items:
            L, _ = oracle.wms_forward(Ht, st, mu32, wx[b][:, :Eb], gx[b][:, :Eb], ex[shot], scale,
                                      all_iters=all_iters)
            tot += L
        return tot

    L0 = total(w32, g32)
    for _ in range(12):
        b, tt = int(rng.integers(0, B.R)), int(rng.integers(0, T))
        k = int(rng.integers(0, int(B.edges[b])))
        for which, got in (("w", gw), ("g", gg)):
            P = (w32 if which == "w" else g32).copy()
            P[b, tt, k] += h
            Lp = total(P, g32) if which == "w" else total(w32, P)
            P[b, tt, k] -= 2 * h
            Lm = total(P, g32) if which == "w" else total(w32, P)
            right, left = (Lp - L0) / h, (L0 - Lm) / h
            if abs(right - left) > 1e-4 * max(abs(right), abs(left), 1e-10):
                continue  # a min or sign switches inside [-h, h]
            fd = (Lp - Lm) / (2 * h)
            assert abs(got[b, tt, k] - fd) <= 1e-3 * abs(fd) + 1e-9, (which, b, tt, k, got[b, tt, k], fd)
            checked += 1
    assert checked >= 16


def test_wms_gradients_on_irregular_code_match_oracle_adjoint():
    """Rows of weight 3 to 6: the kernels' per-row degrees, the parameters and
    gradient sums in the message layout (zeros past a row's degree) and
    their return to edge order, against the FP64 oracle adjoint."""
    import torch
    from paper_2605_14170_gb300 import mbbp
    shots, T, ckpt = 10, 6, 2
    H, B, s, ex, mu, w, g, t = _setup(code="irregular", R=4, shots=shots, T=T, seed=9)
    n = H.shape[1]
    scale = 1.0 / (shots * B.R * n)
    w32, g32, mu32 = (x.astype(np.float32).astype(np.float64) for x in (w, g, mu))
    gw_ref, gg_ref = np.zeros_like(w32), np.zeros_like(g32)
    for shot in range(shots):
        for b in range(B.R):
            Ht, st, wb, gb, Eb = _oracle_item(H, B, s, mu32, w32, g32, ex, shot, b, scale)
            _, gwb, ggb = oracle.wms_backward(Ht, st, mu32, wb, gb, ex[shot], scale, all_iters=True)
            gw_ref[b][:, :Eb] += gwb
            gg_ref[b][:, :Eb] += ggb
    post = torch.empty((shots, B.R, n), dtype=torch.float32, device="cuda")
    ws = torch.empty(mbbp.mbbp_wms_workspace_size(B, shots, T, ckpt), dtype=torch.uint8, device="cuda")
    mbbp.mbbp_wms_forward(B, t["s"], t["mu"], T, t["w"], t["g"], ckpt, t["e"], scale, post, None, ws,
                          all_iters=True)
    gw = torch.zeros_like(t["w"])
    gg = torch.zeros_like(t["g"])
    mbbp.mbbp_wms_backward(B, t["s"], t["mu"], T, t["w"], t["g"], ckpt, t["e"], scale, post, gw, gg, ws,
                           all_iters=True)
    torch.cuda.synchronize()
    gw, gg = gw.cpu().numpy().astype(np.float64), gg.cpu().numpy().astype(np.float64)
    for got, ref in ((gw, gw_ref), (gg, gg_ref)):
        assert np.linalg.norm(got - ref) <= 1e-3 * np.linalg.norm(ref)
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        assert (np.abs(got - ref)[big] <= 1e-3 * np.abs(ref)[big] + 1e-7).mean() >= 0.99
    for b in range(B.R):  # entries past a representation's edges stay untouched
        assert not gw[b][:, int(B.edges[b]):].any() and not gg[b][:, int(B.edges[b]):].any()


def test_checkpoint_interval_does_not_change_gradients():
    import torch
    from paper_2605_14170_gb300 import mbbp
    shots, T = 30, 10
    H, B, s, ex, mu, w, g, t = _setup(shots=shots, T=T, seed=4)
    res = []
    for ckpt in (1, 3, 5, 10):
        post = torch.empty((shots, B.R, 72), dtype=torch.float32, device="cuda")
        ws = torch.empty(mbbp.mbbp_wms_workspace_size(B, shots, T, ckpt), dtype=torch.uint8, device="cuda")
        mbbp.mbbp_wms_forward(B, t["s"], t["mu"], T, t["w"], t["g"], ckpt, t["e"], 1.0, post, None, ws)
        gw = torch.zeros_like(t["w"])
        gg = torch.zeros_like(t["g"])
        mbbp.mbbp_wms_backward(B, t["s"], t["mu"], T, t["w"], t["g"], ckpt, t["e"], 1.0, post, gw, gg, ws)
        res.append((post.clone(), gw, gg))
    for post, gw, gg in res[1:]:
        assert torch.equal(post, res[0][0])
        _same_sums(gw, res[0][1])
        _same_sums(gg, res[0][2])


def test_segment_states_in_global_memory_match_shared_memory():
    """[[144,12,12]] with checkpoint 2 keeps the backward segment states in
    shared memory; checkpoint 12 (one segment of 12 iterations) does not fit
    and keeps them in the per-warp global buffer.  Both give the gradients of
    the FP64 oracle adjoint and of each other."""
    import torch
    from paper_2605_14170_gb300 import mbbp
    shots, T = 6, 12
    H, B, s, ex, mu, w, g, t = _setup(code="bb144", R=2, shots=shots, T=T, seed=6)
    n = H.shape[1]
    scale = 1.0 / (shots * B.R * n)
    res = []
    for ckpt in (2, 12):
        post = torch.empty((shots, B.R, n), dtype=torch.float32, device="cuda")
        ws = torch.empty(mbbp.mbbp_wms_workspace_size(B, shots, T, ckpt), dtype=torch.uint8, device="cuda")
        mbbp.mbbp_wms_forward(B, t["s"], t["mu"], T, t["w"], t["g"], ckpt, t["e"], scale, post, None, ws,
                              all_iters=True)
        gw = torch.zeros_like(t["w"])
        gg = torch.zeros_like(t["g"])
        mbbp.mbbp_wms_backward(B, t["s"], t["mu"], T, t["w"], t["g"], ckpt, t["e"], scale, post, gw, gg, ws,
                               all_iters=True)
        torch.cuda.synchronize()
        res.append((gw.cpu().numpy().astype(np.float64), gg.cpu().numpy().astype(np.float64)))
    w32, g32, mu32 = (x.astype(np.float32).astype(np.float64) for x in (w, g, mu))
    gw_ref, gg_ref = np.zeros_like(w32), np.zeros_like(g32)
    for shot in range(shots):
        for b in range(B.R):
            Ht, st, wb, gb, Eb = _oracle_item(H, B, s, mu32, w32, g32, ex, shot, b, scale)
            _, gwb, ggb = oracle.wms_backward(Ht, st, mu32, wb, gb, ex[shot], scale, all_iters=True)
            gw_ref[b][:, :Eb] += gwb
            gg_ref[b][:, :Eb] += ggb
    for gw, gg in res:
        for got, ref in ((gw, gw_ref), (gg, gg_ref)):
            assert np.linalg.norm(got - ref) <= 1e-3 * np.linalg.norm(ref)
    _same_sums(res[0][0], res[1][0])
    _same_sums(res[0][1], res[1][1])


def test_autograd_function_and_adam():
    import torch
    from paper_2605_14170_gb300 import mbbp
    shots, T = 16, 6
    H, B, s, ex, mu, w, g, t = _setup(shots=shots, T=T, seed=5)
    wt = t["w"].clone().requires_grad_(True)
    gt = t["g"].clone().requires_grad_(True)
    loss = mbbp.wms_loss(wt, gt, B, t["s"], t["mu"], t["e"], ckpt=2, all_iters=True)
    loss.backward()
    post = torch.empty((shots, B.R, 72), dtype=torch.float32, device="cuda")
    ws = torch.empty(mbbp.mbbp_wms_workspace_size(B, shots, T, 2), dtype=torch.uint8, device="cuda")
    scale = 1.0 / (shots * B.R * 72)
    mbbp.mbbp_wms_forward(B, t["s"], t["mu"], T, t["w"], t["g"], 2, t["e"], scale, post, None, ws, all_iters=True)
    gw = torch.zeros_like(t["w"])
    gg = torch.zeros_like(t["g"])
    mbbp.mbbp_wms_backward(B, t["s"], t["mu"], T, t["w"], t["g"], 2, t["e"], scale, post, gw, gg, ws, all_iters=True)
    _same_sums(wt.grad, gw)
    _same_sums(gt.grad, gg)
    # Adam against its definition (Kingma & Ba), clamped to [lo, hi]
    rng = np.random.default_rng(0)
    p0 = rng.uniform(0, 1, 1000).astype(np.float32)
    grads = [rng.normal(0, 1, 1000).astype(np.float32) for _ in range(3)]
    p = torch.from_numpy(p0.copy()).cuda()
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    ref, a, v = p0.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for k, gr in enumerate(grads, start=1):
        mbbp.mbbp_adam_step(p, torch.from_numpy(gr).cuda(), m1, m2, 0.01, 0.9, 0.999, 1e-8, k, 0.1, 0.95)
        a = 0.9 * a + 0.1 * gr
        v = 0.999 * v + 0.001 * gr.astype(np.float64) ** 2
        ref = np.clip(ref - 0.01 * (a / (1 - 0.9 ** k)) / (np.sqrt(v / (1 - 0.999 ** k)) + 1e-8), 0.1, 0.95)
    np.testing.assert_allclose(p.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
