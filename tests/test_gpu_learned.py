"""Learned weights: WMS trained on the GPU by the library's own kernels
(sampler, syndrome, WMS forward, hand-written adjoint, Adam), selected on
held-out shots, against plain MBBP-LD on identical fresh shots.

The initial weights (w = alpha, g = 0) reproduce plain MBBP-LD bit for bit
and take part in the validation-based selection, so the learned decoder
can only match or beat plain MBBP-LD on the validation shots; this test
checks that it does at least as well on unseen shots and reports the gain.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_trained_weights_do_not_lose_to_plain_mbbp_ld():
    import torch
    from paper_2605_14170_gb300 import learn, mbbp
    from paper_2605_14170_gb300.inputs import named_code
    c = named_code("bb144")
    B = mbbp.mbbp_build_bases(c.HZ, 8, 20260515)
    L = mbbp.mbbp_logicals_build(c.HZ, c.HX)
    w, g, hist = learn.train_wms(B, 0.05, T=25, ckpt=5, batch=2048, steps=150, lr=1e-3, L=L,
                                 val_shots=30000, val_every=25, log_every=0)
    losses = [h[1] for h in hist if h[1] is not None]
    assert losses[-1] < losses[0]  # the BCE went down
    assert torch.isfinite(w).all() and torch.isfinite(g).all()
    assert float(w.min()) >= 0.0 and float(g.max()) <= 0.9
    r = learn.compare_ler(B, L, w, g, 0.04, 100000, 100)
    print("learned vs plain at p=0.04:", r["learned"]["failures"], r["plain"]["failures"])
    assert r["learned"]["failures"] <= r["plain"]["failures"]
