"""mbbp_decode_noalloc: the decode entry point for callers that cannot
allocate device memory (for example a decoder inside a real-time control loop,
where an allocation could block or fail mid-run).  Its scratch is a fixed
array inside the library, so this file checks, through the C ABI, that two
calls in a row give exactly what mbbp_decode gives with a caller-owned
workspace, that stale scratch from an earlier call does not leak into a
later one (the third call repeats the first code and size on other shots),
and that a batch too large for the array is refused.  It is collected
last on purpose, and passes alone in a fresh process as well."""
import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import channel_llr, named_code

pytestmark = pytest.mark.gpu


def _outputs(torch, batch, B, dev):
    return {
        "e_hat": torch.full((batch, B.n), 7, dtype=torch.uint8, device=dev),
        "conv": torch.full((batch, B.R), 7, dtype=torch.uint8, device=dev),
        "iters": torch.full((batch, B.R), -1, dtype=torch.int16, device=dev),
        "success": torch.full((batch,), 7, dtype=torch.uint8, device=dev),
        "selected": torch.full((batch,), 99, dtype=torch.int16, device=dev),
    }


def test_noalloc_matches_workspace_decode_on_two_calls():
    import torch
    from paper_2605_14170_gb300 import mbbp
    dev = torch.device("cuda:0")
    # calls in a row: the third repeats the first code and size on other
    # shots, so it reads a scratch region that the first call filled with
    # different candidates (and the second overwrote only in part)
    cases = [("bb144", "HZ", 16, 3000, 0.06, 100, 777), ("bb72", "HX", 4, 1200, 0.05, 50, 777),
             ("bb144", "HZ", 16, 3000, 0.07, 100, 778)]
    for code, which, R, batch, p, iters, seed in cases:
        c = named_code(code)
        H = getattr(c, which)
        ex, ez = oracle.sample(seed, 0, batch, H.shape[1], p, "depolarizing")
        s = oracle.syndrome(H, ex if which == "HZ" else ez)
        llr = torch.from_numpy(channel_llr(H.shape[1], 2 * p / 3).astype(np.float32)).to(dev)
        syn = torch.from_numpy(s).to(dev)
        B = mbbp.mbbp_build_bases(H, R, 5)
        ref = mbbp.decode(B, syn, llr, iters, 0.625)
        got = _outputs(torch, batch, B, dev)
        mbbp.mbbp_decode_noalloc(B, syn, llr, iters, 0.625, mbbp.RULE_NMS, got["e_hat"], got["conv"],
                                 got["success"], iters_run=got["iters"], selected=got["selected"])
        torch.cuda.synchronize()
        for key in ("e_hat", "conv", "iters", "success", "selected"):
            assert torch.equal(got[key], ref[key]), (code, key)


def test_noalloc_rejects_batches_beyond_the_fixed_scratch():
    import torch
    from paper_2605_14170_gb300 import mbbp
    dev = torch.device("cuda:0")
    c = named_code("bb144")
    B = mbbp.mbbp_build_bases(c.HZ, 16, 5)
    batch = 40000  # 40000 * 16 * 5 * 4 bytes > 8 MiB
    syn = torch.zeros((batch, 72), dtype=torch.uint8, device=dev)
    llr = torch.ones(144, dtype=torch.float32, device=dev)
    out = _outputs(torch, batch, B, dev)
    with pytest.raises(mbbp.MBBPError) as err:
        mbbp.mbbp_decode_noalloc(B, syn, llr, 10, 0.625, mbbp.RULE_NMS, out["e_hat"], out["conv"],
                                 out["success"])
    assert err.value.status == 2 and "fixed scratch" in str(err.value)
    torch.cuda.synchronize()
    assert (out["success"] == 7).all()  # nothing was launched
