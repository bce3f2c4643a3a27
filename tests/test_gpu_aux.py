"""GPU sampler, syndrome and logical judge against the oracle (bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2605_14170_gb300.inputs import named_code

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2605_14170_gb300 import mbbp
    return mbbp


@pytest.mark.parametrize("n,noise,p", [(144, "depolarizing", 0.08), (72, "bsc", 0.05),
                                       (882, "depolarizing", 0.03), (37, "bsc", 0.3)])
def test_sampler_matches_oracle(M, n, noise, p):
    import torch
    batch, first = 700, 123456789
    W = (n + 31) // 32
    ex = torch.empty((batch, W), dtype=torch.int32, device="cuda")
    ez = torch.empty((batch, W), dtype=torch.int32, device="cuda")
    M.mbbp_sample_errors(n, batch, first, 42, p, 0 if noise == "bsc" else 1, ex, ez)
    rx, rz = oracle.sample(42, first, batch, n, p, noise)
    assert np.array_equal(M.unpack_words(ex, n), rx)
    assert np.array_equal(M.unpack_words(ez, n), rz)
    # any split of the shots gives the same errors
    part = torch.empty((100, W), dtype=torch.int32, device="cuda")
    M.mbbp_sample_errors(n, 100, first + 250, 42, p, 0 if noise == "bsc" else 1, part)
    assert np.array_equal(M.unpack_words(part, n), rx[250:350])


@pytest.mark.parametrize("code", ["bb72", "bb144", "gb882"])
def test_syndrome_matches_oracle(M, code):
    import torch
    c = named_code(code)
    H = c.HZ
    rng = np.random.default_rng(2)
    e = (rng.random((500, H.shape[1])) < 0.05).astype(np.uint8)
    B = M.mbbp_build_bases_from_sets(H, [[]])
    s = torch.empty((500, H.shape[0]), dtype=torch.uint8, device="cuda")
    M.mbbp_syndrome(B, torch.from_numpy(M.pack_bits(e)).cuda(), s)
    assert np.array_equal(s.cpu().numpy(), oracle.syndrome(H, e))


def test_logicals_count(M):
    for code, k in (("bb72", 12), ("bb144", 12)):
        c = named_code(code)
        L = M.mbbp_logicals_build(c.HZ, c.HX)
        assert L.k == k
        ops = L.ops()
        assert not ((c.HX.astype(int) @ ops.T) % 2).any()  # ops lie in ker(H_X)
        assert oracle.gf2_rank(np.concatenate([c.HZ, ops])) == oracle.gf2_rank(c.HZ) + k


def test_judge_matches_oracle(M):
    import torch
    c = named_code("bb72")
    H, Ho = c.HZ, c.HX
    n = H.shape[1]
    rng = np.random.default_rng(5)
    e = (rng.random((400, n)) < 0.05).astype(np.uint8)
    ehat = e.copy()
    # mix of exact, stabilizer-shifted, random and syndrome-breaking estimates
    for b in range(400):
        kind = b % 4
        if kind == 1:
            ehat[b] ^= Ho[rng.integers(0, Ho.shape[0])]
        elif kind == 2:
            ehat[b] = (rng.random(n) < 0.05).astype(np.uint8)
        elif kind == 3:
            ehat[b, rng.integers(0, n)] ^= 1
    # a few residuals that are X-type logical operators: ker(H_Z) mod rowspace(H_X)
    L = M.mbbp_logicals_build(H, Ho)
    xops = M.mbbp_logicals_build(Ho, H).ops()
    for b in range(0, 400, 37):
        ehat[b] = e[b] ^ xops[b % len(xops)]
    fail = torch.empty(400, dtype=torch.uint8, device="cuda")
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    M.mbbp_judge(L, torch.from_numpy(M.pack_bits(e)).cuda(), torch.from_numpy(ehat).cuda(), fail, counts)
    ref = oracle.judge(H, Ho, e, ehat)
    got = fail.cpu().numpy()
    assert np.array_equal(got, ref)
    assert counts.cpu().numpy().tolist() == np.bincount(ref, minlength=3).tolist()
    assert (ref == 2).sum() >= 5 and (ref == 1).sum() >= 50
