"""Throughput probes (the per-SM rates behind the BP roofline): each launch
reports the work it performs, and the measured rates fall in the range a
GB300 SM can deliver (at most 128 lanes and 128 shared-memory bytes per SM
per clock, at a clock of at most about 2.1 GHz)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_probe_work_and_rate(kind):
    import torch
    from paper_2605_14170_gb300 import mbbp
    dev = torch.device("cuda:0")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    rounds = 512
    work = mbbp.mbbp_probe(kind, rounds, sink)  # first launch sets the kernel attributes
    per_round = 128 if kind == mbbp.PROBE_SMEM else 64
    # 2 blocks of 1024 threads per SM
    assert work == 2 * sms * 1024 * rounds * per_round
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    work = mbbp.mbbp_probe(kind, 4 * rounds, sink)
    e1.record()
    torch.cuda.synchronize()
    per_sm_per_ns = work / (e0.elapsed_time(e1) * 1e6) / sms
    assert 10.0 < per_sm_per_ns < 128 * 2.2
