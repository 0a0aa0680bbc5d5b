"""The FMA throughput probe (the denominator of the arithmetic roofline)
reports a flop count that, divided by its CUDA-event time, lands in the range
GB300's FP32 and FP64 pipes allow: FP32 between 30 and 100 TFLOP/s (nominal
152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5), FP64 between 0.3 and 5
TFLOP/s (nominal about 1.3)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import mgenkf
    return mgenkf


@pytest.mark.parametrize("fp64,lo,hi,iters", [(0, 30e12, 100e12, 4096), (1, 0.3e12, 5e12, 256)])
def test_fma_probe_rate(M, fp64, lo, hi, iters):
    import torch
    n = M.mgk_fma_probe_threads()
    assert n > 0
    sink = torch.zeros(n, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
    M.mgk_fma_probe(fp64, iters, sink)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    flops = M.mgk_fma_probe(fp64, iters, sink)
    e1.record()
    torch.cuda.synchronize()
    rate = flops / (e0.elapsed_time(e1) / 1e3)
    assert lo < rate < hi, rate
    assert torch.isfinite(sink).all()
    with pytest.raises(M.MGEnKFError):
        M.mgk_fma_probe(fp64, 0, sink)
