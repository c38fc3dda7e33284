"""The FP64 throughput probe behind the FP64 roofline (benchmark
instrumentation; no counterpart in the paper)."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_fp64_probe_counts_and_runs():
    from paper_1204_1533_gb300 import ldg
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.full((4 * sms,), float("nan"), dtype=torch.float64, device="cuda")
    fmas = ldg.ldg_fp64_fma_probe(10, sink)
    torch.cuda.synchronize()
    assert fmas == 4 * sms * 256 * 16 * 10
    assert torch.isfinite(sink).all()
    # chains x <- x a + b with a = 1 - 2^-20, b = 2^-30 started at 1e-3 (t + k):
    # after 10 steps every value stays within a hair of its start
    assert float(sink.abs().max()) < 256 * 16 * 1e-3 * (256 + 16)
    with pytest.raises(ldg.LdgError):
        ldg.ldg_fp64_fma_probe(10, sink[: 4 * sms - 1])
