"""Fault paths on the GPU that need no fault: a device allocation that cannot succeed is
reported as TDAGW_ERR_OOM and leaves the device usable."""
import pytest

import workloads as wl

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_build_reports_oom_for_a_kernel_larger_than_device_memory():
    import paper_2502_05635_gb300 as tg
    p = wl.ModelParams(L=400)                      # N = 640000: the dense K needs 3.3 TB
    h = tg.tdagw_create(tg.model_desc(p, tg.C64), torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(tg.TdagwError) as e:
            tg.tdagw_build_kernel(h)
        assert e.value.code == tg.ERR_OOM and "cudaMalloc" in str(e.value)
        with pytest.raises(tg.TdagwError) as e:     # nothing half-built is usable
            tg.tdagw_propagate(h, [tg.make_field(wl.Pulse())], [2], 0.2, tg.FULL)
        assert e.value.code == tg.ERR_NOT_BUILT
    finally:
        tg.tdagw_destroy(h)
    x = torch.ones(8, device="cuda")
    assert float(x.sum()) == 8.0
