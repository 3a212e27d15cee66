"""The unit-rate probe (kkm_probe_unit_rate) on the GPU: the rates it reports
per SM and clock lie within what a Blackwell SM can issue, and its device-wide
rate agrees with the per-SM rate at a plausible SM clock."""
import pytest

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def test_unit_rates_are_plausible():
    torch = torch_cuda()
    from paper_2410_05902_gb300 import kkm
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = kkm.unit_rates()
    # an SM has 4 schedulers issuing one warp instruction per clock: at most
    # 128 lanes per clock for any one pipe, 256 FP32 FMAs for packed f32x2
    assert 2.0 <= r["ex2_per_clk_sm"] <= 128.0
    assert 16.0 <= r["ffma_per_clk_sm"] <= 128.5
    assert 16.0 <= r["ffma2_fp32_per_clk_sm"] <= 256.5
    for key in ("ex2", "ffma"):
        mhz = r[f"{key}_per_s"] / (sms * r[f"{key}_per_clk_sm"]) / 1e6
        assert 300.0 <= mhz <= 2600.0, (key, mhz)


def test_bounded_wait_runs_out_and_reports_a_timeout():
    """Failure detection without a fault: the tcgen05 passes' bounded mbarrier
    wait, on a barrier nothing arrives on, gives up after its limit and the
    host sees KKM_ETIMEOUT; the context stays usable (the control that arrives
    returns KKM_OK on the same device right after)."""
    import time
    torch = torch_cuda()
    from paper_2410_05902_gb300 import kkm
    stream = torch.cuda.current_stream().cuda_stream
    limit_ns = 2_000_000
    t0 = time.perf_counter()
    st = kkm.kkm_probe_bounded_wait(limit_ns, False, stream)
    elapsed = time.perf_counter() - t0
    assert st == kkm.KKM_ETIMEOUT
    assert elapsed >= limit_ns * 1e-9
    assert kkm.kkm_probe_bounded_wait(limit_ns, True, stream) == kkm.KKM_OK
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum().cpu()) == 8.0
