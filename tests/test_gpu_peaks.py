"""The instruction-rate microbenchmarks behind the rooflines (hd_measure_peak):
each kind runs, reports a rate within the physically possible range of a
GB300 (152 SMs at up to 2.07 GHz), and the operand types keep the ratios the
tensor core's kinds have (kind::f8f6f4 runs e2m1 and e4m3 at one rate, about
twice kind::f16)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_16422_gb300 import build, hd as _hd
    build.build()
    return _hd


def test_peaks_in_physical_range(hd):
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    f_max = 2.2e9   # above GB300's 2.07 GHz maximum SM clock
    r = {k: hd.hd_measure_peak(k, 5) for k in ("tc_fp4", "tc_fp8", "tc_bf16", "tc_mxf4", "popc", "lop3")}
    for k, v in r.items():
        assert v["launches"] == 5 and v["best_per_s"] >= v["median_per_s"] > 0, k
    # dense kind::f8f6f4: 8192 multiply-adds per clock per SM at most
    for k in ("tc_fp4", "tc_fp8"):
        assert 0.3 * n_sm * 16384 * 1.0e9 < r[k]["best_per_s"] <= n_sm * 16384 * f_max, (k, r[k])
    assert 0.75 < r["tc_fp4"]["best_per_s"] / r["tc_fp8"]["best_per_s"] < 1.33
    assert 1.5 < r["tc_fp8"]["best_per_s"] / r["tc_bf16"]["best_per_s"] < 2.5
    # block-scaled kind::mxf4 (its warm-up launch verified exact sums): 16384 multiply-adds per clock per SM
    assert 1.5 < r["tc_mxf4"]["best_per_s"] / r["tc_fp8"]["best_per_s"] <= 3.1
    assert r["tc_mxf4"]["best_per_s"] <= n_sm * 3 * 16384 * f_max
    # popcount unit: 16 per clock per SM; logic pipe: 64 per clock per SM
    assert 0.2 * n_sm * 16 * 1.0e9 < r["popc"]["best_per_s"] <= n_sm * 16 * f_max * 1.05
    assert 0.2 * n_sm * 64 * 1.0e9 < r["lop3"]["best_per_s"] <= n_sm * 64 * f_max * 1.05
    with pytest.raises(hd.HDError):
        hd.hd_measure_peak("popc", 0)
