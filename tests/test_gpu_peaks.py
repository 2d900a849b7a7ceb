"""The library's peak-rate microbenchmarks (op_peak_rate), the roofline denominators of
the bench: every rate is positive and of the order the part is built for; the BF16 MMA at
N = 64 (the shape of the FP64 digit products) with a new A tile every MMA runs near half the
N = 256 rate, and with A held in the collector buffer over four MMAs near the full rate."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2511_06788_gb300 as pkg  # noqa: E402


def test_peak_rates_are_sane():
    r = {k: pkg.binding.peak_rate(k) for k in ("fp64_fma", "tf32_mma", "bf16_mma",
                                               "bf16_mma_n64", "bf16_mma_n64_areuse")}
    print(r)
    assert 0.3 < r["fp64_fma"] < 5.0            # TFLOP/s: GB300's FP64 FMA is ~1
    assert 300 < r["bf16_mma"] < 3500
    assert 0.35 < r["tf32_mma"] / r["bf16_mma"] < 0.65
    # N = 64 with a new A tile every MMA: the A reads hold it near half the N = 256 rate
    assert 0.3 < r["bf16_mma_n64"] / r["bf16_mma"] < 0.7
    # A held in the collector buffer over four MMAs lifts N = 64 to most of the N = 256 rate
    assert 1.3 * r["bf16_mma_n64"] < r["bf16_mma_n64_areuse"] < 1.1 * r["bf16_mma"]


def test_peak_rate_rejects_unknown_kinds():
    import ctypes as C
    v = C.c_double()
    assert pkg.lib().op_peak_rate(9, C.byref(v), None) == pkg.binding.OP_ERR_ARG
