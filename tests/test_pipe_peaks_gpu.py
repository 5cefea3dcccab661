"""gfc_measure_pipe_peaks: the measured FP64 FMA, FP32 FMA and binary32
reciprocal rates are positive, repeatable, and ordered as the hardware's
pipes are (the FP32 FMA pipe is many times the FP64 one on this part)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_0752_gb300 as gfc  # noqa: E402


def test_pipe_peaks_are_measured_and_repeatable():
    a = gfc.measure_pipe_peaks(0.05)
    b = gfc.measure_pipe_peaks(0.05)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert a["sm_count"] == sms
    for k in ("dfma_per_s", "dmul_per_s", "dadd_per_s", "ffma_per_s", "rcp32_per_s"):
        assert a[k] > 1e10, (k, a[k])
        assert abs(a[k] - b[k]) <= 0.15 * max(a[k], b[k]), (k, a[k], b[k])
    assert a["ffma_per_s"] > 8 * a["dfma_per_s"]
    # no SM issues more than 128 binary32 FMAs per clock below 3 GHz
    assert a["ffma_per_s"] < sms * 128 * 3.0e9


def test_bad_arguments():
    lib = gfc.load_library()
    assert lib.gfc_measure_pipe_peaks(None, 0.1, None) == -1
    with pytest.raises(gfc.GfcError):
        gfc.measure_pipe_peaks(0.0)
