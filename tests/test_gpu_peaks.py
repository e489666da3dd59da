"""The roofline microbenchmarks (slm_measure_peaks) measure plausible roofs:
FP32 FFMA throughput between a quarter and 1.1x of the nominal rate of 152
SMs x 128 lanes x 2 flop at 2.07 GHz (clocks may run lower under load), and
an L2 read bandwidth above the measured HBM copy rate (the buffer is L2
resident) and below 100 TB/s; a call with both outputs NULL is refused."""
import ctypes
import json
import os

import pytest

pytestmark = pytest.mark.gpu


def test_measured_roofs_are_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07023_gb300 import binding as S
    m = S.measure_peaks(0)
    nominal = 152 * 128 * 2 * 2.07e9 / 1e12
    assert 0.25 * nominal < m["ffma_tflops"] < 1.1 * nominal, m
    hbm = 6000.0
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(root, "MEASURED_PEAKS.json")) as f:
            hbm = float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        pass
    assert hbm < m["l2_read_gbs"] < 100_000.0, (m, hbm)
    assert S.lib().slm_measure_peaks(0, None, None, None) == S.SLM_EINVAL
