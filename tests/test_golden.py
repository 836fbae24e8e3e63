"""Values the paper prints, held against this implementation's workload and
byte accounting (no GPU needed).

tests/golden/data_volume_sec1.txt: the paper's sizing example in Sec. 1 (6,000
channels at 1,500 Hz in single precision, about 3 TB per day).  The
paper-scale workload must have that shape, the chain's sample type must be
4-byte floats, and the benchmark's algorithmic bytes must count the input at
4 bytes per channel-sample, so that a day of pushes reads the printed volume.

tests/golden/ooi_band_sec6.txt: the 15-32 Hz band of the paper's OOI filtering
example (Sec. 6).  A Butterworth bandpass designed by the bilinear transform
with prewarped edges has |H| = 1/sqrt(2) exactly at both edges and 1 at the
image of the geometric centre, for every order and sampling rate; both the
oracle's designer and the library's host designer must show it on this band.
"""
import ctypes as ct
import math
import os

import numpy as np
import pytest

from oracle_pins import sos_response

HERE = os.path.dirname(__file__)


def load_fixture(name: str) -> dict:
    out = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def test_paper_scale_workload_matches_the_sizing_example():
    from paper_2605_20132_gb300 import synth
    g = load_fixture("data_volume_sec1.txt")
    w = synth.PAPER_SCALE
    assert w["n_channels"] == g["channels"]
    assert w["fs"] == g["fs_hz"]
    # one chunk per second of recording, as in the paper's streaming setting
    assert w["chunk"] == g["fs_hz"]


def test_sample_type_and_daily_volume():
    from paper_2605_20132_gb300 import synth
    g = load_fixture("data_volume_sec1.txt")
    assert ct.sizeof(ct.c_float) == g["bytes_per_sample"] == np.dtype(np.float32).itemsize
    x = synth.small_stream(4, 16, seed=1)
    assert x.dtype == np.float32
    per_day = g["channels"] * g["fs_hz"] * g["bytes_per_sample"] * 86400
    assert round(per_day / 1e12) == g["tb_per_day_approx"]


def test_benchmark_counts_the_input_at_the_printed_rate():
    import bench
    g = load_fixture("data_volume_sec1.txt")
    C, T = int(g["channels"]), int(g["fs_hz"])
    b = int(g["bytes_per_sample"])
    # one more sample per channel (windows longer than the push, so the
    # history terms grow too): input, ratio, its history write and the two
    # exiting values read back (STA and LTA windows), each one float
    grow = bench.algorithmic_bytes_per_push(C, T + 1, 8, T + 10, T + 10) - \
        bench.algorithmic_bytes_per_push(C, T, 8, T + 10, T + 10)
    assert grow == 5 * b * C
    # a day of one-second pushes reads the printed volume of input
    assert round(C * b * T * 86400 / 1e12) == g["tb_per_day_approx"]


def _response(sos, f, fs):
    return float(abs(sos_response(sos, np.array([2.0 * np.pi * f / fs]))[0]))


@pytest.mark.parametrize("fs", [100.0, 200.0, 500.0, 1000.0])
@pytest.mark.parametrize("order", [2, 4, 8])
def test_paper_band_edges_and_centre(oracle_mod, fs, order):
    from paper_2605_20132_gb300.chain import butter_bandpass
    g = load_fixture("ooi_band_sec6.txt")
    f1, f2 = g["f1_hz"], g["f2_hz"]
    w1, w2 = (2 * fs * math.tan(math.pi * f / fs) for f in (f1, f2))
    f0 = fs / math.pi * math.atan(math.sqrt(w1 * w2) / (2 * fs))   # centre's image
    for sos in (oracle_mod.butter_bandpass(order, f1, f2, fs), butter_bandpass(order, f1, f2, fs)):
        assert sos.shape == (order, 6)
        for f in (f1, f2):
            assert abs(_response(sos, f, fs) - 1 / math.sqrt(2)) < 1e-9
        assert abs(_response(sos, f0, fs) - 1.0) < 1e-9
        # and it is a bandpass: DC and Nyquist are blocked
        assert _response(sos, 0.0, fs) < 1e-12 and _response(sos, fs / 2, fs) < 1e-12
