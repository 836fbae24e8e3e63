"""The headless display path (row grouping, causal display filter, column
grouping, ring buffer) against the oracle's View, under random chunkings that
leave columns incomplete across pushes and wrap the ring many times."""
import numpy as np
import pytest

from gpu_helpers import TOL, normwise
from paper_2605_20132_gb300 import abi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def run_both(ora, x, chunks, kc, kt, W, mode, sos=None, snapshots=(2, 5)):
    """Push the same chunks through both; compare the images after some pushes."""
    import torch
    from paper_2605_20132_gb300.chain import View
    N, C = x.shape
    v = View(C, kc, kt, W, mode, sos, max_chunk=max(chunks))
    o = ora.View(C, kc, kt, W, mode, sos)
    xd = torch.from_numpy(x).cuda()
    t = 0
    worst = 0.0
    for i, k in enumerate(chunks):
        v.push(xd[t:t + k])
        o.push(x[t:t + k])
        t += k
        if i in snapshots or i == len(chunks) - 1:
            got = v.image().cpu().numpy().astype(np.float64)
            ref = o.image()
            if sos is None and mode != abi.FILARK_VIEW_LINEAR:
                assert np.array_equal(got, ref), (i, mode)
            else:
                worst = max(worst, normwise(got.T, ref.T))
    info = v.info()
    v.close()
    assert info["columns"] == len(o.cols)
    assert info["ring_offset"] == len(o.cols) % W
    return worst


def chunking(rng, N, hi):
    out = []
    while sum(out) < N:
        out.append(int(min(rng.integers(1, hi + 1), N - sum(out))))
    return out


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("kc,kt,W", [(1, 1, 64), (3, 7, 50), (4, 32, 40), (5, 100, 16)])
def test_view_matches_oracle(oracle_mod, mode, kc, kt, W):
    rng = np.random.default_rng(150 + 10 * mode + kt)
    x = synth.small_stream(37, 6000, seed=150 + kt)
    chunks = chunking(rng, 6000, 400)
    worst = run_both(oracle_mod, x, chunks, kc, kt, W, mode)
    assert worst <= 1e-6, worst


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("kc", [1, 2, 3, 5, 6, 8])
def test_view_vector_rows_match_oracle(oracle_mod, mode, kc):
    """Channel counts and row strides that are multiples of 4 (16-byte row
    loads, several rows per thread) with a ragged last group of rows."""
    rng = np.random.default_rng(170 + 10 * mode + kc)
    x = synth.small_stream(44, 3000, seed=170 + kc)
    chunks = chunking(rng, 3000, 500)
    worst = run_both(oracle_mod, x, chunks, kc, 9, 40, mode)
    assert worst <= 1e-6, worst


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_view_display_filter(oracle_mod, mode):
    """Render-time causal display filter (order-4 1-50 Hz bandpass at 1 kHz)
    with its state kept across pushes."""
    rng = np.random.default_rng(160 + mode)
    x = synth.small_stream(48, 8000, seed=160)
    sos = oracle_mod.butter_bandpass(4, 1.0, 50.0, 1000.0)
    chunks = chunking(rng, 8000, 700)
    worst = run_both(oracle_mod, x, chunks, 4, 10, 256, mode, sos)
    print("view with display filter, mode", mode, worst)
    assert worst <= TOL


def test_view_reset_and_errors():
    import torch
    from paper_2605_20132_gb300.chain import View
    x = torch.randn((500, 10), device="cuda")
    v = View(10, 2, 5, 30, abi.FILARK_VIEW_PEAK, max_chunk=500)
    v.push(x)
    a = v.image()
    v.reset()
    assert torch.count_nonzero(v.image()) == 0
    v.push(x)
    assert torch.equal(v.image(), a)
    assert abi.load().filark_view_push(v._h, x.data_ptr(), 10, 501, None) == abi.FILARK_EINVAL
    v.close()
