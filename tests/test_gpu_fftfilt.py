"""Overlap-add FFT filtering against the FP64 oracle's direct FIR (the
exact linear convolution), for filter lengths up to thousands of taps, block
lengths that give every FFT size, odd channel counts (channel pairs share a
transform) and random chunkings."""
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


def run(x, taps, chunks, block_len=0):
    import torch
    from paper_2605_20132_gb300.chain import FFTFilter
    N, C = x.shape
    f = FFTFilter(C, taps, block_len, max_chunk=max(chunks))
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    t = 0
    for k in chunks:
        f.push(xd[t:t + k], yd[t:t + k])
        t += k
    torch.cuda.synchronize()
    info = (f.fft_len, f.block_len)
    f.close()
    return yd.cpu().numpy().astype(np.float64), info


@pytest.mark.parametrize("M,block_len", [(1, 0), (2, 0), (3, 0), (5, 0), (9, 0), (31, 0), (100, 0), (257, 100),
                                         (257, 0), (1001, 0), (1500, 0), (4001, 0), (2000, 6000)])
def test_fftfilt_matches_direct_fir(oracle_mod, M, block_len):
    rng = np.random.default_rng(130 + M)
    C = 9
    x = synth.small_stream(C, 30000, seed=130 + M)
    h = synth.windowed_sinc_bandpass(M, 1.0, 50.0, 1000.0) if M > 1 else np.array([0.7])
    chunks = []
    while sum(chunks) < 30000:
        chunks.append(int(min(rng.integers(1, 9000), 30000 - sum(chunks))))
    got, info = run(x, h, chunks, block_len)
    ref = oracle_mod.TemporalOp(C, oracle_mod.TOP_FIR, M, h.astype(np.float32).astype(np.float64)).push(x)
    err = normwise(got, ref)
    print("fftfilt", M, block_len, info, err)
    assert info[0] >= info[1] + M - 1
    assert err <= TOL


@pytest.mark.parametrize("M", [1, 2, 3, 5, 17, 100, 700])
def test_fftfilt_every_transform_size(oracle_mod, M):
    """Pushes of many lengths make every transform size 2^k and 3 * 2^k
    between M and the largest appear (each block uses the smallest size that
    holds its convolution)."""
    C = 5
    lens = [1, 2, 3, 4, 5, 6, 7, 9, 10, 13, 20, 30, 50, 64, 97, 128, 200, 300, 513, 1000, 1537, 2100]
    N = sum(lens)
    x = synth.small_stream(C, N, seed=150 + M)
    h = synth.windowed_sinc_bandpass(M, 1.0, 50.0, 1000.0) if M > 2 else np.array([0.6, -0.3][:M])
    got, info = run(x, h, lens)
    ref = oracle_mod.TemporalOp(C, oracle_mod.TOP_FIR, M, h.astype(np.float32).astype(np.float64)).push(x)
    err = normwise(got, ref)
    print("sizes", M, info, err)
    assert err <= TOL


def test_fftfilt_reset_and_errors(oracle_mod):
    import torch
    from paper_2605_20132_gb300.chain import FFTFilter
    h = synth.windowed_sinc_bandpass(401, 2.0, 40.0, 1000.0)
    x = torch.from_numpy(synth.small_stream(4, 5000, seed=140)).cuda()
    f = FFTFilter(4, h, max_chunk=5000)
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    f.push(x, y1)
    f.reset()
    f.push(x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    assert abi.filark_fftfilt_push(f._h, x.data_ptr(), 4, 5001, y1.data_ptr(), 4, None) == abi.FILARK_EINVAL
    f.close()
    # a block that does not fit the 8192-point transform is shortened
    g = FFTFilter(4, h, block_len=9000, max_chunk=100)
    assert g.block_len == 8192 - 401 + 1 and g.fft_len == 8192
    g.close()
    st, _ = abi.filark_fftfilt_create(4, np.array([1.0, np.nan]), 0, 100, 0)
    assert st == abi.FILARK_EINVAL


@pytest.mark.parametrize("M,block_len,N", [(4097, 0, 30000), (5000, 0, 30000), (9000, 1000, 30000),
                                           (12289, 0, 24000), (20001, 0, 16000), (3000, 7000, 30000)])
def test_fftfilt_long_filters(oracle_mod, M, block_len, N):
    """Filters beyond the single 8192-point transform: partitions of 4096
    taps (the block transformed once, one inverse transform per partition,
    overhangs completed by the next partition), against the direct FIR; and
    a block too long for a 3000-tap filter, shortened to fit.  Five channels
    (the last pair has one channel), chunks of 1 to 9000 samples, so blocks
    of every length up to 4096 occur."""
    rng = np.random.default_rng(160 + M)
    C = 5
    x = synth.small_stream(C, N, seed=160 + M)
    h = synth.windowed_sinc_bandpass(M, 0.5, 50.0, 1000.0)
    chunks = [1, 4096, 4097]
    while sum(chunks) < N:
        chunks.append(int(min(rng.integers(1, 9000), N - sum(chunks))))
    got, info = run(x, h, chunks, block_len)
    ref = oracle_mod.TemporalOp(C, oracle_mod.TOP_FIR, M, h.astype(np.float32).astype(np.float64)).push(x)
    err = normwise(got, ref)
    print("fftfilt long", M, block_len, info, err)
    assert info[0] <= 8192
    if M > 4096:
        assert info[1] == (block_len or 4096)
    assert err <= TOL
