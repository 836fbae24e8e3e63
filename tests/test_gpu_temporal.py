"""Parity of the stateful temporal operators (FIR, running mean, running AGC,
EMA gain equalisation) with the FP64 oracle, pushed in chunks of many sizes
(the streaming contract), at 1e-5 normwise per channel."""
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


def run_gpu_op(kind, x, chunks, length=1, taps=None, alpha=0.0, ld_in=None, ld_out=None):
    import torch
    from paper_2605_20132_gb300.chain import TemporalOp
    N, C = x.shape
    op = TemporalOp(kind, C, length, taps, alpha, max_chunk=max(chunks))
    li, lo = ld_in or C, ld_out or C
    xd = torch.zeros((N, li), device="cuda")
    xd[:, :C] = torch.from_numpy(x).cuda()
    yd = torch.full((N, lo), float("nan"), device="cuda")
    t = 0
    for k in chunks:
        op.push(xd[t:t + k], yd[t:t + k])
        t += k
    torch.cuda.synchronize()
    op.close()
    if lo > C:
        assert torch.isnan(yd[:, C:]).all()
    return yd[:, :C].cpu().numpy().astype(np.float64)


def run_oracle_op(ora, kind, x, length=1, taps=None, alpha=0.0):
    return ora.TemporalOp(x.shape[1], kind, length, taps, alpha).push(x)


def random_chunks(rng, N, hi):
    out = []
    while sum(out) < N:
        out.append(int(min(rng.integers(1, hi + 1), N - sum(out))))
    return out


@pytest.mark.parametrize("M", [1, 5, 32, 33, 101, 512])
def test_fir_matches_oracle(oracle_mod, M):
    rng = np.random.default_rng(90 + M)
    x = synth.small_stream(70, 6000, seed=90 + M)
    h = rng.standard_normal(M) / np.sqrt(M)
    chunks = random_chunks(rng, 6000, 900)
    got = run_gpu_op(abi.FILARK_TOP_FIR, x, chunks, M, h, ld_in=75, ld_out=72)
    ref = run_oracle_op(oracle_mod, oracle_mod.TOP_FIR, x, M, h.astype(np.float32).astype(np.float64))
    err = normwise(got, ref)
    print("FIR", M, err)
    assert err <= TOL


@pytest.mark.parametrize("M", [7, 101, 300])
def test_fir_aligned_rows_match_oracle(oracle_mod, M):
    """Row strides and channel counts that are multiples of 4 (16-byte tile loads)."""
    rng = np.random.default_rng(95 + M)
    x = synth.small_stream(68, 5000, seed=95 + M)
    h = rng.standard_normal(M) / np.sqrt(M)
    chunks = random_chunks(rng, 5000, 1200)
    got = run_gpu_op(abi.FILARK_TOP_FIR, x, chunks, M, h, ld_in=72, ld_out=76)
    ref = run_oracle_op(oracle_mod, oracle_mod.TOP_FIR, x, M, h.astype(np.float32).astype(np.float64))
    assert normwise(got, ref) <= TOL


@pytest.mark.parametrize("kind", ["mean", "agc"])
@pytest.mark.parametrize("w", [1, 50, 1000, 3000])
def test_window_ops_match_oracle(oracle_mod, kind, w):
    rng = np.random.default_rng(100 + w)
    x = synth.small_stream(96, 12000, seed=100 + w)
    x[7000:9500, :10] = 0.0        # windows that empty out (AGC gives exact zeros)
    chunks = random_chunks(rng, 12000, 2500)
    k = abi.FILARK_TOP_MEAN if kind == "mean" else abi.FILARK_TOP_AGC
    got = run_gpu_op(k, x, chunks, w)
    ref = run_oracle_op(oracle_mod, oracle_mod.TOP_MEAN if kind == "mean" else oracle_mod.TOP_AGC, x, w)
    err = normwise(got, ref)
    print(kind, w, err)
    assert err <= TOL
    if kind == "agc" and w <= 1000:
        assert np.all(got[9500 - 1:9500, :10] == 0.0)


@pytest.mark.parametrize("alpha", [1.0, 0.3, 1e-2, 1e-4, 1e-6])
def test_ema_matches_oracle(oracle_mod, alpha):
    rng = np.random.default_rng(110)
    x = synth.small_stream(40, 20000, seed=111)
    x[:300] = 0.0                  # e = 0 -> y = 0 at the start
    chunks = random_chunks(rng, 20000, 3000)
    got = run_gpu_op(abi.FILARK_TOP_EMA, x, chunks, alpha=alpha)
    ref = run_oracle_op(oracle_mod, oracle_mod.TOP_EMA, x, alpha=alpha)
    err = normwise(got, ref)
    print("EMA", alpha, err)
    assert err <= TOL
    assert np.all(got[:300] == 0.0)


def test_operators_chunk_invariant_and_reset(oracle_mod):
    """Bitwise: the same operator gives the same output for two chunkings
    after a reset."""
    import torch
    from paper_2605_20132_gb300.chain import TemporalOp
    x = torch.from_numpy(synth.small_stream(64, 5000, seed=120)).cuda()
    for kind, kw in [(abi.FILARK_TOP_FIR, dict(length=40, taps=np.linspace(-1, 1, 40))),
                     (abi.FILARK_TOP_MEAN, dict(length=300)), (abi.FILARK_TOP_AGC, dict(length=300)),
                     (abi.FILARK_TOP_EMA, dict(alpha=0.01))]:
        op = TemporalOp(kind, 64, max_chunk=5000, **kw)
        outs = []
        for chunks in ([5000], [1, 999, 2048, 1952]):
            y = torch.empty_like(x)
            t = 0
            for k in chunks:
                op.push(x[t:t + k], y[t:t + k])
                t += k
            outs.append(y.cpu().numpy())
            op.reset()
        op.close()
        ref = run_oracle_op(oracle_mod, kind, x.cpu().numpy(), kw.get("length", 1),
                            None if "taps" not in kw else np.asarray(kw["taps"], np.float32).astype(np.float64),
                            kw.get("alpha", 0.0))
        assert normwise(outs[0].astype(np.float64), ref) <= TOL
        if kind == abi.FILARK_TOP_FIR:
            assert np.array_equal(outs[0], outs[1])
        else:
            assert normwise(outs[1].astype(np.float64), outs[0].astype(np.float64)) <= 1e-6


def test_operator_argument_errors():
    import torch
    st, _ = abi.filark_top_create(abi.FILARK_TOP_FIR, 4, 513, np.ones(513), 0.0, 100, 0)
    assert st == abi.FILARK_EINVAL
    st, _ = abi.filark_top_create(abi.FILARK_TOP_EMA, 4, 1, None, 0.0, 100, 0)
    assert st == abi.FILARK_EINVAL
    st, h = abi.filark_top_create(abi.FILARK_TOP_MEAN, 4, 10, None, 0.0, 100, 0)
    assert st == abi.FILARK_OK
    x = torch.zeros((200, 4), device="cuda")
    assert abi.filark_top_push(h, x.data_ptr(), 4, 101, x.data_ptr(), 4, None) == abi.FILARK_EINVAL
    assert abi.filark_top_push(h, x.data_ptr(), 4, 50, x.data_ptr(), 4, None) == abi.FILARK_EINVAL  # overlap
    abi.filark_top_destroy(h)
