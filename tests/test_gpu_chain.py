"""Parity of the CUDA chain (through the C-ABI) with the FP64 oracle.

Every test feeds both sides the same seeded float32 input and compares the
bandpass output, the spatial mean and the STA/LTA ratio.  Tolerance: 1e-5 max
relative error (normwise per channel; the ratio relative to max(|R|, 1)).
"""
import numpy as np
import pytest

from gpu_helpers import ALL_OUT, TOL, compare, normwise, run_gpu, run_oracle
from paper_2605_20132_gb300 import abi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def small_sos(oracle_mod):
    return oracle_mod.butter_bandpass(4, 1.0, 50.0, 1000.0)


def test_small_workload_parity(oracle_mod):
    """64 ch x 10,000 samples, order-4 1-50 Hz bandpass, 5-channel mean,
    STA/LTA 50/1000, ten pushes of 1,000 samples."""
    cfg = synth.SMALL
    x = synth.small_stream()
    sos = small_sos(oracle_mod)
    chunks = [1000] * 10
    got = run_gpu(x, chunks, sos, K=5, ns=50, nl=1000)
    ref = run_oracle(oracle_mod, x, sos, K=5, ns=50, nl=1000)
    errs = compare(got, ref)
    print("small workload errors:", errs)
    assert all(e <= TOL for e in errs.values()), errs
    assert cfg["chunk"] == 1000


@pytest.mark.parametrize("chunks", [
    [1, 7, 31, 32, 33, 255, 256, 257, 1000, 2047, 2048, 2049, 1],
    [49, 50, 51, 999, 1000, 1001, 5, 2000, 3000, 0, 2018],
    [3000] * 3,
])
def test_chunking_is_invisible(oracle_mod, chunks):
    """Any sequence of push lengths (ragged blocks, launch splits, windows
    straddling pushes) gives the oracle's whole-record output."""
    N = sum(chunks)
    x = synth.small_stream(40, N, seed=3)
    sos = small_sos(oracle_mod)
    got = run_gpu(x, chunks, sos, K=5, ns=50, nl=1000, max_chunk=max(chunks))
    ref = run_oracle(oracle_mod, x, sos, K=5, ns=50, nl=1000)
    errs = compare(got, ref)
    assert all(e <= TOL for e in errs.values()), errs


@pytest.mark.parametrize("C,K", [(1, 1), (3, 3), (57, 5), (56, 9), (131, 9), (200, 17), (97, 33), (64, 1)])
def test_channel_tiles_and_halo(oracle_mod, C, K):
    """Channel counts that leave ragged tiles, every halo width up to the
    maximum, and arrays narrower than one tile."""
    x = synth.small_stream(C, 3000, seed=C + K)
    sos = small_sos(oracle_mod)
    chunks = [1000, 1500, 500]
    got = run_gpu(x, chunks, sos, K=K, ns=20, nl=300)
    ref = run_oracle(oracle_mod, x, sos, K=K, ns=20, nl=300)
    errs = compare(got, ref)
    assert all(e <= TOL for e in errs.values()), (C, K, errs)


@pytest.mark.parametrize("ld_in,ld_out", [(70, 70), (67, 61), (64, 65)])
def test_strided_and_unaligned_buffers(oracle_mod, ld_in, ld_out):
    """Row strides larger than C, including strides that rule out vector
    access (the scalar paths)."""
    C = 60
    x = synth.small_stream(C, 2500, seed=11)
    sos = small_sos(oracle_mod)
    got = run_gpu(x, [700, 1800], sos, K=5, ns=10, nl=200, ld_in=ld_in, ld_out=ld_out)
    ref = run_oracle(oracle_mod, x, sos, K=5, ns=10, nl=200)
    errs = compare(got, ref)
    assert all(e <= TOL for e in errs.values()), errs


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5, 8])
def test_section_counts(oracle_mod, S):
    """Every kernel slot count (padded sections), Butterworth designs of
    several orders."""
    sos = oracle_mod.butter_bandpass(S, 2.0, 120.0, 1000.0)
    x = synth.small_stream(30, 4000, seed=S)
    got = run_gpu(x, [1234, 2766], sos, K=3, ns=25, nl=400)
    ref = run_oracle(oracle_mod, x, sos, K=3, ns=25, nl=400)
    errs = compare(got, ref)
    assert all(e <= TOL for e in errs.values()), (S, errs)


def test_general_sos_real_poles_and_a0(oracle_mod):
    """User SOS that are not Butterworth: real pole pairs, first-order
    sections (a2 = b2 = 0), and a0 != 1."""
    sos = np.array([
        [0.5, 0.2, 0.1, 2.0, -1.0, 0.2],       # real poles 0.25 +- 0.166 after a0 scaling
        [1.0, -0.3, 0.0, 1.0, -0.9, 0.0],      # first order: poles 0.9, 0
        [0.3, 0.0, -0.3, 1.0, -1.6, 0.8],      # complex pair
    ])
    x = synth.small_stream(20, 3000, seed=5)
    got = run_gpu(x, [1500, 1500], sos, K=3, ns=30, nl=500)
    ref = run_oracle(oracle_mod, x, sos, K=3, ns=30, nl=500)
    errs = compare(got, ref)
    assert all(e <= TOL for e in errs.values()), errs


def test_stage_bypasses(oracle_mod):
    """No IIR (S = 0), no spatial stage (K = 1), no detector."""
    x = synth.small_stream(50, 2000, seed=2)
    for sos, K, ns, nl in [(None, 5, 10, 100), (small_sos(oracle_mod), 1, 10, 100), (small_sos(oracle_mod), 5, 0, 0)]:
        got = run_gpu(x, [999, 1001], sos, K=K, ns=ns, nl=nl)
        ref = run_oracle(oracle_mod, x, sos, K=K, ns=ns, nl=nl)
        errs = compare(got, ref)
        assert all(e <= TOL for e in errs.values()), (K, ns, errs)
        if sos is None:
            assert np.array_equal(got["bp"], x)


def test_zero_input_and_empty_push(oracle_mod):
    """All-zero input gives exact zeros (ratio 0: the long window holds only
    zeros); a 0-sample push changes nothing."""
    x = np.zeros((1500, 10), dtype=np.float32)
    got = run_gpu(x, [700, 0, 800], small_sos(oracle_mod), K=3, ns=5, nl=50)
    for k in ("bp", "sp", "ratio"):
        assert np.array_equal(got[k], np.zeros_like(got[k])), k


def test_step_off_gives_exact_zero_ratio(oracle_mod):
    """After a burst, once the long window holds only zero cf the ratio is
    exactly 0, as in the oracle (no running-sum residue)."""
    x = np.zeros((3000, 8), dtype=np.float32)
    x[100:400] = 1.3
    got = run_gpu(x, [1000, 1000, 1000], None, K=1, ns=10, nl=200)
    ref = run_oracle(oracle_mod, x, None, K=1, ns=10, nl=200)
    assert np.array_equal(got["ratio"][700:], ref["ratio"][700:])
    assert np.all(got["ratio"][700:] == 0)
    assert compare(got, ref)["ratio"] <= TOL


@pytest.mark.parametrize("nbc", [0, 1, 3, 4, 5, 6, 7, 8])
def test_blocks_per_cta_choices_match_oracle(oracle_mod, nbc):
    """Every blocks-per-CTA setting (0 = the default, 8) matches the oracle
    over launches of many lengths (ragged, one sample, 2048, split pushes) on
    several channel tiles, and repeats bit for bit."""
    from paper_2605_20132_gb300.chain import Chain
    x = synth.small_stream(300, 7000, seed=31)
    sos = small_sos(oracle_mod)
    chunks = [1500, 2048, 1, 700, 1751, 1000]
    ref = run_oracle(oracle_mod, x, sos, K=5, ns=50, nl=1000)
    outs = []
    for _ in range(2):
        ch = Chain(300, sos, 1000.0, 5, 50, 1000, outputs=ALL_OUT, max_chunk=2048)
        ch.set_blocks_per_cta(nbc)
        outs.append(run_gpu(x, chunks, sos, K=5, ns=50, nl=1000, chain=ch))
        ch.close()
    errs = compare(outs[0], ref)
    print(nbc, errs)
    assert all(e <= TOL for e in errs.values()), errs
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_blocks_per_cta_rejects_out_of_range(oracle_mod):
    from paper_2605_20132_gb300.chain import Chain
    ch = Chain(16, small_sos(oracle_mod), 1000.0, 3, 5, 50, outputs=ALL_OUT, max_chunk=100)
    for bad in (-1, 9):
        assert abi.filark_chain_set_blocks_per_cta(ch._h, bad) == abi.FILARK_EINVAL
    assert abi.filark_chain_set_blocks_per_cta(ch._h, 0) == abi.FILARK_OK
    ch.close()


def test_deterministic(oracle_mod):
    x = synth.small_stream(64, 4000, seed=4)
    a = run_gpu(x, [4000], small_sos(oracle_mod), K=5, ns=50, nl=1000)
    b = run_gpu(x, [4000], small_sos(oracle_mod), K=5, ns=50, nl=1000)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_reset_equals_fresh_chain(oracle_mod):
    x = synth.small_stream(32, 2000, seed=6)
    sos = small_sos(oracle_mod)
    fresh = run_gpu(x, [2000], sos, K=5, ns=20, nl=300)
    _, ch = run_gpu(x[:1200], [1200], sos, K=5, ns=20, nl=300, max_chunk=2000, return_chain=True)
    ch.reset()
    again = run_gpu(x, [2000], sos, K=5, ns=20, nl=300, chain=ch)
    ch.close()
    for k in fresh:
        assert np.array_equal(fresh[k], again[k]), k


def test_checkpoint_resume_is_bitwise(oracle_mod):
    """get_state after some pushes, set_state into a new chain, continue:
    bit-identical to the uninterrupted run; the exported IIR state is the
    canonical TDF-II state, equal to the oracle's."""
    x = synth.small_stream(48, 5000, seed=8)
    sos = small_sos(oracle_mod)
    whole = run_gpu(x, [1700, 1700, 1600], sos, K=5, ns=50, nl=1000, max_chunk=1700)
    first, ch = run_gpu(x[:1700], [1700], sos, K=5, ns=50, nl=1000, max_chunk=1700, return_chain=True)
    state = ch.get_state()
    ch.close()
    # the canonical IIR state vs the oracle's state after 1700 samples
    import struct
    C, S = 48, 4
    hdr = 4 + 4 + 4 * 6 + 8 + 8
    iir = np.frombuffer(state, dtype=np.float64, count=C * 2 * S, offset=hdr).reshape(C, 2 * S)
    o = oracle_mod.Chain(C, sos, 5, 50, 1000)
    o.push(x[:1700])
    z = o.iir_state()
    assert np.max(np.abs(iir - z)) <= TOL * np.max(np.abs(z))
    _, ch2 = run_gpu(x[:0], [0], sos, K=5, ns=50, nl=1000, max_chunk=1700, return_chain=True)
    ch2.set_state(state)
    rest = run_gpu(x[1700:], [1700, 1600], sos, K=5, ns=50, nl=1000, chain=ch2)
    ch2.close()
    for k in whole:
        assert np.array_equal(np.concatenate([first[k], rest[k]]), whole[k]), k
    del struct


def test_host_buffer_push_matches_device_push(oracle_mod):
    from paper_2605_20132_gb300.chain import Chain
    x = synth.small_stream(64, 3000, seed=9)
    sos = small_sos(oracle_mod)
    dev = run_gpu(x, [1000] * 3, sos, K=5, ns=50, nl=1000)
    ch = Chain(64, sos, 1000.0, 5, 50, 1000, outputs=ALL_OUT, max_chunk=1000)
    r = np.zeros((3000, 64), np.float32)
    bp = np.zeros((3000, 64), np.float32)
    sp = np.zeros((3000, 64), np.float32)
    for t in range(0, 3000, 1000):
        ch.push_host(x[t:t + 1000], ratio=r[t:t + 1000], bandpass=bp[t:t + 1000], spatial=sp[t:t + 1000])
    ch.close()
    assert np.array_equal(r, dev["ratio"]) and np.array_equal(bp, dev["bp"]) and np.array_equal(sp, dev["sp"])


@pytest.mark.parametrize("pinned", [True, False])
def test_pipelined_host_push_matches_device_push(oracle_mod, pinned):
    """Pipelined host pushes (three staging slots reused, chunks of mixed
    lengths, outputs at a wider row stride) give bitwise the outputs of device
    pushes, from page-locked and from pageable host memory."""
    import torch
    from paper_2605_20132_gb300.chain import Chain
    x = synth.small_stream(64, 7000, seed=19)
    sos = small_sos(oracle_mod)
    chunks = [1000, 1, 999, 700, 1000, 300, 1000, 1000, 1000]
    dev = run_gpu(x, chunks, sos, K=5, ns=50, nl=1000)
    ch = Chain(64, sos, 1000.0, 5, 50, 1000, outputs=ALL_OUT, max_chunk=1000)
    xt = torch.from_numpy(x)
    outs = [torch.full((7000, 70), float("nan")) for _ in range(3)]
    if pinned:
        xt = xt.pin_memory()
        outs = [o.pin_memory() for o in outs]
    xn = xt.numpy()
    r, bp, sp = (o.numpy() for o in outs)
    for rep in range(2):      # twice, with a reset in between: slots are reused across resets
        t = 0
        for k in chunks:
            ch.push_host_async(xn[t:t + k], ratio=r[t:t + k], bandpass=bp[t:t + k], spatial=sp[t:t + k])
            t += k
        ch.host_sync()
        assert np.array_equal(r[:, :64], dev["ratio"]) and np.array_equal(bp[:, :64], dev["bp"])
        assert np.array_equal(sp[:, :64], dev["sp"])
        assert np.isnan(r[:, 64:]).all()
        ch.reset()
        for o in (r, bp, sp):
            o[:, :64] = np.nan
    ch.close()


def test_abi_argument_errors(oracle_mod):
    import torch
    from paper_2605_20132_gb300.chain import Chain
    ch = Chain(16, small_sos(oracle_mod), 1000.0, 3, 5, 50, outputs=abi.FILARK_OUT_RATIO, max_chunk=100)
    x = torch.zeros((200, 16), device="cuda")
    r = torch.zeros((200, 16), device="cuda")
    h = ch._h
    # too long
    assert abi.filark_chain_push_chunk(h, x.data_ptr(), 16, 101, r.data_ptr(), None, None, 16, None) == abi.FILARK_EINVAL
    # output not enabled
    assert abi.filark_chain_push_chunk(h, x.data_ptr(), 16, 10, None, r.data_ptr(), None, 16, None) == abi.FILARK_EINVAL
    # aliasing input and output
    assert abi.filark_chain_push_chunk(h, x.data_ptr(), 16, 10, x.data_ptr(), None, None, 16, None) == abi.FILARK_EINVAL
    # short strides
    assert abi.filark_chain_push_chunk(h, x.data_ptr(), 15, 10, r.data_ptr(), None, None, 16, None) == abi.FILARK_EINVAL
    # NULL input with samples
    assert abi.filark_chain_push_chunk(h, None, 16, 10, r.data_ptr(), None, None, 16, None) == abi.FILARK_EINVAL
    # 0 samples: no-op
    assert abi.filark_chain_push_chunk(h, None, 16, 0, None, None, None, 16, None) == abi.FILARK_OK
    assert abi.filark_chain_sync_status(h, None) == abi.FILARK_OK
    info = ch.info()
    assert info["samples"] == 0 and info["n_slots"] == 4 and info["halo"] == 1
    ch.close()


# --------------------------------------------------------------------------
# Paper-scale stream: 6,000 ch x 90,000 samples at 1.5 kHz in 60 pushes of
# 1,500 (the benchmark's launch configuration), order-8 0.5-100 Hz bandpass,
# 9-channel mean, STA/LTA 150/3000.  The oracle recomputes sampled channel
# windows (with their 4-channel halos) over the whole record.
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def paper_scale():
    return synth.paper_scale_stream()


def test_paper_scale_parity_sampled(oracle_mod, paper_scale):
    import torch
    from paper_2605_20132_gb300.chain import Chain
    x = paper_scale
    N, C = x.shape
    cfg = synth.PAPER_SCALE
    sos = oracle_mod.butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    K, ns, nl, T = cfg["spatial_width"], cfg["sta"], cfg["lta"], cfg["chunk"]
    ch = Chain(C, sos, cfg["fs"], K, ns, nl, outputs=ALL_OUT, max_chunk=T)
    info = ch.info()
    assert info["precision"] == abi.FILARK_PREC_MODAL32
    xd = torch.from_numpy(x).cuda()
    outs = {k: torch.empty((N, C), device="cuda") for k in ("ratio", "bp", "sp")}
    for t in range(0, N, T):
        ch.push(xd[t:t + T], ratio=outs["ratio"][t:t + T], bandpass=outs["bp"][t:t + T],
                spatial=outs["sp"][t:t + T])
    ch.sync()
    ch.close()
    h = (K - 1) // 2
    worst = {}
    for lo, hi in [(0, 40), (2988, 3012), (5951, 6000)]:
        a, b = max(0, lo - h), min(C, hi + h)
        ref = run_oracle(oracle_mod, np.ascontiguousarray(x[:, a:b]), sos, K=K, ns=ns, nl=nl)
        sel = slice(lo - a, hi - a)
        got = {k: outs[k][:, lo:hi].cpu().numpy() for k in outs}
        errs = compare(got, {k: ref[k][:, sel] for k in ref})
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
    print("paper-scale sampled errors:", worst)
    assert all(e <= TOL for e in worst.values()), worst
    # properties over every channel: finite, ratio >= 0, zero during warm-up
    r = outs["ratio"]
    assert torch.isfinite(r).all() and (r >= 0).all()
    assert (r[: nl - 1] == 0).all()
    assert torch.isfinite(outs["bp"]).all() and torch.isfinite(outs["sp"]).all()
    # spatial mean of the GPU's own bandpass output, every channel, sampled rows
    rows = torch.arange(nl, N, 997, device="cuda")
    bp = outs["bp"][rows].double()
    cs = torch.nn.functional.pad(torch.cumsum(bp, 1), (1, 0))
    idx = torch.arange(C, device="cuda")
    lo_i, hi_i = (idx - h).clamp(min=0), (idx + h).clamp(max=C - 1)
    mean = (cs[:, hi_i + 1] - cs[:, lo_i]) / (hi_i - lo_i + 1).double()
    assert normwise(outs["sp"][rows].double().cpu().numpy(), mean.cpu().numpy()) <= TOL


def test_paper_scale_benchmark_configuration(oracle_mod, paper_scale):
    """The benchmark's own configuration: the paper-scale stream pushed as 60
    chunks of 1,500 samples in the benchmark's lanes and launch length (each
    push cut into launches of at most LAUNCH_SAMPLES samples) with the SOS
    from the library's Butterworth designer and the ratio as the only output,
    as the benchmark line times it.  Its ratio is compared with the FP64
    oracle on sampled channel windows: both array ends, the middle, and every
    boundary between two lanes' tile groups.  A second run with every output
    enabled gives the identical ratio and its bandpass and spatial outputs are
    compared there too."""
    import torch
    from bench import LANES, LAUNCH_SAMPLES
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass
    x = paper_scale
    N, C = x.shape
    cfg = synth.PAPER_SCALE
    sos = butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    K, ns, nl, T = cfg["spatial_width"], cfg["sta"], cfg["lta"], cfg["chunk"]
    xd = torch.from_numpy(x).cuda()

    def run(outputs):
        ch = Chain(C, sos, cfg["fs"], K, ns, nl, outputs=outputs, max_chunk=T)
        ch.set_lanes(LANES)
        ch.set_launch_samples(LAUNCH_SAMPLES)
        assert ch.info()["tile_channels"] == 56
        names = ["ratio"] + (["bp", "sp"] if outputs != abi.FILARK_OUT_RATIO else [])
        outs = {k: torch.full((N, C), float("nan"), device="cuda") for k in names}
        for t in range(0, N, T):
            ch.push(xd[t:t + T], ratio=outs["ratio"][t:t + T],
                    bandpass=outs["bp"][t:t + T] if "bp" in outs else None,
                    spatial=outs["sp"][t:t + T] if "sp" in outs else None)
        ch.join()
        ch.sync()
        ch.close()
        return outs

    bench = run(abi.FILARK_OUT_RATIO)
    full = run(ALL_OUT)
    assert torch.equal(bench["ratio"], full["ratio"])
    h = (K - 1) // 2
    worst = {}
    n_tiles = -(-C // 56)
    bounds = [(n_tiles * l // LANES) * 56 for l in range(1, LANES)]
    for lo, hi in [(0, 24), (2988, 3012), (5976, 6000)] + [(b - 16, b + 16) for b in bounds]:
        a, b = max(0, lo - h), min(C, hi + h)
        ref = run_oracle(oracle_mod, np.ascontiguousarray(x[:, a:b]), sos, K=K, ns=ns, nl=nl)
        sel = slice(lo - a, hi - a)
        got = {k: full[k][:, lo:hi].cpu().numpy() for k in full}
        errs = compare(got, {k: ref[k][:, sel] for k in ref})
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
    print("benchmark configuration, sampled errors:", worst)
    assert set(worst) == {"ratio", "bp", "sp"}
    assert all(e <= TOL for e in worst.values()), worst
    r = bench["ratio"]
    assert torch.isfinite(r).all() and (r >= 0).all() and (r[: nl - 1] == 0).all()


# --------------------------------------------------------------------------
# Dense double-float carry (canonical basis): forced on the small workload, chosen
# automatically for a defective cascade (repeated poles) and for the
# precision-stress bandpass 0.01-1 Hz at 1.5 kHz (poles 8e-6 from z = 1).
# --------------------------------------------------------------------------

def test_dense_mode_small_workload(oracle_mod):
    x = synth.small_stream(64, 4000, seed=12)
    sos = small_sos(oracle_mod)
    got = run_gpu(x, [1000, 1, 999, 2000], sos, K=5, ns=50, nl=1000, precision=abi.FILARK_PREC_DENSE64)
    ref = run_oracle(oracle_mod, x, sos, K=5, ns=50, nl=1000)
    errs = compare(got, ref)
    assert all(e <= TOL for e in errs.values()), errs


def test_repeated_poles_use_dense_carry(oracle_mod):
    from paper_2605_20132_gb300.chain import Chain
    sec = [0.2, 0.0, -0.2, 1.0, -1.6, 0.8]
    sos = np.array([sec, sec, sec])
    ch = Chain(8, sos, 1000.0, 1, 0, 0, outputs=abi.FILARK_OUT_BANDPASS, max_chunk=3000)
    assert ch.info()["precision"] == abi.FILARK_PREC_DENSE64
    ch.close()
    x = synth.small_stream(30, 3000, seed=13)
    got = run_gpu(x, [1700, 1300], sos, K=3, ns=0, nl=0)
    ref = run_oracle(oracle_mod, x, sos, K=3)
    errs = compare(got, ref)
    assert all(e <= TOL for e in errs.values()), errs


def test_precision_stress_sampled(oracle_mod):
    """Order-8 0.01-1 Hz bandpass at 1.5 kHz on 48 channels of the stress
    stream (noise + 0.05 Hz sine), 120 pushes of 1 s: the planner picks the
    dense double-float carry and stays within 1e-5 of the FP64 oracle; carrying in
    FP32 instead (the all-FP32 comparison mode) does not."""
    from paper_2605_20132_gb300.chain import Chain
    cfg = synth.PRECISION
    sos = oracle_mod.butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    chans = np.arange(0, 10_000, 10_000 // 48)[:48]
    n_push = 120
    x = np.concatenate([synth.precision_chunk(i, channels=chans) for i in range(n_push)])
    ch = Chain(len(chans), sos, cfg["fs"], 1, 0, 0, outputs=abi.FILARK_OUT_BANDPASS, max_chunk=cfg["chunk"])
    info = ch.info()
    ch.close()
    assert info["precision"] == abi.FILARK_PREC_DENSE64
    chunks = [cfg["chunk"]] * n_push
    got = run_gpu(x, chunks, sos, K=1)
    ref = run_oracle(oracle_mod, x, sos, K=1)
    err = normwise(got["bp"], ref["bp"])
    got32 = run_gpu(x, chunks, sos, K=1, precision=abi.FILARK_PREC_ALL32)
    err32 = normwise(got32["bp"], ref["bp"])
    # per-chunk report (max over channels) of both modes
    per_chunk = [normwise(got["bp"][i * 1500:(i + 1) * 1500], ref["bp"][i * 1500:(i + 1) * 1500]) for i in range(n_push)]
    print(f"precision stress: dense carry {err:.2e} (worst chunk {max(per_chunk):.2e}), all-FP32 {err32:.2e}")
    assert err <= TOL
    assert err32 > err
