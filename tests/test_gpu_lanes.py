"""Lanes: the chain's channel tiles pushed as independent groups on internal
streams (filark_chain_set_lanes / filark_chain_join).

Every tile carries its halo columns' IIR state itself in this mode, and the
arithmetic of a column does not depend on which tile computes it, so every
output and the checkpointed state must be bit-identical to one lane; one case
is also held against the FP64 oracle.
"""
import numpy as np
import pytest

from gpu_helpers import ALL_OUT, TOL, compare, run_gpu, run_oracle
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


def make_chain(C, sos, lanes, precision=0, max_chunk=3000, K=5, ns=50, nl=1000):
    from paper_2605_20132_gb300.chain import Chain
    ch = Chain(C, sos, 1000.0, K, ns, nl, outputs=ALL_OUT, precision=precision, max_chunk=max_chunk)
    ch.set_lanes(lanes)
    return ch


CHUNKS = [1500, 2048, 1, 700, 3000, 1751, 1000]   # 3000: two launches in one push


@pytest.mark.parametrize("precision", [abi.FILARK_PREC_AUTO, abi.FILARK_PREC_DENSE64, abi.FILARK_PREC_ALL32])
@pytest.mark.parametrize("lanes", [2, 3, 4])
def test_lanes_bit_identical_to_one_lane(oracle_mod, lanes, precision):
    """300 channels = 6 tiles of 56 outputs, pushes of mixed lengths (ragged,
    one sample, two launches in one push): every output of 2-4 lanes equals
    the single-lane output bit for bit, for the modal, dense and all-FP32
    carries."""
    x = synth.small_stream(300, sum(CHUNKS), seed=41)
    sos = small_sos(oracle_mod)
    one = run_gpu(x, CHUNKS, sos, K=5, ns=50, nl=1000, precision=precision, max_chunk=3000)
    ch = make_chain(300, sos, lanes, precision)
    got = run_gpu(x, CHUNKS, sos, K=5, ns=50, nl=1000, chain=ch)
    ch.close()
    for k in one:
        assert np.array_equal(got[k], one[k]), k


def test_lanes_match_oracle(oracle_mod):
    x = synth.small_stream(300, sum(CHUNKS), seed=42)
    sos = small_sos(oracle_mod)
    ch = make_chain(300, sos, 2)
    got = run_gpu(x, CHUNKS, sos, K=5, ns=50, nl=1000, chain=ch)
    ch.close()
    errs = compare(got, run_oracle(oracle_mod, x, sos, K=5, ns=50, nl=1000))
    assert all(e <= TOL for e in errs.values()), errs


def test_lane_count_changes_mid_stream(oracle_mod):
    """Switching 1 -> 2 -> 1 -> 3 -> 4 -> 2 lanes between pushes (tiles move
    between lanes, the per-tile state is rebuilt after single-lane pushes)
    keeps the stream bit-identical."""
    import torch
    x = synth.small_stream(300, 7000, seed=43)
    sos = small_sos(oracle_mod)
    chunks = [1000, 1200, 800, 1500, 1000, 1500]
    plan = [1, 2, 1, 3, 4, 2]
    one = run_gpu(x, chunks, sos, K=5, ns=50, nl=1000, max_chunk=3000)
    ch = make_chain(300, sos, 1)
    xd = torch.from_numpy(x).cuda()
    outs = {k: torch.full(xd.shape, float("nan"), device="cuda") for k in ("ratio", "bp", "sp")}
    t = 0
    for T, lanes in zip(chunks, plan):
        ch.set_lanes(lanes)
        sl = slice(t, t + T)
        ch.push(xd[sl], ratio=outs["ratio"][sl], bandpass=outs["bp"][sl], spatial=outs["sp"][sl])
        t += T
    ch.sync()
    ch.close()
    for k in one:
        assert np.array_equal(outs[k].cpu().numpy(), one[k]), k


def test_lanes_checkpoint_and_reset(oracle_mod):
    """get_state after lane pushes is byte-identical to the single-lane state;
    resuming it in a two-lane chain continues bit for bit; reset then a full
    run equals a fresh chain."""
    x = synth.small_stream(300, 5000, seed=44)
    sos = small_sos(oracle_mod)
    whole = run_gpu(x, [1700, 1700, 1600], sos, K=5, ns=50, nl=1000, max_chunk=3000)
    _, one = run_gpu(x[:1700], [1700], sos, K=5, ns=50, nl=1000, max_chunk=3000, return_chain=True)
    ref_state = one.get_state()
    one.close()
    ch = make_chain(300, sos, 2)
    first = run_gpu(x[:1700], [1700], sos, K=5, ns=50, nl=1000, chain=ch)
    state = ch.get_state()
    assert state == ref_state
    ch2 = make_chain(300, sos, 2)
    ch2.set_state(state)
    rest = run_gpu(x[1700:], [1700, 1600], sos, K=5, ns=50, nl=1000, chain=ch2)
    ch2.close()
    for k in whole:
        assert np.array_equal(np.concatenate([first[k], rest[k]]), whole[k]), k
    ch.reset()
    again = run_gpu(x, [1700, 1700, 1600], sos, K=5, ns=50, nl=1000, chain=ch)
    ch.close()
    for k in whole:
        assert np.array_equal(again[k], whole[k]), k


def test_lanes_with_host_buffer_pushes(oracle_mod):
    """Synchronous and pipelined host-buffer pushes join the lanes after each
    push: their outputs equal the single-lane device pushes."""
    x = synth.small_stream(300, 4000, seed=45)
    sos = small_sos(oracle_mod)
    chunks = [1000, 1000, 500, 1500]
    one = run_gpu(x, chunks, sos, K=5, ns=50, nl=1000, max_chunk=3000)
    for mode in ("sync", "async"):
        ch = make_chain(300, sos, 2)
        r, bp, sp = (np.full((4000, 300), np.nan, np.float32) for _ in range(3))
        t = 0
        for T in chunks:
            sl = slice(t, t + T)
            if mode == "sync":
                ch.push_host(x[sl], ratio=r[sl], bandpass=bp[sl], spatial=sp[sl])
            else:
                ch.push_host_async(x[sl], ratio=r[sl], bandpass=bp[sl], spatial=sp[sl])
            t += T
        if mode == "async":
            ch.host_sync()
        ch.close()
        assert np.array_equal(r, one["ratio"]) and np.array_equal(bp, one["bp"]) and np.array_equal(sp, one["sp"])


def test_join_orders_outputs_on_the_callers_stream(oracle_mod):
    """Pushes enqueued on a side stream with lanes, then join(stream): work
    enqueued on that stream afterwards (a copy of the outputs) sees the
    complete outputs."""
    import torch
    x = synth.small_stream(300, 6000, seed=46)
    sos = small_sos(oracle_mod)
    one = run_gpu(x, [1500] * 4, sos, K=5, ns=50, nl=1000, max_chunk=3000)
    ch = make_chain(300, sos, 2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xd = torch.from_numpy(x).cuda()
        r = torch.full(xd.shape, float("nan"), device="cuda")
        for t in range(0, 6000, 1500):
            ch.push(xd[t:t + 1500], ratio=r[t:t + 1500], stream=s)
        ch.join(s)
        copy = r.clone()
    s.synchronize()
    ch.sync(s)
    ch.close()
    assert np.array_equal(copy.cpu().numpy(), one["ratio"])


def test_lanes_without_iir_and_with_one_tile(oracle_mod):
    """No bandpass (detector on the raw input) and a single-tile chain (the
    lanes collapse to one): equal to one lane."""
    x = synth.small_stream(300, 3000, seed=47)
    one = run_gpu(x, [1000, 2000], None, K=5, ns=50, nl=1000, max_chunk=3000)
    ch = make_chain(300, None, 2)
    got = run_gpu(x, [1000, 2000], None, K=5, ns=50, nl=1000, chain=ch)
    ch.close()
    for k in one:
        assert np.array_equal(got[k], one[k]), k
    xs = x[:, :40].copy()
    sos = small_sos(oracle_mod)
    one = run_gpu(xs, [1000, 2000], sos, K=5, ns=50, nl=1000, max_chunk=3000)
    ch = make_chain(40, sos, 3)
    got = run_gpu(xs, [1000, 2000], sos, K=5, ns=50, nl=1000, chain=ch)
    ch.close()
    for k in one:
        assert np.array_equal(got[k], one[k]), k


def test_set_lanes_rejects_out_of_range(oracle_mod):
    ch = make_chain(16, small_sos(oracle_mod), 1, max_chunk=100)
    for bad in (0, -1, abi.FILARK_MAX_LANES + 1):
        assert abi.filark_chain_set_lanes(ch._h, bad) == abi.FILARK_EINVAL
    assert abi.filark_chain_set_lanes(ch._h, abi.FILARK_MAX_LANES) == abi.FILARK_OK
    assert abi.filark_chain_join(ch._h, None) == abi.FILARK_OK
    ch.close()


def test_lanes_paper_scale_first_pushes_bitwise(oracle_mod):
    """The paper-scale chain (6,000 channels = 108 tiles, two lanes of 54
    tiles; order-8 0.5-100 Hz bandpass from the library's designer, K = 9,
    STA/LTA 150/3000) with pushes longer than one launch right after create
    and right after a reset, where the per-tile state does not exist yet:
    every output equals one lane bit for bit, in both runs."""
    import torch
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass
    cfg = synth.PAPER_SCALE
    C, fs = cfg["n_channels"], cfg["fs"]
    chunks = [3000, 1500, 2500, 1500, 3500]
    N = sum(chunks)
    x = synth.paper_scale_stream(C, N, seed=48)
    sos = butter_bandpass(cfg["order"], *cfg["band"], fs)
    K, ns, nl = cfg["spatial_width"], cfg["sta"], cfg["lta"]
    one = run_gpu(x, chunks, sos, fs=fs, K=K, ns=ns, nl=nl, max_chunk=max(chunks))
    ch = Chain(C, sos, fs, K, ns, nl, outputs=ALL_OUT, max_chunk=max(chunks))
    ch.set_lanes(2)
    xd = torch.from_numpy(x).cuda()
    for rep in range(2):
        outs = {k: torch.full(xd.shape, float("nan"), device="cuda") for k in ("ratio", "bp", "sp")}
        t = 0
        for T in chunks:
            sl = slice(t, t + T)
            ch.push(xd[sl], ratio=outs["ratio"][sl], bandpass=outs["bp"][sl], spatial=outs["sp"][sl])
            t += T
        ch.join()
        ch.sync()
        for k in one:
            assert np.array_equal(outs[k].cpu().numpy(), one[k]), (rep, k)
        ch.reset()
    ch.close()


def test_launch_samples_lanes_bitwise():
    """Pushes cut into launches of at most 1,024 (and 512) samples: three
    lanes equal one lane bit for bit for the same launch length, on the
    paper-scale chain with pushes of 3,000 / 1,500 / 2,500 / 1,024 / 1,500
    samples (ragged last launches); the length must be a multiple of 256 in
    256..2048 (0 restores 2048)."""
    import torch
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass
    cfg = synth.PAPER_SCALE
    C, fs = cfg["n_channels"], cfg["fs"]
    chunks = [3000, 1500, 2500, 1024, 1500]
    N = sum(chunks)
    x = torch.from_numpy(synth.paper_scale_stream(C, N, seed=49)).cuda()
    sos = butter_bandpass(cfg["order"], *cfg["band"], fs)
    K, ns, nl = cfg["spatial_width"], cfg["sta"], cfg["lta"]

    def run(lanes, launch):
        ch = Chain(C, sos, fs, K, ns, nl, outputs=ALL_OUT, max_chunk=max(chunks))
        ch.set_lanes(lanes)
        ch.set_launch_samples(launch)
        outs = {k: torch.full(x.shape, float("nan"), device="cuda") for k in ("ratio", "bp", "sp")}
        t = 0
        for T in chunks:
            sl = slice(t, t + T)
            ch.push(x[sl], ratio=outs["ratio"][sl], bandpass=outs["bp"][sl], spatial=outs["sp"][sl])
            t += T
        ch.join()
        ch.sync()
        ch.close()
        return outs

    for launch in (1024, 512):
        one, three = run(1, launch), run(3, launch)
        for k in one:
            assert torch.equal(one[k], three[k]), (launch, k)
            assert torch.isfinite(one[k]).all(), (launch, k)
    ch = Chain(16, sos, fs, K, ns, nl, outputs=ALL_OUT, max_chunk=100)
    for bad in (-256, 100, 300, 2304):
        assert abi.filark_chain_set_launch_samples(ch._h, bad) == abi.FILARK_EINVAL
    for good in (0, 256, 2048):
        assert abi.filark_chain_set_launch_samples(ch._h, good) == abi.FILARK_OK
    ch.close()


def test_chain_tune_picks_a_candidate_and_resets():
    """The chain's autotuner times lanes x samples per launch x blocks per
    CTA on a push, keeps the fastest and resets the state: a run after tuning
    equals a fresh chain with the chosen settings bit for bit, and within
    rounding (the oracle's bar) the default chain."""
    import torch
    from paper_2605_20132_gb300.chain import Chain, butter_bandpass
    C, fs = 700, 1000.0
    sos = butter_bandpass(4, 1.0, 50.0, fs)
    chunks = [1500, 1500, 700]
    x = torch.from_numpy(synth.small_stream(C, sum(chunks), seed=51)).cuda()

    def run(ch):
        outs = {k: torch.full(x.shape, float("nan"), device="cuda") for k in ("ratio", "bp", "sp")}
        t = 0
        for T in chunks:
            sl = slice(t, t + T)
            ch.push(x[sl], ratio=outs["ratio"][sl], bandpass=outs["bp"][sl], spatial=outs["sp"][sl])
            t += T
        ch.join()
        ch.sync()
        return outs

    tuned = Chain(C, sos, fs, 5, 50, 1000, outputs=ALL_OUT, max_chunk=1500)
    scratch = {k: torch.empty((1500, C), device="cuda") for k in ("ratio", "bp", "sp")}
    res = tuned.tune(x[:1500], ratio=scratch["ratio"], bandpass=scratch["bp"], spatial=scratch["sp"],
                     timed_pushes=2)
    cands, best = res["candidates"], res["chosen"]
    n_tiles = -(-C // tuned.info()["tile_channels"])
    assert len(cands) == min(16, 2 * 2 * min(abi.FILARK_MAX_LANES, n_tiles))
    assert best == min(cands, key=lambda c: c["ms_per_push"])
    got = run(tuned)
    tuned.close()
    ref = Chain(C, sos, fs, 5, 50, 1000, outputs=ALL_OUT, max_chunk=1500)
    ref.set_lanes(best["lanes"])
    ref.set_launch_samples(best["launch_samples"])
    ref.set_blocks_per_cta(best["blocks_per_cta"])
    want = run(ref)
    ref.close()
    for k in want:
        assert torch.equal(got[k], want[k]), k
    plain = Chain(C, sos, fs, 5, 50, 1000, outputs=ALL_OUT, max_chunk=1500)
    base = run(plain)
    plain.close()
    for k in base:
        d = (got[k] - base[k]).abs().max().item()
        assert d <= TOL * base[k].abs().max().item(), (k, d)

