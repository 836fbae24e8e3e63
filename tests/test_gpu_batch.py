"""Parity of the batched chain (one persistent launch per push of many
independent streams) with the FP64 oracle, and with single-stream chains.

Every stream runs the small-workload chain (order-4 1-50 Hz bandpass at 1 kHz,
5-channel mean, STA/LTA 50/1000) on its own channel count and chunk lengths;
each stream's concatenated outputs must equal the oracle's for that stream's
whole record (max relative error 1e-5, as for the single-stream chain).
"""
import numpy as np
import pytest

from gpu_helpers import ALL_OUT, TOL, compare, run_oracle
from paper_2605_20132_gb300 import abi, synth

pytestmark = pytest.mark.gpu

K, NS_, NL = 5, 50, 1000


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def small_sos(ora):
    return ora.butter_bandpass(4, 1.0, 50.0, 1000.0)


def plan_pushes(rng, n_streams, n_pushes, max_chunk, zero_every=0):
    T = rng.integers(1, max_chunk + 1, (n_pushes, n_streams))
    if zero_every:
        T[::zero_every, ::2] = 0
    return T


def run_batch(batch, data, T):
    """Push data[i] ([N_i][C_i] float32) in the chunk lengths T[p][i]."""
    import torch
    n = len(data)
    xs = [torch.from_numpy(d).cuda() for d in data]
    outs = [{k: torch.full(d.shape, float("nan"), device="cuda") for k in ("ratio", "bp", "sp")} for d in data]
    pos = [0] * n
    for row in T:
        sl = []
        for i in range(n):
            sl.append(slice(pos[i], pos[i] + int(row[i])))
            pos[i] += int(row[i])
        batch.push([xs[i][sl[i]] if row[i] else None for i in range(n)],
                   ratios=[outs[i]["ratio"][sl[i]] for i in range(n)],
                   bandpasses=[outs[i]["bp"][sl[i]] for i in range(n)],
                   spatials=[outs[i]["sp"][sl[i]] for i in range(n)])
    batch.sync()
    return [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]


def make_streams(rng, Cs, T):
    tot = T.sum(axis=0)
    return [rng.standard_normal((int(tot[i]), C)).astype(np.float32) * 2.0 for i, C in enumerate(Cs)]


@pytest.fixture(scope="module")
def small_case(oracle_mod):
    rng = np.random.default_rng(70)
    Cs = [70, 130, 257, 33, 5, 64]
    T = plan_pushes(rng, len(Cs), 5, 3000, zero_every=2)
    data = make_streams(rng, Cs, T)
    sos = small_sos(oracle_mod)
    refs = [run_oracle(oracle_mod, d, sos, K=K, ns=NS_, nl=NL) for d in data]
    return Cs, T, data, sos, refs


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_oracle(small_case, cluster, graph):
    """Six streams (5 to 257 channels), five pushes of 1..3000 samples each
    (some streams skip a push), every launch geometry, with and without the
    captured graph."""
    from paper_2605_20132_gb300.chain import Batch
    Cs, T, data, sos, refs = small_case
    b = Batch(Cs, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    b.set_launch(cluster, 0, graph)
    info = b.info()
    assert info["cluster"] == cluster and info["use_graph"] == int(graph) and info["n_clusters"] > 0
    got = run_batch(b, data, T)
    b.close()
    for i in range(len(Cs)):
        errs = compare(got[i], refs[i])
        assert all(e <= TOL for e in errs.values()), (i, Cs[i], errs)


def test_batch_bitwise_equals_single_chains(small_case):
    """With 8 time ranges per cluster, and 8 blocks per CTA on both sides, a
    batched push does exactly the work of the single-stream pushes: the
    outputs agree bit for bit."""
    import torch
    from paper_2605_20132_gb300.chain import Batch, Chain
    Cs, T, data, sos, _ = small_case
    b = Batch(Cs, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    b.set_launch(8, 0, True)
    got = run_batch(b, data, T)
    b.close()
    for i, C in enumerate(Cs):
        ch = Chain(C, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
        ch.set_blocks_per_cta(8)   # the batch's CTAs cover 8 blocks each
        x = torch.from_numpy(data[i]).cuda()
        o = {k: torch.empty(data[i].shape, device="cuda") for k in ("ratio", "bp", "sp")}
        t = 0
        for row in T:
            n = int(row[i])
            ch.push(x[t:t + n], ratio=o["ratio"][t:t + n], bandpass=o["bp"][t:t + n], spatial=o["sp"][t:t + n])
            t += n
        ch.sync()
        ch.close()
        for k in o:
            assert np.array_equal(o[k].cpu().numpy(), got[i][k]), (i, k)


def test_batch_one_cluster_multi_unit_pushes(oracle_mod):
    """One persistent cluster runs every item of a push one after another, so
    a tile's later units finish before its neighbouring tile's first unit
    reads the halo columns' carried state: pushes of 2,500..3,000 samples
    (two units each) must still equal single-stream chains bit for bit, i.e.
    no unit may overwrite the per-channel state that the first units of the
    same launch read."""
    import torch
    from paper_2605_20132_gb300.chain import Batch, Chain
    rng = np.random.default_rng(71)
    Cs = [300, 130]
    T = rng.integers(2500, 3001, (3, len(Cs)))
    data = [synth.small_stream(C, int(T[:, i].sum()), seed=72 + i) for i, C in enumerate(Cs)]
    sos = small_sos(oracle_mod)
    b = Batch(Cs, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    b.set_launch(8, 1, True)
    got = run_batch(b, data, T)
    b.close()
    for i, C in enumerate(Cs):
        ch = Chain(C, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
        ch.set_blocks_per_cta(8)
        x = torch.from_numpy(data[i]).cuda()
        o = {k: torch.empty(data[i].shape, device="cuda") for k in ("ratio", "bp", "sp")}
        t = 0
        for row in T:
            n = int(row[i])
            ch.push(x[t:t + n], ratio=o["ratio"][t:t + n], bandpass=o["bp"][t:t + n], spatial=o["sp"][t:t + n])
            t += n
        ch.sync()
        ch.close()
        for k in o:
            assert np.array_equal(o[k].cpu().numpy(), got[i][k]), (i, k)


def _single_chain_outputs(C, sos, data_i, T_i, blocks):
    import torch
    from paper_2605_20132_gb300.chain import Chain
    ch = Chain(C, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    ch.set_blocks_per_cta(blocks)
    x = torch.from_numpy(data_i).cuda()
    o = {k: torch.empty(data_i.shape, device="cuda") for k in ("ratio", "bp", "sp")}
    t = 0
    for n in T_i:
        n = int(n)
        ch.push(x[t:t + n], ratio=o["ratio"][t:t + n], bandpass=o["bp"][t:t + n], spatial=o["sp"][t:t + n])
        t += n
    ch.sync()
    ch.close()
    return {k: v.cpu().numpy() for k, v in o.items()}


@pytest.mark.parametrize("blocks", [8, 4])
def test_batch_short_pushes_share_clusters(oracle_mod, blocks):
    """Pushes of at most 1,024 samples need fewer time ranges than a cluster
    of 8 CTAs has, so the batched kernel runs 2, 4 or 8 channel tiles of a
    stream in one cluster (ragged tile groups at the array end included).
    With 8 or 4 blocks per CTA on both sides, every stream equals its
    single-stream chain bit for bit; one stream is also held against the
    oracle."""
    from paper_2605_20132_gb300.chain import Batch
    rng = np.random.default_rng(74)
    Cs = [1000, 450, 57, 391]
    # 1..40 samples: one time range; 300: 2 (8 blocks) or 3 (4 blocks); 1024: 4 or 8
    T = np.array([[37, 300, 1024, 129], [1024, 7, 300, 640], [300, 640, 40, 1024], [129, 1024, 700, 1]])
    data = [synth.small_stream(C, int(T[:, i].sum()), seed=75 + i) * np.float32(1.5) for i, C in enumerate(Cs)]
    sos = small_sos(oracle_mod)
    b = Batch(Cs, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    b.set_launch(8, 0, True)
    b.set_blocks_per_cta(blocks)
    assert b.info()["blocks_per_cta"] == blocks
    got = run_batch(b, data, T)
    b.close()
    for i, C in enumerate(Cs):
        ref = _single_chain_outputs(C, sos, data[i], T[:, i], blocks)
        for k in ref:
            assert np.array_equal(ref[k], got[i][k]), (blocks, i, k)
    o = run_oracle(oracle_mod, data[2], sos, K=K, ns=NS_, nl=NL)
    errs = compare(got[2], o)
    assert all(e <= TOL for e in errs.values()), errs


def test_batch_dense_carry_short_pushes():
    """The dense carry (poles next to z = 1) in the batched kernel with tile
    groups: bitwise equal to single-stream chains; it keeps 8 blocks per
    CTA."""
    from paper_2605_20132_gb300.chain import Batch
    st, sos = abi.filark_butter_bandpass_sos(8, 0.01, 1.0, 1500.0)
    assert st == abi.FILARK_OK
    Cs = [300, 61]
    T = np.array([[200, 900], [1024, 33], [500, 1024]])
    data = [synth.small_stream(C, int(T[:, i].sum()), seed=80 + i) for i, C in enumerate(Cs)]
    b = Batch(Cs, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    st, h = abi.filark_batch_stream(b._h, 0)
    st, inf = abi.filark_chain_get_info(h)
    assert inf.precision == abi.FILARK_PREC_DENSE64
    assert abi.filark_batch_set_blocks_per_cta(b._h, 4) == abi.FILARK_ENOSYS
    b.set_launch(8, 0, True)
    got = run_batch(b, data, T)
    b.close()
    for i, C in enumerate(Cs):
        ref = _single_chain_outputs(C, sos, data[i], T[:, i], 8)
        for k in ref:
            assert np.array_equal(ref[k], got[i][k]), (i, k)


def test_batch_tune_then_stream(small_case):
    """The tuner times every geometry, keeps the fastest, and leaves every
    stream reset: streaming afterwards starts from a zero state."""
    import torch
    from paper_2605_20132_gb300.chain import Batch
    Cs, T, data, sos, refs = small_case
    b = Batch(Cs, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    scratch = [torch.zeros((1500, C), device="cuda") for C in Cs]
    info = b.tune(scratch, ratios=[torch.empty_like(s) for s in scratch], timed_pushes=2)
    tuned = info["tuned"]
    assert {t["cluster"] for t in tuned} == {1, 2, 4, 8}
    assert {t["blocks_per_cta"] for t in tuned} == {4, 8}
    best = min(tuned, key=lambda t: t["ms"])
    assert info["cluster"] == best["cluster"] and info["n_clusters"] == best["n_clusters"]
    assert info["blocks_per_cta"] == best["blocks_per_cta"]
    got = run_batch(b, data, T)
    b.close()
    for i in range(len(Cs)):
        errs = compare(got[i], refs[i])
        assert all(e <= TOL for e in errs.values()), (i, errs)


def test_batch_reset_and_stream_handles(small_case):
    """reset_state zeroes every stream; a stream's chain handle reports its
    own sample count."""
    from paper_2605_20132_gb300.chain import Batch
    Cs, T, data, sos, refs = small_case
    b = Batch(Cs, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    run_batch(b, data, T[:2])
    b.reset()
    got = run_batch(b, data, T)
    for i in range(len(Cs)):
        st, h = abi.filark_batch_stream(b._h, i)
        assert st == abi.FILARK_OK
        st, inf = abi.filark_chain_get_info(h)
        assert st == abi.FILARK_OK and inf.samples == int(T[:, i].sum())
        errs = compare(got[i], refs[i])
        assert all(e <= TOL for e in errs.values()), (i, errs)
    b.close()


def test_batch_rejects_bad_descriptor(small_case):
    import torch
    from paper_2605_20132_gb300.chain import Batch
    Cs, _, _, sos, _ = small_case
    b = Batch(Cs, sos, 1000.0, K, NS_, NL, outputs=ALL_OUT, max_chunk=3000)
    xs = [torch.zeros((10, C), device="cuda") for C in Cs]
    d = b._fill(xs)
    d[2].ld_in = Cs[2] - 1
    st = abi.filark_batch_push(b._h, d, None)
    assert st == abi.FILARK_EINVAL and "stream 2" in abi.filark_last_error_string()
    d = b._fill(xs)
    d[1].n_samples = 3001
    assert abi.filark_batch_push(b._h, d, None) == abi.FILARK_EINVAL
    assert abi.filark_batch_set_launch(b._h, 3, 0, 1) == abi.FILARK_EINVAL
    assert abi.filark_batch_set_blocks_per_cta(b._h, 3) == abi.FILARK_EINVAL
    assert abi.filark_batch_set_blocks_per_cta(b._h, 9) == abi.FILARK_EINVAL
    b.close()


def test_batch_workload_sampled(oracle_mod):
    """The batching workload: 32 streams of 500..10,000 channels, chunk
    lengths 200..3,000 drawn per stream and push (two pushes, so the second
    runs on carried state), small-workload data per stream.  Parity on
    channel slices at both ends and the middle of every stream."""
    import torch
    from paper_2605_20132_gb300.chain import Batch
    cfg = synth.BATCH
    specs = synth.batch_streams(cfg["seed"], cfg["n_streams"], cfg["channels"], cfg["chunk"])
    Cs = [s["n_channels"] for s in specs]
    T = synth.batch_chunk_lengths(cfg["seed"], cfg["n_streams"], 2, cfg["chunk"])
    sos = oracle_mod.butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    data = [synth.batch_stream_data(s, int(T[:, i].sum())) for i, s in enumerate(specs)]
    b = Batch(Cs, sos, cfg["fs"], cfg["spatial_width"], cfg["sta"], cfg["lta"], outputs=ALL_OUT,
              max_chunk=cfg["chunk"][1])
    got = run_batch(b, data, T)
    b.close()
    h = (cfg["spatial_width"] - 1) // 2
    worst = {}
    for i, C in enumerate(Cs):
        for lo, hi in [(0, 16), (C // 2 - 8, C // 2 + 8), (C - 16, C)]:
            a, z = max(0, lo - h), min(C, hi + h)
            ref = run_oracle(oracle_mod, np.ascontiguousarray(data[i][:, a:z]), sos, K=cfg["spatial_width"],
                             ns=cfg["sta"], nl=cfg["lta"])
            sel = slice(lo - a, hi - a)
            errs = compare({k: v[:, lo:hi] for k, v in got[i].items()}, {k: r[:, sel] for k, r in ref.items()})
            for k, v in errs.items():
                worst[k] = max(worst.get(k, 0.0), v)
    print("batch workload sampled errors:", worst)
    assert all(e <= TOL for e in worst.values()), worst
