"""Triggers and events on the GPU against the oracle: integer work, so the
trigger lists and the event lists must be identical (after sorting, since the
device appends in no fixed order)."""
import numpy as np
import pytest

from gpu_helpers import ALL_OUT
from paper_2605_20132_gb300 import abi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def sort_records(r):
    r = np.asarray(r, dtype=np.int64)
    return r[np.lexsort(tuple(r[:, k] for k in reversed(range(r.shape[1]))))] if r.size else r


def sort_events(e):
    e = np.asarray(e, dtype=np.int64)
    if e.ndim == 1:
        e = e.reshape(-1, 5)
    return e[np.lexsort((e[:, 3], e[:, 1], e[:, 2], e[:, 0]))] if e.size else e


def blob_ratio(rng, N, C, n_blobs=30, level=5.0):
    R = (rng.random((N, C)) * 2.0).astype(np.float32)
    for _ in range(n_blobs):
        c0, n0 = rng.integers(0, C), rng.integers(0, N)
        w, h, slope = rng.integers(1, 12), rng.integers(3, 120), rng.integers(-3, 4)
        for c in range(max(0, c0 - w), min(C, c0 + w + 1)):
            a = n0 + slope * (c - c0)
            R[max(0, a):max(0, min(N, a + h)), c] = level + rng.random()
    return R


def run_gpu_trigger(R, chunks, on, off, capacity=1 << 18, flush=True, overlap=False):
    import torch
    from paper_2605_20132_gb300.chain import Trigger
    N, C = R.shape
    tr = Trigger(C, on, off, max_chunk=max(chunks), capacity=capacity)
    if overlap:
        tr.set_overlap(True)
    Rd = torch.from_numpy(R).cuda()
    t = 0
    for k in chunks:
        tr.push(Rd[t:t + k])
        t += k
    assert t == N
    if flush:
        tr.flush()
    tr.join()
    torch.cuda.synchronize()
    n = int(tr.count.item())
    recs = tr.triggers() if n <= capacity else None
    return tr, recs, n


def run_oracle_trigger(ora, R, chunks, on, off, flush=True):
    t = ora.Trigger(R.shape[1], on, off)
    parts, pos = [], 0
    for k in chunks:
        parts.append(t.push(R[pos:pos + k]))
        pos += k
    closed = np.concatenate(parts) if parts else np.zeros((0, 3), np.int64)
    opened = t.flush() if flush else np.zeros((0, 3), np.int64)
    return closed, opened


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("C", [300, 301])
def test_triggers_match_oracle_random_chunks(oracle_mod, C, overlap):
    """Blob-shaped ratio images on 300 and 301 channels, pushed in 1..700-sample
    chunks (segments of every phase, pushes shorter than a segment);
    thresholds that are not floats (exact comparison by rounding up); with
    and without the overlap mode (summaries of one push beside the scan and
    emission of the previous one, on the trigger's own streams)."""
    rng = np.random.default_rng(80)
    N = 5000
    R = blob_ratio(rng, N, C)
    on, off = 4.0000001, 1.0000001
    R[10, :5] = np.float32(on)      # equal to neither threshold as a float
    chunks = []
    while sum(chunks) < N:
        chunks.append(int(min(rng.integers(1, 701), N - sum(chunks))))
    tr, got, n = run_gpu_trigger(R, chunks, on, off, overlap=overlap)
    closed, opened = run_oracle_trigger(oracle_mod, R, chunks, on, off)
    want = np.concatenate([np.c_[closed, np.zeros(len(closed), np.int64)],
                           np.c_[opened, np.ones(len(opened), np.int64)]])
    assert n == len(want)
    assert np.array_equal(sort_records(got), sort_records(want))
    tr.close()


def test_trigger_overlap_mode_switches_and_reset(oracle_mod):
    """Pushes in overlap mode, a switch back to stream order in the middle of
    the record and a reset with overlapped pushes pending give the oracle's
    triggers; set_overlap rejects anything but 0 and 1."""
    import torch
    from paper_2605_20132_gb300.chain import Trigger
    rng = np.random.default_rng(81)
    N, C = 4000, 257
    R = blob_ratio(rng, N, C)
    on, off = 4.0, 1.0
    chunks = [500] * 8
    tr = Trigger(C, on, off, max_chunk=500)
    Rd = torch.from_numpy(R).cuda()
    for rep in range(2):
        tr.set_overlap(True)
        for i, k in enumerate(chunks):
            if i == 4:
                tr.set_overlap(False)
            tr.push(Rd[500 * i:500 * i + k])
        tr.flush()
        got = tr.triggers()
        closed, opened = run_oracle_trigger(oracle_mod, R, chunks, on, off)
        want = np.concatenate([np.c_[closed, np.zeros(len(closed), np.int64)],
                               np.c_[opened, np.ones(len(opened), np.int64)]])
        assert np.array_equal(sort_records(got), sort_records(want)), rep
        tr.set_overlap(True)
        tr.push(Rd[:500])                 # pending when reset joins
        tr.reset()
    assert abi.filark_trigger_set_overlap(tr._h, 2) == abi.FILARK_EINVAL
    tr.close()


def test_dense_triggers_match_oracle(oracle_mod):
    """Runs ending in almost every 32-sample segment of every channel (uniform
    ratio around thresholds 1.0 / 0.9): nearly every (channel, segment) pair
    is on the emit list; pushes of mixed lengths."""
    rng = np.random.default_rng(81)
    N, C = 3000, 97
    R = (rng.random((N, C)) * 2.0).astype(np.float32)
    on, off = 1.0, 0.9
    chunks = [1500, 1, 700, 799]
    tr, got, n = run_gpu_trigger(R, chunks, on, off, capacity=1 << 20)
    closed, opened = run_oracle_trigger(oracle_mod, R, chunks, on, off)
    want = np.concatenate([np.c_[closed, np.zeros(len(closed), np.int64)],
                           np.c_[opened, np.ones(len(opened), np.int64)]])
    assert n == len(want) > 50 * C
    assert np.array_equal(sort_records(got), sort_records(want))
    tr.close()


def test_trigger_threshold_edges(oracle_mod):
    """R equal to the on threshold sets, equal to off keeps, the float just
    below off resets; hysteresis across a push boundary of one sample."""
    on, off = 2.5, 0.75
    below = float(np.nextafter(np.float32(off), np.float32(0)))
    R = np.zeros((8, 3), dtype=np.float32)
    R[:, 0] = [0, 2.5, 0.75, 0.75, below, 3, 1, 0]
    R[:, 1] = [2.4999998, 2.5, 2.5, 0, 0, 0, 0, 0]
    R[:, 2] = [3, 0, 3, 0, 3, 0, 3, 0]
    chunks = [1, 1, 3, 1, 2]
    _, got, _ = run_gpu_trigger(R, chunks, on, off)
    closed, opened = run_oracle_trigger(oracle_mod, R, chunks, on, off)
    want = np.concatenate([np.c_[closed, np.zeros(len(closed), np.int64)],
                           np.c_[opened, np.ones(len(opened), np.int64)]])
    assert np.array_equal(sort_records(got), sort_records(want))
    assert sort_records(want)[:3, :3].tolist() == [[0, 1, 4], [0, 5, 7], [1, 1, 3]]


def test_events_match_oracle(oracle_mod):
    """Events merged on the device equal the oracle's for the same triggers
    (closed and open), including the open flag."""
    from paper_2605_20132_gb300.chain import merge_events
    rng = np.random.default_rng(81)
    N, C = 3000, 400
    R = blob_ratio(rng, N, C, n_blobs=60)
    chunks = [1000, 1000, 1000]
    tr, got, n = run_gpu_trigger(R, chunks, 3.0, 1.5)
    ev, m = merge_events(tr.records, n, C)
    closed, opened = run_oracle_trigger(oracle_mod, R, chunks, 3.0, 1.5)
    want = oracle_mod.events_merge(np.concatenate([closed, opened]))
    assert m == len(want)
    assert np.array_equal(sort_events(ev[:, :5]), sort_events(want))
    # an event is flagged open exactly when it holds a run still open, i.e.
    # when it ends at the last sample seen (closed runs end earlier)
    assert np.array_equal(ev[:, 5] == abi.FILARK_TRIGGER_OPEN, ev[:, 1] == N)
    tr.close()


def test_events_merge_bounded_retry_reports_timeout(oracle_mod, monkeypatch):
    """The union-find's retry loop is bounded: with the bound lowered to 0 by
    the test override every union gives up, the merge returns FILARK_ETIMEOUT
    (no hang, no fault), and the next merge with the normal bound is correct."""
    import torch
    rng = np.random.default_rng(83)
    N, C = 2000, 64
    R = blob_ratio(rng, N, C, n_blobs=30)
    tr, _, n = run_gpu_trigger(R, [N], 3.0, 1.5)
    assert n > 10
    wb = abi.filark_events_work_bytes(n, C)
    work = torch.empty(wb + 256, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) // 256 * 256
    ev = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
    n_ev = torch.zeros(1, dtype=torch.int64, device="cuda")
    monkeypatch.setenv("FILARK_TEST_UNION_TRIES", "0")
    st = abi.filark_events_merge(tr.records.data_ptr(), n, C, ev.data_ptr(), n, n_ev.data_ptr(), wp, wb, None)
    assert st == abi.FILARK_ETIMEOUT
    monkeypatch.delenv("FILARK_TEST_UNION_TRIES")
    from paper_2605_20132_gb300.chain import merge_events
    got, m = merge_events(tr.records, n, C)
    closed, opened = run_oracle_trigger(oracle_mod, R, [N], 3.0, 1.5)
    want = oracle_mod.events_merge(np.concatenate([closed, opened]))
    assert m == len(want)
    assert np.array_equal(sort_events(got[:, :5]), sort_events(want))
    tr.close()


def test_trigger_capacity_overflow_counts_everything(oracle_mod):
    rng = np.random.default_rng(82)
    R = blob_ratio(rng, 2000, 64, n_blobs=40)
    closed, opened = run_oracle_trigger(oracle_mod, R, [2000], 3.0, 1.5)
    total = len(closed) + len(opened)
    assert total > 20
    tr, _, n = run_gpu_trigger(R, [2000], 3.0, 1.5, capacity=10)
    assert n == total
    kept = tr.records[:10].cpu().numpy()
    allr = {tuple(r) for r in np.concatenate([closed, opened]).tolist()}
    for w in kept:
        assert (int(w[2] & 0xFFFFFFFF), int(w[0]), int(w[1])) in allr
    tr.close()


def test_events_reject_bad_channel():
    import torch
    recs = torch.zeros((2, 3), dtype=torch.int64, device="cuda")
    recs[1, 2] = 7   # channel 7 of 5
    ev = torch.zeros((2, 4), dtype=torch.int64, device="cuda")
    n_ev = torch.zeros(1, dtype=torch.int64, device="cuda")
    wb = abi.filark_events_work_bytes(2, 5)
    work = torch.empty(wb + 256, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) // 256 * 256
    st = abi.filark_events_merge(recs.data_ptr(), 2, 5, ev.data_ptr(), 2, n_ev.data_ptr(), wp, wb, None)
    assert st == abi.FILARK_EINVAL


def test_chain_ratio_to_events_small_workload(oracle_mod):
    """The small workload end to end on the device: chain -> ratio ->
    triggers -> events, against the oracle trigger and merge run on the same
    ratio (the chain's own parity is covered by the chain tests)."""
    import torch
    from paper_2605_20132_gb300.chain import Chain, Trigger, merge_events
    x = synth.small_stream()
    N, C = x.shape
    sos = oracle_mod.butter_bandpass(4, 1.0, 50.0, 1000.0)
    ch = Chain(C, sos, 1000.0, 5, 50, 1000, outputs=ALL_OUT, max_chunk=1000)
    tr = Trigger(C, 3.0, 1.2, max_chunk=1000, capacity=1 << 16)
    xd = torch.from_numpy(x).cuda()
    r = torch.empty_like(xd)
    for t in range(0, N, 1000):
        ch.push(xd[t:t + 1000], ratio=r[t:t + 1000])
        tr.push(r[t:t + 1000])
    tr.flush()
    ch.sync()
    n = int(tr.count.item())
    got = tr.triggers()
    R = r.cpu().numpy()
    closed, opened = run_oracle_trigger(oracle_mod, R, [1000] * 10, 3.0, 1.2)
    want = np.concatenate([np.c_[closed, np.zeros(len(closed), np.int64)],
                           np.c_[opened, np.ones(len(opened), np.int64)]])
    assert n == len(want) and n > 0
    assert np.array_equal(sort_records(got), sort_records(want))
    ev, m = merge_events(tr.records, n, C)
    ref = oracle_mod.events_merge(np.concatenate([closed, opened]))
    assert np.array_equal(sort_events(ev[:, :5]), sort_events(ref))
    # the three Ricker events span the array: some event covers most channels
    assert max(e[3] - e[2] + 1 for e in ref) >= C // 4
    ch.close()
    tr.close()


def test_paper_scale_triggers_and_events(oracle_mod):
    """Triggers on the paper-scale chain's ratio (6,000 channels, 60 pushes
    of 1,500) and their events, against the oracle on the same ratio."""
    import torch
    from paper_2605_20132_gb300.chain import Chain, Trigger, merge_events
    cfg = synth.PAPER_SCALE
    C, N, T = cfg["n_channels"], cfg["n_samples"], cfg["chunk"]
    x = synth.paper_scale_stream(C, N, cfg["seed"])
    sos = oracle_mod.butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    ch = Chain(C, sos, cfg["fs"], cfg["spatial_width"], cfg["sta"], cfg["lta"], outputs=abi.FILARK_OUT_RATIO,
               max_chunk=T)
    tr = Trigger(C, 6.0, 2.0, max_chunk=T, capacity=1 << 22)
    xd = torch.from_numpy(x).cuda()
    r = torch.empty_like(xd)
    for t in range(0, N, T):
        ch.push(xd[t:t + T], ratio=r[t:t + T])
        tr.push(r[t:t + T])
    tr.flush()
    ch.sync()
    n = int(tr.count.item())
    got = tr.triggers()
    del xd
    R = r.cpu().numpy()
    closed, opened = run_oracle_trigger(oracle_mod, R, [T] * (N // T), 6.0, 2.0)
    want = np.concatenate([np.c_[closed, np.zeros(len(closed), np.int64)],
                           np.c_[opened, np.ones(len(opened), np.int64)]])
    print("paper-scale triggers:", n)
    assert n == len(want) and n > 0
    assert np.array_equal(sort_records(got), sort_records(want))
    ev, m = merge_events(tr.records, n, C)
    ref = oracle_mod.events_merge(np.concatenate([closed, opened]))
    print("paper-scale events:", m)
    assert np.array_equal(sort_events(ev[:, :5]), sort_events(ref))
    ch.close()
    tr.close()


@pytest.mark.parametrize("lanes,overlap", [(1, False), (2, False), (2, True), (3, True), (1, True)])
def test_chain_push_triggers_equals_separate_calls(lanes, overlap):
    """Triggers fused into the chain's detector: the ratio and the trigger
    list equal a chain push followed by a trigger push, on a stream with
    events (the small-workload chain at amplitude 6, thresholds 3 / 1.5),
    pushes of 1..3000 samples (several launches per push, ragged segments),
    in one and two lanes, with and without the trigger's overlap mode."""
    import torch
    from paper_2605_20132_gb300.chain import Chain, Trigger, butter_bandpass
    rng = np.random.default_rng(85)
    C, N = 300, 12000
    x = torch.from_numpy(synth.small_stream(C, N, seed=86) * np.float32(6.0)).cuda()
    sos = butter_bandpass(4, 1.0, 50.0, 1000.0)
    chunks = [1, 3000, 2049, 37] + chunking_fixed(rng, N - 5087, 3000)
    ra, rb = torch.full_like(x, float("nan")), torch.full_like(x, float("nan"))
    ca = Chain(C, sos, 1000.0, 5, 50, 1000, outputs=abi.FILARK_OUT_RATIO, max_chunk=3000)
    cb = Chain(C, sos, 1000.0, 5, 50, 1000, outputs=abi.FILARK_OUT_RATIO, max_chunk=3000)
    cb.set_lanes(lanes)
    ta = Trigger(C, 3.0, 1.5, max_chunk=3000)
    tb = Trigger(C, 3.0, 1.5, max_chunk=3000)
    if overlap:
        tb.set_overlap(True)
    t = 0
    for k in chunks:
        ca.push(x[t:t + k], ratio=ra[t:t + k])
        ta.push(ra[t:t + k])
        cb.push_triggers(x[t:t + k], rb[t:t + k], tb)
        t += k
    assert t == N
    ta.flush()
    tb.flush()
    ca.sync()
    cb.join()
    cb.sync()
    assert torch.equal(ra, rb)
    got, want = tb.triggers(), ta.triggers()
    assert len(want) > 50
    assert np.array_equal(sort_records(got), sort_records(want))
    for o in (ca, cb, ta, tb):
        o.close()


def chunking_fixed(rng, n, hi):
    out = []
    while sum(out) < n:
        out.append(int(min(rng.integers(1, hi + 1), n - sum(out))))
    return out

