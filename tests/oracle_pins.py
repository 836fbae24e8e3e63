"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each ``pin_*`` function runs one check against the oracle module it is given
and returns ``(error, bound)``; the check passes when ``error <= bound``.  The
test module calls them on the oracle as built, and the mutation test calls
them on copies of the oracle with a plausible mistake planted, to show that
every planted mistake makes at least one pin fail.

None of these re-types the oracle's recurrence: they compare it with closed
forms (biquad impulse response, Butterworth magnitude), with a different
algorithm (brute-force convolution with closed-form impulse responses, literal
windows), with invariants (chunk invariance, linearity, adjoint identity) or
with finite differences.
"""
from __future__ import annotations

import numpy as np

from paper_2605_20132_gb300 import synth


def sos_response(sos: np.ndarray, w: np.ndarray) -> np.ndarray:
    """H(e^{jw}) of an SOS cascade, evaluated from its definition as a product
    of ratios of quadratics in z^-1."""
    zi = np.exp(-1j * np.asarray(w, dtype=np.float64))
    H = np.ones_like(zi)
    for b0, b1, b2, a0, a1, a2 in sos:
        H *= (b0 + b1 * zi + b2 * zi * zi) / (a0 + a1 * zi + a2 * zi * zi)
    return H


def butter_bp_mag2(w: np.ndarray, N: int, f1: float, f2: float, fs: float) -> np.ndarray:
    """Closed-form |H|^2 of the N-th order Butterworth bandpass after the
    bilinear transform: 1 / (1 + ((W^2 - W1 W2) / (W (W2 - W1)))^(2N)),
    W = 2 fs tan(w/2), Wi = 2 fs tan(pi fi / fs)."""
    W = 2 * fs * np.tan(np.asarray(w) / 2)
    W1 = 2 * fs * np.tan(np.pi * f1 / fs)
    W2 = 2 * fs * np.tan(np.pi * f2 / fs)
    q = (W * W - W1 * W2) / (W * (W2 - W1))
    return 1.0 / (1.0 + q ** (2 * N))


def biquad_impulse_closed_form(b, r: float, theta: float, n: int) -> np.ndarray:
    """Impulse response of (b0 + b1 z^-1 + b2 z^-2) / (1 - 2 r cos(t) z^-1 + r^2 z^-2):
    g[k] = r^k sin((k+1) t) / sin(t), h[k] = b0 g[k] + b1 g[k-1] + b2 g[k-2]."""
    k = np.arange(n, dtype=np.float64)
    g = r ** k * np.sin((k + 1) * theta) / np.sin(theta)
    h = b[0] * g
    h[1:] += b[1] * g[:-1]
    h[2:] += b[2] * g[:-2]
    return h


def random_sections(rng: np.random.Generator, S: int, rmin=0.5, rmax=0.995):
    secs, poles = [], []
    for _ in range(S):
        r = rng.uniform(rmin, rmax)
        th = rng.uniform(0.05, 3.0)
        b = rng.standard_normal(3)
        secs.append([b[0], b[1], b[2], 1.0, -2 * r * np.cos(th), r * r])
        poles.append((r, th))
    return np.array(secs), poles


def _worst(a, b) -> float:
    """max() that treats NaN or infinity as an infinite error."""
    a, b = float(np.max(a)), float(np.max(b))
    if not (np.isfinite(a) and np.isfinite(b)):
        return float("inf")
    return max(a, b)


def normwise_err(a: np.ndarray, ref: np.ndarray) -> float:
    """max over channels of max_n |a - ref| / max_n |ref| (ref [T][C])."""
    den = np.max(np.abs(ref), axis=0)
    den[den == 0] = 1.0
    return float(np.max(np.max(np.abs(a - ref), axis=0) / den))


# ---------------------------------------------------------------- IIR pins --

def pin_biquad_closed_form(ora):
    """Single biquad (and a0 != 1 scaling) vs its closed-form impulse response,
    through both the single-channel filter and the chunked chain."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(6):
        sos, poles = random_sections(rng, 1)
        r, th = poles[0]
        n = 600
        h_ref = biquad_impulse_closed_form(sos[0, :3], r, th, n)
        imp = np.zeros(n)
        imp[0] = 1.0
        y, _ = ora.sosfilt(sos, imp)
        worst = _worst(worst, np.max(np.abs(y - h_ref)) / np.max(np.abs(h_ref)))
        scaled = sos * 2.5                       # same filter written with a0 = 2.5
        y2, _ = ora.sosfilt(scaled, imp)
        worst = _worst(worst, np.max(np.abs(y2 - h_ref)) / np.max(np.abs(h_ref)))
        # chain, 3 channels (impulse at different delays), pushed in uneven chunks
        x = np.zeros((n, 3), dtype=np.float32)
        x[0, 0] = 1.0
        x[5, 1] = 1.0
        x[17, 2] = -2.0
        ch = ora.Chain(3, sos, 1, 0, 0)
        outs = []
        for a, b in [(0, 1), (1, 40), (40, 40), (40, 333), (333, n)]:
            outs.append(ch.push(x[a:b], want=("bp",))["bp"])
        bp = np.concatenate(outs)
        ref = np.zeros((n, 3))
        ref[:, 0] = h_ref
        ref[5:, 1] = h_ref[: n - 5]
        ref[17:, 2] = -2.0 * h_ref[: n - 17]
        worst = _worst(worst, normwise_err(bp, ref))
    return worst, 1e-12


def _cascade_ir_closed_form(sos, poles, n):
    h = np.zeros(n)
    h[0] = 1.0
    for s, (r, th) in enumerate(poles):
        hs = biquad_impulse_closed_form(sos[s, :3], r, th, n)
        h = np.convolve(h, hs)[:n]
    return h


def pin_bruteforce_convolution(ora):
    """Cascade of 3 random biquads on a tiny 8 x 512 input vs brute-force
    convolution with the product of the closed-form section responses,
    truncated where the tail is below 1e-18."""
    rng = np.random.default_rng(12)
    sos, poles = random_sections(rng, 3, 0.5, 0.95)
    rmax = max(r for r, _ in poles)
    n_ir = int(np.ceil(np.log(1e-18) / np.log(rmax))) + 64
    h = _cascade_ir_closed_form(sos, poles, n_ir)
    x = rng.standard_normal((512, 8)).astype(np.float32)
    ref = np.zeros((512, 8))
    for c in range(8):
        ref[:, c] = np.convolve(x[:, c].astype(np.float64), h)[:512]
    ch = ora.Chain(8, sos, 1, 0, 0)
    bp = np.concatenate([ch.push(x[:100], ("bp",))["bp"], ch.push(x[100:], ("bp",))["bp"]])
    return normwise_err(bp, ref), 1e-11


def pin_butterworth_magnitude(ora):
    """|H(e^{jw})| of the designed SOS vs the closed-form Butterworth bandpass
    magnitude at test tones, including 1/sqrt(2) at both band edges and 1 at
    the digital image of the geometric centre."""
    worst = 0.0
    for N, f1, f2, fs in [(1, 5, 40, 200), (2, 1, 50, 1000), (3, 10, 200, 1000), (4, 1, 50, 1000),
                          (5, 1, 400, 1000), (8, 0.5, 100, 1500), (6, 15, 32, 250)]:
        sos = ora.butter_bandpass(N, f1, f2, fs)
        w = np.concatenate([np.linspace(1e-3, np.pi - 1e-3, 97),
                            [2 * np.pi * f1 / fs, 2 * np.pi * f2 / fs]])
        mag2 = np.abs(sos_response(sos, w)) ** 2
        worst = _worst(worst, np.max(np.abs(mag2 - butter_bp_mag2(w, N, f1, f2, fs))))
        W0 = np.sqrt(2 * fs * np.tan(np.pi * f1 / fs) * 2 * fs * np.tan(np.pi * f2 / fs))
        w0 = 2 * np.arctan(W0 / (2 * fs))
        worst = _worst(worst, abs(abs(sos_response(sos, [w0])[0]) - 1.0))
        worst = _worst(worst, abs(abs(sos_response(sos, [2 * np.pi * f1 / fs])[0]) - 2 ** -0.5))
        # 2N poles, all strictly inside the unit circle; N zeros at z = +1 and
        # N at z = -1 (numerators g*(1,-2,1), g*(1,2,1), or one g*(1,0,-1))
        nplus = nminus = 0
        for row in sos:
            if np.any(np.abs(np.roots(row[3:])) >= 1.0):
                worst = _worst(worst, 1.0)
            b = row[:3] / row[0]
            for zero in np.roots(b):
                if abs(zero - 1) < 1e-6:
                    nplus += 1
                elif abs(zero + 1) < 1e-6:
                    nminus += 1
                else:
                    worst = _worst(worst, 1.0)
        worst = _worst(worst, 0.0 if (nplus == N and nminus == N) else 1.0)
    return worst, 1e-9


def pin_steady_state_tones(ora):
    """The amplitude of the steady-state response to a sine equals |H(e^{jw})|
    from the closed-form Butterworth magnitude (small bandpass, 1 kHz)."""
    sos = ora.butter_bandpass(4, 1.0, 50.0, 1000.0)
    n = 30000
    worst = 0.0
    for f in (0.7, 3.0, 20.0, 50.0, 120.0):
        w = 2 * np.pi * f / 1000.0
        k = np.arange(n)
        y, _ = ora.sosfilt(sos, np.sin(w * k))
        tail = slice(n - 4000, n)
        A = np.stack([np.sin(w * k[tail]), np.cos(w * k[tail])], axis=1)
        coef, *_ = np.linalg.lstsq(A, y[tail], rcond=None)
        amp = np.hypot(*coef)
        worst = _worst(worst, abs(amp - np.sqrt(butter_bp_mag2([w], 4, 1.0, 50.0, 1000.0)[0])))
    return worst, 1e-8


def pin_chunk_invariance(ora):
    """Chunked pushes (including 0- and 1-sample chunks) give bit-identical
    outputs and IIR state to one push of the whole record."""
    rng = np.random.default_rng(13)
    sos = ora.butter_bandpass(4, 1.0, 50.0, 1000.0)
    x = synth.small_stream(12, 2600, seed=5)
    whole = ora.Chain(12, sos, 5, 7, 40)
    ref = whole.push(x)
    worst = 0.0
    for trial in range(3):
        cuts = np.sort(rng.integers(0, 2600, 9))
        cuts = np.concatenate([[0], cuts, [cuts[-1]], [min(cuts[-1] + 1, 2600)], [2600]])
        ch = ora.Chain(12, sos, 5, 7, 40)
        parts = {k: [] for k in ref}
        for a, b in zip(cuts[:-1], cuts[1:]):
            o = ch.push(x[a:b])
            for k in o:
                parts[k].append(o[k])
        for k in ref:
            got = np.concatenate(parts[k])
            if not np.array_equal(got, ref[k]):
                worst = _worst(worst, float(np.max(np.abs(got - ref[k]))) + 1.0)
        if not np.array_equal(ch.iir_state(), whole.iir_state()):
            worst = _worst(worst, 1.0)
    return worst, 0.0


def pin_linearity_time_invariance(ora):
    """The chain's IIR output is linear and shift-invariant: filtering
    a*x1 + b*x2 delayed by d equals the same combination of delayed outputs."""
    rng = np.random.default_rng(14)
    sos = ora.butter_bandpass(4, 1.0, 50.0, 1000.0)
    x1 = rng.standard_normal(3000)
    x2 = rng.standard_normal(3000)
    y1, _ = ora.sosfilt(sos, x1)
    y2, _ = ora.sosfilt(sos, x2)
    d = 37
    comb = np.zeros(3000)
    comb[d:] = 0.5 * x1[:-d] - 1.5 * x2[:-d]
    y, _ = ora.sosfilt(sos, comb)
    ref = np.zeros(3000)
    ref[d:] = 0.5 * y1[:-d] - 1.5 * y2[:-d]
    return float(np.max(np.abs(y - ref)) / np.max(np.abs(ref))), 1e-10


# ------------------------------------------------------------ spatial pins --

def pin_spatial_invariants(ora):
    """With the IIR and detector off: a constant row stays constant; a ramp
    across channels is reproduced exactly in the interior and gives (c+h)/2 at
    the low edge (window [0, c+h]); an impulse on one channel spreads as
    1/|W(c)| over the channels within h of it, with |W| shrunk at the edges."""
    C, K = 23, 7
    h = (K - 1) // 2
    worst = 0.0
    ch = ora.Chain(C, None, K, 0, 0)
    # constant
    out = ch.push(np.full((3, C), 0.75, dtype=np.float32), ("sp",))["sp"]
    worst = _worst(worst, float(np.max(np.abs(out - 0.75))))
    # ramp
    ramp = np.tile(np.arange(C, dtype=np.float32), (2, 1))
    out = ch.push(ramp, ("sp",))["sp"][0]
    for c in range(C):
        lo, hi = max(0, c - h), min(C - 1, c + h)
        worst = _worst(worst, abs(out[c] - (lo + hi) / 2.0))
    # impulse on channel 1 (near the edge) and on channel 12
    for cstar in (1, 12):
        row = np.zeros((1, C), dtype=np.float32)
        row[0, cstar] = 1.0
        out = ch.push(row, ("sp",))["sp"][0]
        for c in range(C):
            lo, hi = max(0, c - h), min(C - 1, c + h)
            want = 1.0 / (hi - lo + 1) if lo <= cstar <= hi else 0.0
            worst = _worst(worst, abs(out[c] - want))
    return worst, 1e-15


# ------------------------------------------------------------ STA/LTA pins --

def pin_stalta_closed_forms(ora):
    """IIR and spatial stage off, so cf = x^2.  Constant input: R = 0 before
    the long window fills, then exactly 1.  Step on at n0: R = STA/LTA with
    STA = a^2 min(n-n0+1, ns)/ns and LTA = a^2 min(n-n0+1, nl)/nl.  Step off:
    once the long window holds only zeros, R is exactly 0."""
    ns, nl = 4, 11
    worst = 0.0
    ch = ora.Chain(1, None, 1, ns, nl)
    R = np.concatenate([ch.push(np.full((k, 1), 1.5, dtype=np.float32), ("ratio",))["ratio"][:, 0]
                        for k in (3, 9, 30)])
    want = np.where(np.arange(42) >= nl - 1, 1.0, 0.0)
    worst = _worst(worst, float(np.max(np.abs(R - want))))
    # step on at n0 = 20, then off at n1 = 60 (exact and inexact amplitudes)
    n0, n1, N = 20, 60, 100
    for a in (2.0, 1.3):
        x = np.zeros((N, 1), dtype=np.float32)
        x[n0:n1, 0] = a
        a2 = float(np.float32(a)) ** 2
        ch = ora.Chain(1, None, 1, ns, nl)
        R = np.concatenate([ch.push(x[:57], ("ratio",))["ratio"], ch.push(x[57:], ("ratio",))["ratio"]])[:, 0]
        for n in range(N):
            on_s = max(0, min(n, n1 - 1) - max(n0, n - ns + 1) + 1)
            on_l = max(0, min(n, n1 - 1) - max(n0, n - nl + 1) + 1)
            sta, lta = a2 * on_s / ns, a2 * on_l / nl
            want = sta / lta if (n >= nl - 1 and on_l > 0) else 0.0
            worst = _worst(worst, abs(R[n] - want))
    return worst, 1e-12


def pin_stalta_vs_literal_windows(ora):
    """Running-sum STA/LTA of the chunked chain vs literal windows (O(window)
    per sample) applied to the chain's own cf = y_sp^2."""
    sos = ora.butter_bandpass(4, 1.0, 50.0, 1000.0)
    x = synth.small_stream(6, 1500, seed=7)
    ns, nl = 9, 61
    ch = ora.Chain(6, sos, 3, ns, nl)
    parts = [ch.push(x[a:b]) for a, b in [(0, 50), (50, 51), (51, 700), (700, 1500)]]
    sp = np.concatenate([p["sp"] for p in parts])
    R = np.concatenate([p["ratio"] for p in parts])
    worst = 0.0
    for c in range(6):
        ref = ora.stalta_naive(sp[:, c] ** 2, ns, nl)
        worst = _worst(worst, float(np.max(np.abs(R[:, c] - ref)) / max(1.0, np.max(np.abs(ref)))))
    # one long channel, past the period at which the running sums are re-added
    rng = np.random.default_rng(8)
    n_long = 140_000
    xl = (rng.standard_normal((n_long, 1)) * np.exp(rng.standard_normal((n_long, 1)))).astype(np.float32)
    ch = ora.Chain(1, None, 1, ns, nl)
    Rl = np.concatenate([ch.push(xl[a:a + 9999], ("ratio",))["ratio"] for a in range(0, n_long, 9999)])[:, 0]
    ref = ora.stalta_naive(xl[:, 0].astype(np.float64) ** 2, ns, nl)
    worst = _worst(worst, float(np.max(np.abs(Rl - ref)) / max(1.0, np.max(np.abs(ref)))))
    return worst, 1e-11



# ------------------------------------------------------ trigger / event pins --

def _sorted_records(r):
    r = np.asarray(r, dtype=np.int64).reshape(-1, 3)
    return r[np.lexsort((r[:, 2], r[:, 1], r[:, 0]))] if r.size else r


def pin_trigger_closed_forms(ora):
    """Hand-built ratio sequences with known runs: a value equal to the on
    threshold sets, equal to the off threshold keeps, just below it resets;
    a run open at the end is reported only by the flush, and a run that spans
    a push boundary keeps its start."""
    on, off = 4.0, 1.5
    lo = float(np.nextafter(np.float32(off), np.float32(0)))
    R = np.zeros((12, 4), dtype=np.float32)
    R[:, 0] = [0, 4, 2, 1.5, 1.5, lo, 0, 5, 0, 0, 0, 0]        # runs [1,5), [7,8)
    R[:, 1] = [3.99, 3.99, 1, 4, 4, 4, 4, 4, 4, 4, 4, 4]       # open from 3
    R[:, 2] = [9, 0, 9, 0, 9, 0, 9, 0, 9, 0, 9, 0]             # six unit runs
    R[:, 3] = [0] * 12                                          # never
    t = ora.Trigger(4, on, off)
    got = np.concatenate([t.push(R[:4]), t.push(R[4:9]), t.push(R[9:])])
    fl = t.flush()
    want = [(0, 1, 5), (0, 7, 8)] + [(2, k, k + 1) for k in range(0, 12, 2)]
    err = 0.0 if np.array_equal(_sorted_records(got), _sorted_records(want)) else 1.0
    err += 0.0 if np.array_equal(_sorted_records(fl), _sorted_records([(1, 3, 12)])) else 1.0
    return err, 0.0


def pin_trigger_last_forcing_sample(ora):
    """The recursion s(n) = set / reset / keep has a non-recursive form: s(n)
    = 1 exactly when the latest sample k <= n with R(k) >= on or R(k) < off
    exists and has R(k) >= on.  Runs of that image, on random ratios pushed
    in random chunks, must equal the oracle's triggers (plus the flush)."""
    rng = np.random.default_rng(31)
    C, N, on, off = 7, 400, 2.0, 1.2
    R = rng.choice(np.array([0.0, 1.0, 1.2, 1.5, 1.99, 2.0, 3.0], dtype=np.float32), size=(N, C),
                   p=[0.15, 0.15, 0.1, 0.3, 0.1, 0.1, 0.1])
    S = np.zeros((N, C), dtype=np.int64)
    for c in range(C):
        forcing = (R[:, c] >= on) | (R[:, c] < off)
        idx = np.where(forcing, np.arange(N), -1)
        last = np.maximum.accumulate(idx)
        S[:, c] = np.where(last >= 0, R[np.maximum(last, 0), c] >= on, False)
    want = []
    for c in range(C):
        d = np.diff(np.concatenate([[0], S[:, c], [0]]))
        for a, b in zip(np.where(d == 1)[0], np.where(d == -1)[0]):
            want.append((c, a, b))
    t = ora.Trigger(C, on, off)
    parts, pos = [], 0
    while pos < N:
        k = int(rng.integers(1, 60))
        parts.append(t.push(R[pos:pos + k]))
        pos += k
    parts.append(t.flush())
    got = np.concatenate(parts)
    return (0.0 if np.array_equal(_sorted_records(got), _sorted_records(want)) else 1.0), 0.0


def _flood_fill_events(S):
    """4-connected components of the binary image S[n][c]: (t_on, t_off,
    c_min, c_max, n_runs) with t_off one past the last sample."""
    N, C = S.shape
    seen = np.zeros_like(S, dtype=bool)
    out = []
    for n0 in range(N):
        for c0 in range(C):
            if not S[n0, c0] or seen[n0, c0]:
                continue
            stack, cells = [(n0, c0)], []
            seen[n0, c0] = True
            while stack:
                n, c = stack.pop()
                cells.append((n, c))
                for dn, dc in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    m, d = n + dn, c + dc
                    if 0 <= m < N and 0 <= d < C and S[m, d] and not seen[m, d]:
                        seen[m, d] = True
                        stack.append((m, d))
            ns = [n for n, _ in cells]
            cs = [c for _, c in cells]
            runs = sum(1 for n, c in cells if n == 0 or not S[n - 1, c])
            out.append((min(ns), max(ns) + 1, min(cs), max(cs), runs))
    out.sort(key=lambda e: (e[0], e[2], e[1], e[3]))
    return np.array(out, dtype=np.int64).reshape(-1, 5)


def pin_events_vs_flood_fill(ora):
    """Events merged from channel triggers (neighbouring channels, intervals
    sharing a sample) equal the 4-connected components of the trigger image
    found by flood fill, on random blob-shaped ratio images."""
    rng = np.random.default_rng(37)
    worst = 0.0
    for trial in range(6):
        C, N = 24, 160
        R = np.zeros((N, C), dtype=np.float32)
        for _ in range(10):
            c0, n0 = rng.integers(0, C), rng.integers(0, N)
            w, h, slope = rng.integers(1, 6), rng.integers(3, 25), rng.integers(-2, 3)
            for c in range(max(0, c0 - w), min(C, c0 + w + 1)):
                a = n0 + slope * (c - c0)
                R[max(0, a):max(0, min(N, a + h)), c] = 5.0
        R[rng.random((N, C)) < 0.03] = 5.0
        t = ora.Trigger(C, 3.0, 3.0)
        recs = np.concatenate([t.push(R[:N // 3]), t.push(R[N // 3:]), t.flush()])
        ev = ora.events_merge(recs)
        ref = _flood_fill_events(R >= 3.0)
        worst = max(worst, 0.0 if np.array_equal(ev, ref) else 1.0)
    return worst, 0.0


# ----------------------------------------------------- temporal-op pins --

def _top_run(ora, x, kind, length=1, taps=None, alpha=0.0, chunks=None):
    op = ora.TemporalOp(x.shape[1], kind, length, taps, alpha)
    if chunks is None:
        return op.push(x)
    out, pos = [], 0
    for k in chunks:
        out.append(op.push(x[pos:pos + k]))
        pos += k
    return np.concatenate(out)


def pin_fir_vs_convolution(ora):
    """Realtime FIR: impulses give the taps back, and random input pushed in
    random chunks equals numpy's full convolution truncated to the input
    length (brute force, independent code)."""
    rng = np.random.default_rng(41)
    worst = 0.0
    for M in (1, 2, 7, 64):
        h = rng.standard_normal(M)
        x = np.zeros((3 * M + 5, 2), dtype=np.float32)
        x[3, 0] = 1.0
        y = _top_run(ora, x, ora.TOP_FIR, M, h)
        worst = _worst(worst, float(np.max(np.abs(y[3:3 + M, 0] - h))))
        worst = _worst(worst, float(np.max(np.abs(y[:3, 0]))) + float(np.max(np.abs(y[:, 1]))))
        x = rng.standard_normal((500, 3)).astype(np.float32)
        chunks, pos = [], 0
        while pos < 500:
            k = int(rng.integers(1, 90))
            chunks.append(min(k, 500 - pos))
            pos += chunks[-1]
        y = _top_run(ora, x, ora.TOP_FIR, M, h, chunks=chunks)
        for c in range(3):
            ref = np.convolve(x[:, c].astype(np.float64), h)[:500]
            worst = _worst(worst, normwise_err(y[:, c:c + 1], ref[:, None]))
    return worst, 1e-13


def pin_window_ops_literal(ora):
    """Running mean and AGC against literal window sums on random input in
    random chunks (past the re-summation period), plus closed forms for a
    constant: mean ramps as c (n+1)/w then stays c; AGC of +-c is w/(n+1) in
    magnitude during the ramp, then +-1."""
    rng = np.random.default_rng(43)
    worst = 0.0
    N, w = 9000, 37
    x = (rng.standard_normal((N, 2)) * rng.uniform(0.1, 3.0, (N, 1))).astype(np.float32)
    x[5000:5100, 0] = 0.0
    chunks = [int(k) for k in rng.integers(1, 700, 40)]
    chunks = [k for k in np.diff(np.unique(np.r_[0, np.cumsum(chunks), N].clip(0, N)))]
    mean = _top_run(ora, x, ora.TOP_MEAN, w, chunks=chunks)
    agc = _top_run(ora, x, ora.TOP_AGC, w, chunks=chunks)
    xd = x.astype(np.float64)
    pad = np.vstack([np.zeros((w - 1, 2)), xd])
    for n in range(0, N, 7):
        win = pad[n:n + w]
        m = win.sum(axis=0) / w
        g = np.abs(win).sum(axis=0) / w
        a = np.where(g > 0, xd[n] / np.where(g > 0, g, 1), 0.0)
        worst = _worst(worst, float(np.max(np.abs(mean[n] - m))) / 3.0)
        worst = _worst(worst, float(np.max(np.abs(agc[n] - a) / np.maximum(1.0, np.abs(a)))))
    c = np.full((3 * w, 1), 2.5, dtype=np.float32)
    c[1::2] *= -1
    m = _top_run(ora, np.abs(c), ora.TOP_MEAN, w)[:, 0]
    n = np.arange(3 * w)
    worst = _worst(worst, float(np.max(np.abs(m - 2.5 * np.minimum(n + 1, w) / w))))
    a = _top_run(ora, c, ora.TOP_AGC, w)[:, 0]
    worst = _worst(worst, float(np.max(np.abs(np.abs(a) - w / np.minimum(n + 1, w)))))
    worst = _worst(worst, float(np.max(np.abs(np.sign(a) - np.sign(c[:, 0])))))
    return worst, 1e-11


def pin_ema_closed_forms(ora):
    """EMA power equalisation: a constant c gives e[n] = c^2 (1 - (1-a)^(n+1))
    and y = 1 / sqrt(1 - (1-a)^(n+1)); an impulse gives y = 1/sqrt(a) then 0;
    chunking does not change the output."""
    worst = 0.0
    for a in (0.5, 0.01, 1e-4):
        n = np.arange(3000)
        y = _top_run(ora, np.full((3000, 1), -1.7, dtype=np.float32), ora.TOP_EMA, alpha=a)[:, 0]
        ref = -1.0 / np.sqrt(1.0 - (1.0 - a) ** (n + 1))
        worst = _worst(worst, float(np.max(np.abs(y - ref) / np.abs(ref))))
        x = np.zeros((50, 1), dtype=np.float32)
        x[4] = 3.0
        y = _top_run(ora, x, ora.TOP_EMA, alpha=a)[:, 0]
        want = np.zeros(50)
        want[4] = 1.0 / np.sqrt(a)
        worst = _worst(worst, float(np.max(np.abs(y - want))) * np.sqrt(a))
    rng = np.random.default_rng(47)
    x = rng.standard_normal((2000, 3)).astype(np.float32)
    whole = _top_run(ora, x, ora.TOP_EMA, alpha=0.003)
    parts = _top_run(ora, x, ora.TOP_EMA, alpha=0.003, chunks=[1, 999, 3, 997])
    worst = _worst(worst, 0.0 if np.array_equal(whole, parts) else 1.0)
    return worst, 1e-12


# ---------------------------------------------------------- display pins --

def pin_view_closed_forms(ora):
    """The headless display buffer on a linear field x[n][c] = 1000 n + c:
    drop gives the group's first sample, linear interpolation the value at
    the group's centre (exact on a linear field), both in the ring order
    (newest column at the right, zeros before the first) for any chunking;
    peak picks an isolated spike, negative or positive."""
    worst = 0.0
    C, N, kc, kt, W = 11, 700, 3, 7, 40
    n = np.arange(N, dtype=np.float64)[:, None]
    c = np.arange(C, dtype=np.float64)[None, :]
    x = (1000.0 * n + c).astype(np.float32)
    ncol = N // kt
    H = -(-C // kc)
    for mode in (ora.VIEW_DROP, ora.VIEW_LINEAR):
        for chunks in ([N], [1, 13, 300, 386]):
            v = ora.View(C, kc, kt, W, mode)
            pos = 0
            for k in chunks:
                v.push(x[pos:pos + k])
                pos += k
            img = v.image()
            want = np.zeros((H, W))
            for i in range(W):
                j = ncol - W + i
                if j < 0:
                    continue
                for r in range(H):
                    k_r = min(C, (r + 1) * kc) - r * kc
                    if mode == ora.VIEW_DROP:
                        want[r, i] = 1000.0 * j * kt + r * kc
                    else:
                        want[r, i] = 1000.0 * (j * kt + (kt - 1) / 2) + r * kc + (k_r - 1) / 2
            worst = _worst(worst, float(np.max(np.abs(img - want))))
    x = np.zeros((70, 9), dtype=np.float32)
    x[12, 4] = -5.0
    x[13, 3] = 4.0
    x[40, 8] = 2.0
    v = ora.View(9, 3, 10, 8, ora.VIEW_PEAK)
    v.push(x)
    img = v.image()
    want = np.zeros((3, 8))
    want[1, 8 - 7 + 1] = -5.0
    want[2, 8 - 7 + 4] = 2.0
    worst = _worst(worst, float(np.max(np.abs(img - want))))
    return worst, 0.0


def pin_view_display_filter(ora):
    """With the causal display filter, drop-mode columns are the filtered
    rows (per-channel SOS filtering of the dropped channels) sampled every kt
    samples, across pushes."""
    rng = np.random.default_rng(53)
    sos = ora.butter_bandpass(2, 5.0, 80.0, 1000.0)
    C, N, kc, kt, W = 8, 900, 2, 5, 200
    x = rng.standard_normal((N, C)).astype(np.float32)
    v = ora.View(C, kc, kt, W, ora.VIEW_DROP, sos)
    for a in range(0, N, 250):
        v.push(x[a:a + 250])
    img = v.image()
    worst = 0.0
    for r in range(C // kc):
        y, _ = ora.sosfilt(sos, x[:, r * kc].astype(np.float64))
        cols = y[0:N - N % kt:kt]
        worst = _worst(worst, normwise_err(img[r, W - len(cols):][:, None], cols[-W:][:, None]))
    return worst, 1e-12

# ------------------------------------------------------------ adjoint pins --

def _loss_and_grads(ora, sos, x, target):
    y, _ = ora.sosfilt(sos, x)
    r = y - target
    L = float(np.mean(r * r))
    gy = 2.0 * r / r.size
    gx, gs = ora.sos_adjoint(sos, x, gy)
    return L, gx, gs


def _central_diff(f, v0, h):
    """Central difference with one Richardson step: O(h^4) truncation."""
    d1 = (f(v0 + h) - f(v0 - h)) / (2 * h)
    d2 = (f(v0 + h / 2) - f(v0 - h / 2)) / h
    return (4 * d2 - d1) / 3


def pin_adjoint_finite_differences(ora):
    """Gradients of L = mean((y - target)^2) with respect to every SOS
    coefficient (a0 included) and to a few input samples vs FP64 central
    finite differences (the coefficient step is small because the sections
    with poles near z = 1 are very sensitive)."""
    rng = np.random.default_rng(15)
    sos = ora.butter_bandpass(4, 1.0, 50.0, 1000.0)
    target_sos = synth.perturb_sos(sos, 0.02, 16)
    x = rng.standard_normal(2000)
    target, _ = ora.sosfilt(target_sos, x)
    _, gx, gs = _loss_and_grads(ora, sos, x, target)
    worst = 0.0
    for s in range(sos.shape[0]):
        for i in range(6):
            def f(v, s=s, i=i):
                q = sos.copy()
                q[s, i] = v
                return _loss_and_grads(ora, q, x, target)[0]
            fd = _central_diff(f, sos[s, i], 1e-7 * max(0.1, abs(sos[s, i])))
            worst = _worst(worst, abs(fd - gs[s, i]) / max(abs(fd), 1e-12 + 1e-6 * np.max(np.abs(gs))))
    for n in (0, 1, 999, 1998, 1999):
        def f(v, n=n):
            q = x.copy()
            q[n] = v
            return _loss_and_grads(ora, sos, q, target)[0]
        fd = _central_diff(f, x[n], 1e-3)
        worst = _worst(worst, abs(fd - gx[n]) / max(abs(fd), 1e-6 * np.max(np.abs(gx))))
    return worst, 1e-5


def pin_adjoint_identity(ora):
    """<H x, g> = <x, H^T g>: the input gradient of the linear map x -> y."""
    rng = np.random.default_rng(17)
    sos = ora.butter_bandpass(4, 1.0, 50.0, 1000.0)
    x = rng.standard_normal(3000)
    g = rng.standard_normal(3000)
    y, _ = ora.sosfilt(sos, x)
    gx, _ = ora.sos_adjoint(sos, x, g)
    a, b = float(np.dot(y, g)), float(np.dot(x, gx))
    return abs(a - b) / max(abs(a), 1e-30), 1e-10


def pin_adjoint_scale_invariance(ora):
    """Scaling all six coefficients of one section by the same factor leaves
    the cascade unchanged, so the loss is homogeneous of degree 0 in each
    section's coefficients and (Euler) sum_k c_k dL/dc_k = 0 per section.
    Checked relative to sum_k |c_k dL/dc_k|; a wrong sign, a swapped lag or a
    dropped term in any of the six gradients breaks it."""
    rng = np.random.default_rng(19)
    sos = ora.butter_bandpass(4, 1.0, 50.0, 1000.0) * np.array([[1.0], [2.5], [0.4], [1.0]])
    target_sos = synth.perturb_sos(sos, 0.02, 20)
    x = rng.standard_normal(2500)
    target, _ = ora.sosfilt(target_sos, x)
    _, _, gs = _loss_and_grads(ora, sos, x, target)
    worst = 0.0
    for s in range(sos.shape[0]):
        terms = sos[s] * gs[s]
        worst = _worst(worst, abs(float(np.sum(terms))) / float(np.sum(np.abs(terms))))
    return worst, 1e-10


def pin_stalta_naive_closed_forms(ora):
    """The literal-window helper itself: constant cf gives R = 1 after the
    warm-up; a single spike of height a at k0 gives STA = a/ns, LTA = a/nl
    while it is inside both windows (R = nl/ns), R = 0 once it has left the
    short window but not the long one, and 0 after both."""
    ns, nl, N = 5, 17, 60
    worst = 0.0
    R = ora.stalta_naive(np.full(N, 2.25), ns, nl)
    worst = _worst(worst, np.max(np.abs(R - np.where(np.arange(N) >= nl - 1, 1.0, 0.0))))
    cf = np.zeros(N)
    k0 = 20
    cf[k0] = 3.0
    R = ora.stalta_naive(cf, ns, nl)
    for n in range(N):
        if n < nl - 1 or n < k0 or n > k0 + nl - 1:
            want = 0.0
        elif n <= k0 + ns - 1:
            want = nl / ns
        else:
            want = 0.0
        worst = _worst(worst, abs(R[n] - want))
    return worst, 1e-12


ALL_PINS = [
    pin_biquad_closed_form,
    pin_bruteforce_convolution,
    pin_butterworth_magnitude,
    pin_steady_state_tones,
    pin_chunk_invariance,
    pin_linearity_time_invariance,
    pin_spatial_invariants,
    pin_stalta_closed_forms,
    pin_stalta_vs_literal_windows,
    pin_stalta_naive_closed_forms,
    pin_adjoint_finite_differences,
    pin_adjoint_identity,
    pin_adjoint_scale_invariance,
    pin_trigger_closed_forms,
    pin_trigger_last_forcing_sample,
    pin_events_vs_flood_fill,
    pin_fir_vs_convolution,
    pin_window_ops_literal,
    pin_ema_closed_forms,
    pin_view_closed_forms,
    pin_view_display_filter,
]
