"""Seeded synthetic DAS streams shaped like the paper's workloads.

This module only makes inputs: Gaussian noise, 1/f (pink) noise and Ricker
wavelets with linear moveout.  It holds none of the filter chain's arithmetic,
and both the CUDA path's tests/benchmark and the oracle's tests draw their
inputs from it, so the two sides always see identical float32 arrays.

The paper's own recordings (three concatenated OOI ocean-cable files,
Sec. 6.2) are not available; these streams stand in for them, with the channel
counts and sampling rates of the paper's sizing example (6,000 channels at
1,500 Hz, float32, Sec. 1).

Layout of every array returned: time-major ``[n_samples][n_channels]`` float32
(the ``nt_nc`` dimension order of the paper's Tape protocol, Sec. 3.5).
"""
from __future__ import annotations

import numpy as np


def ricker(t: np.ndarray, f: float) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f^2 t^2) exp(-pi^2 f^2 t^2), peak frequency f."""
    a = (np.pi * f * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def add_ricker_events(x: np.ndarray, fs: float, t0: np.ndarray, c0: np.ndarray,
                      f: np.ndarray, slope_s: np.ndarray, amp: np.ndarray,
                      t_offset: float = 0.0) -> None:
    """Add events in place.  Event e arrives on channel c at
    t0[e] + slope_s[e] * (c - c0[e]) seconds and lasts |t| <= 1.5 / f[e] around
    it; ``t_offset`` is the time of row 0 of ``x``."""
    N, C = x.shape
    ch = np.arange(C)
    for e in range(len(t0)):
        half = 1.5 / f[e]
        width = int(np.ceil(2 * half * fs)) + 2
        arrival = t0[e] + slope_s[e] * (ch - c0[e]) - t_offset          # [C] seconds
        start = np.floor((arrival - half) * fs).astype(np.int64)         # first row per channel
        rows = start[None, :] + np.arange(width)[:, None]               # [width][C]
        tt = (rows / fs - arrival[None, :]).astype(np.float32)
        w = (amp[e] * ricker(tt, np.float32(f[e]))).astype(np.float32)
        ok = (rows >= 0) & (rows < N) & (np.abs(tt) <= half)
        cols = np.broadcast_to(ch[None, :], rows.shape)
        x[rows[ok], cols[ok]] += w[ok]


def _rfft_shaped_pink(w: np.ndarray, shape: np.ndarray) -> np.ndarray:
    try:
        import scipy.fft as sf
        W = sf.rfft(w, axis=0, workers=1)
        W *= shape[:, None].astype(W.real.dtype)
        return sf.irfft(W, n=w.shape[0], axis=0, workers=1).astype(np.float32)
    except ImportError:
        W = np.fft.rfft(w, axis=0)
        W *= shape[:, None]
        return np.fft.irfft(W, n=w.shape[0], axis=0).astype(np.float32)


def _noise_block(seed: int, b: int, n_samples: int, c0: int, c1: int, pink: bool,
                 shape: np.ndarray | None, out: np.ndarray) -> None:
    rng = np.random.default_rng([seed, 1, b])
    blk = rng.standard_normal((n_samples, c1 - c0), dtype=np.float32)
    if pink:
        p = _rfft_shaped_pink(rng.standard_normal((n_samples, c1 - c0), dtype=np.float32), shape)
        p /= p.std(axis=0, keepdims=True)
        blk += p
    out[:, c0:c1] = blk


NOISE_BLOCK = 128   # channels per independently seeded noise block


def noise_ricker_stream(n_channels: int, n_samples: int, fs: float, n_events: int,
                        amp: float, f_range: tuple[float, float],
                        slope_ms_range: tuple[float, float], seed: int,
                        pink: bool = False, fixed_origin_channel: bool = False,
                        threads: int | None = None) -> np.ndarray:
    """N(0,1) noise (+ unit-sigma pink noise per channel: white noise shaped by
    1/sqrt(f) in the rFFT domain, DC zeroed, scaled to sigma = 1 over the whole
    record) + seeded Ricker events.  Channel blocks of NOISE_BLOCK channels have
    their own seeds, so the result does not depend on the thread count."""
    import concurrent.futures as cf
    import os
    x = np.empty((n_samples, n_channels), dtype=np.float32)
    shape = None
    if pink:
        k = np.arange(n_samples // 2 + 1, dtype=np.float64)
        shape = np.zeros_like(k)
        shape[1:] = 1.0 / np.sqrt(k[1:])
    blocks = [(b, c0, min(n_channels, c0 + NOISE_BLOCK)) for b, c0 in
              enumerate(range(0, n_channels, NOISE_BLOCK))]
    nthr = threads or min(len(blocks), os.cpu_count() or 1, 32)
    with cf.ThreadPoolExecutor(max_workers=max(1, nthr)) as ex:
        list(ex.map(lambda a: _noise_block(seed, a[0], n_samples, a[1], a[2], pink, shape, x), blocks))
    rng = np.random.default_rng([seed, 2])
    dur = n_samples / fs
    if fixed_origin_channel:
        t0 = rng.uniform(0.1 * dur, 0.9 * dur, n_events)
        c0 = np.zeros(n_events)
    else:
        t0 = rng.uniform(0, dur, n_events)
        c0 = rng.uniform(0, n_channels, n_events)
    f = rng.uniform(f_range[0], f_range[1], n_events)
    slope = rng.uniform(slope_ms_range[0], slope_ms_range[1], n_events) * 1e-3
    add_ricker_events(x, fs, t0, c0, f, slope, np.full(n_events, amp))
    return x


# --------------------------------------------------------------------------
# The workloads.  Chain parameters are given in samples (windows) and as
# Butterworth specs (prototype order N, band edges in Hz).
# --------------------------------------------------------------------------

SMALL = dict(name="small-64ch-1kHz", n_channels=64, n_samples=10_000, fs=1000.0, order=4,
             band=(1.0, 50.0), chunk=1000, spatial_width=5, sta=50, lta=1000, seed=1)

PAPER_SCALE = dict(name="paper-scale-6000ch-1500Hz", n_channels=6000, n_samples=90_000, fs=1500.0,
                   order=8, band=(0.5, 100.0), chunk=1500, spatial_width=9, sta=150, lta=3000, seed=2)

BATCH = dict(name="batch-32-streams", n_streams=32, channels=(500, 10_000), chunk=(200, 3000),
             fs=1000.0, order=4, band=(1.0, 50.0), spatial_width=5, sta=50, lta=1000, seed=3)

ADJOINT = dict(name="adjoint-2048ch-30k", n_channels=2048, n_samples=30_000, fs=1000.0, order=4,
               band=(1.0, 50.0), checkpoint=3000, perturb=0.02, seed=4)

PRECISION = dict(name="precision-10000ch-600s", n_channels=10_000, n_samples=900_000, fs=1500.0,
                 order=8, band=(0.01, 1.0), chunk=1500, sine_hz=0.05, sine_amp=0.1, seed=5)


def small_stream(n_channels: int = 64, n_samples: int = 10_000, seed: int = 1) -> np.ndarray:
    """64 ch x 10,000 samples at 1 kHz: N(0,1) + 3 Ricker events (20 Hz peak,
    amplitude 5, 0.5 ms/channel moveout) at seeded times."""
    return noise_ricker_stream(n_channels, n_samples, 1000.0, 3, 5.0, (20.0, 20.0),
                               (0.5, 0.5), seed, pink=False, fixed_origin_channel=True)


def paper_scale_stream(n_channels: int = 6000, n_samples: int = 90_000, seed: int = 2,
                       n_events: int = 200) -> np.ndarray:
    """6,000 ch x 60 s at 1.5 kHz: N(0,1) + unit pink noise + 200 Ricker events
    (amplitude 5, peak 5-80 Hz, moveout -1..1 ms/channel, seeded origin time and
    channel)."""
    return noise_ricker_stream(n_channels, n_samples, 1500.0, n_events, 5.0, (5.0, 80.0),
                               (-1.0, 1.0), seed, pink=True)


def adjoint_stream(n_channels: int = 2048, n_samples: int = 30_000, seed: int = 4) -> np.ndarray:
    """Input of the differentiation workload: 1 kHz float32 N(0,1) noise plus
    Ricker events (amplitude 5, peak 5-50 Hz, moveout -1..1 ms/channel), one
    event per 64 channels."""
    return noise_ricker_stream(n_channels, n_samples, 1000.0, max(1, n_channels // 64), 5.0, (5.0, 50.0),
                               (-1.0, 1.0), seed, pink=False)


def precision_chunk(chunk_index: int, n_channels: int = 10_000, chunk: int = 1500,
                    fs: float = 1500.0, seed: int = 5, sine_hz: float = 0.05,
                    sine_amp: float = 0.1, channels: np.ndarray | None = None) -> np.ndarray:
    """One chunk of the long precision-stress stream: N(0,1) noise plus a
    0.05 Hz sinusoid of amplitude 0.1 with a seeded phase per channel.  Each
    chunk is generated from its own seed, so any chunk (and any subset of
    channels) can be made on its own."""
    phase = np.random.default_rng([seed, 0]).uniform(0, 2 * np.pi, n_channels)
    rng = np.random.default_rng([seed, 1, chunk_index])
    x = rng.standard_normal((chunk, n_channels), dtype=np.float32)
    t = (chunk_index * chunk + np.arange(chunk, dtype=np.float64)) / fs
    if channels is not None:
        x = x[:, channels]
        phase = phase[channels]
    x += (sine_amp * np.sin(2 * np.pi * sine_hz * t[:, None] + phase[None, :])).astype(np.float32)
    return x


def precision_chunk_device(chunk_index: int, n_channels: int = 10_000, chunk: int = 1500,
                           fs: float = 1500.0, seed: int = 5, sine_hz: float = 0.05,
                           sine_amp: float = 0.1, generator=None):
    """The same stream's chunk made on the CUDA device, so that the whole
    600 s record is quick to produce: the noise comes from torch's seeded
    generator (the same N(0,1) distribution as precision_chunk, other
    samples), the sinusoid's phases are precision_chunk's.  Returns a float32
    CUDA tensor of shape (chunk, n_channels)."""
    import torch
    g = generator if generator is not None else torch.Generator(device="cuda")
    g.manual_seed(seed * 1_000_003 + chunk_index)
    x = torch.randn((chunk, n_channels), device="cuda", generator=g, dtype=torch.float32)
    phase = torch.from_numpy(np.random.default_rng([seed, 0]).uniform(0, 2 * np.pi, n_channels)).cuda()
    t = (chunk_index * chunk + torch.arange(chunk, device="cuda", dtype=torch.float64)) / fs
    x += (sine_amp * torch.sin(2 * np.pi * sine_hz * t[:, None] + phase[None, :])).float()
    return x


def batch_streams(seed: int = 3, n_streams: int = 32, channels=(500, 10_000),
                  chunk=(200, 3000)) -> list[dict]:
    """Specs of the independent streams of the batching workload: a channel
    count per stream and a generator of per-push chunk lengths."""
    rng = np.random.default_rng(seed)
    Cs = rng.integers(channels[0], channels[1] + 1, n_streams)
    return [dict(n_channels=int(C), seed=int(seed * 1000 + i)) for i, C in enumerate(Cs)]


def batch_stream_data(spec: dict, n_samples: int) -> np.ndarray:
    """One stream of the batching workload: the small-workload recipe (1 kHz,
    N(0,1) noise plus 3 Ricker events of 20 Hz peak, amplitude 5, moveout
    0.5 ms/channel) at the stream's channel count and seed."""
    return noise_ricker_stream(spec["n_channels"], n_samples, 1000.0, 3, 5.0, (20.0, 20.0), (0.5, 0.5),
                               spec["seed"], pink=False, fixed_origin_channel=True)


def batch_chunk_lengths(seed: int, n_streams: int, n_pushes: int, chunk=(200, 3000)) -> np.ndarray:
    """[n_pushes][n_streams] chunk lengths, uniform in [chunk[0], chunk[1]]."""
    rng = np.random.default_rng([seed, 7])
    return rng.integers(chunk[0], chunk[1] + 1, (n_pushes, n_streams))


def windowed_sinc_bandpass(n_taps: int, f1: float, f2: float, fs: float) -> np.ndarray:
    """Linear-phase FIR bandpass taps (Hamming-windowed ideal bandpass), the
    long filter of the FFT-filtering workload; an input to the operators under
    test, not part of their arithmetic."""
    n = np.arange(n_taps) - (n_taps - 1) / 2.0
    ideal = 2 * f2 / fs * np.sinc(2 * f2 / fs * n) - 2 * f1 / fs * np.sinc(2 * f1 / fs * n)
    return ideal * np.hamming(n_taps)


def perturb_sos(sos: np.ndarray, rel: float, seed: int, max_tries: int = 1000) -> np.ndarray:
    """Multiply every coefficient except a0 by (1+u), u ~ U[-rel, rel]; a
    section is redrawn until its poles lie strictly inside the unit circle."""
    rng = np.random.default_rng(seed)
    out = np.array(sos, dtype=np.float64).copy()
    for s in range(out.shape[0]):
        for _ in range(max_tries):
            u = rng.uniform(-rel, rel, 6)
            u[3] = 0.0
            cand = sos[s] * (1.0 + u)
            if np.all(np.abs(np.roots(cand[3:])) < 1.0):
                out[s] = cand
                break
        else:
            raise RuntimeError("could not draw a stable perturbed section")
    return out
