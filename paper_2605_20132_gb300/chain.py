"""Convenience wrapper of the filark C-ABI for PyTorch users.

PyTorch supplies device memory and streams; each call marshals pointers and
sizes and goes straight to libfilark, where every step runs in CUDA kernels.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import abi


def butter_bandpass(order: int, f1: float, f2: float, fs: float) -> np.ndarray:
    """Butterworth bandpass SOS designed by the library (host code)."""
    st, sos = abi.filark_butter_bandpass_sos(order, f1, f2, fs)
    abi.check(st, "filark_butter_bandpass_sos")
    return sos


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


class Chain:
    """A stateful chain on one GPU: SOS bandpass -> spatial mean -> STA/LTA."""

    def __init__(self, n_channels: int, sos: np.ndarray | None, fs: float = 1.0,
                 spatial_width: int = 1, sta_len: int = 0, lta_len: int = 0,
                 outputs: int = abi.FILARK_OUT_RATIO, precision: int = abi.FILARK_PREC_AUTO,
                 max_chunk: int = 4096, device: int = 0):
        abi.load()
        self._sos = np.ascontiguousarray(np.zeros((0, 6)) if sos is None else sos, dtype=np.float64)
        cfg = abi.filark_chain_config()
        cfg.abi_version = abi.FILARK_ABI_VERSION
        cfg.n_channels = int(n_channels)
        cfg.fs = float(fs)
        cfg.n_sections = int(self._sos.shape[0])
        cfg.sos = self._sos.ctypes.data_as(ct.POINTER(ct.c_double)) if self._sos.size else None
        cfg.spatial_width = int(spatial_width)
        cfg.sta_len = int(sta_len)
        cfg.lta_len = int(lta_len)
        cfg.outputs = int(outputs)
        cfg.precision = int(precision)
        cfg.max_chunk = int(max_chunk)
        self.cfg = cfg
        self.n_channels = int(n_channels)
        self.device = int(device)
        st, h = abi.filark_chain_create(cfg, self.device)
        abi.check(st, "filark_chain_create")
        self._h = h

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "_h", None):
            abi.check(abi.filark_chain_destroy(self._h), "filark_chain_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    # -- streaming
    def push(self, x, ratio=None, bandpass=None, spatial=None, stream=None) -> None:
        """Enqueue one push.  x: CUDA float32 [T][ld_in] (row stride >= C);
        outputs: CUDA float32 [T][ld_out] tensors or None."""
        T = int(x.shape[0])
        ld_in = int(x.stride(0)) if T > 0 else self.n_channels
        outs = [o for o in (ratio, bandpass, spatial) if o is not None]
        ld_out = int(outs[0].stride(0)) if outs else self.n_channels
        st = abi.filark_chain_push_chunk(self._h, _ptr(x), ld_in, T, _ptr(ratio), _ptr(bandpass),
                                         _ptr(spatial), ld_out, _stream_handle(stream))
        abi.check(st, "filark_chain_push_chunk")

    def push_triggers(self, x, ratio, trigger, stream=None) -> None:
        """Push x with the ratio output and the triggers of `trigger` (a
        Trigger) fused into the detector (filark_chain_push_triggers)."""
        T = int(x.shape[0])
        st = abi.filark_chain_push_triggers(self._h, trigger._h, _ptr(x), int(x.stride(0)) if T else self.n_channels,
                                            T, _ptr(ratio), int(ratio.stride(0)) if T else self.n_channels,
                                            _ptr(trigger.records), trigger.capacity, _ptr(trigger.count),
                                            _stream_handle(stream))
        abi.check(st, "filark_chain_push_triggers")

    def push_host(self, x: np.ndarray, ratio: np.ndarray | None = None,
                  bandpass: np.ndarray | None = None, spatial: np.ndarray | None = None,
                  stream=None) -> None:
        """Synchronous push from host arrays (pinned memory is fastest)."""
        T = int(x.shape[0])
        ld_in = int(x.strides[0] // 4) if T > 0 else self.n_channels
        outs = [o for o in (ratio, bandpass, spatial) if o is not None]
        ld_out = int(outs[0].strides[0] // 4) if outs else self.n_channels
        p = lambda a: None if a is None else a.ctypes.data
        st = abi.filark_chain_push_chunk_host(self._h, p(x), ld_in, T, p(ratio), p(bandpass), p(spatial),
                                              ld_out, _stream_handle(stream))
        abi.check(st, "filark_chain_push_chunk_host")

    def push_host_async(self, x: np.ndarray, ratio: np.ndarray | None = None,
                        bandpass: np.ndarray | None = None, spatial: np.ndarray | None = None,
                        stream=None) -> None:
        """Pipelined push from host arrays (page-locked for overlap): enqueues
        and returns; the arrays must stay alive and unmodified, and the
        outputs are valid, only after host_sync()."""
        T = int(x.shape[0])
        ld_in = int(x.strides[0] // 4) if T > 0 else self.n_channels
        outs = [o for o in (ratio, bandpass, spatial) if o is not None]
        ld_out = int(outs[0].strides[0] // 4) if outs else self.n_channels
        p = lambda a: None if a is None else a.ctypes.data
        st = abi.filark_chain_push_host_async(self._h, p(x), ld_in, T, p(ratio), p(bandpass), p(spatial),
                                              ld_out, _stream_handle(stream))
        abi.check(st, "filark_chain_push_host_async")

    def set_blocks_per_cta(self, blocks_per_cta: int) -> None:
        """0: planned per launch (default); 1..8: fixed (see the C header)."""
        abi.check(abi.filark_chain_set_blocks_per_cta(self._h, int(blocks_per_cta)),
                  "filark_chain_set_blocks_per_cta")

    def set_launch_samples(self, samples: int) -> None:
        abi.check(abi.filark_chain_set_launch_samples(self._h, int(samples)), "filark_chain_set_launch_samples")

    def tune(self, x, ratio=None, bandpass=None, spatial=None, timed_pushes: int = 5, stream=None) -> dict:
        """Time the launch geometries on pushes of x (outputs overwritten), keep
        the fastest, reset the state; returns the candidates and the choice."""
        T = int(x.shape[0])
        outs = [o for o in (ratio, bandpass, spatial) if o is not None]
        ld_out = int(outs[0].stride(0)) if outs else self.n_channels
        abi.check(abi.filark_chain_tune(self._h, _ptr(x), int(x.stride(0)), T, _ptr(ratio), _ptr(bandpass),
                                        _ptr(spatial), ld_out, timed_pushes, _stream_handle(stream)),
                  "filark_chain_tune")
        st, t = abi.filark_chain_get_tuning(self._h)
        abi.check(st, "filark_chain_get_tuning")
        rows = [dict(lanes=t.lanes[i], launch_samples=t.launch_samples[i], blocks_per_cta=t.blocks_per_cta[i],
                     ms_per_push=t.ms_per_push[i]) for i in range(t.n_tuned)]
        return {"candidates": rows, "chosen": rows[t.chosen] if t.chosen >= 0 else None}

    def set_lanes(self, lanes: int) -> None:
        """1 (default): every push completes on its stream.  2..FILARK_MAX_LANES:
        channel-tile groups on internal streams; a push's outputs are valid
        only after join(stream) / sync() (see the C header)."""
        abi.check(abi.filark_chain_set_lanes(self._h, int(lanes)), "filark_chain_set_lanes")

    def join(self, stream=None) -> None:
        """Make `stream` (default: the current stream) wait for the lanes."""
        abi.check(abi.filark_chain_join(self._h, _stream_handle(stream)), "filark_chain_join")

    def host_sync(self, stream=None) -> None:
        abi.check(abi.filark_chain_host_sync(self._h, _stream_handle(stream)), "filark_chain_host_sync")

    def reset(self, stream=None) -> None:
        abi.check(abi.filark_chain_reset_state(self._h, _stream_handle(stream)), "filark_chain_reset_state")

    def sync(self, stream=None) -> None:
        abi.check(abi.filark_chain_sync_status(self._h, _stream_handle(stream)), "filark_chain_sync_status")

    # -- checkpoint
    def get_state(self, stream=None) -> bytes:
        n = ct.c_size_t(0)
        abi.check(abi.filark_chain_get_state(self._h, None, n, _stream_handle(stream)), "filark_chain_get_state")
        buf = ct.create_string_buffer(n.value)
        abi.check(abi.filark_chain_get_state(self._h, buf, n, _stream_handle(stream)), "filark_chain_get_state")
        return buf.raw[: n.value]

    def set_state(self, state: bytes, stream=None) -> None:
        buf = ct.create_string_buffer(state, len(state))
        abi.check(abi.filark_chain_set_state(self._h, buf, len(state), _stream_handle(stream)),
                  "filark_chain_set_state")

    def info(self) -> dict:
        st, inf = abi.filark_chain_get_info(self._h)
        abi.check(st, "filark_chain_get_info")
        return {k: getattr(inf, k) for k, _ in inf._fields_}


class Batch:
    """Many independent chains with one configuration (own channel counts,
    chunk lengths and state), pushed together by one persistent launch."""

    def __init__(self, n_channels, sos: np.ndarray | None, fs: float = 1.0, spatial_width: int = 1,
                 sta_len: int = 0, lta_len: int = 0, outputs: int = abi.FILARK_OUT_RATIO,
                 precision: int = abi.FILARK_PREC_AUTO, max_chunk: int = 4096, device: int = 0):
        abi.load()
        self._sos = np.ascontiguousarray(np.zeros((0, 6)) if sos is None else sos, dtype=np.float64)
        cfg = abi.filark_chain_config()
        cfg.abi_version = abi.FILARK_ABI_VERSION
        cfg.n_channels = 1
        cfg.fs = float(fs)
        cfg.n_sections = int(self._sos.shape[0])
        cfg.sos = self._sos.ctypes.data_as(ct.POINTER(ct.c_double)) if self._sos.size else None
        cfg.spatial_width = int(spatial_width)
        cfg.sta_len = int(sta_len)
        cfg.lta_len = int(lta_len)
        cfg.outputs = int(outputs)
        cfg.precision = int(precision)
        cfg.max_chunk = int(max_chunk)
        self.cfg = cfg
        self.n_channels = [int(c) for c in n_channels]
        self.device = int(device)
        st, h = abi.filark_batch_create(cfg, self.n_channels, self.device)
        abi.check(st, "filark_batch_create")
        self._h = h
        self._descs = (abi.filark_chunk_desc * len(self.n_channels))()

    def close(self) -> None:
        if getattr(self, "_h", None):
            abi.check(abi.filark_batch_destroy(self._h), "filark_batch_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _fill(self, xs, ratios=None, bandpasses=None, spatials=None):
        n = len(self.n_channels)
        ratios = ratios or [None] * n
        bandpasses = bandpasses or [None] * n
        spatials = spatials or [None] * n
        for i in range(n):
            d = self._descs[i]
            x = xs[i]
            T = 0 if x is None else int(x.shape[0])
            d.n_samples = T
            d.d_in = _ptr(x) if T else None
            d.ld_in = int(x.stride(0)) if T else self.n_channels[i]
            outs = [o for o in (ratios[i], bandpasses[i], spatials[i]) if o is not None]
            d.ld_out = int(outs[0].stride(0)) if (outs and T) else self.n_channels[i]
            d.d_ratio = _ptr(ratios[i]) if T else None
            d.d_bandpass = _ptr(bandpasses[i]) if T else None
            d.d_spatial = _ptr(spatials[i]) if T else None
        return self._descs

    def push(self, xs, ratios=None, bandpasses=None, spatials=None, stream=None) -> None:
        """xs[i]: CUDA float32 [T_i][ld] (or None for no samples); outputs alike."""
        d = self._fill(xs, ratios, bandpasses, spatials)
        abi.check(abi.filark_batch_push(self._h, d, _stream_handle(stream)), "filark_batch_push")

    def tune(self, xs, ratios=None, bandpasses=None, spatials=None, timed_pushes: int = 5, stream=None) -> dict:
        d = self._fill(xs, ratios, bandpasses, spatials)
        abi.check(abi.filark_batch_tune(self._h, d, timed_pushes, _stream_handle(stream)), "filark_batch_tune")
        return self.info()

    def set_launch(self, cluster: int, n_clusters: int = 0, use_graph: bool = True) -> None:
        abi.check(abi.filark_batch_set_launch(self._h, cluster, n_clusters, int(use_graph)),
                  "filark_batch_set_launch")

    def set_blocks_per_cta(self, blocks: int) -> None:
        abi.check(abi.filark_batch_set_blocks_per_cta(self._h, blocks), "filark_batch_set_blocks_per_cta")

    def reset(self, stream=None) -> None:
        abi.check(abi.filark_batch_reset_state(self._h, _stream_handle(stream)), "filark_batch_reset_state")

    def sync(self, stream=None) -> None:
        abi.check(abi.filark_batch_sync_status(self._h, _stream_handle(stream)), "filark_batch_sync_status")

    def info(self) -> dict:
        st, inf = abi.filark_batch_get_info(self._h)
        abi.check(st, "filark_batch_get_info")
        out = {k: getattr(inf, k) for k, _ in inf._fields_ if not k.startswith("tune_")}
        out["stream_ms"] = inf.tune_stream_ms
        n = inf.n_tuned
        out["tuned"] = [dict(cluster=inf.tune_cluster[i], n_clusters=inf.tune_clusters[i],
                             blocks_per_cta=inf.tune_blocks[i], ms=inf.tune_ms[i]) for i in range(n)]
        return out


class Trigger:
    """Per-channel hysteresis triggers on a ratio stream (device), with the
    triggers collected in a device list of `capacity` records."""

    RECORD_WORDS = 3  # int64 words of one filark_trigger_record (24 bytes)

    def __init__(self, n_channels: int, on: float, off: float, max_chunk: int = 4096, capacity: int = 1 << 20,
                 device: int = 0):
        import torch
        abi.load()
        self.n_channels = int(n_channels)
        self.capacity = int(capacity)
        st, h = abi.filark_trigger_create(n_channels, on, off, max_chunk, device)
        abi.check(st, "filark_trigger_create")
        self._h = h
        dev = torch.device("cuda", device)
        self.records = torch.zeros((self.capacity, self.RECORD_WORDS), dtype=torch.int64, device=dev)
        self.count = torch.zeros(1, dtype=torch.int64, device=dev)

    def close(self) -> None:
        if getattr(self, "_h", None):
            abi.check(abi.filark_trigger_destroy(self._h), "filark_trigger_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, ratio, stream=None) -> None:
        T = int(ratio.shape[0])
        ld = int(ratio.stride(0)) if T else self.n_channels
        st = abi.filark_trigger_push(self._h, _ptr(ratio) if T else None, ld, T, _ptr(self.records), self.capacity,
                                     _ptr(self.count), _stream_handle(stream))
        abi.check(st, "filark_trigger_push")

    def flush(self, stream=None) -> None:
        abi.check(abi.filark_trigger_flush(self._h, _ptr(self.records), self.capacity, _ptr(self.count),
                                           _stream_handle(stream)), "filark_trigger_flush")

    def reset(self, stream=None) -> None:
        abi.check(abi.filark_trigger_reset(self._h, _stream_handle(stream)), "filark_trigger_reset")
        self.count.zero_()

    def set_overlap(self, overlap: bool) -> None:
        abi.check(abi.filark_trigger_set_overlap(self._h, int(bool(overlap))), "filark_trigger_set_overlap")

    def join(self, stream=None) -> None:
        abi.check(abi.filark_trigger_join(self._h, _stream_handle(stream)), "filark_trigger_join")

    def triggers(self) -> np.ndarray:
        """[k][3] = (channel, t_on, t_off, flags folded out) as numpy int64."""
        self.join()
        n = int(self.count.item())
        if n > self.capacity:
            raise RuntimeError(f"{n} triggers exceeded the capacity {self.capacity}")
        raw = self.records[:n].cpu().numpy()
        t_on, t_off = raw[:, 0], raw[:, 1]
        chan = (raw[:, 2] & 0xFFFFFFFF).astype(np.int64)
        flags = (raw[:, 2] >> 32).astype(np.int64)
        return np.stack([chan, t_on, t_off, flags], axis=1)


def merge_events(records_dev, n_triggers: int, n_channels: int, capacity: int | None = None, stream=None):
    """Events of the first n_triggers records of a device record tensor (as
    kept by Trigger): numpy rows (t_on, t_off, c_min, c_max, n_triggers,
    flags), in the library's (unspecified) order."""
    import torch
    dev = records_dev.device
    cap = int(capacity or max(1, n_triggers))
    ev = torch.zeros((cap, 4), dtype=torch.int64, device=dev)
    n_ev = torch.zeros(1, dtype=torch.int64, device=dev)
    wb = abi.filark_events_work_bytes(n_triggers, n_channels)
    work = torch.empty(wb + 256, dtype=torch.uint8, device=dev)
    wp = (work.data_ptr() + 255) // 256 * 256
    st = abi.filark_events_merge(_ptr(records_dev), n_triggers, n_channels, _ptr(ev), cap, _ptr(n_ev), wp, wb,
                                 _stream_handle(stream))
    abi.check(st, "filark_events_merge")
    m = int(n_ev.item())
    raw = ev[:min(m, cap)].cpu().numpy()
    out = np.stack([raw[:, 0], raw[:, 1], raw[:, 2] & 0xFFFFFFFF, raw[:, 2] >> 32,
                    raw[:, 3] & 0xFFFFFFFF, raw[:, 3] >> 32], axis=1).astype(np.int64)
    return out, m


class TemporalOp:
    """A stateful temporal operator on device streams: FIR, running mean,
    running AGC or EMA gain equalisation (include/filark.h, filark_top_*)."""

    def __init__(self, kind: int, n_channels: int, length: int = 1, taps=None, alpha: float = 0.0,
                 max_chunk: int = 4096, device: int = 0):
        abi.load()
        self._taps = None if taps is None else np.ascontiguousarray(taps, dtype=np.float64)
        st, h = abi.filark_top_create(kind, n_channels, length, self._taps, alpha, max_chunk, device)
        abi.check(st, "filark_top_create")
        self._h = h
        self.n_channels = int(n_channels)

    def close(self) -> None:
        if getattr(self, "_h", None):
            abi.check(abi.filark_top_destroy(self._h), "filark_top_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, x, out, stream=None) -> None:
        T = int(x.shape[0])
        ld_in = int(x.stride(0)) if T else self.n_channels
        ld_out = int(out.stride(0)) if T else self.n_channels
        abi.check(abi.filark_top_push(self._h, _ptr(x) if T else None, ld_in, T, _ptr(out) if T else None, ld_out,
                                      _stream_handle(stream)), "filark_top_push")

    def reset(self, stream=None) -> None:
        abi.check(abi.filark_top_reset(self._h, _stream_handle(stream)), "filark_top_reset")


class FFTFilter:
    """Overlap-add FFT filtering with a long FIR (filark_fftfilt_*)."""

    def __init__(self, n_channels: int, taps, block_len: int = 0, max_chunk: int = 4096, device: int = 0):
        abi.load()
        self._taps = np.ascontiguousarray(taps, dtype=np.float64)
        st, h = abi.filark_fftfilt_create(n_channels, self._taps, block_len, max_chunk, device)
        abi.check(st, "filark_fftfilt_create")
        self._h = h
        self.n_channels = int(n_channels)
        st, self.fft_len, self.block_len = abi.filark_fftfilt_get_info(h)
        abi.check(st, "filark_fftfilt_get_info")

    def close(self) -> None:
        if getattr(self, "_h", None):
            abi.check(abi.filark_fftfilt_destroy(self._h), "filark_fftfilt_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, x, out, stream=None) -> None:
        T = int(x.shape[0])
        ld_in = int(x.stride(0)) if T else self.n_channels
        ld_out = int(out.stride(0)) if T else self.n_channels
        abi.check(abi.filark_fftfilt_push(self._h, _ptr(x) if T else None, ld_in, T, _ptr(out) if T else None,
                                          ld_out, _stream_handle(stream)), "filark_fftfilt_push")

    def reset(self, stream=None) -> None:
        abi.check(abi.filark_fftfilt_reset(self._h, _stream_handle(stream)), "filark_fftfilt_reset")


class View:
    """Headless streaming display buffer (filark_view_*)."""

    def __init__(self, n_channels: int, channels_per_row: int, samples_per_column: int, width: int, mode: int,
                 sos: np.ndarray | None = None, max_chunk: int = 4096, device: int = 0):
        import torch
        abi.load()
        self._sos = None if sos is None else np.ascontiguousarray(sos, dtype=np.float64)
        h = ct.c_void_p()
        st = abi.load().filark_view_create(int(n_channels), int(channels_per_row), int(samples_per_column),
                                           int(width), int(mode), 0 if self._sos is None else self._sos.shape[0],
                                           None if self._sos is None else self._sos.ctypes.data, int(max_chunk),
                                           int(device), ct.byref(h))
        abi.check(st, "filark_view_create")
        self._h = h.value
        self.n_channels, self.width = int(n_channels), int(width)
        self.rows = -(-int(n_channels) // int(channels_per_row))
        self.device = torch.device("cuda", device)

    def close(self) -> None:
        if getattr(self, "_h", None):
            abi.check(abi.load().filark_view_destroy(self._h), "filark_view_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, x, stream=None) -> None:
        T = int(x.shape[0])
        ld = int(x.stride(0)) if T else self.n_channels
        abi.check(abi.load().filark_view_push(self._h, _ptr(x) if T else None, ld, T, _stream_handle(stream)),
                  "filark_view_push")

    def image(self, stream=None):
        import torch
        img = torch.empty((self.rows, self.width), dtype=torch.float32, device=self.device)
        abi.check(abi.load().filark_view_image(self._h, _ptr(img), self.width, _stream_handle(stream)),
                  "filark_view_image")
        return img

    def info(self) -> dict:
        r, c, o = ct.c_int(), ct.c_int64(), ct.c_int()
        abi.check(abi.load().filark_view_get_info(self._h, ct.byref(r), ct.byref(c), ct.byref(o)),
                  "filark_view_get_info")
        return {"rows": r.value, "columns": c.value, "ring_offset": o.value}

    def reset(self, stream=None) -> None:
        abi.check(abi.load().filark_view_reset(self._h, _stream_handle(stream)), "filark_view_reset")
