"""ctypes binding of libfilark (include/filark.h), same names as the C-ABI.

Argument marshalling only: every step of the chain runs in the library's CUDA
kernels.  There is no CPU fallback -- if the library cannot be loaded, the
import of the functions below raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

from . import build as _build

FILARK_ABI_VERSION = 1

FILARK_OK = 0
FILARK_EINVAL = 1
FILARK_ENOMEM = 2
FILARK_ECUDA = 3
FILARK_EUNSTABLE = 4
FILARK_ETIMEOUT = 5
FILARK_ESTATE = 6
FILARK_ENOSYS = 7
STATUS_NAMES = {0: "FILARK_OK", 1: "FILARK_EINVAL", 2: "FILARK_ENOMEM", 3: "FILARK_ECUDA",
                4: "FILARK_EUNSTABLE", 5: "FILARK_ETIMEOUT", 6: "FILARK_ESTATE", 7: "FILARK_ENOSYS"}

FILARK_OUT_RATIO = 1
FILARK_OUT_BANDPASS = 2
FILARK_OUT_SPATIAL = 4

FILARK_PREC_AUTO = 0
FILARK_PREC_MODAL32 = 1
FILARK_PREC_DENSE64 = 2
FILARK_PREC_ALL32 = 3

FILARK_MAX_SECTIONS = 8
FILARK_MAX_SPATIAL_WIDTH = 33
FILARK_MAX_LANES = 4
FILARK_HOST_SLOTS = 3

# Every function the header declares (the tests check the library exports them).
EXPORTED = (
    "filark_chain_create", "filark_chain_push_chunk", "filark_chain_push_chunk_host",
    "filark_chain_push_host_async", "filark_chain_host_sync", "filark_chain_set_blocks_per_cta",
    "filark_chain_set_lanes", "filark_chain_join", "filark_chain_set_launch_samples", "filark_chain_tune",
    "filark_chain_get_tuning",
    "filark_chain_reset_state", "filark_chain_destroy", "filark_chain_get_state",
    "filark_chain_set_state", "filark_chain_sync_status", "filark_chain_get_info",
    "filark_butter_bandpass_sos", "filark_last_error_string", "filark_abi_version",
    "filark_chain_run_static", "filark_iir_ckpt_bytes", "filark_iir_work_bytes",
    "filark_iir_forward_ckpt", "filark_iir_backward",
    "filark_batch_create", "filark_batch_push", "filark_batch_tune", "filark_batch_set_launch",
    "filark_batch_set_blocks_per_cta",
    "filark_batch_reset_state", "filark_batch_sync_status", "filark_batch_get_info", "filark_batch_stream",
    "filark_batch_destroy",
    "filark_trigger_create", "filark_trigger_push", "filark_trigger_flush", "filark_trigger_reset",
    "filark_trigger_set_overlap", "filark_trigger_join", "filark_chain_push_triggers",
    "filark_trigger_destroy", "filark_events_work_bytes", "filark_events_merge",
    "filark_top_create", "filark_top_push", "filark_top_reset", "filark_top_destroy",
    "filark_fftfilt_create", "filark_fftfilt_push", "filark_fftfilt_reset", "filark_fftfilt_get_info",
    "filark_fftfilt_destroy",
    "filark_view_create", "filark_view_push", "filark_view_image", "filark_view_get_info", "filark_view_reset",
    "filark_view_destroy",
)

FILARK_VIEW_DROP, FILARK_VIEW_PEAK, FILARK_VIEW_LINEAR = 0, 1, 2

FILARK_TOP_FIR, FILARK_TOP_MEAN, FILARK_TOP_AGC, FILARK_TOP_EMA = 0, 1, 2, 3

FILARK_TRIGGER_OPEN = 1


class filark_chain_config(ct.Structure):
    _fields_ = [
        ("abi_version", ct.c_uint32),
        ("n_channels", ct.c_int32),
        ("fs", ct.c_double),
        ("n_sections", ct.c_int32),
        ("sos", ct.POINTER(ct.c_double)),
        ("spatial_width", ct.c_int32),
        ("sta_len", ct.c_int32),
        ("lta_len", ct.c_int32),
        ("outputs", ct.c_uint32),
        ("precision", ct.c_int32),
        ("max_chunk", ct.c_int64),
    ]


class filark_chain_info(ct.Structure):
    _fields_ = [
        ("precision", ct.c_int32),
        ("block_len", ct.c_int32),
        ("blocks_per_cta", ct.c_int32),
        ("tile_channels", ct.c_int32),
        ("halo", ct.c_int32),
        ("n_slots", ct.c_int32),
        ("modal_condition", ct.c_double),
        ("probe_error", ct.c_double),
        ("ring_len", ct.c_int64),
        ("device_bytes", ct.c_int64),
        ("samples", ct.c_int64),
    ]


class filark_chunk_desc(ct.Structure):
    _fields_ = [
        ("d_in", ct.c_void_p),
        ("ld_in", ct.c_int64),
        ("n_samples", ct.c_int64),
        ("d_ratio", ct.c_void_p),
        ("d_bandpass", ct.c_void_p),
        ("d_spatial", ct.c_void_p),
        ("ld_out", ct.c_int64),
    ]


class filark_chain_tuning(ct.Structure):
    _fields_ = [
        ("n_tuned", ct.c_int32),
        ("chosen", ct.c_int32),
        ("lanes", ct.c_int32 * 16),
        ("launch_samples", ct.c_int32 * 16),
        ("blocks_per_cta", ct.c_int32 * 16),
        ("ms_per_push", ct.c_double * 16),
    ]


class filark_batch_info(ct.Structure):
    _fields_ = [
        ("n_streams", ct.c_int32),
        ("cluster", ct.c_int32),
        ("n_clusters", ct.c_int32),
        ("use_graph", ct.c_int32),
        ("n_tiles", ct.c_int64),
        ("device_bytes", ct.c_int64),
        ("n_tuned", ct.c_int32),
        ("tune_cluster", ct.c_int32 * 16),
        ("tune_clusters", ct.c_int32 * 16),
        ("tune_ms", ct.c_double * 16),
        ("blocks_per_cta", ct.c_int32),
        ("tune_blocks", ct.c_int32 * 16),
        ("tune_stream_ms", ct.c_double),
    ]


class filark_trigger_record(ct.Structure):
    _fields_ = [("t_on", ct.c_int64), ("t_off", ct.c_int64), ("channel", ct.c_int32), ("flags", ct.c_int32)]


class filark_event(ct.Structure):
    _fields_ = [("t_on", ct.c_int64), ("t_off", ct.c_int64), ("c_min", ct.c_int32), ("c_max", ct.c_int32),
                ("n_triggers", ct.c_int32), ("flags", ct.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ct.CDLL:
    """Load libfilark.so (building it in-tree first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"libfilark not built: {path}")
            _build.build()
        lib = ct.CDLL(path)
        vp, i64, f_p = ct.c_void_p, ct.c_int64, ct.POINTER(ct.c_float)
        sig = {
            "filark_chain_create": ([ct.POINTER(filark_chain_config), ct.c_int, ct.POINTER(vp)], ct.c_int),
            "filark_chain_push_chunk": ([vp, vp, i64, i64, vp, vp, vp, i64, vp], ct.c_int),
            "filark_chain_push_chunk_host": ([vp, vp, i64, i64, vp, vp, vp, i64, vp], ct.c_int),
            "filark_chain_push_host_async": ([vp, vp, i64, i64, vp, vp, vp, i64, vp], ct.c_int),
            "filark_chain_host_sync": ([vp, vp], ct.c_int),
            "filark_chain_set_blocks_per_cta": ([vp, ct.c_int], ct.c_int),
            "filark_chain_set_lanes": ([vp, ct.c_int], ct.c_int),
            "filark_chain_set_launch_samples": ([vp, ct.c_int], ct.c_int),
            "filark_chain_tune": ([vp, vp, i64, i64, vp, vp, vp, i64, ct.c_int, vp], ct.c_int),
            "filark_chain_get_tuning": ([vp, ct.POINTER(filark_chain_tuning)], ct.c_int),
            "filark_chain_join": ([vp, vp], ct.c_int),
            "filark_chain_reset_state": ([vp, vp], ct.c_int),
            "filark_chain_destroy": ([vp], ct.c_int),
            "filark_chain_get_state": ([vp, vp, ct.POINTER(ct.c_size_t), vp], ct.c_int),
            "filark_chain_set_state": ([vp, vp, ct.c_size_t, vp], ct.c_int),
            "filark_chain_sync_status": ([vp, vp], ct.c_int),
            "filark_chain_get_info": ([vp, ct.POINTER(filark_chain_info)], ct.c_int),
            "filark_butter_bandpass_sos": ([ct.c_int, ct.c_double, ct.c_double, ct.c_double,
                                            ct.POINTER(ct.c_double)], ct.c_int),
            "filark_last_error_string": ([], ct.c_char_p),
            "filark_abi_version": ([], ct.c_uint32),
            "filark_chain_run_static": ([ct.POINTER(filark_chain_config), vp, i64, i64, vp, vp, vp, i64, vp],
                                        ct.c_int),
            "filark_batch_create": ([ct.POINTER(filark_chain_config), ct.c_int, ct.POINTER(ct.c_int32), ct.c_int,
                                     ct.POINTER(vp)], ct.c_int),
            "filark_batch_push": ([vp, ct.POINTER(filark_chunk_desc), vp], ct.c_int),
            "filark_batch_tune": ([vp, ct.POINTER(filark_chunk_desc), ct.c_int, vp], ct.c_int),
            "filark_batch_set_launch": ([vp, ct.c_int, ct.c_int, ct.c_int], ct.c_int),
            "filark_batch_set_blocks_per_cta": ([vp, ct.c_int], ct.c_int),
            "filark_batch_reset_state": ([vp, vp], ct.c_int),
            "filark_batch_sync_status": ([vp, vp], ct.c_int),
            "filark_batch_get_info": ([vp, ct.POINTER(filark_batch_info)], ct.c_int),
            "filark_batch_stream": ([vp, ct.c_int, ct.POINTER(vp)], ct.c_int),
            "filark_batch_destroy": ([vp], ct.c_int),
            "filark_trigger_create": ([ct.c_int, ct.c_double, ct.c_double, i64, ct.c_int, ct.POINTER(vp)],
                                      ct.c_int),
            "filark_trigger_push": ([vp, vp, i64, i64, vp, i64, vp, vp], ct.c_int),
            "filark_trigger_flush": ([vp, vp, i64, vp, vp], ct.c_int),
            "filark_trigger_reset": ([vp, vp], ct.c_int),
            "filark_trigger_set_overlap": ([vp, ct.c_int], ct.c_int),
            "filark_trigger_join": ([vp, vp], ct.c_int),
            "filark_chain_push_triggers": ([vp, vp, vp, i64, i64, vp, i64, vp, i64, vp, vp], ct.c_int),
            "filark_trigger_destroy": ([vp], ct.c_int),
            "filark_events_work_bytes": ([i64, ct.c_int], ct.c_size_t),
            "filark_events_merge": ([vp, i64, ct.c_int, vp, i64, vp, vp, ct.c_size_t, vp], ct.c_int),
            "filark_top_create": ([ct.c_int, ct.c_int, ct.c_int, vp, ct.c_double, i64, ct.c_int, ct.POINTER(vp)],
                                  ct.c_int),
            "filark_top_push": ([vp, vp, i64, i64, vp, i64, vp], ct.c_int),
            "filark_top_reset": ([vp, vp], ct.c_int),
            "filark_top_destroy": ([vp], ct.c_int),
            "filark_fftfilt_create": ([ct.c_int, ct.c_int, vp, ct.c_int, i64, ct.c_int, ct.POINTER(vp)], ct.c_int),
            "filark_fftfilt_push": ([vp, vp, i64, i64, vp, i64, vp], ct.c_int),
            "filark_fftfilt_reset": ([vp, vp], ct.c_int),
            "filark_fftfilt_get_info": ([vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)], ct.c_int),
            "filark_fftfilt_destroy": ([vp], ct.c_int),
            "filark_view_create": ([ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, vp, i64, ct.c_int,
                                    ct.POINTER(vp)], ct.c_int),
            "filark_view_push": ([vp, vp, i64, i64, vp], ct.c_int),
            "filark_view_image": ([vp, vp, i64, vp], ct.c_int),
            "filark_view_get_info": ([vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int)], ct.c_int),
            "filark_view_reset": ([vp, vp], ct.c_int),
            "filark_view_destroy": ([vp], ct.c_int),
            "filark_iir_ckpt_bytes": ([ct.c_int, ct.c_int, i64, i64], ct.c_size_t),
            "filark_iir_work_bytes": ([ct.c_int, ct.c_int, i64, i64], ct.c_size_t),
            "filark_iir_forward_ckpt": ([vp, ct.c_int, ct.c_int, vp, i64, i64, vp, i64, i64, vp, ct.c_size_t, vp],
                                        ct.c_int),
            "filark_iir_backward": ([vp, ct.c_int, ct.c_int, vp, i64, i64, vp, i64, i64, vp, ct.c_size_t, vp,
                                     ct.c_size_t, vp, i64, vp, vp], ct.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        del f_p
        _lib = lib
        return lib


class FilarkError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().filark_last_error_string().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != FILARK_OK:
        raise FilarkError(status, where)


# Thin wrappers with the C names: raw pointers and sizes in, status out.
def filark_chain_create(cfg: filark_chain_config, cuda_device: int) -> tuple[int, int | None]:
    h = ct.c_void_p()
    st = load().filark_chain_create(ct.byref(cfg), int(cuda_device), ct.byref(h))
    return st, h.value


def filark_chain_push_chunk(h, d_in, ld_in, n, d_ratio, d_bp, d_sp, ld_out, stream) -> int:
    return load().filark_chain_push_chunk(h, d_in, ld_in, n, d_ratio, d_bp, d_sp, ld_out, stream)


def filark_chain_push_chunk_host(h, h_in, ld_in, n, h_ratio, h_bp, h_sp, ld_out, stream) -> int:
    return load().filark_chain_push_chunk_host(h, h_in, ld_in, n, h_ratio, h_bp, h_sp, ld_out, stream)


def filark_chain_push_host_async(h, h_in, ld_in, n, h_ratio, h_bp, h_sp, ld_out, stream) -> int:
    return load().filark_chain_push_host_async(h, h_in, ld_in, n, h_ratio, h_bp, h_sp, ld_out, stream)


def filark_chain_host_sync(h, stream) -> int:
    return load().filark_chain_host_sync(h, stream)


def filark_chain_set_blocks_per_cta(h, blocks_per_cta: int) -> int:
    return load().filark_chain_set_blocks_per_cta(h, blocks_per_cta)


def filark_chain_set_launch_samples(h, samples: int) -> int:
    return load().filark_chain_set_launch_samples(h, samples)


def filark_chain_tune(h, d_in, ld_in: int, n_samples: int, d_ratio, d_bp, d_sp, ld_out: int, timed_pushes: int,
                      stream) -> int:
    return load().filark_chain_tune(h, d_in, ld_in, n_samples, d_ratio, d_bp, d_sp, ld_out, int(timed_pushes), stream)


def filark_chain_get_tuning(h) -> tuple[int, filark_chain_tuning]:
    out = filark_chain_tuning()
    st = load().filark_chain_get_tuning(h, ct.byref(out))
    return st, out


def filark_chain_set_lanes(h, lanes: int) -> int:
    return load().filark_chain_set_lanes(h, lanes)


def filark_chain_join(h, stream) -> int:
    return load().filark_chain_join(h, stream)


def filark_chain_reset_state(h, stream) -> int:
    return load().filark_chain_reset_state(h, stream)


def filark_chain_destroy(h) -> int:
    return load().filark_chain_destroy(h)


def filark_chain_get_state(h, buf, nbytes: ct.c_size_t, stream) -> int:
    return load().filark_chain_get_state(h, buf, ct.byref(nbytes), stream)


def filark_chain_set_state(h, buf, nbytes: int, stream) -> int:
    return load().filark_chain_set_state(h, buf, nbytes, stream)


def filark_chain_sync_status(h, stream) -> int:
    return load().filark_chain_sync_status(h, stream)


def filark_chain_get_info(h) -> tuple[int, filark_chain_info]:
    info = filark_chain_info()
    st = load().filark_chain_get_info(h, ct.byref(info))
    return st, info


def filark_butter_bandpass_sos(order: int, f1: float, f2: float, fs: float):
    import numpy as np
    sos = np.zeros((order, 6), dtype=np.float64)
    st = load().filark_butter_bandpass_sos(order, f1, f2, fs, sos.ctypes.data_as(ct.POINTER(ct.c_double)))
    return st, sos


def filark_chain_run_static(cfg: filark_chain_config, d_in, ld_in, n, d_ratio, d_bp, d_sp, ld_out, stream) -> int:
    return load().filark_chain_run_static(ct.byref(cfg), d_in, ld_in, n, d_ratio, d_bp, d_sp, ld_out, stream)


def filark_iir_ckpt_bytes(n_sections: int, n_channels: int, n_samples: int, ckpt_every: int) -> int:
    return int(load().filark_iir_ckpt_bytes(n_sections, n_channels, n_samples, ckpt_every))


def filark_iir_work_bytes(n_sections: int, n_channels: int, n_samples: int, ckpt_every: int) -> int:
    return int(load().filark_iir_work_bytes(n_sections, n_channels, n_samples, ckpt_every))


def filark_iir_forward_ckpt(sos_host, n_sections, n_channels, d_x, ld_x, n_samples, d_y, ld_y, ckpt_every,
                            d_ckpt, ckpt_size, stream) -> int:
    """sos_host: a C-contiguous float64 numpy array (n_sections, 6)."""
    return load().filark_iir_forward_ckpt(sos_host.ctypes.data, n_sections, n_channels, d_x, ld_x, n_samples, d_y,
                                          ld_y, ckpt_every, d_ckpt, ckpt_size, stream)


def filark_iir_backward(sos_host, n_sections, n_channels, d_x, ld_x, n_samples, d_gy, ld_gy, ckpt_every, d_ckpt,
                        ckpt_size, d_work, work_size, d_gx, ld_gx, d_gsos, stream) -> int:
    """sos_host: a C-contiguous float64 numpy array (n_sections, 6)."""
    return load().filark_iir_backward(sos_host.ctypes.data, n_sections, n_channels, d_x, ld_x, n_samples, d_gy,
                                      ld_gy, ckpt_every, d_ckpt, ckpt_size, d_work, work_size, d_gx, ld_gx, d_gsos,
                                      stream)


def filark_batch_create(cfg: filark_chain_config, n_channels, cuda_device: int) -> tuple[int, int | None]:
    arr = (ct.c_int32 * len(n_channels))(*[int(c) for c in n_channels])
    h = ct.c_void_p()
    st = load().filark_batch_create(ct.byref(cfg), len(n_channels), arr, int(cuda_device), ct.byref(h))
    return st, h.value


def filark_batch_push(b, descs, stream) -> int:
    """descs: a ctypes array of filark_chunk_desc, one per stream."""
    return load().filark_batch_push(b, descs, stream)


def filark_batch_tune(b, descs, timed_pushes: int, stream) -> int:
    return load().filark_batch_tune(b, descs, int(timed_pushes), stream)


def filark_batch_set_launch(b, cluster: int, n_clusters: int, use_graph: int) -> int:
    return load().filark_batch_set_launch(b, int(cluster), int(n_clusters), int(use_graph))


def filark_batch_set_blocks_per_cta(b, blocks: int) -> int:
    return load().filark_batch_set_blocks_per_cta(b, int(blocks))


def filark_batch_reset_state(b, stream) -> int:
    return load().filark_batch_reset_state(b, stream)


def filark_batch_sync_status(b, stream) -> int:
    return load().filark_batch_sync_status(b, stream)


def filark_batch_get_info(b) -> tuple[int, filark_batch_info]:
    info = filark_batch_info()
    st = load().filark_batch_get_info(b, ct.byref(info))
    return st, info


def filark_batch_stream(b, i: int) -> tuple[int, int | None]:
    h = ct.c_void_p()
    st = load().filark_batch_stream(b, int(i), ct.byref(h))
    return st, h.value


def filark_batch_destroy(b) -> int:
    return load().filark_batch_destroy(b)


def filark_trigger_create(n_channels: int, on: float, off: float, max_chunk: int, cuda_device: int):
    h = ct.c_void_p()
    st = load().filark_trigger_create(int(n_channels), float(on), float(off), int(max_chunk), int(cuda_device),
                                      ct.byref(h))
    return st, h.value


def filark_trigger_push(t, d_ratio, ld, n, d_records, capacity, d_count, stream) -> int:
    return load().filark_trigger_push(t, d_ratio, ld, n, d_records, capacity, d_count, stream)


def filark_trigger_flush(t, d_records, capacity, d_count, stream) -> int:
    return load().filark_trigger_flush(t, d_records, capacity, d_count, stream)


def filark_trigger_reset(t, stream) -> int:
    return load().filark_trigger_reset(t, stream)


def filark_trigger_set_overlap(t, overlap: int) -> int:
    return load().filark_trigger_set_overlap(t, int(overlap))


def filark_trigger_join(t, stream) -> int:
    return load().filark_trigger_join(t, stream)


def filark_chain_push_triggers(h, t, d_in, ld_in: int, n_samples: int, d_ratio, ld_out: int, d_records,
                               capacity: int, d_count, stream) -> int:
    return load().filark_chain_push_triggers(h, t, d_in, ld_in, n_samples, d_ratio, ld_out, d_records, capacity,
                                             d_count, stream)


def filark_trigger_destroy(t) -> int:
    return load().filark_trigger_destroy(t)


def filark_events_work_bytes(n_triggers: int, n_channels: int) -> int:
    return int(load().filark_events_work_bytes(int(n_triggers), int(n_channels)))


def filark_events_merge(d_triggers, n_triggers, n_channels, d_events, capacity, d_n_events, d_work, work_bytes,
                        stream) -> int:
    return load().filark_events_merge(d_triggers, n_triggers, n_channels, d_events, capacity, d_n_events, d_work,
                                      work_bytes, stream)


def filark_top_create(kind: int, n_channels: int, length: int, taps, alpha: float, max_chunk: int,
                      cuda_device: int):
    """taps: None or a C-contiguous float64 numpy array."""
    h = ct.c_void_p()
    st = load().filark_top_create(int(kind), int(n_channels), int(length), None if taps is None else taps.ctypes.data,
                                  float(alpha), int(max_chunk), int(cuda_device), ct.byref(h))
    return st, h.value


def filark_top_push(t, d_in, ld_in, n, d_out, ld_out, stream) -> int:
    return load().filark_top_push(t, d_in, ld_in, n, d_out, ld_out, stream)


def filark_top_reset(t, stream) -> int:
    return load().filark_top_reset(t, stream)


def filark_top_destroy(t) -> int:
    return load().filark_top_destroy(t)


def filark_fftfilt_create(n_channels: int, taps, block_len: int, max_chunk: int, cuda_device: int):
    """taps: a C-contiguous float64 numpy array."""
    h = ct.c_void_p()
    st = load().filark_fftfilt_create(int(n_channels), int(taps.shape[0]), taps.ctypes.data, int(block_len),
                                      int(max_chunk), int(cuda_device), ct.byref(h))
    return st, h.value


def filark_fftfilt_push(f, d_in, ld_in, n, d_out, ld_out, stream) -> int:
    return load().filark_fftfilt_push(f, d_in, ld_in, n, d_out, ld_out, stream)


def filark_fftfilt_reset(f, stream) -> int:
    return load().filark_fftfilt_reset(f, stream)


def filark_fftfilt_get_info(f):
    n, l = ct.c_int(), ct.c_int()
    st = load().filark_fftfilt_get_info(f, ct.byref(n), ct.byref(l))
    return st, n.value, l.value


def filark_fftfilt_destroy(f) -> int:
    return load().filark_fftfilt_destroy(f)


def filark_last_error_string() -> str:
    return load().filark_last_error_string().decode(errors="replace")


def filark_abi_version() -> int:
    return int(load().filark_abi_version())
