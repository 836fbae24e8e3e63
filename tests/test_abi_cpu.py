"""C-ABI checks that need no GPU: the library loads, exports every function
include/filark.h declares, designs the Butterworth bandpass, and rejects
invalid configurations before touching CUDA."""
import ctypes as ct
import os
import re
import subprocess

import numpy as np
import pytest

import oracle_pins as P
from paper_2605_20132_gb300 import abi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "filark.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(filark_\w+)\s*\(", text)))


def test_library_loads_and_exports_every_declared_symbol():
    lib = abi.load()
    decl = declared_functions()
    assert decl, "no declarations parsed"
    assert sorted(abi.EXPORTED) == decl
    out = subprocess.run(["nm", "-D", "--defined-only", abi.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (filark_\w+)", out))
    missing = [f for f in decl if f not in exported]
    assert not missing, f"not exported: {missing}"
    for f in decl:
        assert getattr(lib, f) is not None
    assert abi.filark_abi_version() == abi.FILARK_ABI_VERSION


def test_config_struct_layout_matches_header():
    # the ctypes mirror must have the C layout (offsets of the 64-bit members)
    assert abi.filark_chain_config.fs.offset == 8
    assert abi.filark_chain_config.sos.offset == 24
    assert abi.filark_chain_config.max_chunk.offset == 56
    assert ct.sizeof(abi.filark_chain_config) == 64


@pytest.mark.parametrize("spec", [(4, 1.0, 50.0, 1000.0), (8, 0.5, 100.0, 1500.0), (8, 0.01, 1.0, 1500.0),
                                  (3, 10.0, 200.0, 1000.0), (5, 1.0, 400.0, 1000.0), (1, 5.0, 40.0, 200.0)])
def test_butter_design_matches_oracle_and_closed_form(oracle_mod, spec):
    """The library's designer and the oracle's are separate code; both must give
    the closed-form Butterworth magnitude, and the same sections."""
    st, sos = abi.filark_butter_bandpass_sos(*spec)
    assert st == abi.FILARK_OK
    ref = oracle_mod.butter_bandpass(*spec)
    assert np.max(np.abs(sos - ref)) < 1e-9
    N, f1, f2, fs = spec
    w = np.linspace(1e-3, np.pi - 1e-3, 257)
    # evaluating H in double next to poles 8e-6 from the unit circle costs ~1e-9
    bound = 1e-8 if f1 < 0.1 else 1e-9
    assert np.max(np.abs(np.abs(P.sos_response(sos, w)) ** 2 - P.butter_bp_mag2(w, N, f1, f2, fs))) < bound


@pytest.mark.parametrize("bad", [(0, 1.0, 2.0, 10.0), (4, 0.0, 2.0, 10.0), (4, 3.0, 2.0, 10.0), (4, 1.0, 5.0, 10.0)])
def test_butter_design_rejects_bad_arguments(bad):
    st, _ = abi.filark_butter_bandpass_sos(*bad)
    assert st == abi.FILARK_EINVAL
    assert abi.filark_last_error_string()


def _cfg(**kw):
    sos = kw.pop("sos", np.array([[1.0, 0.0, -1.0, 1.0, -1.2, 0.5]]))
    cfg = abi.filark_chain_config()
    cfg.abi_version = kw.pop("abi_version", abi.FILARK_ABI_VERSION)
    cfg.n_channels = kw.pop("n_channels", 16)
    cfg.fs = kw.pop("fs", 1000.0)
    cfg.n_sections = kw.pop("n_sections", sos.shape[0])
    keep = np.ascontiguousarray(sos, dtype=np.float64)
    cfg.sos = keep.ctypes.data_as(ct.POINTER(ct.c_double)) if keep.size else None
    cfg.spatial_width = kw.pop("spatial_width", 5)
    cfg.sta_len = kw.pop("sta_len", 10)
    cfg.lta_len = kw.pop("lta_len", 100)
    cfg.outputs = kw.pop("outputs", abi.FILARK_OUT_RATIO)
    cfg.precision = kw.pop("precision", abi.FILARK_PREC_AUTO)
    cfg.max_chunk = kw.pop("max_chunk", 1000)
    assert not kw
    return cfg, keep


@pytest.mark.parametrize("field,value,expect", [
    ("abi_version", 99, abi.FILARK_EINVAL),
    ("n_channels", 0, abi.FILARK_EINVAL),
    ("fs", -1.0, abi.FILARK_EINVAL),
    ("spatial_width", 4, abi.FILARK_EINVAL),
    ("spatial_width", 0, abi.FILARK_EINVAL),
    ("spatial_width", 35, abi.FILARK_ENOSYS),
    ("sta_len", 200, abi.FILARK_EINVAL),
    ("lta_len", 0, abi.FILARK_EINVAL),
    ("max_chunk", 0, abi.FILARK_EINVAL),
    ("outputs", 8, abi.FILARK_EINVAL),
    ("precision", 9, abi.FILARK_EINVAL),
    ("n_sections", 9, abi.FILARK_ENOSYS),
])
def test_create_rejects_invalid_config(field, value, expect):
    kw = {field: value}
    if field == "n_sections":
        kw["sos"] = np.tile([[1.0, 0.0, -1.0, 1.0, -1.2, 0.5]], (9, 1))
    cfg, _keep = _cfg(**kw)
    st, h = abi.filark_chain_create(cfg, 0)
    assert st == expect
    assert h is None
    assert abi.filark_last_error_string()


def test_create_rejects_ratio_without_detector():
    cfg, _keep = _cfg(sta_len=0, lta_len=0, outputs=abi.FILARK_OUT_RATIO)
    st, h = abi.filark_chain_create(cfg, 0)
    assert st == abi.FILARK_EINVAL and h is None


@pytest.mark.parametrize("row,expect", [
    ([1.0, 0.0, 0.0, 0.0, 0.1, 0.1], abi.FILARK_EINVAL),     # a0 == 0
    ([1.0, 0.0, 0.0, 1.0, -2.0, 1.0], abi.FILARK_EUNSTABLE),  # double pole at z = 1
    ([1.0, 0.0, 0.0, 1.0, 0.0, 1.01], abi.FILARK_EUNSTABLE),  # |p| > 1
    ([1.0, 0.0, 0.0, 2.0, 0.0, 2.2], abi.FILARK_EUNSTABLE),   # unstable after a0 scaling
    ([np.nan, 0.0, 0.0, 1.0, 0.0, 0.1], abi.FILARK_EINVAL),
])
def test_create_rejects_bad_sections(row, expect):
    cfg, _keep = _cfg(sos=np.array([row]))
    st, h = abi.filark_chain_create(cfg, 0)
    assert st == expect and h is None


def test_create_accepts_repeated_poles():
    """Two identical sections make the cascade matrix defective (no modal
    basis); the planner falls back to the dense carry instead of failing
    (without a GPU the call then stops at the device step)."""
    sec = [1.0, 0.0, -1.0, 1.0, -1.2, 0.5]
    cfg, _keep = _cfg(sos=np.array([sec, sec]))
    st, h = abi.filark_chain_create(cfg, 0)
    assert st in (abi.FILARK_OK, abi.FILARK_ECUDA)
    if h:
        abi.filark_chain_destroy(h)


def test_modal_request_with_repeated_poles_is_unsupported():
    sec = [1.0, 0.0, -1.0, 1.0, -1.2, 0.5]
    cfg, _keep = _cfg(sos=np.array([sec, sec]), precision=abi.FILARK_PREC_MODAL32)
    st, h = abi.filark_chain_create(cfg, 0)
    assert st == abi.FILARK_ENOSYS and h is None


def test_destroy_null_is_ok():
    assert abi.filark_chain_destroy(None) == abi.FILARK_OK


def test_chain_calls_reject_a_null_handle():
    """Every chain call that takes a handle reports FILARK_EINVAL for NULL
    before touching a device (lanes, join, geometry, status, state, resets)."""
    import ctypes as ct
    assert abi.filark_chain_set_lanes(None, 2) == abi.FILARK_EINVAL
    assert abi.filark_chain_join(None, None) == abi.FILARK_EINVAL
    assert abi.filark_chain_set_blocks_per_cta(None, 4) == abi.FILARK_EINVAL
    assert abi.filark_chain_sync_status(None, None) == abi.FILARK_EINVAL
    assert abi.filark_chain_host_sync(None, None) == abi.FILARK_EINVAL
    assert abi.filark_chain_reset_state(None, None) == abi.FILARK_EINVAL
    assert abi.filark_chain_get_state(None, None, ct.c_size_t(0), None) == abi.FILARK_EINVAL
    assert abi.filark_chain_set_state(None, None, 0, None) == abi.FILARK_EINVAL
    assert "NULL" in abi.filark_last_error_string()


# ---- differentiable bandpass: host-side sizes and argument checks ----------

def _piece(ckpt):
    import math
    return max(1, min(math.ceil(math.sqrt(2.0 * ckpt)), ckpt))


def _segment(C, N, ckpt):
    """Segment length the library uses: the requested interval, shortened when
    channels x segments are fewer than 2^17 threads, to no fewer than 128
    samples (or the requested interval, if that is shorter)."""
    nt0 = -(-N // ckpt) * C
    if nt0 >= 1 << 17:
        return ckpt
    f = -(-(1 << 17) // nt0)
    return max(min(ckpt, 128), -(-ckpt // f))


@pytest.mark.parametrize("S,C,N,ckpt", [(4, 2048, 30000, 3000), (1, 1, 1, 1), (8, 37, 777, 100), (4, 16, 2000, 5000),
                                        (4, 6000, 90000, 3000), (2, 100, 10**6, 1000)])
def test_iir_buffer_sizes(S, C, N, ckpt):
    """Checkpoints: 2S doubles per channel at every piece start of every
    segment; work: the adjoint states, one piece of section signals and the
    gradient partials per (segment, channel), and 6S x 8 chunk sums of the
    gradient reduction."""
    seg = _segment(C, N, ckpt)
    assert seg <= ckpt
    nseg = -(-N // seg)
    P = _piece(seg)
    npiece = -(-min(seg, N) // P)
    assert abi.filark_iir_ckpt_bytes(S, C, N, ckpt) == 8 * nseg * C * npiece * 2 * S
    assert abi.filark_iir_work_bytes(S, C, N, ckpt) == 8 * (nseg * C * (2 * S + P * S + 6 * S) + 6 * S * 8)


def test_iir_segments_fill_the_gpu_only_when_needed():
    """Large problems keep the requested checkpoint interval; the paper-scale
    differentiation workload (2048 x 30,000, every 3000) is cut finer."""
    assert _segment(6000, 90000, 3000) == 3000
    assert _segment(2048, 30000, 3000) == 429
    # pieces of ceil(sqrt(2 L)) samples: 78 for L = 3000 (39 pieces), 30 for 429 (15)
    assert abi.filark_iir_ckpt_bytes(4, 6000, 90000, 3000) == 8 * 30 * 6000 * 39 * 8
    assert abi.filark_iir_ckpt_bytes(4, 2048, 30000, 3000) == 8 * 70 * 2048 * 15 * 8


@pytest.mark.parametrize("args", [(0, 4, 10, 5), (9, 4, 10, 5), (4, 0, 10, 5), (4, 4, 0, 5), (4, 4, 10, 0)])
def test_iir_buffer_sizes_reject_invalid(args):
    assert abi.filark_iir_ckpt_bytes(*args) == 0
    assert abi.filark_iir_work_bytes(*args) == 0


def test_iir_checkpoint_memory_is_far_below_all_intermediates():
    """The differentiation workload keeps a fraction of the memory that storing
    every section signal in FP64 would take: under a fifth with the segments
    cut finer to fill the GPU, under a tenth at the requested interval."""
    S, C, N, ckpt = 4, 2048, 30000, 3000
    full = 8 * S * C * N
    kept = abi.filark_iir_ckpt_bytes(S, C, N, ckpt) + abi.filark_iir_work_bytes(S, C, N, ckpt)
    assert kept < full / 5
    S, C, N, ckpt = 4, 6000, 90000, 3000
    full = 8 * S * C * N
    kept = abi.filark_iir_ckpt_bytes(S, C, N, ckpt) + abi.filark_iir_work_bytes(S, C, N, ckpt)
    assert kept < full / 10


def test_iir_calls_reject_bad_arguments_before_any_launch():
    """Argument errors return FILARK_EINVAL without touching the device (the
    pointers below are never dereferenced)."""
    sos = np.array([[1.0, 0.0, -1.0, 1.0, -1.9, 0.95]])
    fake = 0x1000
    nb = abi.filark_iir_ckpt_bytes(1, 4, 10, 5)
    wb = abi.filark_iir_work_bytes(1, 4, 10, 5)
    bad_sos = np.array([[1.0, 0.0, -1.0, 0.0, -1.9, 0.95]])
    nan_sos = np.array([[1.0, np.nan, -1.0, 1.0, -1.9, 0.95]])
    for q in (bad_sos, nan_sos):
        assert abi.filark_iir_forward_ckpt(q, 1, 4, fake, 4, 10, fake, 4, 5, fake, nb, None) == abi.FILARK_EINVAL
    assert abi.filark_iir_forward_ckpt(sos, 1, 4, fake, 3, 10, fake, 4, 5, fake, nb, None) == abi.FILARK_EINVAL
    assert abi.filark_iir_forward_ckpt(sos, 1, 4, fake, 4, 10, fake, 4, 5, fake, nb - 8, None) == abi.FILARK_EINVAL
    assert abi.filark_iir_forward_ckpt(sos, 1, 4, None, 4, 10, fake, 4, 5, fake, nb, None) == abi.FILARK_EINVAL
    assert abi.filark_iir_forward_ckpt(sos, 1, 4, fake, 4, 10, fake, 4, 0, fake, nb, None) == abi.FILARK_EINVAL
    assert abi.filark_iir_backward(sos, 1, 4, fake, 4, 10, fake, 4, 5, fake, nb, fake, wb - 8, fake, 4, fake,
                                   None) == abi.FILARK_EINVAL
    assert abi.filark_iir_backward(sos, 1, 4, fake, 4, 10, fake, 4, 5, fake, nb, None, wb, fake, 4, fake,
                                   None) == abi.FILARK_EINVAL
    assert abi.filark_iir_backward(sos, 1, 4, fake, 4, 10, fake, 4, 5, fake, nb, fake, wb, fake, 4, fake + 4,
                                   None) == abi.FILARK_EINVAL
    assert "aligned" in abi.filark_last_error_string()
