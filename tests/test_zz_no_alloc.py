"""The allocation-free entry point, filark_chain_run_static.

It exists for callers that must not call cudaMalloc: a real-time acquisition
thread whose latency budget forbids allocator calls (they can block and
synchronise the device), or a plugin inside a host application that hands out
all device memory from its own pool.  Instead of a chain object with its own
device buffers, the call keeps the chain's working memory in a fixed device
array inside the library, shared by every call.

The entry point runs the same kernel launches as a regular chain that gets the
whole recording in one push, so each call is compared with such a chain bit
for bit.  Consecutive calls use different recordings, channel counts and
windows, the first one loud and wide, so that state or history rows left in
the shared array by an earlier call would change a later result.  This file
is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

from gpu_helpers import TOL, normwise, ratio_err, run_oracle
from paper_2605_20132_gb300 import abi, synth

pytestmark = pytest.mark.gpu

ALL = abi.FILARK_OUT_RATIO | abi.FILARK_OUT_BANDPASS | abi.FILARK_OUT_SPATIAL


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def _config(C, sos, K, ns, nl, max_chunk, precision=abi.FILARK_PREC_AUTO, outputs=ALL):
    keep = np.ascontiguousarray(sos, dtype=np.float64)
    cfg = abi.filark_chain_config()
    cfg.abi_version = abi.FILARK_ABI_VERSION
    cfg.n_channels = C
    cfg.fs = 1000.0
    cfg.n_sections = keep.shape[0]
    cfg.sos = keep.ctypes.data_as(ct.POINTER(ct.c_double))
    cfg.spatial_width = K
    cfg.sta_len = ns
    cfg.lta_len = nl
    cfg.outputs = outputs
    cfg.precision = precision
    cfg.max_chunk = max_chunk
    return cfg, keep


def _chain_reference(cfg, xd):
    """The regular chain (own device buffers) with the recording in one push."""
    import torch
    lib = abi.load()
    N, C = xd.shape
    st, h = abi.filark_chain_create(cfg, torch.cuda.current_device())
    assert st == abi.FILARK_OK, abi.filark_last_error_string()
    ref = {k: torch.full((N, C), float("nan"), device="cuda") for k in ("ratio", "bp", "sp")}
    sh = torch.cuda.current_stream().cuda_stream
    st = lib.filark_chain_push_chunk(h, xd.data_ptr(), C, N, ref["ratio"].data_ptr(), ref["bp"].data_ptr(),
                                     ref["sp"].data_ptr(), C, sh)
    assert st == abi.FILARK_OK, abi.filark_last_error_string()
    assert lib.filark_chain_sync_status(h, sh) == abi.FILARK_OK
    abi.filark_chain_destroy(h)
    return {k: v.cpu().numpy() for k, v in ref.items()}


def _run_static(cfg, xd):
    import torch
    N, C = xd.shape
    out = {k: torch.full((N, C), float("nan"), device="cuda") for k in ("ratio", "bp", "sp")}
    sh = torch.cuda.current_stream().cuda_stream
    st = abi.filark_chain_run_static(cfg, xd.data_ptr(), C, N, out["ratio"].data_ptr(), out["bp"].data_ptr(),
                                     out["sp"].data_ptr(), C, sh)
    assert st == abi.FILARK_OK, abi.filark_last_error_string()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _case(C, N, seed, amp, sos, K, ns, nl, precision=abi.FILARK_PREC_AUTO):
    import torch
    x = synth.small_stream(C, N, seed=seed) * np.float32(amp)
    cfg, keep = _config(C, sos, K, ns, nl, N, precision)
    return x, torch.from_numpy(x).cuda(), cfg, keep


def test_static_calls_in_a_row_match_the_chain_bitwise(oracle_mod):
    """Three calls in a row on different recordings: a loud, wide one (200
    channels, 5,000 samples, long window 1,500), then a quiet, narrower one
    (64 channels, 3,000 samples, long window 1,000) whose history rows lie
    inside the region the first call filled, then the first one again.  Each
    call equals the regular chain bit for bit; the second is also held
    against the FP64 oracle."""
    st, sos = abi.filark_butter_bandpass_sos(4, 1.0, 50.0, 1000.0)
    assert st == abi.FILARK_OK
    cases = [_case(200, 5000, 31, 40.0, sos, 7, 60, 1500), _case(64, 3000, 32, 0.25, sos, 5, 50, 1000)]
    cases.append(cases[0])
    for i, (x, xd, cfg, keep) in enumerate(cases):
        got = _run_static(cfg, xd)
        ref = _chain_reference(cfg, xd)
        for k in ref:
            assert np.array_equal(got[k], ref[k], equal_nan=False), (i, k)
        if i == 1:
            o = run_oracle(oracle_mod, x, sos, K=5, ns=50, nl=1000)
            errs = {"bp": normwise(got["bp"], o["bp"]), "sp": normwise(got["sp"], o["sp"]),
                    "ratio": ratio_err(got["ratio"], o["ratio"])}
            assert all(e <= TOL for e in errs.values()), errs
    del cases


def test_static_dense_carry_and_short_recording(oracle_mod):
    """The dense carry (forced) and a recording shorter than one launch
    (700 samples: history ring of lta_len + 700 rows), each bitwise equal to
    the regular chain."""
    st, sos = abi.filark_butter_bandpass_sos(4, 1.0, 50.0, 1000.0)
    for C, N, prec, seed in [(96, 2600, abi.FILARK_PREC_DENSE64, 33), (80, 700, abi.FILARK_PREC_AUTO, 34)]:
        x, xd, cfg, keep = _case(C, N, seed, 3.0, sos, 5, 40, 500, prec)
        got = _run_static(cfg, xd)
        ref = _chain_reference(cfg, xd)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (prec, N, k)
        del keep


def test_static_argument_checks():
    """Zero samples do nothing; an output that overlaps the input or another
    output, or that the output mask does not enable, is rejected; a
    recording whose working memory exceeds the static array is rejected."""
    import torch
    st, sos = abi.filark_butter_bandpass_sos(4, 1.0, 50.0, 1000.0)
    cfg, keep = _config(16, sos, 3, 5, 50, 100)
    x = torch.zeros((100, 16), device="cuda")
    a = torch.full((100, 16), float("nan"), device="cuda")
    b = torch.full((100, 16), float("nan"), device="cuda")
    run = abi.filark_chain_run_static
    assert run(cfg, x.data_ptr(), 16, 0, a.data_ptr(), None, None, 16, None) == abi.FILARK_OK
    torch.cuda.synchronize()
    assert torch.isnan(a).all()
    assert run(cfg, x.data_ptr(), 16, 100, x.data_ptr(), None, None, 16, None) == abi.FILARK_EINVAL
    assert run(cfg, x.data_ptr(), 16, 100, a.data_ptr(), a[50].data_ptr(), None, 16, None) == abi.FILARK_EINVAL
    assert run(cfg, x.data_ptr(), 16, 100, a.data_ptr(), None, None, 15, None) == abi.FILARK_EINVAL
    cfg_r, keep_r = _config(16, sos, 3, 5, 50, 100, outputs=abi.FILARK_OUT_RATIO)
    assert run(cfg_r, x.data_ptr(), 16, 100, a.data_ptr(), b.data_ptr(), None, 16, None) == abi.FILARK_EINVAL
    assert "not enabled" in abi.filark_last_error_string()
    assert run(cfg_r, x.data_ptr(), 16, 100, a.data_ptr(), None, None, 16, None) == abi.FILARK_OK
    torch.cuda.synchronize()
    assert torch.isfinite(a).all()
    # 6000 channels with a 3000-sample long window need ~120 MB of history
    big, keep_b = _config(6000, sos, 9, 150, 3000, 1500)
    xb = torch.zeros((1500, 6000), device="cuda")
    rb = torch.zeros((1500, 6000), device="cuda")
    assert run(big, xb.data_ptr(), 6000, 1500, rb.data_ptr(), None, None, 6000, None) == abi.FILARK_EINVAL
    assert "static" in abi.filark_last_error_string()
    del keep, keep_r, keep_b
