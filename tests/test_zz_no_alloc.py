"""The allocation-free entry point, filark_chain_run_static.

It exists for callers that must not call cudaMalloc: a real-time acquisition
thread whose latency budget forbids allocator calls (they can block and
synchronise the device), or a plugin inside a host application that hands out
all device memory from its own pool.  Instead of a chain object with its own
device buffers, the call keeps the chain's working memory in a fixed device
array inside the library.

The test runs it twice in a row on one recording and checks both results
against the regular chain (filark_chain_create + pushes) within the tolerance
the other GPU tests use; the second call shows that the shared array is
cleared between calls.  This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

from gpu_helpers import TOL, normwise, ratio_err
from paper_2605_20132_gb300 import abi, synth

pytestmark = pytest.mark.gpu


def _config(C, sos, K, ns, nl, max_chunk):
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
    cfg.outputs = abi.FILARK_OUT_RATIO | abi.FILARK_OUT_BANDPASS | abi.FILARK_OUT_SPATIAL
    cfg.precision = abi.FILARK_PREC_AUTO
    cfg.max_chunk = max_chunk
    return cfg, keep


def test_static_entry_point_matches_chain():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = abi.load()
    C, N, K, ns, nl = 64, 3000, 5, 50, 1000
    st, sos = abi.filark_butter_bandpass_sos(4, 1.0, 50.0, 1000.0)
    assert st == abi.FILARK_OK
    x = torch.from_numpy(synth.small_stream(C, N, seed=21)).cuda()

    # reference: the regular chain, pushed in three chunks
    cfg, keep = _config(C, sos, K, ns, nl, 1000)
    st, h = abi.filark_chain_create(cfg, torch.cuda.current_device())
    assert st == abi.FILARK_OK, abi.filark_last_error_string()
    ref = {k: torch.empty((N, C), device="cuda") for k in ("ratio", "bp", "sp")}
    sh = torch.cuda.current_stream().cuda_stream
    for t in range(0, N, 1000):
        st = lib.filark_chain_push_chunk(h, x[t].data_ptr(), C, 1000, ref["ratio"][t].data_ptr(),
                                         ref["bp"][t].data_ptr(), ref["sp"][t].data_ptr(), C, sh)
        assert st == abi.FILARK_OK, abi.filark_last_error_string()
    assert lib.filark_chain_sync_status(h, sh) == abi.FILARK_OK
    abi.filark_chain_destroy(h)
    ref = {k: v.cpu().numpy().astype(np.float64) for k, v in ref.items()}

    for call in range(2):
        out = {k: torch.full((N, C), float("nan"), device="cuda") for k in ("ratio", "bp", "sp")}
        st = abi.filark_chain_run_static(cfg, x.data_ptr(), C, N, out["ratio"].data_ptr(), out["bp"].data_ptr(),
                                         out["sp"].data_ptr(), C, sh)
        assert st == abi.FILARK_OK, abi.filark_last_error_string()
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
        errs = {"bp": normwise(got["bp"], ref["bp"]), "sp": normwise(got["sp"], ref["sp"]),
                "ratio": ratio_err(got["ratio"], ref["ratio"])}
        assert all(e <= TOL for e in errs.values()), (call, errs)
    del keep


def test_static_entry_point_rejects_oversized_recording():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # 6000 channels with a 3000-sample long window need ~120 MB of history
    st, sos = abi.filark_butter_bandpass_sos(4, 1.0, 50.0, 1000.0)
    cfg, keep = _config(6000, sos, 9, 150, 3000, 1500)
    x = torch.zeros((1500, 6000), device="cuda")
    r = torch.zeros((1500, 6000), device="cuda")
    st = abi.filark_chain_run_static(cfg, x.data_ptr(), 6000, 1500, r.data_ptr(), None, None, 6000, None)
    assert st == abi.FILARK_EINVAL
    assert "static" in abi.filark_last_error_string()
    del keep
