"""Shared helpers of the GPU tests: run the CUDA chain through the C-ABI and
the FP64 oracle on the same seeded float32 input, and compare them."""
from __future__ import annotations

import numpy as np

from paper_2605_20132_gb300 import abi
from paper_2605_20132_gb300.chain import Chain

# Tolerance of the FP32 path against the FP64 oracle (max relative error).
TOL = 1e-5

ALL_OUT = abi.FILARK_OUT_RATIO | abi.FILARK_OUT_BANDPASS | abi.FILARK_OUT_SPATIAL


def normwise(got: np.ndarray, ref: np.ndarray) -> float:
    """max over channels of max_t |got - ref| / max_t |ref| (zero columns: absolute)."""
    got = np.asarray(got, dtype=np.float64)
    den = np.max(np.abs(ref), axis=0)
    den = np.where(den > 0, den, 1.0)
    err = np.max(np.abs(got - ref), axis=0) / den
    if not np.all(np.isfinite(got)):
        return float("inf")
    return float(np.max(err)) if err.size else 0.0


def ratio_err(got: np.ndarray, ref: np.ndarray) -> float:
    """max over channels of max_t |R - R_ref| / max(max_t |R_ref|, 1)."""
    got = np.asarray(got, dtype=np.float64)
    den = np.maximum(np.max(np.abs(ref), axis=0), 1.0)
    if not np.all(np.isfinite(got)):
        return float("inf")
    return float(np.max(np.max(np.abs(got - ref), axis=0) / den)) if got.size else 0.0


def run_gpu(x: np.ndarray, chunks, sos, fs=1000.0, K=1, ns=0, nl=0, outputs=None, precision=0,
            ld_in=None, ld_out=None, max_chunk=None, chain=None, return_chain=False):
    """Push x [N][C] (float32) in the given chunk lengths; returns dict of outputs."""
    import torch
    N, C = x.shape
    det = nl > 0
    if outputs is None:
        outputs = (abi.FILARK_OUT_BANDPASS | abi.FILARK_OUT_SPATIAL | (abi.FILARK_OUT_RATIO if det else 0))
    mc = max_chunk or max(max(chunks), 1)
    ch = chain or Chain(C, sos, fs, K, ns, nl, outputs=outputs, precision=precision, max_chunk=mc)
    ldi = ld_in or C
    ldo = ld_out or C
    xd = torch.zeros((N, ldi), dtype=torch.float32, device="cuda")
    xd[:, :C] = torch.from_numpy(x).cuda()
    outs = {}
    if outputs & abi.FILARK_OUT_RATIO:
        outs["ratio"] = torch.full((N, ldo), float("nan"), dtype=torch.float32, device="cuda")
    if outputs & abi.FILARK_OUT_BANDPASS:
        outs["bp"] = torch.full((N, ldo), float("nan"), dtype=torch.float32, device="cuda")
    if outputs & abi.FILARK_OUT_SPATIAL:
        outs["sp"] = torch.full((N, ldo), float("nan"), dtype=torch.float32, device="cuda")
    t = 0
    for T in chunks:
        sl = slice(t, t + T)
        ch.push(xd[sl], ratio=outs["ratio"][sl] if "ratio" in outs else None,
                bandpass=outs["bp"][sl] if "bp" in outs else None,
                spatial=outs["sp"][sl] if "sp" in outs else None)
        t += T
    assert t == N
    ch.sync()
    res = {k: v[:, :C].cpu().numpy() for k, v in outs.items()}
    # padding columns beyond C must be untouched
    for k, v in outs.items():
        if ldo > C:
            assert torch.isnan(v[:, C:]).all(), f"{k}: wrote past n_channels"
    if return_chain:
        return res, ch
    if chain is None:
        ch.close()
    return res


def run_oracle(oracle_mod, x: np.ndarray, sos, K=1, ns=0, nl=0, chunks=None):
    ch = oracle_mod.Chain(x.shape[1], sos, K, ns, nl)
    if chunks is None:
        return ch.push(x)
    parts = []
    t = 0
    for T in chunks:
        parts.append(ch.push(x[t:t + T]))
        t += T
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def compare(got: dict, ref: dict) -> dict:
    errs = {}
    if "bp" in got:
        errs["bp"] = normwise(got["bp"], ref["bp"])
    if "sp" in got:
        errs["sp"] = normwise(got["sp"], ref["sp"])
    if "ratio" in got:
        errs["ratio"] = ratio_err(got["ratio"], ref["ratio"])
    return errs
