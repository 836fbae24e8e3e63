"""The precision-stress workload at full width: order-8 Butterworth bandpass
0.01-1 Hz at 1.5 kHz (poles within 1e-4 of z = 1) on 10,000 channels of
N(0,1) noise plus a 0.05 Hz sine of amplitude 0.1, pushed in 1 s chunks.

The planner's path (FP32 block scan with double-float carries -- the dense carry for
this filter) and the all-FP32 comparison mode run on all 10,000 channels; the
FP64 oracle runs on 64 evenly spaced channels.  For every chunk the max
relative error (normwise per channel, over the 64 channels) of both modes is
computed; the planner's path must stay within 1e-5 in every chunk.

By default the whole 600 s record (600 chunks) is run, its chunks made on the
device (synth.precision_chunk_device); FILARK_PRECISION_PUSHES=n runs the
first n.  With FILARK_REPORT_DIR set, the per-chunk errors are written there
as JSON.
"""
import json
import os

import numpy as np
import pytest

from gpu_helpers import TOL
from paper_2605_20132_gb300 import abi, synth

pytestmark = pytest.mark.gpu


def test_precision_stress_per_chunk_report(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_20132_gb300.chain import Chain
    cfg = synth.PRECISION
    C, T = cfg["n_channels"], cfg["chunk"]
    # the whole 600 s record by default (FILARK_PRECISION_PUSHES shortens it)
    n_push = min(cfg["n_samples"] // T, int(os.environ.get("FILARK_PRECISION_PUSHES", "600")))
    sos = oracle_mod.butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    sel = np.linspace(0, C - 1, 64).round().astype(np.int64)
    sel_t = torch.from_numpy(sel).cuda()
    chains = {
        "fp32_scan_df_carry": Chain(C, sos, cfg["fs"], outputs=abi.FILARK_OUT_BANDPASS, max_chunk=T),
        "all_fp32": Chain(C, sos, cfg["fs"], outputs=abi.FILARK_OUT_BANDPASS, max_chunk=T,
                          precision=abi.FILARK_PREC_ALL32),
    }
    modes = {k: {1: "modal32", 2: "dense64", 3: "all32"}[c.info()["precision"]] for k, c in chains.items()}
    assert modes["fp32_scan_df_carry"] == "dense64"
    ora = oracle_mod.Chain(len(sel), sos, 1, 0, 0)
    got = {k: np.empty((n_push * T, len(sel))) for k in chains}
    ref = np.empty((n_push * T, len(sel)))
    y = torch.empty((T, C), device="cuda")

    gen = torch.Generator(device="cuda")
    for i in range(n_push):
        # the chunk is made on the device; the oracle gets the same values of
        # its 64 channels
        xd = synth.precision_chunk_device(i, C, T, cfg["fs"], cfg["seed"], cfg["sine_hz"], cfg["sine_amp"], gen)
        xs = np.ascontiguousarray(xd.index_select(1, sel_t).cpu().numpy())
        for k, ch in chains.items():
            ch.push(xd, bandpass=y)
            got[k][i * T:(i + 1) * T] = y.index_select(1, sel_t).double().cpu().numpy()
        ref[i * T:(i + 1) * T] = ora.push(xs, want=("bp",))["bp"]
    for ch in chains.values():
        ch.close()
    den = np.max(np.abs(ref), axis=0)
    den = np.where(den > 0, den, 1.0)
    report = {"workload": cfg["name"], "pushes": n_push, "channels": C, "oracle_channels": len(sel), "modes": {}}
    per = {}
    for k in chains:
        e = np.abs(got[k] - ref).reshape(n_push, T, len(sel)).max(axis=1) / den[None, :]
        per[k] = e.max(axis=1)
        report["modes"][k] = {"mode": modes[k], "max": float(per[k].max()), "median": float(np.median(per[k])),
                              "first": float(per[k][0]), "last": float(per[k][-1]),
                              "chunks_over_1e-5": int((per[k] > TOL).sum()),
                              "per_chunk": [float(v) for v in per[k]]}
    short = {k: {q: v for q, v in m.items() if q != "per_chunk"} for k, m in report["modes"].items()}
    print("precision stress per-chunk report:", json.dumps(short))
    out_dir = os.environ.get("FILARK_REPORT_DIR")
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "precision_stress_report.json"), "w") as f:
            json.dump(report, f)
    assert per["fp32_scan_df_carry"].max() <= TOL
    # the comparison mode drifts: its worst chunk is far above the planner's
    assert per["all_fp32"].max() > 10 * per["fp32_scan_df_carry"].max()
