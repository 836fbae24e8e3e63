"""The FP64 oracle against its pins (CPU only).

Also: the oracle's own rounding error, bounded by the long double build of the
same source, and an independent library cross-check (SciPy), and a mutation
test showing that each planted mistake in the oracle fails at least one pin.
"""
import os
import re
import shutil

import numpy as np
import pytest

import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=[f.__name__ for f in P.ALL_PINS])
def test_pin(oracle_mod, pin):
    err, bound = pin(oracle_mod)
    assert err <= bound, f"{pin.__name__}: {err:.3e} > {bound:.1e}"


@pytest.mark.parametrize("spec,n,bound", [
    ((4, 1.0, 50.0, 1000.0), 20_000, 1e-10),      # small bandpass
    ((8, 0.5, 100.0, 1500.0), 90_000, 1e-10),      # paper-scale bandpass, 60 s
    ((8, 0.01, 1.0, 1500.0), 300_000, 1e-8),       # precision-stress bandpass, 200 s
])
def test_oracle_rounding_vs_long_double(oracle_mod, spec, n, bound):
    """The double build's own error, measured against the long double build of
    the same source.  With each section's double zero facing its poles the
    TDF-II states stay small even 8e-6 from the unit circle."""
    sos = oracle_mod.butter_bandpass(*spec)
    x = np.random.default_rng(0).standard_normal(n)
    yd, _ = oracle_mod.sosfilt(sos, x)
    yl, _ = oracle_mod.sosfilt(sos, x, long_double=True)
    err = np.max(np.abs(yd - yl)) / np.max(np.abs(yl))
    assert err <= bound


def test_long_double_build_agrees_on_design(oracle_mod):
    for spec in [(4, 1.0, 50.0, 1000.0), (8, 0.5, 100.0, 1500.0), (8, 0.01, 1.0, 1500.0)]:
        a = oracle_mod.butter_bandpass(*spec)
        b = oracle_mod.butter_bandpass(*spec, long_double=True)
        assert np.max(np.abs(a - b)) < 1e-12


def test_scipy_crosscheck(oracle_mod):
    """SciPy (an independent implementation) designs the same transfer
    function, and its sosfilt agrees with the oracle chain's IIR stage."""
    ss = pytest.importorskip("scipy.signal")
    from paper_2605_20132_gb300 import synth
    for N, f1, f2, fs in [(4, 1.0, 50.0, 1000.0), (8, 0.5, 100.0, 1500.0)]:
        ours = oracle_mod.butter_bandpass(N, f1, f2, fs)
        ref = ss.butter(N, [f1, f2], btype="band", fs=fs, output="sos")
        w = np.linspace(1e-3, np.pi - 1e-3, 301)
        assert np.max(np.abs(P.sos_response(ours, w) - P.sos_response(ref, w))) < 1e-11
        x = synth.small_stream(4, 3000, seed=9)
        ch = oracle_mod.Chain(4, ref, 1, 0, 0)
        bp = np.concatenate([ch.push(x[:1234], ("bp",))["bp"], ch.push(x[1234:], ("bp",))["bp"]])
        want = ss.sosfilt(ref, x.astype(np.float64), axis=0)
        assert P.normwise_err(bp, want) < 1e-13


# Plausible mistakes planted in a copy of the oracle source: (name, old, new).
MUTANTS = [
    ("tdf2_sign_a1", "zs[0] = k[1] * u - k[3] * y + zs[1];", "zs[0] = k[1] * u + k[3] * y + zs[1];"),
    ("tdf2_drop_b2", "zs[1] = k[2] * u - k[4] * y;", "zs[1] = - k[4] * y;"),
    ("tdf2_drop_z2", "zs[0] = k[1] * u - k[3] * y + zs[1];", "zs[0] = k[1] * u - k[3] * y;"),
    ("swap_a1_a2", "c[5 * s + 3] = (real)sos[6 * s + 4] / a0;", "c[5 * s + 3] = (real)sos[6 * s + 5] / a0;"),
    ("no_a0_norm_b0", "c[5 * s + 0] = (real)sos[6 * s + 0] / a0;", "c[5 * s + 0] = (real)sos[6 * s + 0];"),
    ("no_prewarp", "const real W1 = two_fs * R_TAN(pi * (real)f1 / (real)fs);",
     "const real W1 = two_fs * (pi * (real)f1 / (real)fs);"),
    ("gain_inverted", "real g = R_POW(1 / c_abs(H), (real)1 / (real)N);", "real g = R_POW(c_abs(H), (real)1 / (real)N);"),
    ("zero_pair_sign", "else { num[s][0] = 1; num[s][1] = 2; num[s][2] = 1; }", "else { num[s][0] = 1; num[s][1] = -2; num[s][2] = 1; }"),
    ("bilinear_sign", "cplx z = c_div(c_add(c_make(two_fs, 0), s), c_sub(c_make(two_fs, 0), s));",
     "cplx z = c_div(c_sub(c_make(two_fs, 0), s), c_add(c_make(two_fs, 0), s));"),
    ("proto_angle", "real ang = pi * (real)(2 * k + N - 1) / (real)(2 * N);",
     "real ang = pi * (real)(2 * k + N + 1) / (real)(2 * N);"),
    ("spatial_window_short", "int hi = c + hw > C - 1 ? C - 1 : c + hw;", "int hi = c + hw - 1 > C - 1 ? C - 1 : c + hw - 1;"),
    ("spatial_divide_K", "real ysp = acc / (real)(hi - lo + 1);", "real ysp = acc / (real)h->K;"),
    ("sta_exit_off_by_one", "real out_s = (n - h->ns >= 0) ? hist_at(h, c, n - h->ns) : 0;",
     "real out_s = (n - h->ns + 1 >= 0) ? hist_at(h, c, n - h->ns + 1) : 0;"),
    ("warmup_off_by_one", "if (n >= h->nl - 1 && h->nz[c] > 0)", "if (n >= h->nl && h->nz[c] > 0)"),
    ("lta_zero_test_dropped", "if (n >= h->nl - 1 && h->nz[c] > 0)", "if (n >= h->nl - 1)"),
    ("ratio_inverted", "r = (h->sta[c] / (real)h->ns) / (h->lta[c] / (real)h->nl);",
     "r = (h->lta[c] / (real)h->nl) / (h->sta[c] / (real)h->ns);"),
    ("hist_index_by_chunk", "h->hist[(size_t)c * (size_t)h->nl + (size_t)(n % h->nl)] = cf;",
     "h->hist[(size_t)c * (size_t)h->nl + (size_t)(t % h->nl)] = cf;"),
    ("resum_window_short", "for (long m = h->n - h->nl; m < h->n; ++m) if (m >= 0) l += hist_at(h, c, m);",
     "for (long m = h->n - h->nl + 1; m < h->n; ++m) if (m >= 0) l += hist_at(h, c, m);"),
    ("adjoint_sign_a", "ga[i] -= w[n] * y[n - i];", "ga[i] += w[n] * y[n - i];"),
    ("adjoint_index", "if (n + 1 < N) acc -= a1 * w[n + 1];", "if (n + 1 < N) acc -= a2 * w[n + 1];"),
    ("adjoint_input_grad_b", "if (n + 2 < N) acc += b2 * w[n + 2];", "if (n + 2 < N) acc += b1 * w[n + 2];"),
    ("trigger_on_strict", "if (r >= t->on) s = 1;", "if (r > t->on) s = 1;"),
    ("trigger_off_inclusive", "else if (r < t->off) s = 0;", "else if (r <= t->off) s = 0;"),
    ("trigger_no_hysteresis", "else if (r < t->off) s = 0;", "else s = 0;"),
    ("trigger_flush_end", "roff[k] = t->n;", "roff[k] = t->n - 1;"),
    ("events_touching_merge", "if (lo >= hi) continue;", "if (lo > hi) continue;"),
    ("events_skip_a_channel", "if (dc != 1 && dc != -1) continue;", "if (dc != 2 && dc != -2) continue;"),
    ("events_one_side_only", "if (dc != 1 && dc != -1) continue;", "if (dc != 1) continue;"),
    ("fir_skip_current", "for (int k = 0; k < t->M; ++k) acc += t->h[k] * top_hist(t, c, n - k);",
     "for (int k = 0; k < t->M; ++k) acc += t->h[k] * top_hist(t, c, n - k - 1);"),
    ("window_exit_early", "const double old = top_hist(t, c, n - t->M);",
     "const double old = top_hist(t, c, n - t->M + 1);"),
    ("agc_no_abs", "const double u = t->kind == 1 ? v : fabs(v);", "const double u = v;"),
    ("ema_swapped", "t->e[c] = (1 - t->a) * t->e[c] + t->a * v * v;",
     "t->e[c] = t->a * t->e[c] + (1 - t->a) * v * v;"),
    ("window_resum_short", "for (long m = n - t->M + 1; m <= n; ++m) s += top_hist(t, c, m);",
     "for (long m = n - t->M + 2; m <= n; ++m) s += top_hist(t, c, m);"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle_mod, tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle_mod.__file__), "filark_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    cpath = tmp_path / "mutant.c"
    cpath.write_text(mutated)
    lib = str(tmp_path / "libmutant.so")
    oracle_mod.compile_source(str(cpath), lib)
    failed = []
    with oracle_mod.use_library(lib):
        for pin in P.ALL_PINS:
            try:
                with np.errstate(all="ignore"):
                    err, bound = pin(oracle_mod)
                ok = bool(err <= bound)
            except Exception:
                ok = False
            if not ok:
                failed.append(pin.__name__)
    assert failed, f"no pin caught mutant {name}"


# The display-path oracle is numpy code: plant mistakes by swapping its group
# reduction and check a pin fails.
def _bad_linear(v, mode):
    import numpy as _np
    if mode == 2:
        return float(v[(v.shape[0] - 1) // 2])          # no interpolation
    return _ORIG_REDUCE(v, mode)


def _bad_peak(v, mode):
    import numpy as _np
    if mode == 1:
        return float(v[int(_np.argmax(v))])              # largest value, not magnitude
    return _ORIG_REDUCE(v, mode)


def _bad_drop(v, mode):
    if mode == 0:
        return float(v[-1])                              # last sample of the group
    return _ORIG_REDUCE(v, mode)


_ORIG_REDUCE = None


@pytest.mark.parametrize("bad", [_bad_linear, _bad_peak, _bad_drop], ids=["linear", "peak", "drop"])
def test_planted_display_mistake_is_caught(oracle_mod, monkeypatch, bad):
    global _ORIG_REDUCE
    _ORIG_REDUCE = oracle_mod._reduce_group
    monkeypatch.setattr(oracle_mod, "_reduce_group", bad)
    failed = False
    for pin in (P.pin_view_closed_forms, P.pin_view_display_filter):
        try:
            err, bound = pin(oracle_mod)
            failed |= not (err <= bound)
        except Exception:
            failed = True
    assert failed
