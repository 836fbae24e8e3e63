"""FP64 CPU oracle of the chunked DAS operator chain -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product library never loads it, and it
shares no code with the CUDA path.  See ``filark_oracle.c`` for what each
function computes and which passage of the paper it follows.

Two builds of the same C source are made: ``ora_*`` (double) and ``orald_*``
(long double, used only to bound the rounding error of the double build).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "filark_oracle.c")
_OUT = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict = {}

_dp = ct.POINTER(ct.c_double)
_fp = ct.POINTER(ct.c_float)


def _lib_path(long_double: bool) -> str:
    return os.path.join(_OUT, "libfilark_oracle_ld.so" if long_double else "libfilark_oracle.so")


def compile_source(src: str, out: str, long_double: bool = False) -> None:
    """gcc a copy of the oracle source into a shared library (plain C11, no
    target-specific flags, no floating-point contraction)."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]
    if long_double:
        cmd.append("-DORA_LONG_DOUBLE")
    tmp = out + f".tmp{os.getpid()}"
    cmd += ["-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> None:
    """Compile both oracle builds."""
    os.makedirs(_OUT, exist_ok=True)
    for ld in (False, True):
        out = _lib_path(ld)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        compile_source(_SRC, out, ld)


def _bind(path: str, long_double: bool):
    lib = ct.CDLL(path)
    p = "orald_" if long_double else "ora_"
    f = getattr(lib, p + "butter_bandpass")
    f.argtypes = [ct.c_int, ct.c_double, ct.c_double, ct.c_double, _dp]
    f.restype = ct.c_int
    f = getattr(lib, p + "sosfilt")
    f.argtypes = [_dp, ct.c_int, _dp, ct.c_long, _dp, _dp]
    f.restype = None
    f = getattr(lib, p + "chain_new")
    f.argtypes = [ct.c_int, ct.c_int, _dp, ct.c_int, ct.c_int, ct.c_int]
    f.restype = ct.c_void_p
    for name in ("chain_free", "chain_reset"):
        f = getattr(lib, p + name)
        f.argtypes = [ct.c_void_p]
        f.restype = None
    f = getattr(lib, p + "chain_samples")
    f.argtypes = [ct.c_void_p]
    f.restype = ct.c_long
    f = getattr(lib, p + "chain_push")
    f.argtypes = [ct.c_void_p, _fp, ct.c_long, ct.c_long, _dp, _dp, _dp, ct.c_long]
    f.restype = ct.c_int
    f = getattr(lib, p + "chain_get_iir_state")
    f.argtypes = [ct.c_void_p, _dp]
    f.restype = None
    f = getattr(lib, p + "stalta_naive")
    f.argtypes = [_dp, ct.c_long, ct.c_int, ct.c_int, _dp]
    f.restype = None
    f = getattr(lib, p + "sos_adjoint")
    f.argtypes = [_dp, ct.c_int, _dp, ct.c_long, _dp, _dp, _dp]
    f.restype = None
    if not long_double:
        _lp = ct.POINTER(ct.c_long)
        f = lib.ora_trig_new
        f.argtypes = [ct.c_int, ct.c_double, ct.c_double]
        f.restype = ct.c_void_p
        f = lib.ora_trig_free
        f.argtypes = [ct.c_void_p]
        f.restype = None
        f = lib.ora_trig_push
        f.argtypes = [ct.c_void_p, _fp, ct.c_long, ct.c_long, _lp, _lp, _lp, ct.c_long]
        f.restype = ct.c_long
        f = lib.ora_trig_flush
        f.argtypes = [ct.c_void_p, _lp, _lp, _lp, ct.c_long]
        f.restype = ct.c_long
        f = lib.ora_events_merge
        f.argtypes = [_lp, _lp, _lp, ct.c_long, _lp]
        f.restype = ct.c_long
        f = lib.ora_top_new
        f.argtypes = [ct.c_int, ct.c_int, ct.c_int, _dp, ct.c_double]
        f.restype = ct.c_void_p
        f = lib.ora_top_free
        f.argtypes = [ct.c_void_p]
        f.restype = None
        f = lib.ora_top_push
        f.argtypes = [ct.c_void_p, _fp, ct.c_long, ct.c_long, _dp, ct.c_long]
        f.restype = None
    return lib, p


def _load(long_double: bool = False):
    with _LOCK:
        if long_double not in _LIBS:
            build()
            _LIBS[long_double] = _bind(_lib_path(long_double), long_double)
        return _LIBS[long_double]


class use_library:
    """Context manager: route the double-precision API through another build of
    the oracle source (the tests use it to run the pins on planted mistakes)."""

    def __init__(self, path: str):
        self._path = path

    def __enter__(self):
        with _LOCK:
            self._saved = _LIBS.get(False)
            _LIBS[False] = _bind(self._path, False)
        return self

    def __exit__(self, *exc):
        with _LOCK:
            if self._saved is None:
                _LIBS.pop(False, None)
            else:
                _LIBS[False] = self._saved
        return False


def _fn(name: str, long_double: bool = False):
    lib, p = _load(long_double)
    return getattr(lib, p + name)


def _ptr(a: np.ndarray | None, typ=_dp):
    if a is None:
        return ct.cast(None, typ)
    return a.ctypes.data_as(typ)


def butter_bandpass(order: int, f1: float, f2: float, fs: float, long_double: bool = False) -> np.ndarray:
    """Butterworth bandpass as ``order`` SOS rows {b0,b1,b2,a0,a1,a2}."""
    sos = np.zeros((order, 6), dtype=np.float64)
    rc = _fn("butter_bandpass", long_double)(order, f1, f2, fs, _ptr(sos))
    if rc != 0:
        raise ValueError("invalid Butterworth bandpass parameters")
    return sos


def sosfilt(sos: np.ndarray, x: np.ndarray, zi: np.ndarray | None = None,
            long_double: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Filter one channel with the TDF-II cascade; returns (y, final state)."""
    sos = np.ascontiguousarray(sos, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    S = sos.shape[0]
    z = np.zeros(2 * S) if zi is None else np.array(zi, dtype=np.float64).copy()
    y = np.empty_like(x)
    _fn("sosfilt", long_double)(_ptr(sos), S, _ptr(x), x.shape[0], _ptr(y), _ptr(z))
    return y, z


class Chain:
    """Stateful oracle chain: IIR -> spatial mean -> STA/LTA (all FP64)."""

    def __init__(self, n_channels: int, sos: np.ndarray | None, spatial_width: int = 1,
                 sta_len: int = 0, lta_len: int = 0, long_double: bool = False):
        self._ld = long_double
        sos = np.zeros((0, 6)) if sos is None else np.ascontiguousarray(sos, dtype=np.float64)
        self._sos = sos
        self.C = int(n_channels)
        self.S = int(sos.shape[0])
        self.detector = lta_len > 0
        lib, p = _load(long_double)
        self._f = {k: getattr(lib, p + k) for k in
                   ("chain_new", "chain_free", "chain_reset", "chain_samples", "chain_push",
                    "chain_get_iir_state")}
        self._h = self._f["chain_new"](self.C, self.S, _ptr(sos if self.S else np.zeros(6)),
                                       int(spatial_width), int(sta_len), int(lta_len))
        if not self._h:
            raise ValueError("invalid oracle chain configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._f["chain_free"](h)
            self._h = None

    def reset(self) -> None:
        self._f["chain_reset"](self._h)

    @property
    def samples(self) -> int:
        return int(self._f["chain_samples"](self._h))

    def push(self, x: np.ndarray, want=("bp", "sp", "ratio")) -> dict:
        """Push a time-major float32 chunk [T][C]; returns the requested outputs
        as float64 arrays [T][C]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        if x.ndim != 2 or x.shape[1] != self.C:
            raise ValueError("chunk must be [T][C]")
        T = x.shape[0]
        out = {k: np.zeros((T, self.C), dtype=np.float64) for k in want
               if k != "ratio" or self.detector}
        rc = self._f["chain_push"](self._h, _ptr(x, _fp), self.C, T,
                                         _ptr(out.get("bp")), _ptr(out.get("sp")),
                                         _ptr(out.get("ratio")), self.C)
        if rc != 0:
            raise ValueError("oracle push failed")
        return out

    def iir_state(self) -> np.ndarray:
        z = np.zeros((self.C, 2 * self.S), dtype=np.float64)
        self._f["chain_get_iir_state"](self._h, _ptr(z))
        return z


def stalta_naive(cf: np.ndarray, sta_len: int, lta_len: int, long_double: bool = False) -> np.ndarray:
    """Literal-window STA/LTA of one channel's cf sequence (O(window) per sample)."""
    cf = np.ascontiguousarray(cf, dtype=np.float64)
    R = np.zeros_like(cf)
    _fn("stalta_naive", long_double)(_ptr(cf), cf.shape[0], int(sta_len), int(lta_len), _ptr(R))
    return R


def sos_adjoint(sos: np.ndarray, x: np.ndarray, gy: np.ndarray, long_double: bool = False):
    """Adjoint of the SOS cascade for one channel: returns (dL/dx, dL/dsos)."""
    sos = np.ascontiguousarray(sos, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    gy = np.ascontiguousarray(gy, dtype=np.float64)
    gx = np.zeros_like(x)
    gs = np.zeros_like(sos)
    _fn("sos_adjoint", long_double)(_ptr(sos), sos.shape[0], _ptr(x), x.shape[0], _ptr(gy),
                                    _ptr(gx), _ptr(gs))
    return gx, gs


# ------------------------------------------------------ triggers and events --

_lp = ct.POINTER(ct.c_long)


class Trigger:
    """Per-channel on/off hysteresis on the detector ratio, carried across
    pushes; reports each channel trigger [t_on, t_off) when it ends."""

    def __init__(self, C: int, on: float, off: float):
        lib, _ = _load(False)
        self._f = {k: getattr(lib, "ora_" + k) for k in ("trig_new", "trig_free", "trig_push", "trig_flush")}
        self.C = int(C)
        self._h = self._f["trig_new"](self.C, float(on), float(off))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._f["trig_free"](h)
            self._h = None

    @staticmethod
    def _records(call, cap):
        while True:
            rc, ron, roff = (np.zeros(cap, dtype=np.int64) for _ in range(3))
            n = call(rc, ron, roff, cap)
            if n <= cap:
                return np.stack([rc[:n], ron[:n], roff[:n]], axis=1)
            cap = int(n)

    def push(self, R: np.ndarray) -> np.ndarray:
        """R: [T][C] float32.  Returns the triggers that ended, [k][3] =
        (channel, t_on, t_off)."""
        R = np.ascontiguousarray(R, dtype=np.float32)
        if R.ndim != 2 or R.shape[1] != self.C:
            raise ValueError("R must be [T][C]")
        T = R.shape[0]
        # at most one trigger can end per channel every second sample
        cap = min(T * self.C // 2 + 16, 64 * self.C + 100_000)
        rc, ron, roff = (np.zeros(cap, dtype=np.int64) for _ in range(3))
        n = self._f["trig_push"](self._h, _ptr(R, _fp), self.C, T, _ptr(rc, _lp), _ptr(ron, _lp),
                                 _ptr(roff, _lp), cap)
        if n > cap:
            raise RuntimeError("more triggers ended in one push than the oracle buffer holds")
        return np.stack([rc[:n], ron[:n], roff[:n]], axis=1)

    def flush(self) -> np.ndarray:
        """The runs still open, with t_off = samples seen (state kept)."""
        return self._records(lambda a, b, c, cap: self._f["trig_flush"](
            self._h, _ptr(a, _lp), _ptr(b, _lp), _ptr(c, _lp), cap), max(16, self.C))


def events_merge(records: np.ndarray) -> np.ndarray:
    """Events from channel triggers [k][3] = (channel, t_on, t_off): rows
    (t_on, t_off, c_min, c_max, n_triggers), sorted by (t_on, c_min, t_off,
    c_max)."""
    r = np.ascontiguousarray(records, dtype=np.int64).reshape(-1, 3)
    rc, ron, roff = (np.ascontiguousarray(r[:, i]) for i in range(3))
    ev = np.zeros((max(1, r.shape[0]), 5), dtype=np.int64)
    m = _fn("events_merge")(_ptr(rc, _lp), _ptr(ron, _lp), _ptr(roff, _lp), r.shape[0], _ptr(ev, _lp))
    return ev[:m].copy()


# ------------------------------------------------------- temporal operators --

TOP_FIR, TOP_MEAN, TOP_AGC, TOP_EMA = 0, 1, 2, 3


class TemporalOp:
    """Stateful temporal operator per channel (x before the stream start is 0):
    FIR y = sum_k h[k] x[n-k]; MEAN y = window mean of x over the last w
    samples; AGC y = x / (window mean of |x|) (0 if that mean is 0); EMA e =
    (1-a) e + a x^2, y = x / sqrt(e) (0 if e = 0)."""

    def __init__(self, C: int, kind: int, length: int = 1, taps=None, alpha: float = 0.0):
        lib, _ = _load(False)
        self._f = {k: getattr(lib, "ora_" + k) for k in ("top_new", "top_free", "top_push")}
        self.C = int(C)
        h = None if taps is None else np.ascontiguousarray(taps, dtype=np.float64)
        self._h = self._f["top_new"](self.C, int(kind), int(length), _ptr(h), float(alpha))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._f["top_free"](h)
            self._h = None

    def push(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        if x.ndim != 2 or x.shape[1] != self.C:
            raise ValueError("x must be [T][C]")
        y = np.zeros(x.shape, dtype=np.float64)
        self._f["top_push"](self._h, _ptr(x, _fp), self.C, x.shape[0], _ptr(y), self.C)
        return y


# ------------------------------------------------- headless display path --

VIEW_DROP, VIEW_PEAK, VIEW_LINEAR = 0, 1, 2


def _reduce_group(v: np.ndarray, mode: int) -> float:
    """One display value from a group of samples (consecutive channels or
    consecutive times): drop = the first; peak = the value of largest
    magnitude (first on ties); linear = interpolation at the group's centre."""
    n = v.shape[0]
    if mode == VIEW_DROP:
        return float(v[0])
    if mode == VIEW_PEAK:
        return float(v[int(np.argmax(np.abs(v)))])
    p = (n - 1) / 2.0
    i0 = int(np.floor(p))
    f = p - i0
    return float(v[i0]) if f == 0 else float((1 - f) * v[i0] + f * v[i0 + 1])


class View:
    """Streaming display buffer (test infrastructure): channels grouped by kc
    into display rows, an optional causal SOS display filter on the rows at
    the source rate (state carried), times grouped by kt into columns, the
    last W columns kept in a ring; image() returns them oldest to newest, the
    newest at the right, zeros before the first column."""

    def __init__(self, C: int, kc: int, kt: int, W: int, mode: int, sos=None):
        self.C, self.kc, self.kt, self.W, self.mode = int(C), int(kc), int(kt), int(W), int(mode)
        self.H = -(-self.C // self.kc)
        self.filt = None if sos is None else Chain(self.H, sos)
        self.pending = np.zeros((0, self.H))
        self.cols: list[np.ndarray] = []

    def push(self, x: np.ndarray) -> None:
        x = np.asarray(x, dtype=np.float32)
        T = x.shape[0]
        rows = np.zeros((T, self.H))
        for n in range(T):
            for r in range(self.H):
                rows[n, r] = _reduce_group(x[n, r * self.kc:min(self.C, (r + 1) * self.kc)].astype(np.float64),
                                           self.mode)
        if self.filt is not None:
            rows = self.filt.push(rows.astype(np.float32), want=("bp",))["bp"]
        self.pending = np.vstack([self.pending, rows])
        while self.pending.shape[0] >= self.kt:
            grp = self.pending[:self.kt]
            self.cols.append(np.array([_reduce_group(grp[:, r], self.mode) for r in range(self.H)]))
            self.pending = self.pending[self.kt:]

    def image(self) -> np.ndarray:
        img = np.zeros((self.H, self.W))
        last = self.cols[-self.W:]
        for i, col in enumerate(last):
            img[:, self.W - len(last) + i] = col
        return img
