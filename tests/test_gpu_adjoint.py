"""Parity of the differentiable SOS cascade (forward with checkpoints and the
reverse-time adjoint) with the FP64 oracle and with FP64 finite differences.

The CUDA side runs in FP64 and returns float32 signals, so y and dL/dx are
compared normwise per channel and the coefficient gradients elementwise; the
bars are the 1e-5 budget of the float32 path unless a test states a tighter
one derived from the FP64 arithmetic.
"""
import concurrent.futures as cf

import numpy as np
import pytest

from gpu_helpers import TOL, normwise
from oracle_pins import random_sections
from paper_2605_20132_gb300 import abi, synth

pytestmark = pytest.mark.gpu

# FP64 on both sides; what is left is float32 rounding of the stored signals
# (2^-24 ~ 6e-8 relative) and summation order.
TIGHT = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi.load()


def gpu_fwd_bwd(sos, x, gy, ckpt, ld=None, want_y=True, want_gx=True):
    """Forward with checkpoints and backward through the C-ABI."""
    import torch
    sos = np.ascontiguousarray(sos, dtype=np.float64)
    N, C = x.shape
    S = sos.shape[0]
    ld = ld or C
    xd = torch.zeros((N, ld), dtype=torch.float32, device="cuda")
    xd[:, :C] = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    gyd = torch.zeros((N, ld), dtype=torch.float32, device="cuda")
    gyd[:, :C] = torch.from_numpy(np.ascontiguousarray(gy, dtype=np.float32)).cuda()
    nb = abi.filark_iir_ckpt_bytes(S, C, N, ckpt)
    wb = abi.filark_iir_work_bytes(S, C, N, ckpt)
    assert nb > 0 and wb > 0
    ck = torch.empty(nb, dtype=torch.uint8, device="cuda")
    wk = torch.empty(wb, dtype=torch.uint8, device="cuda")
    y = torch.full((N, ld), float("nan"), dtype=torch.float32, device="cuda")
    gx = torch.full((N, ld), float("nan"), dtype=torch.float32, device="cuda")
    gs = torch.full((S, 6), float("nan"), dtype=torch.float64, device="cuda")
    sh = torch.cuda.current_stream().cuda_stream
    st = abi.filark_iir_forward_ckpt(sos, S, C, xd.data_ptr(), ld, N, y.data_ptr() if want_y else None, ld, ckpt,
                                     ck.data_ptr(), nb, sh)
    assert st == abi.FILARK_OK, abi.filark_last_error_string()
    st = abi.filark_iir_backward(sos, S, C, xd.data_ptr(), ld, N, gyd.data_ptr(), ld, ckpt, ck.data_ptr(), nb,
                                 wk.data_ptr(), wb, gx.data_ptr() if want_gx else None, ld, gs.data_ptr(), sh)
    assert st == abi.FILARK_OK, abi.filark_last_error_string()
    torch.cuda.synchronize()
    if ld > C:
        if want_y:
            assert torch.isnan(y[:, C:]).all()
        assert torch.isnan(gx[:, C:]).all()
    return (y[:, :C].cpu().numpy().astype(np.float64), gx[:, :C].cpu().numpy().astype(np.float64),
            gs.cpu().numpy())


def oracle_fwd_bwd(ora, sos, x, gy, threads=16):
    """Per-channel oracle forward and adjoint; coefficient gradients summed."""
    C = x.shape[1]

    def one(c):
        y, _ = ora.sosfilt(sos, x[:, c].astype(np.float64))
        gx, gs = ora.sos_adjoint(sos, x[:, c].astype(np.float64), gy[:, c].astype(np.float64))
        return y, gx, gs

    with cf.ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, range(C)))
    y = np.stack([r[0] for r in res], axis=1)
    gx = np.stack([r[1] for r in res], axis=1)
    gs = np.sum([r[2] for r in res], axis=0)
    return y, gx, gs


def grad_err(got, ref):
    """Elementwise relative error of the coefficient gradients, floored at
    1e-6 of the largest entry (entries that cancel to ~0)."""
    den = np.maximum(np.abs(ref), 1e-6 * np.max(np.abs(ref)))
    if not np.all(np.isfinite(got)):
        return float("inf")
    return float(np.max(np.abs(got - ref) / den))


@pytest.mark.parametrize("ckpt", [1, 2, 7, 300, 1999, 2000, 5000])
def test_adjoint_vs_oracle_checkpoint_intervals(oracle_mod, ckpt):
    """16 ch x 2000 samples, order-4 1-50 Hz bandpass, random input and
    output gradient; every checkpoint interval gives the oracle's answer
    (ragged last segments, single-sample segments, one segment)."""
    rng = np.random.default_rng(40 + ckpt)
    sos = oracle_mod.butter_bandpass(4, 1.0, 50.0, 1000.0)
    x = rng.standard_normal((2000, 16)).astype(np.float32)
    gy = rng.standard_normal((2000, 16)).astype(np.float32)
    y, gx, gs = gpu_fwd_bwd(sos, x, gy, ckpt)
    ry, rgx, rgs = oracle_fwd_bwd(oracle_mod, sos, x, gy)
    errs = dict(y=normwise(y, ry), gx=normwise(gx, rgx), gsos=grad_err(gs, rgs))
    print(ckpt, errs)
    assert errs["y"] <= TIGHT and errs["gx"] <= TIGHT and errs["gsos"] <= TIGHT, errs


@pytest.mark.parametrize("S", [1, 3, 8])
def test_adjoint_general_sections(oracle_mod, S):
    """Random stable sections (poles 0.5..0.995, raw a0 != 1), odd sizes and a
    strided layout (leading dimension > n_channels)."""
    rng = np.random.default_rng(50 + S)
    sos, _ = random_sections(rng, S)
    sos *= rng.uniform(0.5, 2.0, (S, 1))  # a0 != 1: the a0 division is exercised
    N, C = 777, 37
    x = rng.standard_normal((N, C)).astype(np.float32)
    gy = rng.standard_normal((N, C)).astype(np.float32)
    y, gx, gs = gpu_fwd_bwd(sos, x, gy, 100, ld=45)
    ry, rgx, rgs = oracle_fwd_bwd(oracle_mod, sos, x, gy)
    errs = dict(y=normwise(y, ry), gx=normwise(gx, rgx), gsos=grad_err(gs, rgs))
    print(S, errs)
    assert max(errs.values()) <= TIGHT, errs


def test_adjoint_degenerate_sizes(oracle_mod):
    """One sample, one channel, and optional outputs left out."""
    rng = np.random.default_rng(60)
    sos = oracle_mod.butter_bandpass(2, 5.0, 40.0, 1000.0)
    for N, C, ckpt in [(1, 1, 1), (1, 5, 3), (3, 1, 2), (64, 1, 64)]:
        x = rng.standard_normal((N, C)).astype(np.float32)
        gy = rng.standard_normal((N, C)).astype(np.float32)
        y, gx, gs = gpu_fwd_bwd(sos, x, gy, ckpt)
        ry, rgx, rgs = oracle_fwd_bwd(oracle_mod, sos, x, gy, threads=1)
        assert normwise(y, ry) <= TIGHT and normwise(gx, rgx) <= TIGHT
        assert grad_err(gs, rgs) <= TIGHT, (N, C, gs, rgs)
    x = rng.standard_normal((500, 8)).astype(np.float32)
    gy = rng.standard_normal((500, 8)).astype(np.float32)
    _, _, gs = gpu_fwd_bwd(sos, x, gy, 50, want_y=False, want_gx=False)
    _, _, rgs = oracle_fwd_bwd(oracle_mod, sos, x, gy)
    assert grad_err(gs, rgs) <= TIGHT


def _mse_loss_fp64(ora, sos, x, target):
    L = 0.0
    for c in range(x.shape[1]):
        y, _ = ora.sosfilt(sos, x[:, c].astype(np.float64))
        L += float(np.sum((y - target[:, c]) ** 2))
    return L / x.size


def test_adjoint_finite_differences_slice(oracle_mod):
    """The differentiation workload's check: on a 16 x 2000 slice, the GPU
    gradients of L = mean((y - target)^2) (target = the input filtered with
    the coefficients perturbed by up to 2%) against FP64 central finite
    differences of L for all 4 x 6 coefficients and a few input samples."""
    cfg = synth.ADJOINT
    sos = oracle_mod.butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    tsos = synth.perturb_sos(sos, cfg["perturb"], cfg["seed"])
    x = synth.adjoint_stream(16, 2000, seed=cfg["seed"]).astype(np.float64)
    target = np.stack([oracle_mod.sosfilt(tsos, x[:, c])[0] for c in range(16)], axis=1)
    ry = np.stack([oracle_mod.sosfilt(sos, x[:, c])[0] for c in range(16)], axis=1)
    gy = 2.0 * (ry - target) / x.size
    _, gx, gs = gpu_fwd_bwd(sos, x.astype(np.float32), gy, 300)

    def central(f, v0, h):
        d1 = (f(v0 + h) - f(v0 - h)) / (2 * h)
        d2 = (f(v0 + h / 2) - f(v0 - h / 2)) / h
        return (4 * d2 - d1) / 3

    worst = 0.0
    for s in range(sos.shape[0]):
        for i in range(6):
            def f(v, s=s, i=i):
                q = sos.copy()
                q[s, i] = v
                return _mse_loss_fp64(oracle_mod, q, x, target)
            fd = central(f, sos[s, i], 1e-7 * max(0.1, abs(sos[s, i])))
            worst = max(worst, abs(fd - gs[s, i]) / max(abs(fd), 1e-6 * np.max(np.abs(gs))))
    for (n, c) in [(0, 0), (1, 3), (999, 7), (1998, 15), (1999, 2)]:
        def f(v, n=n, c=c):
            q = x.copy()
            q[n, c] = v
            return _mse_loss_fp64(oracle_mod, sos, q, target)
        # L is quadratic in x, so a large step has no truncation error and
        # keeps the rounding error of L (~1e-16 L / h) small
        fd = central(f, x[n, c], 0.1)
        worst = max(worst, abs(fd - gx[n, c]) / max(abs(fd), 1e-6 * np.max(np.abs(gx))))
    print("finite-difference worst relative error", worst)
    assert worst <= TOL


def test_autograd_function_matches_abi(oracle_mod):
    """FilarkSOS.apply inside a torch loss gives the C-ABI's gradients, and a
    small step along minus the gradient lowers the FP64 loss."""
    import torch
    from paper_2605_20132_gb300.adjoint import FilarkSOS
    cfg = synth.ADJOINT
    sos = oracle_mod.butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    tsos = synth.perturb_sos(sos, cfg["perturb"], cfg["seed"])
    x = synth.adjoint_stream(64, 4000, seed=7)
    target = np.stack([oracle_mod.sosfilt(tsos, x[:, c].astype(np.float64))[0] for c in range(64)], axis=1)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    st = torch.from_numpy(sos.copy()).cuda().requires_grad_(True)
    tt = torch.from_numpy(target).cuda()
    y = FilarkSOS.apply(xt, st, 1000)
    loss = ((y.double() - tt) ** 2).mean()
    loss.backward()
    gy = (2.0 * (y.detach().double() - tt) / y.numel()).float().cpu().numpy()
    _, gx, gs = gpu_fwd_bwd(sos, x, gy, 1000)
    assert normwise(xt.grad.cpu().numpy().astype(np.float64), gx) <= 1e-6
    assert grad_err(st.grad.cpu().numpy(), gs) <= 1e-6
    L0 = _mse_loss_fp64(oracle_mod, sos, x, target)
    g = st.grad.cpu().numpy()
    step = 1e-3 * L0 / float(np.sum(g * g))
    L1 = _mse_loss_fp64(oracle_mod, sos - step * g, x, target)
    assert L1 < L0, (L0, L1)
    # torch's own check: the input gradient is the adjoint of the linear map x -> y
    v = torch.randn_like(xt)
    with torch.no_grad():
        Hv = FilarkSOS.apply(v, st.detach(), 1000)
    xt2 = xt.detach().clone().requires_grad_(True)
    u = torch.randn_like(xt)
    (FilarkSOS.apply(xt2, st.detach(), 1000) * u).sum().backward()
    # <H v, u> = <v, H^T u>
    a = float((Hv.double() * u.double()).sum())
    b = float((v.double() * xt2.grad.double()).sum())
    assert abs(a - b) <= 1e-5 * max(abs(a), 1e-30)


def test_adjoint_full_size_parity(oracle_mod):
    """The differentiation workload at full size: 2048 ch x 30,000 samples,
    order-4 1-50 Hz bandpass, checkpoints every 3,000 samples, MSE against the
    input filtered with 2%-perturbed coefficients.  y and dL/dx against the
    oracle on every channel, the summed coefficient gradients elementwise."""
    cfg = synth.ADJOINT
    C, N, ckpt = cfg["n_channels"], cfg["n_samples"], cfg["checkpoint"]
    sos = oracle_mod.butter_bandpass(cfg["order"], *cfg["band"], cfg["fs"])
    tsos = synth.perturb_sos(sos, cfg["perturb"], cfg["seed"])
    x = synth.adjoint_stream(C, N, seed=cfg["seed"])

    def filt(c, q):
        return oracle_mod.sosfilt(q, x[:, c].astype(np.float64))[0]

    with cf.ThreadPoolExecutor(16) as ex:
        target = np.stack(list(ex.map(lambda c: filt(c, tsos), range(C))), axis=1)
        ry = np.stack(list(ex.map(lambda c: filt(c, sos), range(C))), axis=1)
    gy = (2.0 * (ry - target) / ry.size).astype(np.float32)
    y, gx, gs = gpu_fwd_bwd(sos, x, gy, ckpt)
    _, rgx, rgs = oracle_fwd_bwd(oracle_mod, sos, x, gy)
    errs = dict(y=normwise(y, ry), gx=normwise(gx, rgx), gsos=grad_err(gs, rgs))
    print("full-size adjoint errors:", errs)
    assert max(errs.values()) <= TOL, errs
