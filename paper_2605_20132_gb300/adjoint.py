"""Differentiable SOS bandpass for PyTorch: ``FilarkSOS.apply(x, sos, ckpt_every)``.

The forward and the backward are the library's CUDA kernels
(filark_iir_forward_ckpt / filark_iir_backward); this module only allocates
the checkpoint and work buffers with torch and marshals pointers.  The
forward keeps the cascade state at the start of every piece of about
sqrt(2 L) samples of segments of at most ``ckpt_every`` samples (shorter when
the channels are too few to fill the GPU) and nothing else; the backward
recomputes the section signals piece by piece from those checkpoints and runs
the reverse-time adjoint (Sec. 3.4, the SOS filter, differentiated).

x: (n_samples, n_channels) float32 CUDA tensor, time-major (row stride >=
n_channels, unit channel stride).  sos: (n_sections, 6) float64 tensor of raw
rows {b0,b1,b2,a0,a1,a2} on any device.  Returns y with x's shape; the
gradient with respect to sos is float64 on sos's device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import abi


def _stream(device) -> int | None:
    return torch.cuda.current_stream(device).cuda_stream or None


def _time_major(t: torch.Tensor) -> torch.Tensor:
    if t.dim() != 2:
        raise ValueError("expected a (n_samples, n_channels) tensor")
    if t.stride(1) != 1 or t.stride(0) < t.shape[1]:
        t = t.contiguous()
    return t


class FilarkSOS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, sos: torch.Tensor, ckpt_every: int = 3000):
        if not x.is_cuda or x.dtype != torch.float32:
            raise TypeError("x must be a float32 CUDA tensor")
        x = _time_major(x)
        N, C = x.shape
        sos_host = np.ascontiguousarray(sos.detach().to("cpu", torch.float64).numpy())
        if sos_host.ndim != 2 or sos_host.shape[1] != 6:
            raise ValueError("sos must have shape (n_sections, 6)")
        S = sos_host.shape[0]
        ckpt_every = int(min(max(int(ckpt_every), 1), max(N, 1)))
        y = torch.empty((N, C), dtype=torch.float32, device=x.device)
        if N == 0:
            ctx.empty = True
            ctx.save_for_backward(x)
            ctx.sos_meta = (sos_host, sos.device, sos.dtype)
            return y
        ctx.empty = False
        nbytes = abi.filark_iir_ckpt_bytes(S, C, N, ckpt_every)
        if nbytes == 0:
            raise ValueError("invalid sizes for filark_iir_ckpt_bytes")
        ckpt = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
        with torch.cuda.device(x.device):
            st = abi.filark_iir_forward_ckpt(sos_host, S, C, x.data_ptr(), x.stride(0), N, y.data_ptr(), C,
                                             ckpt_every, ckpt.data_ptr(), nbytes, _stream(x.device))
        abi.check(st, "filark_iir_forward_ckpt")
        ctx.save_for_backward(x, ckpt)
        ctx.sos_meta = (sos_host, sos.device, sos.dtype)
        ctx.ckpt_every = ckpt_every
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        sos_host, sos_device, sos_dtype = ctx.sos_meta
        S = sos_host.shape[0]
        if ctx.empty:
            (x,) = ctx.saved_tensors
            return torch.zeros_like(x), torch.zeros((S, 6), dtype=sos_dtype, device=sos_device), None
        x, ckpt = ctx.saved_tensors
        N, C = x.shape
        gy = _time_major(gy.to(torch.float32))
        wbytes = abi.filark_iir_work_bytes(S, C, N, ctx.ckpt_every)
        work = torch.empty(wbytes, dtype=torch.uint8, device=x.device)
        gx = torch.empty((N, C), dtype=torch.float32, device=x.device) if ctx.needs_input_grad[0] else None
        gsos = torch.empty((S, 6), dtype=torch.float64, device=x.device)
        with torch.cuda.device(x.device):
            st = abi.filark_iir_backward(sos_host, S, C, x.data_ptr(), x.stride(0), N, gy.data_ptr(), gy.stride(0),
                                         ctx.ckpt_every, ckpt.data_ptr(), ckpt.numel(), work.data_ptr(), wbytes,
                                         None if gx is None else gx.data_ptr(), C, gsos.data_ptr(),
                                         _stream(x.device))
        abi.check(st, "filark_iir_backward")
        gs = gsos.to(device=sos_device, dtype=sos_dtype) if ctx.needs_input_grad[1] else None
        return gx, gs, None


def sos_filter(x: torch.Tensor, sos: torch.Tensor, ckpt_every: int = 3000) -> torch.Tensor:
    """y = the SOS cascade applied to every channel of x, differentiable in x and sos."""
    return FilarkSOS.apply(x, sos, ckpt_every)
