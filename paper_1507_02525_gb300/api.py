"""PyTorch front end of the MrDFT library: device memory and streams from torch,
all arithmetic in the CUDA kernels behind the C ABI.

    y = mrdft(x)                     # x [B, N] or [N] complex64/float32 (cuda)
                                     # -> [B, m, N] or [m, N] complex64
    gx = mrdft_adjoint(gy)           # gy [B, m, N] -> [B, N] complex64
    y = MrDFT.apply(x)               # differentiable (backward = adjoint)
    y = mrdft_ragged(x_flat, lengths)  # uneven power-of-two lengths, one launch set
"""
from __future__ import annotations

import threading

import torch

from . import _lib

_cache_lock = threading.Lock()
_plans: dict = {}


def get_plan(lengths, batch: int, real_input: bool, graph: bool = False, device=None,
             tune: bool = False) -> _lib.Plan:
    """Plan for the given signal lengths (cached per device and configuration).

    With tune=True the execution options come from the autotuner (timed once
    per configuration and device, then read from its JSON cache)."""
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    key = (tuple(int(v) for v in lengths), int(batch), bool(real_input), bool(graph), dev, bool(tune))
    with _cache_lock:
        p = _plans.get(key)
        if p is None:
            with torch.cuda.device(dev):
                opts = {}
                if tune:
                    from . import autotune
                    opts = autotune.tune_plan(list(key[0]), batch, real_input, objective="both")
                p = _lib.Plan(list(key[0]), batch=batch, real_input=real_input, graph=graph, opts=opts)
            _plans[key] = p
        return p


def clear_plans() -> None:
    with _cache_lock:
        for p in _plans.values():
            p.close()
        _plans.clear()


def _stream_ptr() -> int:
    return torch.cuda.current_stream().cuda_stream


def _check_input(x: torch.Tensor) -> torch.Tensor:
    if not x.is_cuda:
        raise ValueError("mrdft: input must be a CUDA tensor (there is no CPU path)")
    if x.dtype not in (torch.complex64, torch.float32):
        raise TypeError(f"mrdft: input dtype must be complex64 or float32, got {x.dtype}")
    return x.contiguous()


def _log2(n: int) -> int:
    m = int(n).bit_length() - 1
    if n < 2 or (1 << m) != n:
        raise ValueError(f"mrdft: signal length must be a power of two >= 2, got {n}")
    return m


def mrdft(x: torch.Tensor, graph: bool = False) -> torch.Tensor:
    """Forward MrDFT (Eq. 1 of Andreatto & Cariow) of each row of x."""
    x = _check_input(x)
    squeeze = x.dim() == 1
    xb = x.unsqueeze(0) if squeeze else x
    if xb.dim() != 2:
        raise ValueError("mrdft: x must be [N] or [B, N]")
    B, N = xb.shape
    m = _log2(N)
    plan = get_plan([N], B, xb.dtype == torch.float32, graph, xb.device)
    y = torch.empty((B, m, N), dtype=torch.complex64, device=xb.device)
    plan.forward(xb.data_ptr(), y.data_ptr(), _stream_ptr())
    return y[0] if squeeze else y


def mrdft_adjoint(gy: torch.Tensor, graph: bool = False) -> torch.Tensor:
    """Conjugate transpose of Eq. 1: gy [B, m, N] (or [m, N]) -> [B, N] complex64."""
    if not gy.is_cuda or gy.dtype != torch.complex64:
        raise TypeError("mrdft_adjoint: gy must be a complex64 CUDA tensor")
    gy = gy.contiguous()
    squeeze = gy.dim() == 2
    g = gy.unsqueeze(0) if squeeze else gy
    B, m, N = g.shape
    if _log2(N) != m:
        raise ValueError("mrdft_adjoint: gy must have m = log2(N) levels")
    plan = get_plan([N], B, False, graph, g.device)
    gx = torch.empty((B, N), dtype=torch.complex64, device=g.device)
    plan.adjoint(g.data_ptr(), gx.data_ptr(), _stream_ptr())
    return gx[0] if squeeze else gx


def mrdft_loss_grad(x: torch.Tensor, t: torch.Tensor, graph: bool = False):
    """Fused loss and gradient for fitting the level spectra to targets t:
    L = sum_i 2^-i ||Y^(i) - T^(i)||^2 with Y = MrDFT(x).

    x: [B, N] (or [N]) complex64 or float32 CUDA; t: [B, m, N] (or [m, N])
    complex64.  Returns (L as a 0-d float64 CUDA tensor, Y [B, m, N], gx):
    gx is dL/dx* (complex64 [B, N]); for real x the gradient is its real part
    (returned as float32).  The adjoint reads Y and T directly.
    """
    x = _check_input(x)
    squeeze = x.dim() == 1
    xb = x.unsqueeze(0) if squeeze else x
    B, N = xb.shape
    m = _log2(N)
    if not t.is_cuda or t.dtype != torch.complex64:
        raise TypeError("mrdft_loss_grad: t must be a complex64 CUDA tensor")
    tb = (t.unsqueeze(0) if squeeze else t).contiguous()
    if tuple(tb.shape) != (B, m, N):
        raise ValueError(f"mrdft_loss_grad: t must have shape {(B, m, N)}")
    real = xb.dtype == torch.float32
    plan = get_plan([N], B, real, graph, xb.device)
    y = torch.empty((B, m, N), dtype=torch.complex64, device=xb.device)
    gx = torch.empty((B, N), dtype=torch.complex64, device=xb.device)
    loss = torch.zeros((), dtype=torch.float64, device=xb.device)
    plan.loss_grad(xb.data_ptr(), tb.data_ptr(), y.data_ptr(), gx.data_ptr(), loss.data_ptr(), _stream_ptr())
    g = gx.real.contiguous() if real else gx
    if squeeze:
        return loss, y[0], g[0]
    return loss, y, g


def mrdft_ragged(x: torch.Tensor, lengths, graph: bool = False) -> torch.Tensor:
    """Forward MrDFT of signals of uneven power-of-two lengths, concatenated in x.

    Returns the flat complex64 output: signal s contributes m_s * N_s values,
    level-major (level i of signal s at [(i-1) N_s, i N_s) of its block).
    """
    x = _check_input(x).reshape(-1)
    lengths = [int(v) for v in lengths]
    for n in lengths:
        _log2(n)
    if sum(lengths) != x.numel():
        raise ValueError("mrdft_ragged: sum(lengths) must equal x.numel()")
    plan = get_plan(lengths, len(lengths), x.dtype == torch.float32, graph, x.device)
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device=x.device)
    plan.forward(x.data_ptr(), y.data_ptr(), _stream_ptr())
    return y


def mrdft_ragged_adjoint(gy: torch.Tensor, lengths, graph: bool = False) -> torch.Tensor:
    lengths = [int(v) for v in lengths]
    plan = get_plan(lengths, len(lengths), False, graph, gy.device)
    gy = gy.contiguous().reshape(-1)
    if gy.dtype != torch.complex64 or gy.numel() != plan.out_elems:
        raise ValueError("mrdft_ragged_adjoint: gy must be complex64 with sum(m_s N_s) elements")
    gx = torch.empty(plan.in_elems, dtype=torch.complex64, device=gy.device)
    plan.adjoint(gy.data_ptr(), gx.data_ptr(), _stream_ptr())
    return gx


class MrDFT(torch.autograd.Function):
    """Differentiable MrDFT: forward = Eq. 1, backward = its conjugate transpose.

    For a real-valued loss L of the complex output Y, torch passes
    dL/dY* -style gradients (conjugate Wirtinger); the adjoint maps them to the
    input gradient, and for float32 inputs the real part is returned.
    """

    @staticmethod
    def forward(ctx, x: torch.Tensor) -> torch.Tensor:
        ctx.real_input = x.dtype == torch.float32
        return mrdft(x)

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        gx = mrdft_adjoint(gy.contiguous().to(torch.complex64))
        return gx.real.contiguous() if ctx.real_input else gx
