"""PyTorch-facing wrapper around the C ABI: torch provides device memory and
streams; every step of a transform runs in the CUDA library.

Layouts (see include/soft.h): a grid is a complex128 tensor of shape
(2B, 2B, 2B) indexed [j][i][k] = f(alpha_i, beta_j, gamma_k); coefficients are
a complex128 vector of length B(4B^2-1)/3 in (m, m')-run order.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi

_DTYPES = {"fp64": capi.SOFT_FP64, "bf16x3": capi.SOFT_MIXED_BF16X3, "tf32": capi.SOFT_MIXED_TF32,
           "fp64_tc": capi.SOFT_FP64_TC}


def num_coeffs(B: int) -> int:
    return B * (4 * B * B - 1) // 3


def _stream_ptr(device: torch.device, stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return int(s.cuda_stream)


def _check_tensor(t: torch.Tensor, numel: int, device: torch.device, what: str,
                  dtype: torch.dtype = torch.complex128) -> None:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{what} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{what} must have {numel} elements, got {t.numel()}")


class Plan:
    """A transform plan for bandwidth B on one CUDA device (soft_plan_create)."""

    def __init__(self, B: int, dtype: str = "fp64", device=None):
        if dtype not in _DTYPES:
            raise ValueError(f"dtype must be one of {sorted(_DTYPES)}")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.device.type != "cuda":
            raise ValueError("Plan needs a CUDA device")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.B = int(B)
        self.dtype = dtype
        self.n = 2 * self.B
        self.ncoef = num_coeffs(self.B)
        with torch.cuda.device(self.device):
            self._h = capi.soft_plan_create(self.B, _DTYPES[dtype])

    # -- lifetime -----------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None):
            capi.soft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        if not self._h:
            raise RuntimeError("plan is closed")
        return self._h

    def sync(self) -> None:
        capi.soft_plan_sync(self.handle)

    def tune(self, reps: int = 3, use_cache: bool = True) -> dict:
        """Pick the fastest DWT / iDWT tile shapes for this plan (cached per GPU, B, mode)."""
        from . import autotune
        return autotune.tune(self, reps=reps, use_cache=use_cache)

    def set_variant(self, kernel: int, variant: int) -> None:
        """Select tile-shape variant `variant` of kernel 0 (DWT) or 1 (iDWT)."""
        capi.check(capi.load().soft_plan_set_variant(self.handle, kernel, variant), "soft_plan_set_variant")

    def num_variants(self, kernel: int) -> int:
        return capi.load().soft_plan_num_variants(self.handle, kernel)

    # -- allocation helpers ---------------------------------------------------
    def empty_grid(self) -> torch.Tensor:
        return torch.empty((self.n,) * 3, dtype=torch.complex128, device=self.device)

    def empty_coef(self) -> torch.Tensor:
        return torch.empty(self.ncoef, dtype=torch.complex128, device=self.device)

    # -- transforms ------------------------------------------------------------
    def forward(self, grid: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """FSOFT: grid (2B,2B,2B) -> coefficients (soft_forward)."""
        _check_tensor(grid, self.n ** 3, self.device, "grid")
        out = self.empty_coef() if out is None else out
        _check_tensor(out, self.ncoef, self.device, "out")
        capi.check(capi.soft_forward(self.handle, grid.data_ptr(), out.data_ptr(), _stream_ptr(self.device, stream)),
                   "soft_forward")
        return out

    def inverse(self, coef: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """iFSOFT: coefficients -> grid (2B,2B,2B) (soft_inverse)."""
        _check_tensor(coef, self.ncoef, self.device, "coef")
        out = self.empty_grid() if out is None else out
        _check_tensor(out, self.n ** 3, self.device, "out")
        capi.check(capi.soft_inverse(self.handle, coef.data_ptr(), out.data_ptr(), _stream_ptr(self.device, stream)),
                   "soft_inverse")
        return out

    def forward_real(self, grid: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """FSOFT of a real grid: float64 (2B,2B,2B) -> complex coefficients (soft_forward_real).
        FP64 and FP64-TC plans with power-of-two 2B."""
        _check_tensor(grid, self.n ** 3, self.device, "grid", torch.float64)
        out = self.empty_coef() if out is None else out
        _check_tensor(out, self.ncoef, self.device, "out")
        capi.check(capi.soft_forward_real(self.handle, grid.data_ptr(), out.data_ptr(),
                                          _stream_ptr(self.device, stream)), "soft_forward_real")
        return out

    def inverse_real(self, coef: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """iFSOFT to a real grid: coefficients of a real function -> float64 (2B,2B,2B)
        (soft_inverse_real; reads one partner of each conjugate pair)."""
        _check_tensor(coef, self.ncoef, self.device, "coef")
        out = torch.empty((self.n,) * 3, dtype=torch.float64, device=self.device) if out is None else out
        _check_tensor(out, self.n ** 3, self.device, "out", torch.float64)
        capi.check(capi.soft_inverse_real(self.handle, coef.data_ptr(), out.data_ptr(),
                                          _stream_ptr(self.device, stream)), "soft_inverse_real")
        return out

    def forward_adjoint(self, coef: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Adjoint of ``forward``: coefficients -> grid (soft_forward_adjoint)."""
        _check_tensor(coef, self.ncoef, self.device, "coef")
        out = self.empty_grid() if out is None else out
        _check_tensor(out, self.n ** 3, self.device, "out")
        capi.check(capi.soft_forward_adjoint(self.handle, coef.data_ptr(), out.data_ptr(),
                                             _stream_ptr(self.device, stream)), "soft_forward_adjoint")
        return out

    def inverse_adjoint(self, grid: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Adjoint of ``inverse``: grid -> coefficients (soft_inverse_adjoint)."""
        _check_tensor(grid, self.n ** 3, self.device, "grid")
        out = self.empty_coef() if out is None else out
        _check_tensor(out, self.ncoef, self.device, "out")
        capi.check(capi.soft_inverse_adjoint(self.handle, grid.data_ptr(), out.data_ptr(),
                                             _stream_ptr(self.device, stream)), "soft_inverse_adjoint")
        return out

    def correlation_coeffs(self, f_sh: torch.Tensor, g_sh: torch.Tensor, out: torch.Tensor | None = None,
                           stream=None) -> torch.Tensor:
        """c(l,m,m') = g_lm conj(f_lm') (soft_correlation_coeffs); f_sh, g_sh: B^2 complex128."""
        _check_tensor(f_sh, self.B * self.B, self.device, "f_sh")
        _check_tensor(g_sh, self.B * self.B, self.device, "g_sh")
        out = self.empty_coef() if out is None else out
        _check_tensor(out, self.ncoef, self.device, "out")
        capi.check(capi.load().soft_correlation_coeffs(self.handle, f_sh.data_ptr(), g_sh.data_ptr(), out.data_ptr(),
                                                       _stream_ptr(self.device, stream)), "soft_correlation_coeffs")
        return out

    def correlate(self, f_sh: torch.Tensor, g_sh: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """C(R) on the Euler grid and the arg-max of Re C (soft_correlate).
        Returns (grid, best_index tensor, best_value tensor), all on the device."""
        _check_tensor(f_sh, self.B * self.B, self.device, "f_sh")
        _check_tensor(g_sh, self.B * self.B, self.device, "g_sh")
        out = self.empty_grid() if out is None else out
        _check_tensor(out, self.n ** 3, self.device, "out")
        idx = torch.empty(1, dtype=torch.int64, device=self.device)
        val = torch.empty(1, dtype=torch.float64, device=self.device)
        capi.check(capi.load().soft_correlate(self.handle, f_sh.data_ptr(), g_sh.data_ptr(), out.data_ptr(),
                                              idx.data_ptr(), val.data_ptr(), _stream_ptr(self.device, stream)),
                   "soft_correlate")
        return out, idx, val

    def dwt_forward(self, S: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """DWT step only: S[j][m mod 2B][m' mod 2B] -> coefficients (soft_dwt_forward)."""
        _check_tensor(S, self.n ** 3, self.device, "S")
        out = self.empty_coef() if out is None else out
        _check_tensor(out, self.ncoef, self.device, "out")
        capi.check(capi.soft_dwt_forward(self.handle, S.data_ptr(), out.data_ptr(), _stream_ptr(self.device, stream)),
                   "soft_dwt_forward")
        return out

    def dwt_inverse(self, coef: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """iDWT step only: coefficients -> S (soft_dwt_inverse)."""
        _check_tensor(coef, self.ncoef, self.device, "coef")
        out = self.empty_grid() if out is None else out
        _check_tensor(out, self.n ** 3, self.device, "out")
        capi.check(capi.soft_dwt_inverse(self.handle, coef.data_ptr(), out.data_ptr(), _stream_ptr(self.device, stream)),
                   "soft_dwt_inverse")
        return out

    def forward_host(self, grid: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
        """FSOFT on host buffers (soft_forward_host): copies in, transforms, copies out."""
        g = np.ascontiguousarray(grid, dtype=np.complex128)
        if g.size != self.n ** 3:
            raise ValueError("grid has the wrong size")
        out = np.empty(self.ncoef, dtype=np.complex128) if out is None else out
        with torch.cuda.device(self.device):
            capi.check(capi.soft_forward_host(self.handle, g.ctypes.data, out.ctypes.data,
                                              _stream_ptr(self.device)), "soft_forward_host")
        return out

    def inverse_host(self, coef: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
        """iFSOFT on host buffers (soft_inverse_host)."""
        c = np.ascontiguousarray(coef, dtype=np.complex128)
        if c.size != self.ncoef:
            raise ValueError("coef has the wrong size")
        out = np.empty((self.n,) * 3, dtype=np.complex128) if out is None else out
        with torch.cuda.device(self.device):
            capi.check(capi.soft_inverse_host(self.handle, c.ctypes.data, out.ctypes.data,
                                              _stream_ptr(self.device)), "soft_inverse_host")
        return out


class _SoftForwardFn(torch.autograd.Function):
    """grid -> coefficients; backward applies the adjoint E^H W T^T V."""

    @staticmethod
    def forward(ctx, grid, plan):
        ctx.plan = plan
        ctx.shape = grid.shape
        return plan.forward(grid.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.forward_adjoint(g.contiguous()).reshape(ctx.shape), None


class _SoftInverseFn(torch.autograd.Function):
    """coefficients -> grid; backward applies the adjoint T E."""

    @staticmethod
    def forward(ctx, coef, plan):
        ctx.plan = plan
        ctx.shape = coef.shape
        return plan.inverse(coef.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.inverse_adjoint(g.contiguous()).reshape(ctx.shape), None


def soft_forward(grid: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable forward transform (complex128 grid of shape (2B,)*3)."""
    return _SoftForwardFn.apply(grid, plan)


def soft_inverse(coef: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable inverse transform (complex128 coefficient vector)."""
    return _SoftInverseFn.apply(coef, plan)


def _ptr_array(ts):
    import ctypes
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def _plan_array(plans):
    import ctypes
    return (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])


def _same_device(plans):
    dev = plans[0].device
    if any(p.device != dev for p in plans):
        raise ValueError("all plans of a batch must be on one device")
    return dev


def batched_inverse(plans, coefs, grids=None, stream=None):
    """Inverse transforms of a batch (soft_batched_inverse), one distinct plan per entry."""
    dev = _same_device(plans)
    grids = [p.empty_grid() for p in plans] if grids is None else grids
    for p, c, g in zip(plans, coefs, grids):
        _check_tensor(c, p.ncoef, dev, "coef")
        _check_tensor(g, p.n ** 3, dev, "grid")
    capi.check(capi.load().soft_batched_inverse(len(plans), _plan_array(plans), _ptr_array(coefs), _ptr_array(grids),
                                                _stream_ptr(dev, stream)), "soft_batched_inverse")
    return grids


def batched_forward(plans, grids, coefs=None, stream=None):
    """Forward transforms of a batch (soft_batched_forward)."""
    dev = _same_device(plans)
    coefs = [p.empty_coef() for p in plans] if coefs is None else coefs
    for p, g, c in zip(plans, grids, coefs):
        _check_tensor(g, p.n ** 3, dev, "grid")
        _check_tensor(c, p.ncoef, dev, "coef")
    capi.check(capi.load().soft_batched_forward(len(plans), _plan_array(plans), _ptr_array(grids), _ptr_array(coefs),
                                                _stream_ptr(dev, stream)), "soft_batched_forward")
    return coefs


def batched_correlate(plans, f_shs, g_shs, grids=None, best_index=None, best_value=None, stream=None):
    """Rotational correlations of a batch (soft_batched_correlate).
    Returns (grids, best_index (n,) int64, best_value (n,) float64) on the device."""
    dev = _same_device(plans)
    n = len(plans)
    grids = [p.empty_grid() for p in plans] if grids is None else grids
    best_index = torch.empty(n, dtype=torch.int64, device=dev) if best_index is None else best_index
    best_value = torch.empty(n, dtype=torch.float64, device=dev) if best_value is None else best_value
    for p, f, g, gr in zip(plans, f_shs, g_shs, grids):
        _check_tensor(f, p.B * p.B, dev, "f_sh")
        _check_tensor(g, p.B * p.B, dev, "g_sh")
        _check_tensor(gr, p.n ** 3, dev, "grid")
    capi.check(capi.load().soft_batched_correlate(n, _plan_array(plans), _ptr_array(f_shs), _ptr_array(g_shs),
                                                  _ptr_array(grids), best_index.data_ptr(), best_value.data_ptr(),
                                                  _stream_ptr(dev, stream)), "soft_batched_correlate")
    return grids, best_index, best_value
