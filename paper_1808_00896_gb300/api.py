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

_DTYPES = {"fp64": capi.SOFT_FP64, "bf16x3": capi.SOFT_MIXED_BF16X3, "tf32": capi.SOFT_MIXED_TF32}


def num_coeffs(B: int) -> int:
    return B * (4 * B * B - 1) // 3


def _stream_ptr(device: torch.device, stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return int(s.cuda_stream)


def _check_tensor(t: torch.Tensor, numel: int, device: torch.device, what: str) -> None:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch.Tensor")
    if t.dtype != torch.complex128:
        raise TypeError(f"{what} must be complex128, got {t.dtype}")
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
