"""``FlycooTensor``: an owning Python handle over the C ABI.

It only holds the handle and forwards calls; each method is one C call (or
one per mode for ``all_modes``).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _native as nat


def _as_cuda(x, dtype) -> torch.Tensor:
    if isinstance(x, np.ndarray):
        if dtype == torch.int32 and x.dtype == np.uint32:
            x = x.view(np.int32)
        x = torch.from_numpy(np.ascontiguousarray(x))
    return x.to(device="cuda", dtype=dtype).contiguous()


class FlycooTensor:
    """A sparse tensor in the FLYCOO format on the current CUDA device.

    ``idx``: [N, nnz] coordinates (uint32/int32, numpy or torch), ``vals``:
    [nnz] float32, ``dims``: mode sizes.  ``m``, ``g``, ``bins`` are the
    partition parameters of ``flycoo_params`` (0 = default); ``schedule``
    is ``SCHEDULE_LPT`` (Algorithm 3, the default) or
    ``SCHEDULE_BLOCK_CYCLIC``; ``order`` is ``ORDER_KEY`` (the default) or
    ``ORDER_MORTON`` (Z-Morton order inside the super-shards).
    """

    def __init__(self, idx, vals, dims: Sequence[int], m: Optional[Sequence[int]] = None, g: int = 0,
                 bins: int = 0, stream=None, schedule: int = 0, order: int = 0):
        idx_t = _as_cuda(idx, torch.int32)
        vals_t = _as_cuda(vals, torch.float32)
        self.N = int(idx_t.shape[0])
        self.nnz = int(idx_t.shape[1])
        self.dims = [int(d) for d in dims]
        self.h = None
        self.h = nat.flycoo_create(self.N, self.dims, self.nnz, idx_t, vals_t,
                                   nat.make_params(m, g, bins, schedule, order), stream)

    def close(self):
        if self.h:
            nat.flycoo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ info
    @property
    def info(self) -> dict:
        return nat.flycoo_get_info(self.h)

    @property
    def layout_mode(self) -> int:
        return self.info["layout_mode"]

    # --------------------------------------------------------------- compute
    def spmttkrp(self, mode: int, factors: Sequence[Optional[torch.Tensor]], out: Optional[torch.Tensor] = None,
                 remap: bool = True, stream=None) -> torch.Tensor:
        """spMTTKRP of ``mode``; with ``remap`` the tensor moves to the next
        mode's layout in the same pass.  Remaps first if it is elsewhere."""
        R = next(f.shape[1] for w, f in enumerate(factors) if w != mode and f is not None)
        if out is None:
            out = torch.empty((self.dims[mode], R), dtype=torch.float32, device="cuda")
        if self.layout_mode != mode:
            nat.flycoo_remap(self.h, mode, stream)
        nat.flycoo_spmttkrp(self.h, mode, factors, out, (mode + 1) % self.N if remap else -1, stream)
        return out

    def all_modes(self, factors: Sequence[torch.Tensor], outs: Optional[List[torch.Tensor]] = None,
                  stream=None) -> List[torch.Tensor]:
        """spMTTKRP of modes 0..N-1 in turn, each fused with the remap to the
        next mode (Algorithm 2); the tensor ends in layout L_0 again."""
        if self.layout_mode != 0:
            nat.flycoo_remap(self.h, 0, stream)
        R = factors[0].shape[1]
        if outs is None:
            outs = [torch.empty((d, R), dtype=torch.float32, device="cuda") for d in self.dims]
        for n in range(self.N):
            nat.flycoo_spmttkrp(self.h, n, factors, outs[n], (n + 1) % self.N, stream)
        return outs

    def cp_als_step(self, factors: Sequence[torch.Tensor], lam: Optional[torch.Tensor] = None,
                    stream=None):
        """One CP-ALS iteration (Algorithm 1 with the least-squares update),
        factors updated in place; returns ``(lambda, fit)``."""
        R = factors[0].shape[1]
        if lam is None:
            lam = torch.empty(R, dtype=torch.float64, device=factors[0].device)
        fit = nat.flycoo_cp_als_step(self.h, factors, lam, stream)
        return lam, fit

    def cp_als(self, factors: Sequence[torch.Tensor], iters: int, tol: float = 0.0, stream=None):
        """CP-ALS iterations until ``iters`` are done or the fit changes by
        less than ``tol``; returns ``(lambda, fits)``.  Without a tolerance
        the iterations run in one library call."""
        R = factors[0].shape[1]
        if tol <= 0.0:
            lam = torch.empty(R, dtype=torch.float64, device=factors[0].device)
            return lam, nat.flycoo_cp_als(self.h, factors, lam, iters, stream)
        fits: List[float] = []
        lam = None
        for _ in range(iters):
            lam, fit = self.cp_als_step(factors, lam, stream)
            fits.append(fit)
            if len(fits) > 1 and abs(fits[-1] - fits[-2]) < tol:
                break
        return lam, fits

    def cp_als_state(self, factors: Sequence[torch.Tensor], lam: Optional[torch.Tensor], fits: List[float]) -> dict:
        """Everything needed to resume CP-ALS: the factors, lambda, the fits so
        far and the layout the tensor is in (a handle rebuilt from the same COO
        input has the same layouts, so resuming is bitwise identical)."""
        return {"factors": [f.detach().cpu().clone() for f in factors],
                "lambda": None if lam is None else lam.detach().cpu().clone(),
                "fits": list(fits), "iteration": len(fits), "layout_mode": self.layout_mode,
                "dims": list(self.dims), "nnz": self.nnz}

    @staticmethod
    def save_cp_als_state(path: str, state: dict) -> None:
        torch.save(state, path)

    @staticmethod
    def load_cp_als_state(path: str, device="cuda"):
        """Returns ``(factors on device, lambda on device or None, fits)``."""
        state = torch.load(path, map_location="cpu")
        facs = [f.to(device).contiguous() for f in state["factors"]]
        lam = None if state["lambda"] is None else state["lambda"].to(device)
        return facs, lam, list(state["fits"])

    def remap(self, next_mode: int, stream=None) -> None:
        nat.flycoo_remap(self.h, next_mode, stream)

    # --------------------------------------------------------------- exports
    def export_layout(self, stream=None):
        return nat.flycoo_export_layout(self.h, stream)

    def export_partition(self, mode: int):
        return nat.flycoo_export_partition(self.h, mode)

    def export_schedule(self, mode: int, which: int):
        return nat.flycoo_export_schedule(self.h, mode, which)

    def export_next(self, mode: int, stream=None) -> torch.Tensor:
        return nat.flycoo_export_next(self.h, mode, stream)

    def export_tile_order(self, mode: int, stage: int, stream=None) -> torch.Tensor:
        return nat.flycoo_export_tile_order(self.h, mode, stage, stream)

    # ---------------------------------------------------------------- timing
    def timing_enable(self, enable: bool = True) -> None:
        nat.flycoo_timing_enable(self.h, enable)

    def timing_read(self):
        return nat.flycoo_timing_read(self.h)
