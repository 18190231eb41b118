"""Staged 3D FFT on one GB300 (sm_103a): Python front end of libgbfft.

The transform is the paper's (arxiv 2601.12209) pencil sequence -- batched 1D
FFTs along x, a redistribution, along y, a redistribution, along z
(Section III-A, Algorithm 1) -- or its slab variant, all computed by the
hand-written CUDA kernels of libgbfft.so behind the C ABI of include/gbfft.h.
PyTorch only provides device memory and streams. There is no CPU fallback:
without the built library or a CUDA device every call raises.

    plan = Plan(512, 512, 512)                 # C2C, pencil, persistent launch
    X = plan.forward(x)                        # x: complex64 [nz, ny, nx] on cuda
    x2 = plan.inverse(X)                       # scaled by 1/N
    X = rfftn(x)                               # real [.., nz, ny, nx] -> [.., nz, ny, nx//2+1]
    phi = poisson(f)                           # periodic Poisson solve
    FFT3.apply(x), RFFT3.apply(x), IRFFT3.apply(h, nx), Poisson.apply(f)   # differentiable
"""
from __future__ import annotations

import torch

from . import abi
from .abi import (GBFFT_C2C, GBFFT_R2C, GBFFT_OP_FORWARD, GBFFT_OP_INVERSE, GBFFT_OP_ADJOINT,  # noqa: F401
                  GBFFT_OP_INVERSE_ADJOINT, GbfftError)

__all__ = ["Plan", "ManyPlan", "fftn", "ifftn", "rfftn", "irfftn", "poisson", "FFT3", "RFFT3", "IRFFT3", "Poisson",
           "abi", "GbfftError"]


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _check_tensor(t: torch.Tensor, dtype, shape, what: str):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (no CPU path exists)")
    if t.dtype != dtype:
        raise ValueError(f"{what} must be {dtype}, got {t.dtype}")
    if tuple(t.shape[-3:]) != tuple(shape[-3:]) or t.numel() != int(torch.Size(shape).numel()):
        raise ValueError(f"{what} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")


class Plan:
    """A gbfft plan for `batch` grids of nx x ny x nz (x fastest).

    kind: "c2c" or "r2c"; slab: plane-wise x,y then z (else pencil);
    transposed_out: pencil forward output left as [b][kx][ky][kz];
    staged: one launch per stage instead of the persistent launch;
    tma=False: staged launches load tiles with thread loads instead of tensor copies;
    precision: "fp32", or "fp16_split" / "bf16_split" (c2c only: radix-16 passes
    on the tensor cores with hi/lo operand pairs, warp-level mma.sync; storage stays
    complex64), or "fp16_split_tc5" / "bf16_split_tc5" (the same products as
    tcgen05.mma on the 5th-generation tensor cores, accumulators in tensor memory).
    """

    _PRECISIONS = {"fp32": abi.GBFFT_FP32, "fp16_split": abi.GBFFT_FP16_SPLIT, "bf16_split": abi.GBFFT_BF16_SPLIT,
                   "fp16_split_tc5": abi.GBFFT_FP16_SPLIT_TC5, "bf16_split_tc5": abi.GBFFT_BF16_SPLIT_TC5}

    def __init__(self, nx: int, ny: int, nz: int, kind: str = "c2c", batch: int = 1, slab: bool = False,
                 transposed_out: bool = False, staged: bool = False, debug_timeout: bool = False,
                 cached: bool = False, tma: bool = True, precision: str = "fp32"):
        self.nx, self.ny, self.nz, self.batch = int(nx), int(ny), int(nz), int(batch)
        self.kind = kind
        k = GBFFT_R2C if kind == "r2c" else GBFFT_C2C
        if kind not in ("c2c", "r2c"):
            raise ValueError("kind must be 'c2c' or 'r2c'")
        flags = (abi.GBFFT_SLAB if slab else 0) | (abi.GBFFT_TRANSPOSED_OUT if transposed_out else 0) | \
                (abi.GBFFT_STAGED if staged else 0) | (abi.GBFFT_DEBUG_TIMEOUT if debug_timeout else 0) | \
                (0 if tma else abi.GBFFT_NO_TMA)
        self.flags = flags
        self.transposed_out = transposed_out
        self._cached = cached
        mk = abi.gbfft_plan_get_cached if cached else abi.gbfft_plan_create
        if precision not in self._PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(self._PRECISIONS)}")
        self.precision = precision
        self.handle = mk(self.nx, self.ny, self.nz, k, self._PRECISIONS[precision], self.batch, flags)
        self.nxc = self.nx // 2 + 1 if kind == "r2c" else self.nx
        self._ws = None

    # shapes of the two sides
    def real_shape(self):
        return (self.batch, self.nz, self.ny, self.nx)

    def spectrum_shape(self):
        if self.transposed_out:
            return (self.batch, self.nxc, self.ny, self.nz)
        return (self.batch, self.nz, self.ny, self.nxc)

    def _io(self, op: int):
        """(in dtype, in shape, out dtype, out shape) of an operation."""
        spec = (torch.complex64, self.spectrum_shape())
        if self.kind == "c2c":
            nat = (torch.complex64, (self.batch, self.nz, self.ny, self.nx))
            if op in (GBFFT_OP_FORWARD, GBFFT_OP_INVERSE_ADJOINT):
                return nat + spec
            return spec + nat
        real = (torch.float32, self.real_shape())
        if op in (GBFFT_OP_FORWARD, GBFFT_OP_INVERSE_ADJOINT):
            return real + spec
        if op == abi.GBFFT_OP_POISSON:
            return real + real
        return spec + real

    def exec(self, op: int, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        idt, ishape, odt, oshape = self._io(op)
        _check_tensor(x, idt, ishape, "input")
        if out is None:
            out = torch.empty(oshape, dtype=odt, device=x.device)
            if x.dim() == 3 and self.batch == 1:
                out = out.view(oshape[1:])
        else:
            _check_tensor(out, odt, oshape, "out")
        s = _stream_handle(stream)
        if op == abi.GBFFT_OP_POISSON:
            abi.gbfft_exec_poisson(self.handle, x.data_ptr(), out.data_ptr(), s)
        else:
            abi.gbfft_exec(self.handle, op, x.data_ptr(), out.data_ptr(), s)
        return out

    def forward(self, x, out=None, stream=None):
        return self.exec(GBFFT_OP_FORWARD, x, out, stream)

    def inverse(self, x, out=None, stream=None):
        return self.exec(GBFFT_OP_INVERSE, x, out, stream)

    def adjoint(self, x, out=None, stream=None):
        return self.exec(GBFFT_OP_ADJOINT, x, out, stream)

    def inverse_adjoint(self, x, out=None, stream=None):
        return self.exec(GBFFT_OP_INVERSE_ADJOINT, x, out, stream)

    def r2r_z(self, x, kind: str = "dct", inverse: bool = False, out=None, stream=None):
        """Real-to-real transform along z (kind "dct": DCT-II / DCT-III, "dst": DST-II / DST-III) with
        Fourier x and y: forward takes the forward op's input to its spectrum shape; inverse undoes it."""
        if kind not in ("dct", "dst"):
            raise ValueError("kind must be 'dct' or 'dst'")
        return self.r2r(x, (None, None, kind), inverse, out, stream)

    def r2r(self, x, kinds=(None, None, "dct"), inverse: bool = False, out=None, stream=None):
        """Per-axis transform (axes x, y, z): None = DFT, "dct" = DCT-II / DCT-III, "dst" = DST-II / DST-III."""
        code = {None: abi.GBFFT_R2R_NONE, "dct": abi.GBFFT_R2R_DCT, "dst": abi.GBFFT_R2R_DST}
        if len(kinds) != 3 or any(k not in code for k in kinds):
            raise ValueError("kinds: three of None, 'dct', 'dst'")
        op = abi.GBFFT_OP_INVERSE if inverse else abi.GBFFT_OP_FORWARD
        idt, ishape, odt, oshape = self._io(op)
        _check_tensor(x, idt, ishape, "input")
        if out is None:
            out = torch.empty(oshape, dtype=odt, device=x.device)
            if x.dim() == 3 and self.batch == 1:
                out = out.view(oshape[1:])
        else:
            _check_tensor(out, odt, oshape, "out")
        abi.gbfft_exec_r2r(self.handle, *(code[k] for k in kinds), inverse, x.data_ptr(), out.data_ptr(),
                           _stream_handle(stream))
        return out

    def poisson(self, f, out=None, stream=None, bounded: bool = False):
        """Periodic Poisson solve; bounded=True: z bounded by Neumann walls (cosine expansion)."""
        if self.kind != "r2c":
            raise ValueError("poisson needs an r2c plan")
        if not bounded:
            return self.exec(abi.GBFFT_OP_POISSON, f, out, stream)
        idt, ishape, odt, oshape = self._io(abi.GBFFT_OP_POISSON)
        _check_tensor(f, idt, ishape, "input")
        if out is None:
            out = torch.empty_like(f)
        else:
            _check_tensor(out, odt, oshape, "out")
        abi.gbfft_exec_poisson_bounded(self.handle, f.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def set_host_chunks(self, chunks: int) -> None:
        """exec_host in `chunks` slabs whose copies overlap the first and last stages (1 = plain)."""
        abi.gbfft_plan_set_host_chunks(self.handle, chunks)

    def exec_host(self, op: int, host_in: torch.Tensor, host_out: torch.Tensor) -> torch.Tensor:
        """End-to-end on host tensors (pinned recommended): H2D copy, op, D2H copy, wait."""
        for t in (host_in, host_out):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("exec_host takes contiguous CPU tensors")
        abi.gbfft_exec_host(self.handle, int(op), host_in.data_ptr(), host_out.data_ptr())
        return host_out

    def debug_run(self, step: int, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        for t in (x, out):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("debug_run takes contiguous CUDA tensors")
        abi.gbfft_debug_run(self.handle, int(step), x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def autotune(self, stream=None) -> dict:
        """Time the kernel variants per stage and the persistent launch; keep the fastest."""
        abi.gbfft_plan_autotune(self.handle, _stream_handle(stream))
        return {name: abi.gbfft_plan_get_tuning(self.handle, k)
                for k, name in enumerate(("forward", "inverse", "poisson")) if k < 2 or self.kind == "r2c"}

    def workspace_size(self) -> int:
        return abi.gbfft_workspace_size(self.handle)

    def set_workspace(self, t: torch.Tensor) -> None:
        if not t.is_cuda:
            raise ValueError("workspace must be a CUDA tensor")
        abi.gbfft_set_workspace(self.handle, t.data_ptr(), t.numel() * t.element_size())
        self._ws = t  # keep alive

    def device_error(self) -> int:
        return abi.gbfft_get_device_error(self.handle)

    def close(self):
        if getattr(self, "handle", None) and not self._cached:
            abi.gbfft_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ManyPlan:
    """Many C2C grids of different sizes, transformed by one persistent launch.

    shapes: list of (nx, ny, nz). Data is packed back to back (pack/unpack helpers
    below); exec() runs one launch (capturable in a CUDA graph), exec_separate()
    one plan per grid for comparison.
    """

    def __init__(self, shapes, debug_timeout: bool = False):
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.handle = abi.gbfft_many_create(self.shapes, abi.GBFFT_DEBUG_TIMEOUT if debug_timeout else 0)
        self.offsets = [abi.gbfft_many_layout(self.handle, g)[0] for g in range(len(self.shapes))]
        self.total = abi.gbfft_many_layout(self.handle, 0)[1]

    def empty(self, device="cuda") -> torch.Tensor:
        return torch.zeros(self.total, dtype=torch.complex64, device=device)

    def pack(self, grids, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.empty(grids[0].device) if out is None else out
        for (nx, ny, nz), off, g in zip(self.shapes, self.offsets, grids):
            out[off:off + nx * ny * nz].copy_(g.reshape(-1))
        return out

    def unpack(self, packed: torch.Tensor):
        return [packed[off:off + nx * ny * nz].view(nz, ny, nx) for (nx, ny, nz), off in zip(self.shapes, self.offsets)]

    def exec(self, op: int, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        abi.gbfft_many_exec(self.handle, int(op), x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def exec_staged(self, op: int, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """Three launches, one per stage over all grids (no dependency waits)."""
        abi.gbfft_many_exec_staged(self.handle, int(op), x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def exec_separate(self, op: int, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        abi.gbfft_many_exec_separate(self.handle, int(op), x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def autotune(self, stream=None) -> dict:
        """Pick the tiles per ticket of every axis length for both directions (times the one launch)."""
        abi.gbfft_many_autotune(self.handle, _stream_handle(stream))
        return self.tuning()

    def tuning(self) -> dict:
        out = {}
        for k, name in enumerate(("forward", "inverse")):
            out[name] = abi.gbfft_many_get_tuning(self.handle, k)
            out[name]["lag"] = abi.gbfft_many_get_lag(self.handle, k)
        return out

    def set_lag(self, pipeline: int, lag: int) -> None:
        abi.gbfft_many_set_lag(self.handle, pipeline, lag)

    def set_tuning(self, pipeline: int, teams: dict) -> None:
        abi.gbfft_many_set_tuning(self.handle, pipeline, teams)

    def device_error(self) -> int:
        return abi.gbfft_many_get_device_error(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            abi.gbfft_many_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_plans: dict = {}


def _plan_for(shape, kind: str, slab: bool = False) -> Plan:
    *lead, nz, ny, nx = shape
    batch = 1
    for v in lead:
        batch *= int(v)
    key = (torch.cuda.current_device(), nx, ny, nz, kind, batch, slab)
    p = _plans.get(key)
    if p is None:
        p = Plan(nx, ny, nz, kind=kind, batch=batch, slab=slab, cached=True)
        _plans[key] = p
    return p


def fftn(x: torch.Tensor, slab: bool = False) -> torch.Tensor:
    """Forward C2C 3D FFT over the last three dims (unnormalised, sign -)."""
    p = _plan_for(x.shape, "c2c", slab)
    return p.forward(x.contiguous()).view(x.shape)


def ifftn(x: torch.Tensor, slab: bool = False) -> torch.Tensor:
    """Inverse C2C 3D FFT over the last three dims, scaled by 1/N."""
    p = _plan_for(x.shape, "c2c", slab)
    return p.inverse(x.contiguous()).view(x.shape)


def rfftn(x: torch.Tensor, slab: bool = False) -> torch.Tensor:
    """R2C 3D FFT: real [..., nz, ny, nx] -> complex [..., nz, ny, nx//2+1]."""
    p = _plan_for(x.shape, "r2c", slab)
    return p.forward(x.contiguous()).view(*x.shape[:-1], x.shape[-1] // 2 + 1)


def irfftn(h: torch.Tensor, nx: int, slab: bool = False) -> torch.Tensor:
    """C2R 3D FFT scaled by 1/N: complex [..., nz, ny, nx//2+1] -> real [..., nz, ny, nx]."""
    shape = (*h.shape[:-1], nx)
    p = _plan_for(shape, "r2c", slab)
    return p.inverse(h.contiguous()).view(shape)


def poisson(f: torch.Tensor, slab: bool = False) -> torch.Tensor:
    """Periodic Poisson solve: C2R(-R2C(f)/|k|^2, k=0 -> 0)/N on a 2 pi box."""
    p = _plan_for(f.shape, "r2c", slab)
    return p.poisson(f.contiguous()).view(f.shape)


# ------------------------------------------------------------------ autograd
# Hand-written adjoints: for a linear map y = A x, PyTorch asks for
# A^H grad_y (complex) or A^T grad_y (real-linear maps); libgbfft computes
# them with exec_adjoint / exec_inverse_adjoint, and the Poisson operator is
# symmetric.

class FFT3(torch.autograd.Function):
    """y = fftn(x) (C2C, unnormalised); backward = F^H grad = unscaled inverse."""

    @staticmethod
    def forward(ctx, x):
        ctx.shape = x.shape
        return fftn(x)

    @staticmethod
    def backward(ctx, g):
        p = _plan_for(ctx.shape, "c2c")
        return p.adjoint(g.contiguous()).view(ctx.shape)


class RFFT3(torch.autograd.Function):
    """y = rfftn(x); backward = R^T grad (C2R of grad with interior x-bins halved, unscaled)."""

    @staticmethod
    def forward(ctx, x):
        ctx.shape = x.shape
        return rfftn(x)

    @staticmethod
    def backward(ctx, g):
        p = _plan_for(ctx.shape, "r2c")
        return p.adjoint(g.contiguous()).view(ctx.shape)


class IRFFT3(torch.autograd.Function):
    """x = irfftn(h, nx); backward = (C/N)^T grad (R2C with interior bins doubled, / N)."""

    @staticmethod
    def forward(ctx, h, nx: int):
        ctx.shape = (*h.shape[:-1], int(nx))
        return irfftn(h, nx)

    @staticmethod
    def backward(ctx, g):
        p = _plan_for(ctx.shape, "r2c")
        return p.inverse_adjoint(g.contiguous()).view(*ctx.shape[:-1], ctx.shape[-1] // 2 + 1), None


class Poisson(torch.autograd.Function):
    """phi = poisson(f); the operator is real, symmetric (even multiplier), so backward = poisson(grad)."""

    @staticmethod
    def forward(ctx, f):
        return poisson(f)

    @staticmethod
    def backward(ctx, g):
        return poisson(g.contiguous())
