"""Seeded synthetic inputs for the staged 3D FFT.

This module is the only code shared between the FP64 oracle's tests and the
CUDA path's tests and benchmark. It draws random numbers and builds input
grids; it contains none of the transform's arithmetic (no DFT, no twiddle, no
layout permutation).

Every generator draws in float64 on the CPU from ``torch.Generator`` seeded by
the caller, then rounds once to the storage precision. The oracle consumes the
rounded values upcast to float64, so both sides see bit-identical inputs.

Workload recipes (the paper's workloads are synthetic grids of unstated
content, Section VI):
  * complex grids: real and imaginary parts i.i.d. uniform[-1, 1];
  * real grids: i.i.d. N(0, 1);
  * Poisson right-hand side: 32 periodic Gaussian blobs, mean removed;
  * batched grids: each axis drawn from {32,48,60,64,80,96,120,128,160,192,256};
  * precision grids: uniform[-1,1] noise plus 16 integer-wavenumber plane waves.
"""
from __future__ import annotations

import math

import numpy as np
import torch

BATCH_AXIS_SIZES = (32, 48, 60, 64, 80, 96, 120, 128, 160, 192, 256)


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def uniform_complex(shape, seed: int) -> torch.Tensor:
    """complex64 tensor with Re, Im i.i.d. uniform[-1, 1] (drawn in fp64)."""
    g = _gen(seed)
    shape = tuple(int(s) for s in shape)
    re = torch.rand(shape, generator=g, dtype=torch.float64) * 2.0 - 1.0
    im = torch.rand(shape, generator=g, dtype=torch.float64) * 2.0 - 1.0
    return torch.complex(re.float(), im.float())


def normal_real(shape, seed: int) -> torch.Tensor:
    """float32 tensor with i.i.d. N(0, 1) entries (drawn in fp64)."""
    g = _gen(seed)
    shape = tuple(int(s) for s in shape)
    return torch.randn(shape, generator=g, dtype=torch.float64).float()


def integer_complex(shape, seed: int, lo: int = -1000, hi: int = 1000) -> torch.Tensor:
    """complex64 tensor with small distinct-looking integer parts.

    Used by the bit-exact layout tests: every value is exactly representable,
    so any index mix-up shows as a changed bit pattern.
    """
    g = _gen(seed)
    shape = tuple(int(s) for s in shape)
    re = torch.randint(lo, hi, shape, generator=g, dtype=torch.int64).float()
    im = torch.randint(lo, hi, shape, generator=g, dtype=torch.int64).float()
    return torch.complex(re, im)


def poisson_rhs(n: int, seed: int, n_blobs: int = 32) -> tuple[torch.Tensor, dict]:
    """Right-hand side f on an n^3 periodic grid: sum of Gaussian blobs, mean removed.

    Blob b has centre c_b ~ U[0, n)^3 (cells), width sigma_b ~ U[2, 8] cells,
    amplitude A_b ~ N(0, 1); the distance is the periodic minimum-image one.
    Returns the float32 grid [z][y][x] and the blob parameters.
    """
    g = _gen(seed)
    centres = torch.rand((n_blobs, 3), generator=g, dtype=torch.float64) * n
    sigmas = torch.rand((n_blobs,), generator=g, dtype=torch.float64) * 6.0 + 2.0
    amps = torch.randn((n_blobs,), generator=g, dtype=torch.float64)
    idx = torch.arange(n, dtype=torch.float64)
    f = torch.zeros((n, n, n), dtype=torch.float64)
    for b in range(n_blobs):
        cx, cy, cz = (float(v) for v in centres[b])
        def per(d):
            d = torch.remainder(d + n / 2.0, float(n)) - n / 2.0
            return d * d
        dx2 = per(idx - cx)
        dy2 = per(idx - cy)
        dz2 = per(idx - cz)
        s2 = 2.0 * float(sigmas[b]) ** 2
        gx = torch.exp(-dx2 / s2)
        gy = torch.exp(-dy2 / s2)
        gz = torch.exp(-dz2 / s2)
        f += float(amps[b]) * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    f -= f.mean()
    params = {"centres": centres.numpy(), "sigmas": sigmas.numpy(), "amps": amps.numpy()}
    return f.float(), params


def batched_sizes(count: int, seed: int, choices=BATCH_AXIS_SIZES) -> list[tuple[int, int, int]]:
    """`count` grid shapes (nx, ny, nz), each axis drawn independently from `choices`."""
    g = _gen(seed)
    idx = torch.randint(0, len(choices), (count, 3), generator=g)
    return [tuple(int(choices[int(i)]) for i in row) for row in idx]


def batched_grids(count: int, seed: int) -> tuple[list[tuple[int, int, int]], list[torch.Tensor]]:
    """Shapes from `batched_sizes` and one uniform complex grid [nz][ny][nx] per shape."""
    shapes = batched_sizes(count, seed)
    grids = [uniform_complex((nz, ny, nx), seed * 1000 + i) for i, (nx, ny, nz) in enumerate(shapes)]
    return shapes, grids


def plane_wave_spec(n: int, seed: int, count: int = 16) -> tuple[np.ndarray, np.ndarray]:
    """`count` distinct integer wavevectors k_m in [0, n)^3 and amplitudes a_m.

    |a_m| = (m + 1) / 4 with a uniformly random phase.
    Returns (k: int64 [count, 3] as (kx, ky, kz), a: complex128 [count]).
    """
    g = _gen(seed)
    ks: list[tuple[int, int, int]] = []
    while len(ks) < count:
        k = tuple(int(v) for v in torch.randint(0, n, (3,), generator=g))
        if k not in ks:
            ks.append(k)
    phases = torch.rand((count,), generator=g, dtype=torch.float64) * 2.0 * math.pi
    mags = (torch.arange(count, dtype=torch.float64) + 1.0) / 4.0
    a = (mags * torch.cos(phases)).numpy() + 1j * (mags * torch.sin(phases)).numpy()
    return np.asarray(ks, dtype=np.int64), a.astype(np.complex128)


def uniform_complex_slabs(shape, seed: int, planes: int = 64) -> torch.Tensor:
    """complex64 grid [nz][ny][nx] with Re, Im i.i.d. uniform[-1, 1], drawn slab by slab.

    Slab s (z-planes [s*planes, (s+1)*planes)) draws Re then Im in fp64 from a
    generator seeded with seed * 1_000_003 + s, so a 2^30-point grid never
    needs an fp64 copy of the whole grid.
    """
    nz, ny, nx = (int(s) for s in shape)
    out = torch.empty((nz, ny, nx), dtype=torch.complex64)
    view = torch.view_as_real(out)
    for s, z0 in enumerate(range(0, nz, planes)):
        z1 = min(nz, z0 + planes)
        g = _gen(int(seed) * 1_000_003 + s)
        view[z0:z1, ..., 0] = (torch.rand((z1 - z0, ny, nx), generator=g, dtype=torch.float64) * 2.0 - 1.0).float()
        view[z0:z1, ..., 1] = (torch.rand((z1 - z0, ny, nx), generator=g, dtype=torch.float64) * 2.0 - 1.0).float()
    return out


def add_plane_waves(grid: torch.Tensor, ks: np.ndarray, amps: np.ndarray, planes: int = 64) -> torch.Tensor:
    """Add the input signal sum_m a_m exp(+2 pi i (kx x + ky y + kz z) / n) to a cubic
    complex64 grid [n][n][n] in place (on the grid's device).

    Each wave is built in fp64 from its integer phase (k . r) mod n, as the
    product of its three 1D factors, and rounded once into the grid. Its 3D DFT
    is n^3 a_m at bin k_m and zero elsewhere (up to the grid's rounding).
    """
    n = grid.shape[-1]
    assert grid.shape == (n, n, n) and grid.dtype == torch.complex64
    dev = grid.device
    r = torch.arange(n, dtype=torch.int64, device=dev)

    def factor(k):
        ang = ((int(k) * r) % n).to(torch.float64) * (2.0 * math.pi / n)
        return torch.complex(torch.cos(ang), torch.sin(ang))

    for z0 in range(0, n, planes):
        z1 = min(n, z0 + planes)
        acc = torch.zeros((z1 - z0, n, n), dtype=torch.complex128, device=dev)
        for (kx, ky, kz), a in zip(np.asarray(ks).tolist(), np.asarray(amps).tolist()):
            ex, ey, ez = factor(kx), factor(ky), factor(kz)[z0:z1]
            acc += (complex(a) * ez)[:, None, None] * ey[None, :, None] * ex[None, None, :]
        grid[z0:z1] += acc.to(torch.complex64)
    return grid
