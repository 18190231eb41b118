"""FP64 CPU oracle for the staged 3D FFT -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA library
(``paper_2601_12209_gb300``) and imports nothing from it.

Contents, each citing the passage it follows:
  * ``fft3`` / ``ifft3``: the 3D DFT of Section III-A evaluated separably, x then
    y then z (Section III-A list; Algorithm 1), by the C library
    ``fft_oracle.c`` (recursive mixed-radix FFT, or the naive DFT).
  * ``rfft3`` / ``irfft3``: real-to-complex transforms (Section V-B: R2C exploits
    Hermitian symmetry). R2C keeps the first nx/2+1 x-bins; C2R projects the
    kx = 0 and kx = nx/2 planes onto their Hermitian part first (a reading:
    the paper does not define C2R on non-Hermitian input).
  * adjoints of the four linear maps, written from their definitions (not in
    the paper; they serve the differentiation direction of the project).
  * ``poisson``: the periodic FFT Poisson solve of Section VI-B restricted to
    the (Periodic, Periodic, Periodic) topology.
  * ``layout_*``: the stage layouts A -> B -> C -> natural, each an explicit
    integer index map (Algorithm 1's distributions D1/D2/D3 made concrete).
  * ``dft_matrix`` / ``dft3_naive``: pure numpy naive DFT for tiny grids.

Arrays are numpy, row-major [..., z, y, x] (x fastest). All arithmetic is FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle-" + __import__("platform").machine() + ".so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (plain C99, no host-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            D = ctypes.POINTER(ctypes.c_double)
            L = ctypes.c_long
            I = ctypes.c_int
            lib.oracle_fft1d.argtypes = [D, L, L, I, I, I]
            lib.oracle_fft3d.argtypes = [D, L, L, L, L, I, I, I, I]
            lib.oracle_rfft3d.argtypes = [D, D, L, L, L, L, I]
            lib.oracle_irfft3d.argtypes = [D, D, L, L, L, L, I]
            lib.oracle_dft3d_bins.argtypes = [D, L, L, L, ctypes.POINTER(ctypes.c_long), L, I, D]
            lib.oracle_dft3d_bins_c64.argtypes = [ctypes.POINTER(ctypes.c_float), L, L, L,
                                                  ctypes.POINTER(ctypes.c_long), L, I, D, I]
            for f in ("oracle_fft1d", "oracle_fft3d", "oracle_rfft3d", "oracle_irfft3d",
                      "oracle_dft3d_bins", "oracle_dft3d_bins_c64"):
                getattr(lib, f).restype = ctypes.c_int
            lib.oracle_name.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_c128(x) -> np.ndarray:
    if hasattr(x, "detach"):  # torch tensor -> numpy without importing torch here
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _as_f64(x) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed (rc={rc})")


def _split3(shape):
    if len(shape) < 3:
        raise ValueError("need at least 3 dims [..., z, y, x]")
    nz, ny, nx = shape[-3:]
    batch = int(np.prod(shape[:-3])) if len(shape) > 3 else 1
    return nx, ny, nz, batch


# ----------------------------------------------------------------- 1D / 3D C2C

def fft1(x, sign: int = -1, naive: bool = False, threads: int | None = None) -> np.ndarray:
    """Unscaled 1D DFT along the last axis: y[k] = sum_j x[j] exp(sign 2 pi i jk/n)."""
    a = _as_c128(x).copy()
    n = a.shape[-1]
    count = a.size // n if n else 0
    _check(_load().oracle_fft1d(_dptr(a), n, count, int(sign), int(naive), threads or default_threads()),
           "fft1d")
    return a


def fft3(x, sign: int = -1, naive: bool = False, order: int = 0, threads: int | None = None) -> np.ndarray:
    """Unscaled 3D DFT of Section III-A over the last three axes (x, then y, then z)."""
    a = _as_c128(x).copy()
    nx, ny, nz, batch = _split3(a.shape)
    _check(_load().oracle_fft3d(_dptr(a), nx, ny, nz, batch, int(sign), int(naive), int(order),
                                threads or default_threads()), "fft3d")
    return a


def ifft3(x, threads: int | None = None) -> np.ndarray:
    """Inverse 3D DFT, sign +, scaled by 1/N so that ifft3(fft3(x)) = x."""
    a = fft3(x, sign=+1, threads=threads)
    nx, ny, nz, _ = _split3(a.shape)
    return a / float(nx * ny * nz)


# ------------------------------------------------------------------- R2C / C2R

def rfft3(x, threads: int | None = None) -> np.ndarray:
    """R2C: the first nx//2+1 x-bins of fft3 of the real input (x is the halved axis)."""
    a = _as_f64(x)
    nx, ny, nz, batch = _split3(a.shape)
    out = np.empty(a.shape[:-1] + (nx // 2 + 1,), dtype=np.complex128)
    _check(_load().oracle_rfft3d(_dptr(a), _dptr(out), nx, ny, nz, batch, threads or default_threads()),
           "rfft3d")
    return out


def c2r_unscaled(h, nx: int, threads: int | None = None) -> np.ndarray:
    """Unscaled C2R: real part of the inverse DFT of the Hermitian-completed spectrum.

    The kx = 0 and kx = nx/2 planes are first replaced by their Hermitian part
    (h(ky,kz) + conj(h(-ky,-kz)))/2.
    """
    a = _as_c128(h)
    if a.shape[-1] != nx // 2 + 1:
        raise ValueError("last axis must be nx//2+1")
    _, ny, nz, batch = _split3(a.shape)
    out = np.empty(a.shape[:-1] + (nx,), dtype=np.float64)
    _check(_load().oracle_irfft3d(_dptr(a), _dptr(out), nx, ny, nz, batch, threads or default_threads()),
           "irfft3d")
    return out


def irfft3(h, nx: int, threads: int | None = None) -> np.ndarray:
    """C2R inverse, scaled by 1/N: irfft3(rfft3(x), nx) = x."""
    out = c2r_unscaled(h, nx, threads=threads)
    ny, nz = out.shape[-2], out.shape[-3]
    return out / float(nx * ny * nz)


# -------------------------------------------------------------------- adjoints
# Each map is real-linear; the adjoint is taken for the real inner product
# <a, b> = Re sum conj(a) b. Not in the paper: derived here from the definitions.

def c2c_adjoint(y, threads: int | None = None) -> np.ndarray:
    """F^H y: conjugate transpose of the unscaled forward DFT (sign +, no 1/N)."""
    return fft3(y, sign=+1, threads=threads)


def c2c_inverse_adjoint(y, threads: int | None = None) -> np.ndarray:
    """(F^-1)^H y = F y / N."""
    a = fft3(y, sign=-1, threads=threads)
    nx, ny, nz, _ = _split3(a.shape)
    return a / float(nx * ny * nz)


def r2c_adjoint(g, nx: int, threads: int | None = None) -> np.ndarray:
    """R^T g for R = rfft3: Re(F^H P^T g), P^T zero-pads the half spectrum to nx bins."""
    a = _as_c128(g)
    full = np.zeros(a.shape[:-1] + (nx,), dtype=np.complex128)
    full[..., : nx // 2 + 1] = a
    return np.ascontiguousarray(fft3(full, sign=+1, threads=threads).real)


def c2r_adjoint(y, threads: int | None = None) -> np.ndarray:
    """C^T y for C = c2r_unscaled: H^T F y, H the Hermitian completion with projection.

    H^T Y[k] = Y[k] + conj(Y[-k]) for 0 < kx < nx/2, and (Y[k] + conj(Y[-k]))/2
    on the kx = 0 and kx = nx/2 planes.
    """
    r = _as_f64(y)
    nx = r.shape[-1]
    Y = fft3(r.astype(np.complex128), sign=-1, threads=threads)
    # Y[-k]: index (-kz, -ky, -kx) mod n
    Ym = np.roll(np.flip(Y, axis=(-3, -2, -1)), shift=(1, 1, 1), axis=(-3, -2, -1))
    M = nx // 2
    half = np.empty(Y.shape[:-1] + (M + 1,), dtype=np.complex128)
    for kx in range(M + 1):
        s = Y[..., kx] + np.conj(Ym[..., kx])
        if kx == 0 or (kx == M and nx % 2 == 0):
            s = s / 2.0
        half[..., kx] = s
    return half


def c2r_scaled_adjoint(y, threads: int | None = None) -> np.ndarray:
    """Adjoint of irfft3 (= c2r_unscaled / N): c2r_adjoint(y) / N."""
    r = _as_f64(y)
    nz, ny, nx = r.shape[-3:]
    return c2r_adjoint(r, threads=threads) / float(nx * ny * nz)


# --------------------------------------------------------------------- Poisson

def wavenumbers(n: int) -> np.ndarray:
    """Integer wavenumbers for a periodic axis of length 2 pi: k = j (j <= n/2) else j - n."""
    j = np.arange(n)
    return np.where(j <= n // 2, j, j - n).astype(np.float64)


def poisson_multiplier(nx: int, ny: int, nz: int) -> np.ndarray:
    """m(k) = -1/|k|^2 on the R2C half spectrum [nz][ny][nx//2+1], m(0) = 0."""
    kx = np.arange(nx // 2 + 1, dtype=np.float64)
    ky = wavenumbers(ny)
    kz = wavenumbers(nz)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    m = np.zeros_like(k2)
    nz_mask = k2 > 0
    m[nz_mask] = -1.0 / k2[nz_mask]
    return m


def poisson(f, threads: int | None = None) -> np.ndarray:
    """Periodic Poisson solve (Section VI-B, (P,P,P)): phi = C2R(m * R2C(f)) / N."""
    r = _as_f64(f)
    nz, ny, nx = r.shape[-3:]
    F = rfft3(r, threads=threads)
    F *= poisson_multiplier(nx, ny, nz)
    return irfft3(F, nx, threads=threads)


# ------------------------------------------------- bounded z: real-to-real DCT
# Section V-B lists real-to-real transforms (DCT, DST); Section VI-B solves the
# Poisson equation on the (Periodic, Periodic, Bounded) topology. Reading: the
# bounded axis z holds nz cell centres z_n = (n + 1/2) pi / nz of a box of
# height pi between walls with zero normal derivative (Neumann), so the
# cosines cos(k z_n), k = 0..nz-1, diagonalise the Laplacian with eigenvalue
# -k^2 -- integer wavenumbers, like the periodic axes of length 2 pi.

def _cos_matrix(n: int) -> np.ndarray:
    """C[k, m] = cos(pi k (2m + 1) / 2n), from the integer argument reduced mod 4n."""
    k = np.arange(n)[:, None]
    m = np.arange(n)[None, :]
    t = (k * (2 * m + 1)) % (4 * n)
    return np.cos(2.0 * np.pi * t / (4.0 * n))


def dct2_z(x) -> np.ndarray:
    """DCT-II (REDFT10) along z (axis -3): Y_k = 2 sum_n x_n cos(pi k (2n + 1) / 2 nz)."""
    a = np.asarray(x.detach().cpu().numpy() if hasattr(x, "detach") else x)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    C = _cos_matrix(a.shape[-3])
    return 2.0 * np.einsum("kn,...nyx->...kyx", C, a)


def dct3_z(y) -> np.ndarray:
    """DCT-III (REDFT01) along z: x_n = Y_0 + 2 sum_{k>0} Y_k cos(pi k (2n + 1) / 2 nz); dct3(dct2(x)) = 2 nz x."""
    a = np.asarray(y.detach().cpu().numpy() if hasattr(y, "detach") else y)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    n = a.shape[-3]
    w = np.full(n, 2.0)
    w[0] = 1.0
    C = _cos_matrix(n)
    return np.einsum("kn,...kyx->...nyx", C * w[:, None], a)


def _sin_matrix(n: int) -> np.ndarray:
    """S[k, m] = sin(pi (k + 1) (2m + 1) / 2n), from the integer argument reduced mod 4n."""
    k = np.arange(n)[:, None]
    m = np.arange(n)[None, :]
    t = ((k + 1) * (2 * m + 1)) % (4 * n)
    return np.sin(2.0 * np.pi * t / (4.0 * n))


def dst2_z(x) -> np.ndarray:
    """DST-II (RODFT10) along z: Y_k = 2 sum_n x_n sin(pi (k + 1) (2n + 1) / 2 nz)."""
    a = np.asarray(x.detach().cpu().numpy() if hasattr(x, "detach") else x)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    return 2.0 * np.einsum("kn,...nyx->...kyx", _sin_matrix(a.shape[-3]), a)


def dst3_z(y) -> np.ndarray:
    """DST-III (RODFT01) along z: x_n = (-1)^n Y_(nz-1) + 2 sum_{k<nz-1} Y_k sin(pi (k + 1) (2n + 1) / 2 nz)."""
    a = np.asarray(y.detach().cpu().numpy() if hasattr(y, "detach") else y)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    n = a.shape[-3]
    w = np.full(n, 2.0)
    w[-1] = 1.0
    return np.einsum("kn,...kyx->...nyx", _sin_matrix(n) * w[:, None], a)


def _along(a: np.ndarray, axis: int, fn) -> np.ndarray:
    """Apply fn (acting on the last axis) along `axis`."""
    return np.moveaxis(fn(np.moveaxis(a, axis, -1)), -1, axis)


def _r2r_1d(a: np.ndarray, kind: str, inverse: bool) -> np.ndarray:
    """DCT-II / DST-II (forward) or DCT-III / DST-III (inverse) along the last axis (matrix definitions)."""
    n = a.shape[-1]
    if kind == "dct":
        M = _cos_matrix(n)
        if inverse:
            w = np.full(n, 2.0)
            w[0] = 1.0
            return np.einsum("...k,kn->...n", a, M * w[:, None])
        return 2.0 * np.einsum("...n,kn->...k", a, M)
    M = _sin_matrix(n)
    if inverse:
        w = np.full(n, 2.0)
        w[-1] = 1.0
        return np.einsum("...k,kn->...n", a, M * w[:, None])
    return 2.0 * np.einsum("...n,kn->...k", a, M)


def r2r(x, kinds=(None, None, "dct"), inverse: bool = False, nx: int | None = None,
        threads: int | None = None) -> np.ndarray:
    """Per-axis mixed transform of a grid [..., z, y, x]: kinds[axis] (axes x, y, z) is None (DFT),
    "dct" (DCT-II forward, DCT-III inverse) or "dst" (DST-II / DST-III). Forward: unscaled, the x
    axis of real input as R2C (bins 0..nx/2). Inverse: the transposed-order inverse of each axis,
    C2R along x when `nx` is given, scaled by 1 / prod(2n for R2R axes, n for DFT axes)."""
    kx, ky, kz = kinds
    a = np.asarray(x.detach().cpu().numpy() if hasattr(x, "detach") else x)
    if not inverse:
        real = not np.iscomplexobj(a)
        a = a.astype(np.float64 if real else np.complex128)
        # x
        if kx is None:
            n = a.shape[-1]
            a = fft1(a, threads=threads)
            if real:
                a = a[..., : n // 2 + 1]
        else:
            a = _r2r_1d(a, kx, False)
        for axis, k in ((-2, ky), (-3, kz)):
            a = _along(a, axis, (lambda v: fft1(v, threads=threads)) if k is None else
                       (lambda v, k=k: _r2r_1d(v, k, False)))
        return a
    a = a.astype(np.complex128)
    scale = 1.0
    for axis, k in ((-3, kz), (-2, ky)):
        n = a.shape[axis]
        scale *= n if k is None else 2 * n
        a = _along(a, axis, (lambda v: fft1(v, sign=+1, threads=threads)) if k is None else
                   (lambda v, k=k: _r2r_1d(v, k, True)))
    if kx is None and nx is not None:
        lead = a.shape[:-1]
        a = c2r_unscaled(a.reshape((-1, 1, 1, a.shape[-1])), nx, threads=threads).reshape(lead + (nx,))
        scale *= nx
    elif kx is None:
        scale *= a.shape[-1]
        a = fft1(a, sign=+1, threads=threads)
    else:
        scale *= 2 * a.shape[-1]
        a = _r2r_1d(a, kx, True)
    return a / scale


def r2r_z(x, kind: str = "dct", inverse: bool = False, nx: int | None = None, threads: int | None = None):
    """Fourier along x (R2C for real input) and y, real-to-real along z: `r2r` with kinds (None, None, kind)."""
    return r2r(x, (None, None, kind), inverse=inverse, nx=nx, threads=threads)


def poisson_bounded_multiplier(nx: int, ny: int, nz: int) -> np.ndarray:
    """m = -1/(kx^2 + ky^2 + kz^2) on [nz][ny][nx] with kx, ky periodic integers and kz = 0..nz-1; m(0) = 0."""
    kx = wavenumbers(nx)
    ky = wavenumbers(ny)
    kz = np.arange(nz, dtype=np.float64)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    m = np.zeros_like(k2)
    m[k2 > 0] = -1.0 / k2[k2 > 0]
    return m


def poisson_bounded(f, threads: int | None = None) -> np.ndarray:
    """(P,P,Bounded) Poisson solve: phi = DCT3_z(F_xy^-1(m * F_xy(DCT2_z(f)))) / (2 nx ny nz).

    F_xy is the 2D DFT of every z-plane (the separable 3D oracle on planes of
    depth 1); the mean (k = 0) mode is set to zero.
    """
    r = _as_f64(f)
    nz, ny, nx = r.shape[-3:]
    lead = r.shape[:-3]
    Y = dct2_z(r).reshape((-1, 1, ny, nx))       # z-planes as a batch of depth-1 grids
    S = fft3(Y.astype(np.complex128), threads=threads).reshape(lead + (nz, ny, nx))
    S *= poisson_bounded_multiplier(nx, ny, nz)
    T = fft3(S.reshape((-1, 1, ny, nx)), sign=+1, threads=threads).reshape(lead + (nz, ny, nx))
    return np.ascontiguousarray(dct3_z(T).real / (2.0 * nx * ny * nz))


# ---------------------------------------------------------------- stage layouts
# Algorithm 1 keeps three arrays, each with its transform axis complete and
# contiguous. Concretely (a reading: the paper leaves the order of the other
# two axes open):
#   A[b][z][y][x]  (x contiguous)  -- natural layout, stage-x input
#   B[b][z][x][y]  (y contiguous)  -- after the first redistribution
#   C[b][x][y][z]  (z contiguous)  -- after the second redistribution
# Each map below is the explicit index definition: dst.flat[d] = src.flat[s(d)].

def _gather(src: np.ndarray, shape_dst, src_index) -> np.ndarray:
    flat = src.reshape(-1)
    return flat[src_index].reshape(shape_dst)


def layout_a_to_b(a: np.ndarray) -> np.ndarray:
    """B[b][z][x][y] = A[b][z][y][x]."""
    *lead, nz, ny, nx = a.shape
    batch = int(np.prod(lead)) if lead else 1
    b, z, x, y = np.meshgrid(np.arange(batch), np.arange(nz), np.arange(nx), np.arange(ny), indexing="ij")
    s = ((b * nz + z) * ny + y) * nx + x
    return _gather(a, tuple(lead) + (nz, nx, ny), s.reshape(-1))


def layout_b_to_c(bb: np.ndarray) -> np.ndarray:
    """C[b][x][y][z] = B[b][z][x][y]."""
    *lead, nz, nx, ny = bb.shape
    batch = int(np.prod(lead)) if lead else 1
    b, x, y, z = np.meshgrid(np.arange(batch), np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    s = ((b * nz + z) * nx + x) * ny + y
    return _gather(bb, tuple(lead) + (nx, ny, nz), s.reshape(-1))


def layout_c_to_a(c: np.ndarray) -> np.ndarray:
    """A[b][z][y][x] = C[b][x][y][z] (the natural-layout un-permute of the last stage)."""
    *lead, nx, ny, nz = c.shape
    batch = int(np.prod(lead)) if lead else 1
    b, z, y, x = np.meshgrid(np.arange(batch), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = ((b * nx + x) * ny + y) * nz + z
    return _gather(c, tuple(lead) + (nz, ny, nx), s.reshape(-1))


def layout_a_to_c(a: np.ndarray) -> np.ndarray:
    """C[b][x][y][z] = A[b][z][y][x] (the two redistributions composed)."""
    return layout_b_to_c(layout_a_to_b(a))


# ------------------------------------------------- pure numpy naive DFT (tiny)

def dft_matrix(n: int, sign: int = -1) -> np.ndarray:
    """W[k, j] = exp(sign 2 pi i (jk mod n)/n), the DFT definition as a matrix."""
    j = np.arange(n)
    t = np.outer(j, j) % n
    return np.exp(sign * 2j * np.pi * t / n)


def dft3_naive(x, sign: int = -1) -> np.ndarray:
    """3D DFT by applying the 1D DFT matrix along x, y and z (tiny grids only)."""
    a = _as_c128(x)
    nz, ny, nx = a.shape[-3:]
    a = np.einsum("kx,...x->...k", dft_matrix(nx, sign), a)
    a = np.einsum("ky,...yx->...kx", dft_matrix(ny, sign), a)
    a = np.einsum("kz,...zyx->...kyx", dft_matrix(nz, sign), a)
    return a


def dft3_bins(x, bins, sign: int = -1) -> np.ndarray:
    """Direct triple-sum DFT (no factorisation) at the given (kx, ky, kz) bins of one grid."""
    a = _as_c128(x)
    if a.ndim != 3:
        raise ValueError("one grid [z][y][x]")
    nz, ny, nx = a.shape
    b = np.ascontiguousarray(np.asarray(bins, dtype=np.int64).reshape(-1, 3)).astype(np.int_)
    out = np.empty(2 * b.shape[0], dtype=np.float64)
    _check(_load().oracle_dft3d_bins(_dptr(a), nx, ny, nz,
                                     b.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), b.shape[0],
                                     int(sign), _dptr(out)), "dft3d_bins")
    return out[0::2] + 1j * out[1::2]


# --------------------------------------------------------------------- metrics

def dft3_bins_c64(x, bins, sign: int = -1, threads: int | None = None) -> np.ndarray:
    """`dft3_bins` of a complex64 grid [z][y][x] read in place (values upcast to FP64
    term by term; bins split across threads). Equal to dft3_bins on the upcast grid."""
    a = x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    if a.dtype != np.complex64 or a.ndim != 3:
        raise ValueError("one complex64 grid [z][y][x]")
    a = np.ascontiguousarray(a)
    nz, ny, nx = a.shape
    b = np.ascontiguousarray(np.asarray(bins, dtype=np.int64).reshape(-1, 3)).astype(np.int_)
    if b.size and (b[:, 0].min() < 0 or b[:, 0].max() >= nx):
        raise ValueError("kx must lie in [0, nx)")
    out = np.empty(2 * b.shape[0], dtype=np.float64)
    _check(_load().oracle_dft3d_bins_c64(a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), nx, ny, nz,
                                         b.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), b.shape[0],
                                         int(sign), _dptr(out), int(threads or default_threads())),
           "dft3d_bins_c64")
    return out[0::2] + 1j * out[1::2]


def rel_l2(y, y_ref) -> float:
    """||y - y_ref||_2 / ||y_ref||_2 accumulated in FP64."""
    a = np.asarray(y.detach().cpu().numpy() if hasattr(y, "detach") else y)
    b = np.asarray(y_ref.detach().cpu().numpy() if hasattr(y_ref, "detach") else y_ref)
    a = a.astype(np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = b.astype(a.dtype)
    num = np.sqrt(np.sum(np.abs(a - b) ** 2))
    den = np.sqrt(np.sum(np.abs(b) ** 2))
    return float(num / den) if den > 0 else float(num)
