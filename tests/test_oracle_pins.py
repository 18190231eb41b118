"""Pins the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: hand-derived textbook values (tests/golden), closed forms (delta, plane
wave, constant), brute force on tiny inputs (the naive DFT), identities
(Parseval, linearity, round trip, axis-order independence, adjoint dot
products) and an independent library routine (numpy.fft, pocketfft). A
dropped term, a wrong sign, a wrong twiddle index or a transposed axis in the
oracle fails at least one of them.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dft_textbook.txt")


def _read_golden():
    cases, cur = [], None
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "name":
                cur = {"name": vals[0]}
                cases.append(cur)
            elif key == "shape":
                cur["shape"] = tuple(int(v) for v in vals)
            elif key == "input":
                cur["input"] = np.array([float(v) for v in vals])
            elif key == "output":
                v = np.array([float(t) for t in vals])
                cur["output"] = v[0::2] + 1j * v[1::2]
    return cases


@pytest.mark.parametrize("case", _read_golden(), ids=lambda c: c["name"])
@pytest.mark.parametrize("naive", [False, True])
def test_golden_textbook(case, naive):
    """Hand-derived DFT values (Section III-A definition, forward sign -1)."""
    x = case["input"].reshape(case["shape"]).astype(np.complex128)
    got = oracle.fft3(x, naive=naive).reshape(-1)
    np.testing.assert_allclose(got, case["output"], atol=1e-12, rtol=0)
    got2 = oracle.dft3_naive(x).reshape(-1)
    np.testing.assert_allclose(got2, case["output"], atol=1e-12, rtol=0)


SIZES_1D = list(range(1, 65)) + [80, 96, 120, 128, 160, 192, 256, 77, 91, 98, 127]


@pytest.mark.parametrize("n", SIZES_1D)
def test_fft1_matches_naive_dft(n):
    """Brute force: the recursive mixed-radix FFT equals the O(n^2) DFT."""
    x = synth.uniform_complex((3, n), seed=100 + n).numpy()
    fast = oracle.fft1(x, naive=False)
    slow = oracle.fft1(x, naive=True)
    np.testing.assert_allclose(fast, slow, atol=1e-11 * max(1, n), rtol=0)
    # pure numpy matrix form of the definition (independent code path)
    ref = x.astype(np.complex128) @ oracle.dft_matrix(n).T
    np.testing.assert_allclose(fast, ref, atol=1e-11 * max(1, n), rtol=0)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 12, 60, 64])
def test_delta_constant_planewave_1d(n):
    """Closed forms: delta -> phase ramp, constant -> n delta_k0, plane wave -> n a delta_k,k0."""
    j0 = n // 3
    d = np.zeros(n, complex)
    d[j0] = 1.0
    k = np.arange(n)
    np.testing.assert_allclose(oracle.fft1(d), np.exp(-2j * np.pi * ((k * j0) % n) / n), atol=1e-13)
    c = np.full(n, 2.5 - 1j)
    exp = np.zeros(n, complex)
    exp[0] = n * (2.5 - 1j)
    np.testing.assert_allclose(oracle.fft1(c), exp, atol=1e-12)
    k0 = (n - 1) // 2
    a = 0.75 + 0.25j
    w = a * np.exp(2j * np.pi * k0 * k / n)
    exp = np.zeros(n, complex)
    exp[k0] = n * a
    np.testing.assert_allclose(oracle.fft1(w), exp, atol=1e-12)


SHAPES_3D = [(2, 3, 4), (4, 4, 4), (8, 8, 8), (5, 6, 10), (12, 15, 9), (16, 8, 32), (7, 11, 3)]


@pytest.mark.parametrize("shape", SHAPES_3D)
def test_fft3_vs_numpy(shape):
    """Independent library routine: numpy.fft.fftn over (z, y, x) in FP64."""
    x = synth.uniform_complex(shape, seed=7).numpy().astype(np.complex128)
    got = oracle.fft3(x)
    ref = np.fft.fftn(x, axes=(-3, -2, -1))
    np.testing.assert_allclose(got, ref, atol=1e-11 * np.sqrt(x.size), rtol=0)


@pytest.mark.parametrize("shape", [(4, 6, 5), (8, 8, 8)])
def test_fft3_matches_naive_and_bins(shape):
    """3D brute force: separable recursive FFT == naive per-axis DFT == direct triple sum."""
    x = synth.uniform_complex(shape, seed=8).numpy()
    fast = oracle.fft3(x)
    np.testing.assert_allclose(fast, oracle.fft3(x, naive=True), atol=1e-11, rtol=0)
    np.testing.assert_allclose(fast, oracle.dft3_naive(x), atol=1e-11, rtol=0)
    nz, ny, nx = shape
    bins = [(kx, ky, kz) for kz in range(nz) for ky in range(ny) for kx in range(nx)]
    direct = oracle.dft3_bins(x, bins)
    np.testing.assert_allclose(direct, fast.reshape(-1), atol=1e-11, rtol=0)


def test_fft3_identities():
    """Parseval, linearity, round trip, axis-order independence, batch independence."""
    shape = (2, 12, 10, 16)
    x = synth.uniform_complex(shape, seed=11).numpy().astype(np.complex128)
    y = synth.uniform_complex(shape, seed=12).numpy().astype(np.complex128)
    X = oracle.fft3(x)
    N = 12 * 10 * 16
    np.testing.assert_allclose(np.sum(np.abs(X) ** 2, axis=(-3, -2, -1)),
                               N * np.sum(np.abs(x) ** 2, axis=(-3, -2, -1)), rtol=1e-13)
    a, b = 0.3 - 1.2j, -2.0 + 0.5j
    np.testing.assert_allclose(oracle.fft3(a * x + b * y), a * X + b * oracle.fft3(y), atol=1e-11)
    np.testing.assert_allclose(oracle.ifft3(X), x, atol=1e-14 * 50)
    np.testing.assert_allclose(oracle.fft3(x, order=1), X, atol=1e-11)
    np.testing.assert_allclose(oracle.fft3(x[1]), X[1], atol=0, rtol=0)


def test_fft3_delta_and_planewave_3d():
    """3D closed forms: delta at (a,b,c) -> exp(-2 pi i (kx a/nx + ky b/ny + kz c/nz));
    plane wave exp(+2 pi i k0.r) -> N delta_{k,k0}."""
    nz, ny, nx = 6, 10, 12
    a, b, c = 5, 3, 4
    d = np.zeros((nz, ny, nx), complex)
    d[c, b, a] = 1.0
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = (kx * a % nx) / nx + (ky * b % ny) / ny + (kz * c % nz) / nz
    np.testing.assert_allclose(oracle.fft3(d), np.exp(-2j * np.pi * ph), atol=1e-13)
    k0 = (7, 2, 5)  # (kx, ky, kz)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    w = np.exp(2j * np.pi * (k0[0] * x / nx + k0[1] * y / ny + k0[2] * z / nz))
    exp = np.zeros((nz, ny, nx), complex)
    exp[k0[2], k0[1], k0[0]] = nx * ny * nz
    np.testing.assert_allclose(oracle.fft3(w), exp, atol=1e-10)


# --------------------------------------------------------------- R2C / C2R

@pytest.mark.parametrize("shape", [(4, 6, 8), (8, 8, 8), (6, 10, 12), (3, 5, 16), (2, 4, 6, 10)])
def test_rfft3_relation_and_numpy(shape):
    """R2C == first nx/2+1 bins of C2C (exact relation) == numpy.fft.rfftn."""
    x = synth.normal_real(shape, seed=21).numpy().astype(np.float64)
    nx = shape[-1]
    got = oracle.rfft3(x)
    full = oracle.fft3(x.astype(np.complex128))
    np.testing.assert_allclose(got, full[..., : nx // 2 + 1], atol=1e-11)
    np.testing.assert_allclose(got, np.fft.rfftn(x, axes=(-3, -2, -1)), atol=1e-11)


@pytest.mark.parametrize("shape", [(4, 6, 8), (6, 10, 12), (2, 4, 6, 10)])
def test_irfft3_roundtrip_and_projection(shape):
    """C2R(R2C(x))/N = x; on a NON-Hermitian half spectrum the projection reading
    agrees with numpy.fft.irfftn (which drops the imaginary part of the kx = 0 and
    kx = nx/2 lines after the inverse along the other axes)."""
    x = synth.normal_real(shape, seed=22).numpy().astype(np.float64)
    nx = shape[-1]
    np.testing.assert_allclose(oracle.irfft3(oracle.rfft3(x), nx), x, atol=1e-13)
    h = synth.uniform_complex(shape[:-1] + (nx // 2 + 1,), seed=23).numpy().astype(np.complex128)
    got = oracle.irfft3(h, nx)
    ref = np.fft.irfftn(h, s=shape[-3:], axes=(-3, -2, -1))
    np.testing.assert_allclose(got, ref, atol=1e-13)


# ----------------------------------------------------------------- adjoints

def _rdot(a, b):
    return float(np.real(np.vdot(a, b)))


def test_adjoint_dot_products():
    """<A x, y> = <x, A^T y> for the four maps and the scaled inverses (real inner product)."""
    shape = (6, 4, 8)
    nx = shape[-1]
    N = np.prod(shape)
    xc = synth.uniform_complex(shape, seed=31).numpy().astype(np.complex128)
    yc = synth.uniform_complex(shape, seed=32).numpy().astype(np.complex128)
    xr = synth.normal_real(shape, seed=33).numpy().astype(np.float64)
    yr = synth.normal_real(shape, seed=34).numpy().astype(np.float64)
    gh = synth.uniform_complex(shape[:-1] + (nx // 2 + 1,), seed=35).numpy().astype(np.complex128)
    # C2C forward and inverse
    assert abs(_rdot(oracle.fft3(xc), yc) - _rdot(xc, oracle.c2c_adjoint(yc))) < 1e-9
    assert abs(_rdot(oracle.ifft3(xc), yc) - _rdot(xc, oracle.c2c_inverse_adjoint(yc))) < 1e-9
    # F^H = N F^-1
    np.testing.assert_allclose(oracle.c2c_adjoint(yc), N * oracle.ifft3(yc), atol=1e-10)
    # R2C
    assert abs(_rdot(oracle.rfft3(xr), gh) - _rdot(xr, oracle.r2c_adjoint(gh, nx))) < 1e-9
    # unscaled C2R (with projection) and the scaled inverse
    assert abs(_rdot(oracle.c2r_unscaled(gh, nx), yr) - _rdot(gh, oracle.c2r_adjoint(yr))) < 1e-9
    assert abs(_rdot(oracle.irfft3(gh, nx), yr) - _rdot(gh, oracle.c2r_scaled_adjoint(yr))) < 1e-9


def test_adjoint_closed_forms():
    """R^T g equals the unscaled C2R of g with interior x-bins halved; C^T y equals
    R2C(y) with interior x-bins doubled (both follow from Hermitian completion)."""
    shape = (6, 4, 8)
    nx, M = shape[-1], shape[-1] // 2
    gh = synth.uniform_complex(shape[:-1] + (M + 1,), seed=36).numpy().astype(np.complex128)
    half = gh.copy()
    half[..., 1:M] *= 0.5
    np.testing.assert_allclose(oracle.r2c_adjoint(gh, nx), oracle.c2r_unscaled(half, nx), atol=1e-10)
    yr = synth.normal_real(shape, seed=37).numpy().astype(np.float64)
    dbl = oracle.rfft3(yr)
    dbl[..., 1:M] *= 2.0
    np.testing.assert_allclose(oracle.c2r_adjoint(yr), dbl, atol=1e-10)


# ------------------------------------------------------------------ Poisson

def test_poisson_single_mode_closed_form():
    """f = sin(k0 . r) on [0, 2 pi)^3 -> phi = -sin(k0 . r)/|k0|^2 exactly (Section VI-B, periodic)."""
    n = 16
    r = 2 * np.pi * np.arange(n) / n
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    for k0 in [(1, 0, 0), (0, 2, 0), (0, 0, 3), (2, -3, 1), (8, 1, -2)]:
        arg = k0[0] * x + k0[1] * y + k0[2] * z
        f = np.sin(arg) + 0.5 * np.cos(arg)
        k2 = sum(k * k for k in k0)
        np.testing.assert_allclose(oracle.poisson(f), -f / k2, atol=1e-12)


def test_poisson_spectral_laplacian():
    """Applying -|k|^2 (numpy FFT) to phi returns f minus its mean; phi has zero mean."""
    f, _ = synth.poisson_rhs(16, seed=4)
    f = f.numpy().astype(np.float64) + 0.3  # nonzero mean must be removed by the k=0 rule
    phi = oracle.poisson(f)
    assert abs(phi.mean()) < 1e-14
    k = np.fft.fftfreq(16, d=1.0 / 16)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    lap = np.real(np.fft.ifftn(-(kx ** 2 + ky ** 2 + kz ** 2) * np.fft.fftn(phi)))
    np.testing.assert_allclose(lap, f - f.mean(), atol=1e-12)


def test_poisson_self_adjoint():
    """The multiplier is real and even, so <P f, w> = <f, P w>."""
    f = synth.normal_real((8, 12, 10), seed=41).numpy().astype(np.float64)
    w = synth.normal_real((8, 12, 10), seed=42).numpy().astype(np.float64)
    assert abs(_rdot(oracle.poisson(f), w) - _rdot(f, oracle.poisson(w))) < 1e-12


# ------------------------------------------------------------ stage layouts

@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 8, 6, 10), (16, 16, 16)])
def test_layout_maps(shape):
    """The explicit index maps equal numpy axis permutations and are bijections."""
    a = synth.integer_complex(shape, seed=51).numpy()
    b = oracle.layout_a_to_b(a)
    c = oracle.layout_b_to_c(b)
    np.testing.assert_array_equal(b, np.swapaxes(a, -1, -2))
    np.testing.assert_array_equal(c, np.moveaxis(a, -3, -1).swapaxes(-3, -2))
    np.testing.assert_array_equal(oracle.layout_c_to_a(c), a)
    assert len(np.unique(oracle.layout_a_to_b(np.arange(a.size).reshape(a.shape)))) == a.size
    # B[z][x][y] and C[x][y][z] element checks straight from the definition
    A = a.reshape((-1,) + shape[-3:])
    B = b.reshape((-1,) + b.shape[-3:])
    C = c.reshape((-1,) + c.shape[-3:])
    nz, ny, nx = shape[-3:]
    for (bb, z, y, x) in [(0, 0, 0, 0), (0, nz - 1, ny - 1, nx - 1), (A.shape[0] - 1, 1 % nz, 2 % ny, 3 % nx)]:
        assert B[bb, z, x, y] == A[bb, z, y, x]
        assert C[bb, x, y, z] == A[bb, z, y, x]


def test_separable_stage_sequence():
    """Algorithm 1 on explicit stage arrays (x on A, redistribute, y on B, redistribute,
    z on C, un-permute) equals the 3D DFT."""
    shape = (6, 10, 8)
    x = synth.uniform_complex(shape, seed=61).numpy().astype(np.complex128)
    A = oracle.fft1(x)
    B = oracle.fft1(oracle.layout_a_to_b(A))
    C = oracle.fft1(oracle.layout_b_to_c(B))
    np.testing.assert_allclose(oracle.layout_c_to_a(C), np.fft.fftn(x), atol=1e-11)


def test_dft3_bins_c64_equals_fp64_version():
    """The threaded complex64 bin sum reads the same values and adds the same terms in the same
    order as the FP64 one, so it agrees bit for bit; both agree with the separable FFT."""
    x = synth.uniform_complex((6, 10, 12), seed=21)
    nz, ny, nx = 6, 10, 12
    bins = [(kx, ky, kz) for kz in range(nz) for ky in range(0, ny, 3) for kx in range(nx)]
    a = oracle.dft3_bins_c64(x, bins, threads=3)
    b = oracle.dft3_bins(x.numpy().astype(np.complex128), bins)
    assert np.array_equal(a, b)
    full = oracle.fft3(x.numpy())
    ref = np.array([full[kz, ky, kx] for kx, ky, kz in bins])
    np.testing.assert_allclose(a, ref, atol=1e-11, rtol=0)
    with pytest.raises(ValueError):
        oracle.dft3_bins_c64(x, [(nx, 0, 0)])


def test_plane_waves_closed_form():
    """Waves-only grid: the DFT is n^3 a_m at k_m and ~0 elsewhere (the 1024^3 precision pin,
    at n = 24); also the slab-wise noise generator is deterministic and in range."""
    n = 24
    ks, amps = synth.plane_wave_spec(n, seed=7, count=16)
    assert len({tuple(k) for k in ks.tolist()}) == 16
    np.testing.assert_allclose(np.abs(amps), (np.arange(16) + 1) / 4, rtol=1e-15)
    g = torch.zeros((n, n, n), dtype=torch.complex64)
    synth.add_plane_waves(g, ks, amps, planes=5)
    X = oracle.fft3(g.numpy())
    N = n ** 3
    peaks = np.array([X[kz, ky, kx] for kx, ky, kz in ks.tolist()])
    np.testing.assert_allclose(peaks, N * amps, rtol=2e-7, atol=0)
    rest = X.copy()
    for kx, ky, kz in ks.tolist():
        rest[kz, ky, kx] = 0
    assert np.sqrt(np.sum(np.abs(rest) ** 2)) < 1e-6 * np.sqrt(np.sum(np.abs(peaks) ** 2))
    np.testing.assert_allclose(oracle.dft3_bins_c64(g, ks), peaks, rtol=1e-12, atol=1e-6)
    u = synth.uniform_complex_slabs((9, 5, 4), seed=3, planes=4)
    assert torch.equal(u, synth.uniform_complex_slabs((9, 5, 4), seed=3, planes=4))
    r = torch.view_as_real(u)
    assert float(r.abs().max()) <= 1.0 and u.dtype == torch.complex64


def test_dct_z_against_library_and_inverse():
    """DCT-II / DCT-III along z: against scipy.fft.dct (an independent library), the
    inverse pair identity, and a cosine basis vector (closed form N at its own bin)."""
    sf = pytest.importorskip("scipy.fft")
    x = synth.normal_real((2, 9, 5, 4), seed=31).numpy().astype(np.float64)
    np.testing.assert_allclose(oracle.dct2_z(x), sf.dct(x, type=2, axis=-3), atol=1e-12)
    np.testing.assert_allclose(oracle.dct3_z(x), sf.dct(x, type=3, axis=-3), atol=1e-12)
    np.testing.assert_allclose(oracle.dct3_z(oracle.dct2_z(x)), 2 * 9 * x, atol=1e-12)
    n, k0 = 12, 5
    e = np.cos(np.pi * k0 * (2 * np.arange(n) + 1) / (2 * n))[:, None, None]
    y = oracle.dct2_z(e)[:, 0, 0]
    ref = np.zeros(n)
    ref[k0] = n
    np.testing.assert_allclose(y, ref, atol=1e-12)


def test_poisson_bounded_single_mode_and_symmetry():
    """(P,P,Bounded): a single cosine-in-z, Fourier-in-xy mode solves to -f/|k|^2 exactly;
    the operator is symmetric; the mean mode is removed."""
    nx, ny, nz = 16, 12, 10
    i, j, n = np.arange(nx), np.arange(ny), np.arange(nz)
    for kx, ky, kz in [(3, -2, 4), (0, 5, 1), (8, 0, 9), (1, 1, 0)]:
        f = (np.cos(kz * (n + 0.5) * np.pi / nz)[:, None, None]
             * np.cos(kx * 2 * np.pi * i / nx + ky * 2 * np.pi * j[:, None] / ny)[None, :, :])
        np.testing.assert_allclose(oracle.poisson_bounded(f), -f / (kx * kx + ky * ky + kz * kz), atol=1e-13)
    a = synth.normal_real((nz, ny, nx), seed=32).numpy().astype(np.float64)
    b = synth.normal_real((nz, ny, nx), seed=33).numpy().astype(np.float64)
    np.testing.assert_allclose(np.sum(oracle.poisson_bounded(a) * b), np.sum(a * oracle.poisson_bounded(b)),
                               rtol=1e-12)
    np.testing.assert_allclose(oracle.poisson_bounded(np.ones((nz, ny, nx))), 0.0, atol=1e-14)


def test_dst_z_and_r2r_z_round_trip():
    """DST-II / DST-III along z against scipy.fft.dst; the mixed Fourier-xy / R2R-z transform
    and its inverse are exact inverses (real and complex input), and a single
    sin-in-z, Fourier-in-xy mode lands on one bin with the closed-form value."""
    sf = pytest.importorskip("scipy.fft")
    x = synth.normal_real((2, 9, 5, 4), seed=34).numpy().astype(np.float64)
    np.testing.assert_allclose(oracle.dst2_z(x), sf.dst(x, type=2, axis=-3), atol=1e-12)
    np.testing.assert_allclose(oracle.dst3_z(x), sf.dst(x, type=3, axis=-3), atol=1e-12)
    r = synth.normal_real((6, 8, 10), seed=35).numpy().astype(np.float64)
    c = synth.uniform_complex((6, 8, 10), seed=36).numpy().astype(np.complex128)
    for kind in ("dct", "dst"):
        np.testing.assert_allclose(oracle.r2r_z(oracle.r2r_z(r, kind), kind, inverse=True, nx=10), r, atol=1e-12)
        np.testing.assert_allclose(oracle.r2r_z(oracle.r2r_z(c, kind), kind, inverse=True), c, atol=1e-12)
    nx, ny, nz, kx, ky, kz = 8, 6, 5, 2, 1, 3
    i, j, n = np.arange(nx), np.arange(ny), np.arange(nz)
    f = (np.sin((kz + 1) * (n + 0.5) * np.pi / nz)[:, None, None]
         * np.exp(2j * np.pi * (kx * i / nx + ky * j[:, None] / ny))[None, :, :])
    Y = oracle.r2r_z(f, "dst")
    ref = np.zeros_like(Y)
    ref[kz, ky, kx] = nz * nx * ny
    np.testing.assert_allclose(Y, ref, atol=1e-10)


@pytest.mark.parametrize("kinds", [("dct", None, None), (None, "dct", None), ("dst", None, None), (None, "dst", None),
                                   ("dst", "dct", None), ("dct", "dst", "dst"), ("dct", "dct", "dct")],
                         ids=lambda k: "-".join(str(v) for v in k))
def test_r2r_x_and_y_axes_against_library(kinds):
    """The per-axis mixed transform with DCT / DST on the x and y axes: every R2R axis against
    scipy.fft's dct / dst (an independent library; types II forward, III inverse), every Fourier
    axis against numpy.fft, forward unscaled and inverse scaled by prod(2n R2R, n DFT)."""
    sf = pytest.importorskip("scipy.fft")
    kx, ky, kz = kinds
    c = synth.uniform_complex((5, 6, 8), seed=37).numpy().astype(np.complex128)
    fwd = c
    for axis, k in ((-1, kx), (-2, ky), (-3, kz)):
        fwd = np.fft.fft(fwd, axis=axis) if k is None else \
            (sf.dct if k == "dct" else sf.dst)(fwd, type=2, axis=axis)
    np.testing.assert_allclose(oracle.r2r(c, kinds), fwd, atol=1e-11)
    inv = c
    for axis, k in ((-3, kz), (-2, ky), (-1, kx)):
        inv = np.fft.ifft(inv, axis=axis) if k is None else \
            (sf.dct if k == "dct" else sf.dst)(inv, type=3, axis=axis) / (2 * c.shape[axis])
    np.testing.assert_allclose(oracle.r2r(c, kinds, inverse=True), inv, atol=1e-12)


def test_r2r_y_axis_of_real_input_against_library():
    """Real input with the x axis Fourier (R2C, bins 0..nx/2) and R2R along y and z: numpy.fft.rfft
    along x, scipy.fft dct / dst along y and z; the inverse with nx given returns the real grid."""
    sf = pytest.importorskip("scipy.fft")
    r = synth.normal_real((4, 6, 10), seed=38).numpy().astype(np.float64)
    for ky, kz in (("dct", None), ("dst", "dct"), ("dct", "dst")):
        ref = np.fft.rfft(r, axis=-1)
        ref = (sf.dct if ky == "dct" else sf.dst)(ref, type=2, axis=-2)
        ref = np.fft.fft(ref, axis=-3) if kz is None else (sf.dct if kz == "dct" else sf.dst)(ref, type=2, axis=-3)
        got = oracle.r2r(r, (None, ky, kz))
        np.testing.assert_allclose(got, ref, atol=1e-11)
        np.testing.assert_allclose(oracle.r2r(got, (None, ky, kz), inverse=True, nx=10), r, atol=1e-12)
