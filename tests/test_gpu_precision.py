"""Split-precision tensor-core radix-16 passes (C2C): parity with the FP64 oracle, for the
warp-level products (mma.sync, modes *_split) and the 5th-generation ones (tcgen05.mma with
accumulators in tensor memory, modes *_split_tc5; lengths whose butterflies do not fill 128-row
operand tiles fall back to the warp-level kernel of the same operand type).

Bounds, from the operand splits (each real operand a = hi + lo, three products
hi.hi + hi.lo + lo.hi, FP32 accumulation, one power-of-two scale per butterfly):
  * FP16 pairs carry 22 significant bits: representation and dropped lo.lo
    terms are ~2^-22 of the column scale per pass, far inside the FP32 bound
    of 1e-5 (rel-L2 vs FP64), which the test keeps.
  * BF16 pairs carry 16 bits: ~2^-16 = 1.5e-5 per pass. The grids here have at
    most 6 radix-16 passes (two per axis at lengths 256 and 768), so the bound is
    6 * 2^-16 = 9.2e-5 < 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp16_split": 1e-5, "bf16_split": 1e-4, "fp16_split_tc5": 1e-5, "bf16_split_tc5": 1e-4}
SPLIT_MODES = ["fp16_split", "bf16_split", "fp16_split_tc5", "bf16_split_tc5"]


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_12209_gb300 import _build
    _build.build()
    import paper_2601_12209_gb300 as gbmod
    return gbmod


# lengths with radix-16 passes (48, 80, 128, 240, 256, 384, 640, 768, 1024), ragged
# 16-pencil tiles, and axes without one (24, 60) that keep the FP32 butterflies
SHAPES = [(256, 48, 80), (1024, 24, 60), (128, 240, 48), (80, 768, 16), (640, 40, 48), (384, 96, 32)]


@pytest.mark.parametrize("precision", SPLIT_MODES)
@pytest.mark.parametrize("shape", SHAPES)
def test_split_forward_inverse(gb, precision, shape):
    nx, ny, nz = shape
    x = synth.uniform_complex((nz, ny, nx), seed=40 + nx)
    ref = oracle.fft3(x.numpy())
    p = gb.Plan(nx, ny, nz, precision=precision)
    y = p.forward(x.cuda())
    z = p.inverse(y)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    e = oracle.rel_l2(y.cpu().numpy(), ref)
    e_inv = oracle.rel_l2(z.cpu().numpy(), x.numpy())
    e32 = oracle.rel_l2(gb.Plan(nx, ny, nz).forward(x.cuda()).cpu().numpy(), ref)
    print(f"[precision] {precision} {shape}: fwd rel-L2 {e:.3e} (fp32 path {e32:.3e}), round trip {e_inv:.3e}")
    assert e < TOL[precision] and e_inv < TOL[precision]


@pytest.mark.parametrize("precision", SPLIT_MODES)
def test_split_adjoint_and_slab(gb, precision):
    """The adjoint (+ sign, unscaled) and the slab schedule take the same passes."""
    nx, ny, nz = 256, 80, 48
    x = synth.uniform_complex((nz, ny, nx), seed=77)
    p = gb.Plan(nx, ny, nz, precision=precision)
    a = p.adjoint(x.cuda())
    ps = gb.Plan(nx, ny, nz, precision=precision, slab=True)
    ys = ps.forward(x.cuda())
    torch.cuda.synchronize()
    e_adj = oracle.rel_l2(a.cpu().numpy(), oracle.c2c_adjoint(x.numpy()))
    e_slab = oracle.rel_l2(ys.cpu().numpy(), oracle.fft3(x.numpy()))
    print(f"[precision] {precision} adjoint {e_adj:.3e}, slab {e_slab:.3e}")
    assert e_adj < TOL[precision] and e_slab < TOL[precision]


@pytest.mark.parametrize("precision", SPLIT_MODES)
@pytest.mark.parametrize("shape", [(64, 256, 48), (40, 80, 768), (256, 1024, 16)], ids=lambda s: "x".join(map(str, s)))
def test_split_r2c_c2r_and_poisson(gb, precision, shape):
    """R2C plans in the split modes: the complex y and z stages take the tensor-core radix-16 passes
    (the real x stage and the fused Poisson z stage keep FP32); forward, inverse, adjoint and the
    Poisson solve against the FP64 oracle."""
    nx, ny, nz = shape
    r = synth.normal_real((nz, ny, nx), seed=50 + ny)
    p = gb.Plan(nx, ny, nz, kind="r2c", precision=precision)
    s = p.forward(r.cuda())
    back = p.inverse(s)
    adj = p.adjoint(s)
    phi = p.poisson(r.cuda())
    torch.cuda.synchronize()
    assert p.device_error() == 0
    sh = s.cpu().numpy().astype("complex128")
    e = oracle.rel_l2(s.cpu().numpy(), oracle.rfft3(r.numpy()))
    e_rt = oracle.rel_l2(back.cpu().numpy(), r.numpy())
    e_adj = oracle.rel_l2(adj.cpu().numpy(), oracle.r2c_adjoint(sh, nx))
    e_p = oracle.rel_l2(phi.cpu().numpy(), oracle.poisson(r.numpy()))
    print(f"[precision] r2c {precision} {shape}: fwd {e:.3e}, round trip {e_rt:.3e}, adjoint {e_adj:.3e}, "
          f"poisson {e_p:.3e}")
    tol = TOL[precision]
    assert e < tol and e_rt < tol and e_adj < tol and e_p < tol


def test_split_rejected_for_unknown_precision(gb):
    with pytest.raises(ValueError):
        gb.Plan(64, 64, 64, precision="fp8")


def test_split_cube_256(gb):
    """256^3: two radix-16 passes per axis, errors of all three modes on one input."""
    n = 256
    x = synth.uniform_complex((n, n, n), seed=3)
    ref = oracle.fft3(x.numpy())
    xd = x.cuda()
    for precision in ["fp32"] + SPLIT_MODES:
        y = gb.Plan(n, n, n, precision=precision).forward(xd)
        e = oracle.rel_l2(y.cpu().numpy(), ref)
        print(f"[precision] 256^3 {precision}: rel-L2 {e:.3e}")
        assert e < TOL[precision]


def _rel_l2_dev(a: torch.Tensor, b: torch.Tensor) -> float:
    """rel-L2 on the device in FP64 (test-side check of two device tensors)."""
    num = torch.linalg.vector_norm((a.to(torch.complex128) - b.to(torch.complex128)).reshape(-1))
    return float(num / torch.linalg.vector_norm(b.to(torch.complex128).reshape(-1)))


def test_precision_1024_plane_waves(gb):
    """1024^3 C2C: uniform[-1,1] noise plus 16 plane waves (|a_m| = (m+1)/4).

    Per mode: sampled bins against the FP64 direct sum of the same complex64
    input (the 16 peaks relative to their size, 16 random bins relative to the
    spectrum's rms); the waves alone against their closed
    form n^3 a_m at k_m (and the energy that leaks elsewhere); the round trip.
    """
    n = 1024
    N = n ** 3
    ks, amps = synth.plane_wave_spec(n, seed=7)
    rng = np.random.default_rng(5)
    bins = np.concatenate([ks, rng.integers(0, n, size=(16, 3))])
    x = synth.uniform_complex_slabs((n, n, n), seed=7).cuda()
    synth.add_plane_waves(x, ks, amps)
    xh = x.cpu()
    ref = oracle.dft3_bins_c64(xh, bins)
    del xh
    waves = torch.zeros_like(x)
    synth.add_plane_waves(waves, ks, amps)
    kx = torch.as_tensor(bins[:, 0], device="cuda")
    ky = torch.as_tensor(bins[:, 1], device="cuda")
    kz = torch.as_tensor(bins[:, 2], device="cuda")
    pk = torch.as_tensor(ks, device="cuda")
    for precision in ["fp32"] + SPLIT_MODES:
        p = gb.Plan(n, n, n, precision=precision)
        y = p.forward(x)
        got = y[kz, ky, kx].cpu().numpy().astype(np.complex128)
        rms = float(torch.sqrt(torch.mean(torch.abs(y.to(torch.complex128)) ** 2)))
        # a peak carries its own rounding (relative to its size); elsewhere the error is
        # the spread of all the rounding, relative to the spectrum's rms
        e_bins = max(float(np.max(np.abs(got[:16] - ref[:16]) / np.abs(ref[:16]))),
                     float(np.max(np.abs(got[16:] - ref[16:]))) / rms)
        z = p.inverse(y)
        e_rt = _rel_l2_dev(z, x)
        del z
        w = p.forward(waves, out=y)
        peaks = w[pk[:, 2], pk[:, 1], pk[:, 0]].cpu().numpy().astype(np.complex128)
        e_peak = float(np.max(np.abs(peaks - N * amps) / np.abs(N * amps)))
        w[pk[:, 2], pk[:, 1], pk[:, 0]] = 0
        leak = float(torch.linalg.vector_norm(w.reshape(-1).to(torch.complex128))) / float(
            np.sqrt(np.sum(np.abs(N * amps) ** 2)))
        torch.cuda.synchronize()
        assert p.device_error() == 0
        print(f"[precision] 1024^3 {precision}: sampled bins {e_bins:.3e}, peaks rel {e_peak:.3e}, "
              f"leak {leak:.3e}, round trip {e_rt:.3e}")
        del y, w
        tol = TOL[precision]
        assert e_bins < tol and e_peak < tol and leak < tol and e_rt < tol


@pytest.mark.parametrize("precision", ["fp16_split_tc5", "bf16_split_tc5"])
def test_tc5_staged_transposed_and_batch(gb, precision):
    """The tcgen05 passes in every stage position: row and column input, pass 0 reading HBM
    directly, the last pass writing HBM directly (length 256: radix-16 passes 0 and 1),
    transposed output, two batch entries; bitwise equal on a repeated call (no state carried
    between calls in tensor memory or the completion barrier)."""
    nx, ny, nz = 256, 1024, 128
    x = synth.uniform_complex((2, nz, ny, nx), seed=91)
    ref = oracle.fft3(x.numpy())
    p = gb.Plan(nx, ny, nz, batch=2, precision=precision, transposed_out=True)
    y = p.forward(x.cuda())
    y2 = p.forward(x.cuda())
    back = p.inverse(y)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    assert torch.equal(y, y2)
    e = oracle.rel_l2(y.cpu().numpy(), np.transpose(ref, (0, 3, 2, 1)))
    e_rt = oracle.rel_l2(back.cpu().numpy(), x.numpy())
    print(f"[precision] tc5 {precision} 256x1024x128 batch 2 transposed: fwd {e:.3e}, round trip {e_rt:.3e}")
    assert e < TOL[precision] and e_rt < TOL[precision]
