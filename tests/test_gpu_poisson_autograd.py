"""Differentiation: the periodic Poisson solve and the autograd adjoints.

The hand-written backward passes (exec_adjoint, exec_inverse_adjoint, the
symmetric Poisson operator) are checked against the FP64 oracle's adjoints,
against FP64 central finite differences of the oracle loss, and by
dot-product identities on the GPU results.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_12209_gb300 import _build
    _build.build()
    import paper_2601_12209_gb300 as gbmod
    return gbmod


def err(name, got, ref):
    e = oracle.rel_l2(got, ref)
    print(f"[parity-poisson] {name}: rel-L2 {e:.3e}")
    return e


@pytest.mark.parametrize("shape", [(64, 64, 64), (32, 48, 40), (16, 16, 16)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("slab", [False, True], ids=["pencil", "slab"])
def test_poisson_vs_oracle(gb, shape, slab):
    nx, ny, nz = shape
    f = synth.normal_real((nz, ny, nx), seed=61)
    plan = gb.Plan(nx, ny, nz, kind="r2c", slab=slab)
    phi = plan.poisson(f.cuda())
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    assert err(f"poisson {shape} {'slab' if slab else 'pencil'}", phi.cpu().numpy(), oracle.poisson(f.numpy())) < TOL


def test_poisson_single_mode_closed_form(gb):
    n = 32
    r = 2 * np.pi * np.arange(n) / n
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    arg = 3 * x - 2 * y + 5 * z
    f = (np.sin(arg) + 0.5 * np.cos(arg)).astype(np.float32)
    phi = gb.poisson(torch.from_numpy(f).cuda()).cpu().numpy()
    assert err("poisson single mode", phi, -f.astype(np.float64) / 38.0) < TOL


def test_config3_poisson_256_gradient(gb):
    """256^3 Gaussian-blob RHS, loss = sum(w * phi): the autograd gradient equals
    the FP64 oracle P(w) (P is symmetric), and phi equals the oracle solve."""
    n = 256
    f, _ = synth.poisson_rhs(n, seed=4)
    w = synth.normal_real((n, n, n), seed=4)
    fd = f.cuda().requires_grad_(True)
    phi = gb.Poisson.apply(fd)
    loss = (w.cuda() * phi).sum()
    loss.backward()
    assert err("cfg3 phi 256", phi.detach().cpu().numpy(), oracle.poisson(f.numpy())) < TOL
    assert err("cfg3 grad 256", fd.grad.cpu().numpy(), oracle.poisson(w.numpy())) < TOL


def test_config3_finite_differences_64_directions(gb):
    """Central finite differences in FP64 of the oracle loss on 64 random
    directions against <grad, v> from the GPU autograd gradient."""
    n = 32
    f, _ = synth.poisson_rhs(n, seed=14)
    w = synth.normal_real((n, n, n), seed=15)
    fd = f.cuda().requires_grad_(True)
    (w.cuda() * gb.Poisson.apply(fd)).sum().backward()
    g = fd.grad.cpu().numpy().astype(np.float64)
    f64, w64 = f.numpy().astype(np.float64), w.numpy().astype(np.float64)
    eps = 1e-3
    worst = 0.0
    for k in range(64):
        v = synth.normal_real((n, n, n), seed=1000 + k).numpy().astype(np.float64)
        lp = np.sum(w64 * oracle.poisson(f64 + eps * v))
        lm = np.sum(w64 * oracle.poisson(f64 - eps * v))
        fdv = (lp - lm) / (2 * eps)
        an = float(np.sum(g * v))
        rel = abs(fdv - an) / max(abs(fdv), 1e-30)
        worst = max(worst, rel)
    print(f"[parity-poisson] FD 64 directions: worst relative deviation {worst:.3e}")
    assert worst < 1e-4


def _rdot(a, b):
    return float(np.real(np.vdot(np.asarray(a, dtype=np.complex128), np.asarray(b, dtype=np.complex128))))


def test_autograd_fft3_rfft3_irfft3(gb):
    n = (20, 24, 32)  # (nz, ny, nx)
    nz, ny, nx = n
    # C2C: backward = F^H g
    x = synth.uniform_complex(n, seed=71).cuda().requires_grad_(True)
    gy = synth.uniform_complex(n, seed=72)
    y = gb.FFT3.apply(x)
    y.backward(gy.cuda())
    assert err("FFT3 backward", x.grad.cpu().numpy(), oracle.c2c_adjoint(gy.numpy())) < TOL
    # R2C: backward = R^T g
    r = synth.normal_real(n, seed=73).cuda().requires_grad_(True)
    gh = synth.uniform_complex((nz, ny, nx // 2 + 1), seed=74)
    gb.RFFT3.apply(r).backward(gh.cuda())
    assert err("RFFT3 backward", r.grad.cpu().numpy(), oracle.r2c_adjoint(gh.numpy(), nx)) < TOL
    # C2R (scaled): backward = (C/N)^T g
    h = synth.uniform_complex((nz, ny, nx // 2 + 1), seed=75).cuda().requires_grad_(True)
    gr = synth.normal_real(n, seed=76)
    gb.IRFFT3.apply(h, nx).backward(gr.cuda())
    assert err("IRFFT3 backward", h.grad.cpu().numpy(), oracle.c2r_scaled_adjoint(gr.numpy())) < TOL
    # dot-product identity on the GPU results themselves
    xr = synth.normal_real(n, seed=77)
    Rx = gb.rfftn(xr.cuda()).cpu().numpy()
    RTg = gb.Plan(nx, ny, nz, kind="r2c").adjoint(gh.cuda()).cpu().numpy()
    lhs, rhs = _rdot(Rx, gh.numpy()), _rdot(xr.numpy(), RTg)
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_torch_autograd_matches_torch_fft_gradients(gb):
    """Cross-check against PyTorch's own FFT autograd (a library routine) on the GPU."""
    n = (16, 12, 20)
    x = synth.uniform_complex(n, seed=81).cuda()
    g = synth.uniform_complex(n, seed=82).cuda()
    a = x.clone().requires_grad_(True)
    gb.FFT3.apply(a).backward(g)
    b = x.clone().requires_grad_(True)
    torch.fft.fftn(b, dim=(-3, -2, -1)).backward(g)
    assert err("FFT3 vs torch.fft grad", a.grad.cpu().numpy(), b.grad.cpu().numpy()) < TOL
