"""Fused slab plane launches: a thread-block cluster per xy-plane runs both in-plane stages.

Checked against the FP64 oracle, and bit for bit against the same slab pipeline
run as one launch per stage (the fused kernel runs the same tile arithmetic).
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


def _plane_bits(gb, plan):
    from paper_2601_12209_gb300 import abi
    return [abi.gbfft_plan_get_tuning(plan.handle, k)["tma_mask"] >> 8 for k in (0, 1)]


@pytest.mark.parametrize("shape", [(512, 512, 8), (256, 256, 24), (256, 256, 2)])
def test_plane_c2c(gb, shape):
    nx, ny, nz = shape
    x = synth.uniform_complex((2, nz, ny, nx), seed=90 + nz)
    fused = gb.Plan(nx, ny, nz, batch=2, slab=True)
    staged = gb.Plan(nx, ny, nz, batch=2, slab=True, staged=True)
    xd = x.cuda()
    y = fused.forward(xd)
    z = fused.inverse(y)
    y2 = staged.forward(xd)
    z2 = staged.inverse(y2)
    torch.cuda.synchronize()
    assert fused.device_error() == 0
    ref = oracle.fft3(x.numpy())
    e = oracle.rel_l2(y.cpu().numpy(), ref)
    e_rt = oracle.rel_l2(z.cpu().numpy(), x.numpy())
    print(f"[plane] c2c {shape} x2: fwd {e:.3e}, round trip {e_rt:.3e}")
    assert e < TOL and e_rt < TOL
    assert torch.equal(y, y2) and torch.equal(z, z2)


@pytest.mark.parametrize("shape", [(512, 512, 8), (256, 256, 16)])
def test_plane_r2c_c2r(gb, shape):
    nx, ny, nz = shape
    r = synth.normal_real((nz, ny, nx), seed=95 + nz)
    fused = gb.Plan(nx, ny, nz, kind="r2c", slab=True)
    staged = gb.Plan(nx, ny, nz, kind="r2c", slab=True, staged=True)
    rd = r.cuda()
    s = fused.forward(rd)
    back = fused.inverse(s)
    s2 = staged.forward(rd)
    back2 = staged.inverse(s2)
    a = fused.adjoint(s)
    a2 = staged.adjoint(s)
    torch.cuda.synchronize()
    assert fused.device_error() == 0
    e = oracle.rel_l2(s.cpu().numpy(), oracle.rfft3(r.numpy()))
    e_rt = oracle.rel_l2(back.cpu().numpy(), r.numpy())
    print(f"[plane] r2c {shape}: fwd {e:.3e}, round trip {e_rt:.3e}")
    assert e < TOL and e_rt < TOL
    assert torch.equal(s, s2) and torch.equal(back, back2) and torch.equal(a, a2)


def test_plane_poisson_256(gb):
    n = 256
    f, _ = synth.poisson_rhs(n, seed=4)
    fused = gb.Plan(n, n, n, kind="r2c", slab=True)
    staged = gb.Plan(n, n, n, kind="r2c", slab=True, staged=True)
    fd = f.cuda()
    phi = fused.poisson(fd)
    phi2 = staged.poisson(fd)
    torch.cuda.synchronize()
    e = oracle.rel_l2(phi.cpu().numpy(), oracle.poisson(f.numpy()))
    print(f"[plane] poisson 256^3 slab: {e:.3e}")
    assert e < TOL and torch.equal(phi, phi2)


def test_plane_autotune_and_pinned_choice(gb):
    """The autotuner may keep the fused launch; pinning it by hand gives the same bits."""
    from paper_2601_12209_gb300 import abi
    nx = ny = 256
    nz = 32
    x = synth.uniform_complex((nz, ny, nx), seed=99).cuda()
    p = gb.Plan(nx, ny, nz, slab=True)
    ref = p.forward(x)
    p.autotune()
    print(f"[plane] autotune plane bits {_plane_bits(gb, p)}")
    assert torch.equal(p.forward(x), ref)
    q = gb.Plan(nx, ny, nz, slab=True)
    abi.gbfft_plan_set_tuning(q.handle, 0, 0, 1 << 8)  # stages 0 and 1 fused, stage 2 thread loads
    assert _plane_bits(gb, q)[0] == 1
    assert torch.equal(q.forward(x), ref)
    abi.gbfft_plan_set_tuning(q.handle, 0, 0, 0)  # plain stage launches
    assert torch.equal(q.forward(x), ref)
