"""Real-to-real transforms along z (DCT-II/III, DST-II/III as one length-nz FFT each) with
Fourier x and y: against the FP64 oracle, and forward-inverse round trips."""
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


@pytest.mark.parametrize("kind", ["dct", "dst"])
@pytest.mark.parametrize("plan_kind,shape,slab", [("r2c", (64, 48, 40), False), ("r2c", (32, 24, 15), True),
                                                  ("c2c", (40, 30, 64), False), ("c2c", (24, 20, 5), True),
                                                  ("r2c", (512, 128, 512), False)])
def test_r2r_z(gb, kind, plan_kind, shape, slab):
    nx, ny, nz = shape
    if plan_kind == "r2c":
        x = synth.normal_real((nz, ny, nx), seed=90 + nz)
    else:
        x = synth.uniform_complex((nz, ny, nx), seed=90 + nz)
    p = gb.Plan(nx, ny, nz, kind=plan_kind, slab=slab)
    y = p.r2r_z(x.cuda(), kind)
    back = p.r2r_z(y, kind, inverse=True)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    ref = oracle.r2r_z(x.numpy(), kind)
    e = oracle.rel_l2(y.cpu().numpy(), ref)
    ref_inv = oracle.r2r_z(y.cpu().numpy(), kind, inverse=True, nx=nx if plan_kind == "r2c" else None)
    e_inv = oracle.rel_l2(back.cpu().numpy(), ref_inv)
    e_rt = oracle.rel_l2(back.cpu().numpy(), x.numpy())
    print(f"[r2r] {kind} {plan_kind} {shape} slab={slab}: fwd {e:.3e}, inverse {e_inv:.3e}, round trip {e_rt:.3e}")
    assert e < TOL and e_inv < TOL and e_rt < TOL


@pytest.mark.parametrize("kinds", [("dct", "dst", None), ("dst", "dct", "dct"), (None, "dst", "dst"),
                                   ("dct", "dct", "dct")])
@pytest.mark.parametrize("shape,slab", [((40, 30, 24), False), ((15, 32, 20), True), ((256, 64, 32), False)])
def test_r2r_per_axis_c2c(gb, kinds, shape, slab):
    """Any axis real-to-real on complex data (C2C plans), against the per-axis oracle."""
    nx, ny, nz = shape
    x = synth.uniform_complex((nz, ny, nx), seed=95 + nx)
    p = gb.Plan(nx, ny, nz, slab=slab)
    y = p.r2r(x.cuda(), kinds)
    back = p.r2r(y, kinds, inverse=True)
    torch.cuda.synchronize()
    e = oracle.rel_l2(y.cpu().numpy(), oracle.r2r(x.numpy(), kinds))
    e_rt = oracle.rel_l2(back.cpu().numpy(), x.numpy())
    print(f"[r2r] {kinds} c2c {shape} slab={slab}: fwd {e:.3e}, round trip {e_rt:.3e}")
    assert e < TOL and e_rt < TOL


def test_r2r_y_on_r2c_and_rejections(gb):
    from paper_2601_12209_gb300 import abi
    nx, ny, nz = 64, 48, 40
    r = synth.normal_real((nz, ny, nx), seed=97)
    p = gb.Plan(nx, ny, nz, kind="r2c")
    y = p.r2r(r.cuda(), (None, "dct", "dst"))
    back = p.r2r(y, (None, "dct", "dst"), inverse=True)
    torch.cuda.synchronize()
    assert oracle.rel_l2(y.cpu().numpy(), oracle.r2r(r.numpy(), (None, "dct", "dst"))) < TOL
    assert oracle.rel_l2(back.cpu().numpy(), r.numpy()) < TOL
    with pytest.raises(Exception):  # x is the real axis of an R2C plan
        p.r2r(r.cuda(), ("dct", None, None))
