"""Slab plane launches with each plane's intermediate in distributed shared memory.

R2C plans of 512-point rows (ny = 512 or 256): an 8-CTA cluster per xy-plane runs the
x and y stages with the plane held in the cluster's shared memory (tuning bit 27 plus
the plane bits of the in-plane pairs). Every op is checked against the FP64 oracle,
including an inverse of a non-Hermitian spectrum (the packed real-bin columns must
reproduce the C2R projection), the adjoints and the Poisson solve; the per-launch
timing confirms that each in-plane pair ran as one launch.
"""
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
DSM = 1 << 27


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_12209_gb300 import _build
    _build.build()
    import paper_2601_12209_gb300 as gbmod
    return gbmod


def _pin_dsm(plan):
    """Forward X,Y | Z: pair at stage 0; inverse Z | Y,X: pair at 1; Poisson X,Y | PZ | Yi,Xi: 0 and 3."""
    from paper_2601_12209_gb300 import abi
    abi.gbfft_plan_set_tuning(plan.handle, 0, False, DSM | (1 << 8))
    abi.gbfft_plan_set_tuning(plan.handle, 1, False, DSM | (1 << 9))
    abi.gbfft_plan_set_tuning(plan.handle, 2, False, DSM | (1 << 8) | (1 << 11))


def _segments(plan, pipeline, fn):
    from paper_2601_12209_gb300 import abi
    abi.gbfft_plan_time_stages(plan.handle, True)
    out = fn()
    torch.cuda.synchronize()
    abi.gbfft_plan_time_stages(plan.handle, False)
    seg, ncalls = abi.gbfft_plan_stage_times(plan.handle, pipeline)
    return out, len(seg), ncalls


@pytest.mark.parametrize("shape,batch", [((512, 512, 8), 1), ((512, 256, 6), 2), ((512, 512, 3), 1),
                                         ((512, 256, 40), 1)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else f"b{v}")
def test_plane_dsm_r2c_ops(gb, shape, batch):
    nx, ny, nz = shape
    nxc = nx // 2 + 1
    r = synth.normal_real((batch, nz, ny, nx), seed=120 + ny + nz)
    h = synth.uniform_complex((batch, nz, ny, nxc), seed=121 + nz)  # not Hermitian
    p = gb.Plan(nx, ny, nz, kind="r2c", batch=batch, slab=True)
    _pin_dsm(p)
    rd, hd = r.cuda(), h.cuda()
    s, nseg_f, nc_f = _segments(p, 0, lambda: p.forward(rd))
    back, nseg_i, nc_i = _segments(p, 1, lambda: p.inverse(s))
    assert (nseg_f, nc_f, nseg_i, nc_i) == (2, 1, 2, 1)  # plane launch + z stage, each way
    inv_h = p.inverse(hd)
    adj = p.adjoint(hd)
    iadj = p.inverse_adjoint(rd)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    rn, hn = r.numpy(), h.numpy().astype("complex128")
    errs = {
        "forward": oracle.rel_l2(s.cpu().numpy(), oracle.rfft3(rn)),
        "round trip": oracle.rel_l2(back.cpu().numpy(), rn),
        "inverse non-Hermitian": oracle.rel_l2(inv_h.cpu().numpy(), oracle.irfft3(hn, nx)),
        "adjoint": oracle.rel_l2(adj.cpu().numpy(), oracle.r2c_adjoint(hn, nx)),
        "inverse adjoint": oracle.rel_l2(iadj.cpu().numpy(), oracle.c2r_scaled_adjoint(rn)),
    }
    if batch == 1:
        f = r[0] - r[0].mean()
        phi, nseg_p, _ = _segments(p, 2, lambda: p.poisson(f.contiguous().cuda()))
        assert nseg_p == 3  # two plane launches + the fused Poisson z stage
        errs["poisson"] = oracle.rel_l2(phi.cpu().numpy(), oracle.poisson(f.numpy()))
    print(f"[plane dsm] {shape} batch={batch}: " + ", ".join(f"{k} {v:.3e}" for k, v in errs.items()))
    assert all(v < TOL for v in errs.values()), errs
    # the same plan without the distributed-shared-memory launches (plain stage launches) agrees
    from paper_2601_12209_gb300 import abi
    for pipe in (0, 1, 2):
        abi.gbfft_plan_set_tuning(p.handle, pipe, False, 0)
    s2 = p.forward(rd)
    torch.cuda.synchronize()
    assert oracle.rel_l2(s.cpu().numpy(), s2.cpu().numpy()) < TOL


def test_plane_dsm_512_cube(gb):
    """The benchmark's grid: 512^3 R2C slab forward and round trip through the DSM plane launches."""
    n = 512
    r = synth.normal_real((n, n, n), seed=7)
    p = gb.Plan(n, n, n, kind="r2c", slab=True)
    _pin_dsm(p)
    rd = r.cuda()
    s = p.forward(rd)
    back = p.inverse(s)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    e_f = oracle.rel_l2(s.cpu().numpy(), oracle.rfft3(r.numpy()))
    e_rt = oracle.rel_l2(back.cpu().numpy(), r.numpy())
    print(f"[plane dsm] 512^3: forward {e_f:.3e}, round trip {e_rt:.3e}")
    assert e_f < TOL and e_rt < TOL


def test_plane_dsm_autotune_candidate(gb):
    """The autotuner times the DSM plane launch among the slab candidates; whatever it keeps is correct."""
    from paper_2601_12209_gb300 import abi
    nx, ny, nz = 512, 512, 32
    r = synth.normal_real((nz, ny, nx), seed=8)
    p = gb.Plan(nx, ny, nz, kind="r2c", slab=True)
    t = p.autotune()
    bits = [abi.gbfft_plan_get_tuning(p.handle, k)["tma_mask"] for k in (0, 1)]
    print(f"[plane dsm] autotune 512x512x32: dsm {[(b >> 27) & 1 for b in bits]}, "
          f"plane {[(b >> 8) & 0xFF for b in bits]}, ms {[t['forward']['ms'], t['inverse']['ms']]}")
    rd = r.cuda()
    s = p.forward(rd)
    back = p.inverse(s)
    torch.cuda.synchronize()
    assert oracle.rel_l2(s.cpu().numpy(), oracle.rfft3(r.numpy())) < TOL
    assert oracle.rel_l2(back.cpu().numpy(), r.numpy()) < TOL
