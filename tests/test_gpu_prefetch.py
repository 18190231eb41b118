"""C2R x stage with the next tile's column-side half spectrum prefetched by cp.async into a
second shared-memory buffer: the inverse, the adjoint (interior bins scaled) and the Poisson
solve of R2C plans, pinned to that kernel through the tuning bits, against the FP64 oracle.
Ragged tiles (ny not a multiple of 16) take the kernel's synchronous fused load for their last
chunk; batch entries and half-spectrum lengths 128, 256 and 512 are covered."""
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


@pytest.mark.parametrize("shape,batch", [((512, 48, 40), 1), ((512, 40, 24), 2), ((256, 24, 20), 1),
                                         ((1024, 32, 16), 1), ((512, 512, 64), 1)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else f"b{v}")
def test_prefetch_c2r_x_stage(gb, shape, batch):
    from paper_2601_12209_gb300 import abi
    nx, ny, nz = shape
    r = synth.normal_real((batch, nz, ny, nx), seed=90 + ny + nz)
    p = gb.Plan(nx, ny, nz, kind="r2c", batch=batch, staged=True)
    for pipe in (1, 2):  # inverse (INVERSE, ADJOINT) and Poisson pipelines: every eligible stage prefetches
        abi.gbfft_plan_set_tuning(p.handle, pipe, False, 0xF << 28)
    assert abi.gbfft_plan_get_tuning(p.handle, 1)["tma_mask"] >> 28 == 0xF
    s = p.forward(r.cuda())
    back = p.inverse(s)
    adj = p.adjoint(s)
    phi = p.poisson(r.cuda()) if batch == 1 else None
    torch.cuda.synchronize()
    assert p.device_error() == 0
    sh = s.cpu().numpy()
    e_rt = oracle.rel_l2(back.cpu().numpy(), r.numpy())
    e_inv = oracle.rel_l2(back.cpu().numpy(), oracle.irfft3(sh.astype("complex128"), nx))
    e_adj = oracle.rel_l2(adj.cpu().numpy(), oracle.r2c_adjoint(sh.astype("complex128"), nx))
    msg = f"[prefetch] {shape} batch={batch}: inverse {e_inv:.3e}, round trip {e_rt:.3e}, adjoint {e_adj:.3e}"
    assert e_rt < TOL and e_inv < TOL and e_adj < TOL
    if phi is not None:
        e_p = oracle.rel_l2(phi.cpu().numpy(), oracle.poisson(r.numpy()))
        msg += f", poisson {e_p:.3e}"
        assert e_p < TOL
    print(msg)
