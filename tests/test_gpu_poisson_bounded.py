"""(Periodic, Periodic, Bounded) Poisson solve: DCT-II / DCT-III along z fused into the z
stage (each one length-nz complex FFT), against the FP64 oracle and the closed form."""
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


@pytest.mark.parametrize("shape,slab", [((64, 64, 64), False), ((64, 64, 64), True), ((32, 24, 15), False),
                                        ((40, 30, 48), True), ((48, 20, 5), False), ((256, 256, 256), False)])
def test_poisson_bounded_vs_oracle(gb, shape, slab):
    nx, ny, nz = shape
    f, _ = synth.poisson_rhs(nx, seed=4) if nx == ny == nz else (synth.normal_real((nz, ny, nx), seed=81), None)
    p = gb.Plan(nx, ny, nz, kind="r2c", slab=slab)
    phi = p.poisson(f.cuda(), bounded=True)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    e = oracle.rel_l2(phi.cpu().numpy(), oracle.poisson_bounded(f.numpy()))
    print(f"[poisson-bounded] {shape} slab={slab}: rel-L2 {e:.3e}")
    assert e < TOL


def test_poisson_bounded_closed_form_and_host(gb):
    from paper_2601_12209_gb300 import abi
    nx, ny, nz = 64, 48, 40
    i, j, n = np.arange(nx), np.arange(ny), np.arange(nz)
    kx, ky, kz = 5, -3, 7
    f = (np.cos(kz * (n + 0.5) * np.pi / nz)[:, None, None]
         * np.cos(kx * 2 * np.pi * i / nx + ky * 2 * np.pi * j[:, None] / ny)[None, :, :])
    ft = torch.from_numpy(f.astype(np.float32))
    p = gb.Plan(nx, ny, nz, kind="r2c")
    phi = p.poisson(ft.cuda(), bounded=True).cpu().numpy()
    exact = -f / (kx * kx + ky * ky + kz * kz)
    e = oracle.rel_l2(phi, exact)
    print(f"[poisson-bounded] closed form mode {(kx, ky, kz)}: rel-L2 {e:.3e}")
    assert e < TOL
    h_out = torch.empty_like(ft).pin_memory()
    p.exec_host(abi.GBFFT_OP_POISSON_BOUNDED, ft.pin_memory(), h_out)
    assert torch.equal(h_out, torch.from_numpy(phi))
