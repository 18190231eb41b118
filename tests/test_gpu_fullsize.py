"""Full-size parity at the benchmark's sizes, in the launch configurations the
benchmark times (the autotuned pencil plan it publishes, the persistent and
staged pencil launches, the slab variant): every output element against the
FP64 oracle, plus direct triple-sum DFT samples.
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
    print(f"[parity-full] {name}: rel-L2 {e:.3e}")
    return e


def _tuned(plan, mode):
    """The autotuned plan is the one the benchmark times: tune it the same way."""
    if mode == "pencil_tuned":
        tuning = plan.autotune()
        print(f"[parity-full] tuning {tuning}")


@pytest.mark.parametrize("mode", ["pencil_tuned", "pencil", "pencil_staged", "slab"])
def test_r2c_c2r_512(gb, mode):
    """Config: R2C forward and C2R inverse at 512^3 FP32, real N(0,1) input."""
    n = 512
    slab = mode == "slab"
    r = synth.normal_real((n, n, n), seed=2)
    plan = gb.Plan(n, n, n, kind="r2c", slab=slab, staged=(mode == "pencil_staged"))
    _tuned(plan, mode)
    rd = r.cuda()
    H = plan.forward(rd)
    r2 = plan.inverse(H)
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    Hh = H.cpu().numpy()
    ref = oracle.rfft3(r.numpy())
    assert err(f"r2c 512 fwd {mode}", Hh, ref) < TOL
    # direct triple-sum DFT at sampled bins (no factorisation involved)
    rng = np.random.default_rng(5)
    bins = [(int(rng.integers(0, n // 2 + 1)), int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(4)]
    direct = oracle.dft3_bins(r.numpy().astype(np.complex128), bins)
    got = np.array([Hh[kz, ky, kx] for (kx, ky, kz) in bins])
    assert err("r2c 512 direct-DFT samples", got, direct) < TOL
    del ref, Hh
    assert err(f"r2c 512 roundtrip {mode}", r2.cpu().numpy(), r.numpy()) < TOL


@pytest.mark.parametrize("mode", ["pencil_tuned", "pencil", "pencil_staged", "slab"])
def test_c2c_512(gb, mode):
    """C2C forward+inverse at 512^3, complex64 uniform[-1,1] (the headline C2C configuration)."""
    n = 512
    slab = mode == "slab"
    x = synth.uniform_complex((n, n, n), seed=3)
    plan = gb.Plan(n, n, n, slab=slab, staged=(mode == "pencil_staged"))
    _tuned(plan, mode)
    X = plan.forward(x.cuda())
    torch.cuda.synchronize()
    Xh = X.cpu().numpy()
    ref = oracle.fft3(x.numpy())
    assert err(f"c2c 512 fwd {mode}", Xh, ref) < TOL
    del ref
    xr = plan.inverse(X)
    assert err(f"c2c 512 roundtrip {mode}", xr.cpu().numpy(), x.numpy()) < TOL
    assert plan.device_error() == 0


def test_c2r_512_non_hermitian_projection(gb):
    n = 512
    h = synth.uniform_complex((n, n, n // 2 + 1), seed=8)
    plan = gb.Plan(n, n, n, kind="r2c")
    got = plan.inverse(h.cuda())
    assert err("c2r 512 non-Hermitian", got.cpu().numpy(), oracle.irfft3(h.numpy(), n)) < TOL
