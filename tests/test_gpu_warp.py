"""Warp-per-pencil stage kernels (L = R1 x 32 in registers, a per-warp transpose and
lane shuffles; lengths 512 and 256, and the length-256 R2C split / C2R merge x stages):
every stage position (row/column input and output, in place in the slab schedule)
against the FP64 oracle, pinned through the tuning bits."""
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


def _pin_warp(plan, pipes=(0, 1)):
    from paper_2601_12209_gb300 import abi
    for k in pipes:
        abi.gbfft_plan_set_tuning(plan.handle, k, False, 0x1F << 20)  # every eligible stage: warp kernel


@pytest.mark.parametrize("shape,slab,batch", [((512, 24, 20), False, 1), ((24, 512, 20), False, 2),
                                              ((20, 24, 512), False, 1), ((512, 512, 4), True, 1),
                                              ((48, 512, 512), False, 1), ((256, 40, 24), False, 1),
                                              ((24, 256, 40), False, 2), ((40, 24, 256), False, 1),
                                              ((256, 256, 6), True, 1)])
def test_warp512_c2c(gb, shape, slab, batch):
    nx, ny, nz = shape
    x = synth.uniform_complex((batch, nz, ny, nx), seed=60 + nx + ny)
    p = gb.Plan(nx, ny, nz, batch=batch, slab=slab)
    _pin_warp(p)
    y = p.forward(x.cuda())
    z = p.inverse(y)
    a = p.adjoint(x.cuda())
    torch.cuda.synchronize()
    assert p.device_error() == 0
    e = oracle.rel_l2(y.cpu().numpy(), oracle.fft3(x.numpy()))
    e_rt = oracle.rel_l2(z.cpu().numpy(), x.numpy())
    e_adj = oracle.rel_l2(a.cpu().numpy(), oracle.c2c_adjoint(x.numpy()))
    print(f"[warp] {shape} slab={slab} batch={batch}: fwd {e:.3e}, round trip {e_rt:.3e}, adjoint {e_adj:.3e}")
    assert e < TOL and e_rt < TOL and e_adj < TOL


def test_warp512_r2c_512_cube(gb):
    """The 512^3 R2C configuration with the y and z stages on the warp kernel."""
    n = 512
    r = synth.normal_real((n, n, n), seed=2)
    p = gb.Plan(n, n, n, kind="r2c", staged=True)
    _pin_warp(p)
    s = p.forward(r.cuda())
    back = p.inverse(s)
    torch.cuda.synchronize()
    e = oracle.rel_l2(s.cpu().numpy(), oracle.rfft3(r.numpy()))
    e_rt = oracle.rel_l2(back.cpu().numpy(), r.numpy())
    print(f"[warp] r2c 512^3: fwd {e:.3e}, round trip {e_rt:.3e}")
    assert e < TOL and e_rt < TOL


@pytest.mark.parametrize("shape,slab", [((512, 48, 40), False), ((512, 40, 24), True), ((512, 256, 16), False)])
def test_warp_r2c_x_stage(gb, shape, slab):
    """The length-256 real x stages (R2C split after, C2R merge before the transform),
    with the Poisson pipeline and the adjoints that scale the interior bins."""
    nx, ny, nz = shape
    r = synth.normal_real((nz, ny, nx), seed=70 + ny)
    p = gb.Plan(nx, ny, nz, kind="r2c", slab=slab)
    _pin_warp(p, pipes=(0, 1, 2))
    s = p.forward(r.cuda())
    back = p.inverse(s)
    adj = p.adjoint(s)
    phi = p.poisson(r.cuda())
    torch.cuda.synchronize()
    assert p.device_error() == 0
    e = oracle.rel_l2(s.cpu().numpy(), oracle.rfft3(r.numpy()))
    e_rt = oracle.rel_l2(back.cpu().numpy(), r.numpy())
    e_adj = oracle.rel_l2(adj.cpu().numpy(), oracle.r2c_adjoint(s.cpu().numpy().astype("complex128"), nx))
    e_p = oracle.rel_l2(phi.cpu().numpy(), oracle.poisson(r.numpy()))
    print(f"[warp] r2c {shape} slab={slab}: fwd {e:.3e}, round trip {e_rt:.3e}, adjoint {e_adj:.3e}, poisson {e_p:.3e}")
    assert e < TOL and e_rt < TOL and e_adj < TOL and e_p < TOL


@pytest.mark.parametrize("shape,slab,batch", [((20, 24, 512), False, 2), ((40, 6, 256), False, 1),
                                              ((48, 20, 256), True, 2), ((30, 512, 512), False, 1)])
def test_warp_merged_z_pencils(gb, shape, slab, batch):
    """z stages whose spectrum side is the natural [z][y][kx] layout run with the outer (y)
    and group (kx) indices merged into one pencil axis of ny * (nx/2+1) pencils: chunks that
    cross a y row, a ragged last chunk, batch entries, and the in-place slab z stage."""
    nx, ny, nz = shape
    r = synth.normal_real((batch, nz, ny, nx), seed=80 + nx + nz)
    p = gb.Plan(nx, ny, nz, kind="r2c", batch=batch, slab=slab)
    _pin_warp(p)
    s = p.forward(r.cuda())
    back = p.inverse(s)
    adj = p.adjoint(s)
    torch.cuda.synchronize()
    assert p.device_error() == 0
    e = oracle.rel_l2(s.cpu().numpy(), oracle.rfft3(r.numpy()))
    e_rt = oracle.rel_l2(back.cpu().numpy(), r.numpy())
    e_adj = oracle.rel_l2(adj.cpu().numpy(), oracle.r2c_adjoint(s.cpu().numpy().astype("complex128"), nx))
    print(f"[warp] merged z {shape} slab={slab} batch={batch}: fwd {e:.3e}, round trip {e_rt:.3e}, "
          f"adjoint {e_adj:.3e}")
    assert e < TOL and e_rt < TOL and e_adj < TOL


def test_persistent_launch_with_warp_body_c2c_512_cube(gb):
    """The persistent ticket-queue launch (one launch per transform, bounded per-chunk dependency
    waits) running the warp-per-pencil tile body on its length-512 stages: the same bits as the
    staged warp-per-pencil launches, and the FP64 oracle, forward and inverse at 512^3 C2C."""
    from paper_2601_12209_gb300 import abi
    n = 512
    x = synth.uniform_complex((n, n, n), seed=3)
    xd = x.cuda()
    s = gb.Plan(n, n, n, staged=True)
    _pin_warp(s)
    ys = s.forward(xd)
    zs = s.inverse(ys)
    p = gb.Plan(n, n, n)
    for log_t in (0, 1, 2):  # 1, 2, 4 tiles per ticket
        for pipe in (0, 1):
            abi.gbfft_plan_set_tuning(p.handle, pipe, True, (0x7 << 20) | (log_t << 25))
        t = abi.gbfft_plan_get_tuning(p.handle, 0)
        assert t["persistent"] and (t["tma_mask"] >> 20) & 0x7 == 0x7 and (t["tma_mask"] >> 25) & 0x3 == log_t
        y = p.forward(xd)
        z = p.inverse(y)
        torch.cuda.synchronize()
        assert p.device_error() == 0
        assert torch.equal(y, ys) and torch.equal(z, zs), log_t
    e = oracle.rel_l2(y.cpu().numpy(), oracle.fft3(x.numpy()))
    e_rt = oracle.rel_l2(z.cpu().numpy(), x.numpy())
    print(f"[warp] persistent warp body c2c 512^3: fwd {e:.3e}, round trip {e_rt:.3e}")
    assert e < TOL and e_rt < TOL


@pytest.mark.parametrize("shape,slab,batch", [((1024, 24, 20), False, 1), ((24, 1024, 20), False, 2),
                                              ((20, 24, 1024), False, 1), ((1024, 1024, 2), True, 1),
                                              ((48, 1024, 40), False, 1)])
def test_warp1024_c2c(gb, shape, slab, batch):
    """Length-1024 warp-per-pencil stages (32 values per lane, radix 32 in registers twice): every
    stage position (row and column input and output, in place in the slab schedule, merged z
    pencils), forward, inverse and adjoint against the FP64 oracle."""
    nx, ny, nz = shape
    x = synth.uniform_complex((batch, nz, ny, nx), seed=95 + nx + ny)
    p = gb.Plan(nx, ny, nz, batch=batch, slab=slab)
    _pin_warp(p)
    y = p.forward(x.cuda())
    z = p.inverse(y)
    a = p.adjoint(x.cuda())
    torch.cuda.synchronize()
    assert p.device_error() == 0
    e = oracle.rel_l2(y.cpu().numpy(), oracle.fft3(x.numpy()))
    e_rt = oracle.rel_l2(z.cpu().numpy(), x.numpy())
    e_adj = oracle.rel_l2(a.cpu().numpy(), oracle.c2c_adjoint(x.numpy()))
    print(f"[warp] 1024 {shape} slab={slab} batch={batch}: fwd {e:.3e}, round trip {e_rt:.3e}, adjoint {e_adj:.3e}")
    assert e < TOL and e_rt < TOL and e_adj < TOL


@pytest.mark.parametrize("kind", ["c2c", "r2c"])
def test_persistent_tiles_per_ticket_bitwise(gb, kind):
    """Tickets of 1, 2 and 4 consecutive tiles in the persistent launch (Stockham tile bodies): the same
    bits in every case, forward, inverse and (R2C) the five-stage Poisson pipeline; the FP64 oracle."""
    from paper_2601_12209_gb300 import abi
    n = 64
    x = (synth.normal_real((2, n, n, n), seed=97) if kind == "r2c" else synth.uniform_complex((2, n, n, n), seed=97))
    p = gb.Plan(n, n, n, kind=kind, batch=2)
    outs = []
    for log_t in (0, 1, 2):
        for pipe in ((0, 1, 2) if kind == "r2c" else (0, 1)):
            abi.gbfft_plan_set_tuning(p.handle, pipe, True, log_t << 25)
        y = p.forward(x.cuda())
        z = p.inverse(y)
        ph = p.poisson(x.cuda()) if kind == "r2c" else None
        torch.cuda.synchronize()
        assert p.device_error() == 0
        outs.append((y, z, ph))
    for y, z, ph in outs[1:]:
        assert torch.equal(y, outs[0][0]) and torch.equal(z, outs[0][1])
        if ph is not None:
            assert torch.equal(ph, outs[0][2])
    ref = oracle.rfft3(x.numpy()) if kind == "r2c" else oracle.fft3(x.numpy())
    assert oracle.rel_l2(outs[0][0].cpu().numpy(), ref) < TOL
    assert oracle.rel_l2(outs[0][1].cpu().numpy(), x.numpy()) < TOL
    with pytest.raises(abi.GbfftError):
        abi.gbfft_plan_set_tuning(p.handle, 0, True, 3 << 25)  # 8 tiles per ticket: not built


@pytest.mark.parametrize("kind", ["c2c", "r2c"])
def test_persistent_repeated_equals_staged(gb, kind):
    """Repeated one-launch transforms against the stage launches, bit for bit. The last stage of a pencil
    pipeline overwrites the buffer its middle stage reads (and the Poisson pipeline's inverse y stage the
    forward y stage's input), so inside one launch it must wait for that whole stage; a tile that ran ahead
    would corrupt data another tile had not yet read. 60 launches per tile-per-ticket choice."""
    from paper_2601_12209_gb300 import abi
    n = 64
    x = (synth.normal_real((2, n, n, n), seed=98) if kind == "r2c" else synth.uniform_complex((2, n, n, n), seed=98))
    xd = x.cuda()
    ref = gb.Plan(n, n, n, kind=kind, batch=2, staged=True)
    y0 = ref.forward(xd)
    z0 = ref.inverse(y0)
    p = gb.Plan(n, n, n, kind=kind, batch=2)
    pipes = (0, 1, 2) if kind == "r2c" else (0, 1)
    ph0 = None
    if kind == "r2c":
        rp = gb.Plan(n, n, n, kind=kind, staged=True)
        pq = gb.Plan(n, n, n, kind=kind)
        ph0 = rp.poisson(xd[0])
    for log_t in (0, 2):
        for pipe in pipes:
            abi.gbfft_plan_set_tuning(p.handle, pipe, True, log_t << 25)
        if kind == "r2c":
            abi.gbfft_plan_set_tuning(pq.handle, 2, True, log_t << 25)
        for _ in range(60):
            y = p.forward(xd)
            z = p.inverse(y)
            assert torch.equal(y, y0) and torch.equal(z, z0)
            if kind == "r2c":
                assert torch.equal(pq.poisson(xd[0]), ph0)
    torch.cuda.synchronize()
    assert p.device_error() == 0
