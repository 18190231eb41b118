"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Floating point: relative L2 error <= 1e-5 over the whole output (the bound
stated for FP32 C2C/R2C at 512^3); every error is printed. Index maps: the
redistribution-alone debug steps must reproduce bit patterns exactly.
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


def dev():
    return torch.device("cuda:0")


def err(name, got, ref):
    e = oracle.rel_l2(got, ref)
    print(f"[parity] {name}: rel-L2 {e:.3e}")
    return e


C2C_SHAPES = [  # (nx, ny, nz, batch)
    (8, 8, 8, 1), (16, 12, 10, 2), (64, 64, 64, 1), (60, 48, 80, 1), (24, 40, 30, 2), (32, 128, 20, 1),
    (256, 16, 8, 1), (5, 6, 3, 1), (1024, 4, 2, 1), (30, 160, 96, 1),
]


MODES = ["pencil", "pencil_staged", "pencil_staged_lsu", "slab", "slab_staged"]


def make_plan(gb, nx, ny, nz, mode, **kw):
    """pencil: persistent launch; *_staged: one launch per stage (tensor-copy loads where the
    layout allows); *_lsu: staged with thread loads only."""
    return gb.Plan(nx, ny, nz, slab=mode.startswith("slab"), staged="staged" in mode, tma=not mode.endswith("lsu"),
                   **kw)


@pytest.mark.parametrize("shape", C2C_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("mode", MODES)
def test_c2c_forward_inverse(gb, shape, mode):
    nx, ny, nz, b = shape
    x = synth.uniform_complex((b, nz, ny, nx), seed=1 + nx + ny + nz)
    plan = make_plan(gb, nx, ny, nz, mode, batch=b)
    xd = x.to(dev())
    X = plan.forward(xd)
    xr = plan.inverse(X)
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    ref = oracle.fft3(x.numpy())
    assert err(f"c2c fwd {shape} {mode}", X.cpu().numpy(), ref) < TOL
    assert err(f"c2c roundtrip {shape} {mode}", xr.cpu().numpy(), x.numpy()) < TOL
    # inverse alone against the oracle inverse of the same input
    xi = plan.inverse(xd)
    assert err(f"c2c inv {shape} {mode}", xi.cpu().numpy(), oracle.ifft3(x.numpy())) < TOL
    assert torch.equal(xd.cpu(), x)  # input untouched (out-of-place)


def test_config1_tiny_c2c_64(gb):
    """64^3 complex64 uniform[-1,1]: round trip, Parseval, naive DFT on 8x8x8 blocks."""
    x = synth.uniform_complex((64, 64, 64), seed=1)
    plan = gb.Plan(64, 64, 64)
    X = plan.forward(x.to(dev()))
    xr = plan.inverse(X)
    Xh = X.cpu().numpy().astype(np.complex128)
    assert err("cfg1 roundtrip", xr.cpu().numpy(), x.numpy()) < TOL
    xn = x.numpy().astype(np.complex128)
    parseval = abs(np.sum(np.abs(Xh) ** 2) / (64 ** 3 * np.sum(np.abs(xn) ** 2)) - 1.0)
    print(f"[parity] cfg1 Parseval relative deviation {parseval:.3e}")
    assert parseval < 1e-5
    bins = [(kx, ky, kz) for kz in range(8) for ky in range(8) for kx in range(8)]
    off = (37, 21, 50)
    bins += [((kx + off[0]) % 64, (ky + off[1]) % 64, (kz + off[2]) % 64)
             for kz in range(8) for ky in range(8) for kx in range(8)]
    direct = oracle.dft3_bins(xn, bins)
    got = np.array([Xh[kz, ky, kx] for (kx, ky, kz) in bins])
    assert err("cfg1 naive DFT 2x8^3 bins", got, direct) < TOL
    assert err("cfg1 fwd full", Xh, oracle.fft3(xn)) < TOL


# odd ny (odd column strides, odd spectrum size per batch entry) and a ragged last tile after
# full ones: the real x stages switch between their two-pencil and one-pencil access paths
R2C_SHAPES = [(8, 8, 8, 1), (64, 64, 64, 1), (16, 12, 10, 2), (60, 48, 80, 1), (32, 20, 24, 1), (128, 30, 16, 1),
              (256, 16, 8, 1), (32, 15, 5, 2), (16, 40, 3, 2)]


@pytest.mark.parametrize("shape", R2C_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("mode", MODES)
def test_r2c_c2r(gb, shape, mode):
    nx, ny, nz, b = shape
    r = synth.normal_real((b, nz, ny, nx), seed=2 + nx)
    plan = make_plan(gb, nx, ny, nz, mode, kind="r2c", batch=b)
    H = plan.forward(r.to(dev()))
    r2 = plan.inverse(H)
    torch.cuda.synchronize()
    assert plan.device_error() == 0
    assert err(f"r2c fwd {shape} {mode}", H.cpu().numpy(), oracle.rfft3(r.numpy())) < TOL
    assert err(f"r2c roundtrip {shape} {mode}", r2.cpu().numpy(), r.numpy()) < TOL
    # C2R of a NON-Hermitian half spectrum: the Hermitian-projection reading
    h = synth.uniform_complex((b, nz, ny, nx // 2 + 1), seed=3 + nx)
    got = plan.inverse(h.to(dev()))
    assert err(f"c2r non-Hermitian {shape} {mode}", got.cpu().numpy(), oracle.irfft3(h.numpy(), nx)) < TOL


@pytest.mark.parametrize("kind", ["c2c", "r2c"])
@pytest.mark.parametrize("slab", [False, True])
def test_adjoint_ops(gb, kind, slab):
    nx, ny, nz = 16, 24, 20
    plan = gb.Plan(nx, ny, nz, kind=kind, slab=slab)
    if kind == "c2c":
        y = synth.uniform_complex((nz, ny, nx), seed=5)
        a = plan.adjoint(y.to(dev()))
        assert err("c2c adjoint", a.cpu().numpy(), oracle.c2c_adjoint(y.numpy())) < TOL
        ia = plan.inverse_adjoint(y.to(dev()))
        assert err("c2c inverse-adjoint", ia.cpu().numpy(), oracle.c2c_inverse_adjoint(y.numpy())) < TOL
    else:
        g = synth.uniform_complex((nz, ny, nx // 2 + 1), seed=6)
        a = plan.adjoint(g.to(dev()))
        assert err("r2c adjoint", a.cpu().numpy(), oracle.r2c_adjoint(g.numpy(), nx)) < TOL
        y = synth.normal_real((nz, ny, nx), seed=7)
        ia = plan.inverse_adjoint(y.to(dev()))
        assert err("c2r scaled adjoint", ia.cpu().numpy(), oracle.c2r_scaled_adjoint(y.numpy())) < TOL


def test_transposed_out(gb):
    nx, ny, nz = 32, 24, 16
    x = synth.uniform_complex((nz, ny, nx), seed=9)
    plan = gb.Plan(nx, ny, nz, transposed_out=True)
    C = plan.forward(x.to(dev()))
    assert C.shape[-3:] == (nx, ny, nz)
    ref = oracle.layout_a_to_c(oracle.fft3(x.numpy()))
    assert err("transposed-out fwd", C.cpu().numpy(), ref) < TOL
    xr = plan.inverse(C)
    assert err("transposed-out roundtrip", xr.cpu().numpy(), x.numpy()) < TOL


# ----------------------------------------------------- index maps (bit-exact)

@pytest.mark.parametrize("shape", [(16, 16, 16), (60, 48, 80), (120, 24, 40), (32, 20, 24), (8, 8, 8)],
                         ids=lambda s: "x".join(map(str, s)))
def test_redistribution_maps_bit_exact(gb, shape):
    """Debug steps 2/4/6 and 12/14/16 move data only; they must equal the oracle's
    explicit index maps bit for bit (integer-valued inputs)."""
    nx, ny, nz = shape
    plan = gb.Plan(nx, ny, nz)
    A = synth.integer_complex((nz, ny, nx), seed=11)
    Ad = A.to(dev())
    B = torch.empty((nz, nx, ny), dtype=torch.complex64, device=dev())
    plan.debug_run(2, Ad, B)
    assert torch.equal(B.cpu(), torch.from_numpy(oracle.layout_a_to_b(A.numpy())))
    C = torch.empty((nx, ny, nz), dtype=torch.complex64, device=dev())
    plan.debug_run(4, B, C)
    assert torch.equal(C.cpu(), torch.from_numpy(oracle.layout_b_to_c(B.cpu().numpy())))
    N = torch.empty((nz, ny, nx), dtype=torch.complex64, device=dev())
    plan.debug_run(6, C, N)
    assert torch.equal(N.cpu(), A)
    C2 = torch.empty_like(C)
    plan.debug_run(12, N, C2)
    assert torch.equal(C2.cpu(), C.cpu())
    B2 = torch.empty_like(B)
    plan.debug_run(14, C2, B2)
    assert torch.equal(B2.cpu(), B.cpu())
    A2 = torch.empty_like(Ad)
    plan.debug_run(16, B2, A2)
    assert torch.equal(A2.cpu(), A)


def test_redistribution_maps_r2c_halved_axis(gb):
    """Same bit-exact check for the y/z redistributions of an R2C plan (nx/2+1 bins)."""
    nx, ny, nz = 64, 20, 24
    nxc = nx // 2 + 1
    plan = gb.Plan(nx, ny, nz, kind="r2c")
    Bh = synth.integer_complex((nz, nxc, ny), seed=12)
    C = torch.empty((nxc, ny, nz), dtype=torch.complex64, device=dev())
    plan.debug_run(4, Bh.to(dev()), C)
    assert torch.equal(C.cpu(), torch.from_numpy(oracle.layout_b_to_c(Bh.numpy())))
    N = torch.empty((nz, ny, nxc), dtype=torch.complex64, device=dev())
    plan.debug_run(6, C, N)
    assert torch.equal(N.cpu(), torch.from_numpy(oracle.layout_c_to_a(C.cpu().numpy())))


@pytest.mark.parametrize("shape", [(32, 24, 20), (60, 48, 16)], ids=lambda s: "x".join(map(str, s)))
def test_each_stage_alone(gb, shape):
    """Each FFT stage alone (debug steps 1,3,5,11,13,15) equals the oracle 1D FFT
    along its axis composed with the stage's layout map."""
    nx, ny, nz = shape
    plan = gb.Plan(nx, ny, nz)
    A = synth.uniform_complex((nz, ny, nx), seed=13)
    An = A.numpy().astype(np.complex128)
    B = torch.empty((nz, nx, ny), dtype=torch.complex64, device=dev())
    plan.debug_run(1, A.to(dev()), B)
    assert err("stage x", B.cpu().numpy(), oracle.layout_a_to_b(oracle.fft1(An))) < TOL
    Bn = B.cpu().numpy().astype(np.complex128)
    C = torch.empty((nx, ny, nz), dtype=torch.complex64, device=dev())
    plan.debug_run(3, B, C)
    assert err("stage y", C.cpu().numpy(), oracle.layout_b_to_c(oracle.fft1(Bn))) < TOL
    Cn = C.cpu().numpy().astype(np.complex128)
    N = torch.empty((nz, ny, nx), dtype=torch.complex64, device=dev())
    plan.debug_run(5, C, N)
    assert err("stage z", N.cpu().numpy(), oracle.layout_c_to_a(oracle.fft1(Cn))) < TOL
    # inverse steps (unscaled, sign +)
    C2 = torch.empty_like(C)
    plan.debug_run(11, A.to(dev()), C2)
    assert err("stage z inv", C2.cpu().numpy(), oracle.fft1(oracle.layout_a_to_c(An), sign=+1)) < TOL
    B2 = torch.empty_like(B)
    plan.debug_run(13, C, B2)
    # y-inverse on C[x][y][z] along y, written as B[z][x][y]
    yinv = np.swapaxes(oracle.fft1(np.swapaxes(Cn, -1, -2).copy(), sign=+1), -1, -2)  # [x][y][z]
    ref = np.transpose(yinv, (2, 0, 1))  # B[z][x][y]
    assert err("stage y inv", B2.cpu().numpy(), ref) < TOL
    A2 = torch.empty_like(A.to(dev()))
    plan.debug_run(15, B, A2)
    xinv = oracle.fft1(Bn.swapaxes(-1, -2).copy(), sign=+1)  # [z][y][x]
    assert err("stage x inv", A2.cpu().numpy(), xinv) < TOL


def test_persistent_equals_staged_bitwise(gb):
    """The persistent launch, the staged launches with tensor-copy loads and the staged
    launches with thread loads run the same tile arithmetic: identical bits."""
    for kind, shape in (("c2c", (64, 64, 64)), ("r2c", (64, 64, 64)), ("c2c", (512, 64, 32)),
                        ("r2c", (512, 32, 64))):
        nx, ny, nz = shape
        x = synth.uniform_complex((nz, ny, nx), seed=21) if kind == "c2c" else synth.normal_real((nz, ny, nx), 22)
        p1 = gb.Plan(nx, ny, nz, kind=kind)
        p2 = gb.Plan(nx, ny, nz, kind=kind, staged=True)
        p3 = gb.Plan(nx, ny, nz, kind=kind, staged=True, tma=False)
        a = p1.forward(x.to(dev()))
        b = p2.forward(x.to(dev()))
        c = p3.forward(x.to(dev()))
        assert torch.equal(a, b) and torch.equal(a, c)
        assert torch.equal(p1.inverse(a), p2.inverse(b)) and torch.equal(p1.inverse(a), p3.inverse(c))
        assert p1.device_error() == 0 and p2.device_error() == 0 and p3.device_error() == 0


def test_device_timeout_is_reported_not_hung(gb):
    """Dependency waits are bounded: with the debug flag every wait targets one
    completion too many, times out after ~20 ms, and the error is returned."""
    plan = gb.Plan(64, 64, 64, debug_timeout=True)
    x = synth.uniform_complex((64, 64, 64), seed=31).to(dev())
    plan.forward(x)
    from paper_2601_12209_gb300 import abi
    assert plan.device_error() == abi.GBFFT_ERR_TIMEOUT
    assert plan.device_error() == 0  # read-and-clear
    ok = gb.Plan(64, 64, 64)
    X = ok.forward(x)
    assert err("after timeout", X.cpu().numpy(), oracle.fft3(x.cpu().numpy())) < TOL


def test_error_paths(gb):
    from paper_2601_12209_gb300 import abi
    plan = gb.Plan(16, 16, 16)
    x = torch.zeros((16, 16, 16), dtype=torch.complex64, device=dev())
    with pytest.raises(abi.GbfftError) as e:
        abi.gbfft_exec(plan.handle, 0, x.data_ptr(), x.data_ptr(), 0)
    assert e.value.code == abi.GBFFT_ERR_INPLACE
    y = torch.zeros(16 ** 3 + 2, dtype=torch.complex64, device=dev())
    with pytest.raises(abi.GbfftError) as e:
        abi.gbfft_exec(plan.handle, 0, x.data_ptr(), y.data_ptr() + 8, 0)
    assert e.value.code == abi.GBFFT_ERR_ALIGNMENT
    with pytest.raises(abi.GbfftError) as e:
        abi.gbfft_exec(plan.handle, 9, x.data_ptr(), y.data_ptr(), 0)
    assert e.value.code == abi.GBFFT_ERR_INVALID_ARG
    with pytest.raises(abi.GbfftError) as e:
        gb.Plan(14, 16, 16)
    assert e.value.code == abi.GBFFT_ERR_UNSUPPORTED_SIZE
    with pytest.raises(abi.GbfftError) as e:
        abi.gbfft_exec_poisson(plan.handle, x.data_ptr(), y.data_ptr(), 0)
    assert e.value.code == abi.GBFFT_ERR_INVALID_ARG


def test_caller_workspace(gb):
    plan = gb.Plan(32, 32, 32, kind="r2c")
    n = plan.workspace_size()
    assert n >= 2 * 17 * 32 * 32 * 8
    ws = torch.empty(n, dtype=torch.uint8, device=dev())
    plan.set_workspace(ws)
    r = synth.normal_real((32, 32, 32), seed=41)
    H = plan.forward(r.to(dev()))
    assert err("r2c with caller workspace", plan.inverse(H).cpu().numpy(), r.numpy()) < TOL


def test_exec_host_end_to_end(gb):
    """Pinned buffers (kernels read and write host memory directly) and pageable buffers
    (staging copies) give the device path's bits, for every op and both layouts."""
    from paper_2601_12209_gb300 import abi
    plan = gb.Plan(64, 48, 32)
    x = synth.uniform_complex((32, 48, 64), seed=51).pin_memory()
    out = torch.empty_like(x).pin_memory()
    plan.exec_host(abi.GBFFT_OP_FORWARD, x, out)
    assert err("exec_host fwd", out.numpy(), oracle.fft3(x.numpy())) < TOL
    for kind, shape, slab in (("c2c", (64, 48, 32), False), ("r2c", (64, 64, 48), False), ("r2c", (256, 256, 8), True),
                              ("c2c", (256, 256, 8), True)):
        nx, ny, nz = shape
        p = gb.Plan(nx, ny, nz, kind=kind, slab=slab)
        src = synth.normal_real((nz, ny, nx), seed=52) if kind == "r2c" else synth.uniform_complex((nz, ny, nx), seed=52)
        ref_f = p.forward(src.to(dev()))
        ref_i = p.inverse(ref_f)
        ops = [(abi.GBFFT_OP_FORWARD, src, ref_f), (abi.GBFFT_OP_INVERSE, ref_f.cpu(), ref_i),
               (abi.GBFFT_OP_ADJOINT, ref_f.cpu(), p.adjoint(ref_f))]
        if kind == "r2c":
            ops.append((4, src, p.poisson(src.to(dev()))))
        for op, hin, ref in ops:
            for pinned in (True, False):
                h_in = hin.contiguous().pin_memory() if pinned else hin.contiguous().clone()
                h_out = torch.empty(ref.shape, dtype=ref.dtype)
                h_out = h_out.pin_memory() if pinned else h_out
                p.exec_host(op, h_in, h_out)
                assert torch.equal(h_out, ref.cpu()), (kind, shape, slab, op, pinned)


@pytest.mark.parametrize("kind,shape,batch,tune", [("c2c", (64, 48, 32), 1, False), ("r2c", (64, 48, 40), 2, False),
                                                    ("r2c", (512, 48, 24), 1, True), ("c2c", (30, 20, 6), 2, False),
                                                    ("r2c", (32, 15, 5), 2, False), ("c2c", (24, 512, 20), 1, True)])
def test_exec_host_staged(gb, kind, shape, batch, tune):
    """Host buffers through plans run as stage launches: the bits equal the device path's for
    ops 0-3, pinned and pageable, with autotuned launch choices, batch entries of odd size
    and short z axes."""
    from paper_2601_12209_gb300 import abi
    nx, ny, nz = shape
    p = gb.Plan(nx, ny, nz, kind=kind, batch=batch, staged=True)
    if tune:
        p.autotune()
    r2c = kind == "r2c"
    src = synth.normal_real((batch, nz, ny, nx), seed=53) if r2c else \
        synth.uniform_complex((batch, nz, ny, nx), seed=53)
    src_d = src.to(dev())
    spec = p.forward(src_d)
    cases = [(abi.GBFFT_OP_FORWARD, src, spec), (abi.GBFFT_OP_INVERSE, spec.cpu(), p.inverse(spec)),
             (abi.GBFFT_OP_ADJOINT, spec.cpu(), p.adjoint(spec)),
             (abi.GBFFT_OP_INVERSE_ADJOINT, src, p.inverse_adjoint(src_d))]
    for op, hin, ref in cases:
        for pinned in (True, False):
            h_in = hin.contiguous().pin_memory() if pinned else hin.contiguous().clone()
            h_out = torch.empty(ref.shape, dtype=ref.dtype)
            h_out = h_out.pin_memory() if pinned else h_out
            p.exec_host(op, h_in, h_out)
            assert torch.equal(h_out, ref.cpu()), (kind, shape, batch, op, pinned)
    assert p.device_error() == 0
    e = oracle.rel_l2(spec.cpu().numpy(), (oracle.rfft3 if r2c else oracle.fft3)(src.numpy()))
    print(f"[parity] exec_host staged {kind} {shape} x{batch} tuned={tune}: fwd {e:.3e}")
    assert e < TOL


@pytest.mark.parametrize("kind,shape", [("c2c", (64, 48, 32)), ("r2c", (64, 64, 64)), ("c2c", (128, 128, 128))])
def test_autotuned_plan(gb, kind, shape):
    """The autotuner times the variants and keeps one; results stay within tolerance,
    and per-launch timing inside exec reports one segment per launch."""
    from paper_2601_12209_gb300 import abi
    nx, ny, nz = shape
    plan = gb.Plan(nx, ny, nz, kind=kind)
    t = plan.autotune()
    assert all(v["tuned"] and v["ms"] > 0 for v in t.values())
    x = synth.uniform_complex((nz, ny, nx), seed=91) if kind == "c2c" else synth.normal_real((nz, ny, nx), 92)
    abi.gbfft_plan_time_stages(plan.handle, True)
    X = plan.forward(x.to(dev()))
    xr = plan.inverse(X)
    abi.gbfft_plan_time_stages(plan.handle, False)
    seg, ncalls = abi.gbfft_plan_stage_times(plan.handle, 0)
    assert ncalls == 1 and len(seg) == (1 if t["forward"]["persistent"] else 3) and all(v > 0 for v in seg)
    ref = oracle.fft3(x.numpy()) if kind == "c2c" else oracle.rfft3(x.numpy())
    assert err(f"autotuned {kind} {shape} fwd {t['forward']}", X.cpu().numpy(), ref) < TOL
    assert err(f"autotuned {kind} {shape} roundtrip", xr.cpu().numpy(), x.numpy()) < TOL
    assert plan.device_error() == 0


def test_graph_capture_of_staged_launches(gb):
    """Stage launches (programmatic dependent launch, warp-per-pencil and tensor-copy kernels pinned) captured in a
    CUDA graph and replayed give the eager results bit for bit."""
    from paper_2601_12209_gb300 import abi
    n = 256
    r = synth.normal_real((n, n, n), seed=61).to(dev())
    p = gb.Plan(n, n, n, kind="r2c")
    abi.gbfft_plan_set_tuning(p.handle, 0, False, 0x600000)  # x Stockham, y and z warp-per-pencil
    abi.gbfft_plan_set_tuning(p.handle, 1, False, 0x300004)  # z and y warp-per-pencil, x tensor copies
    spec = p.forward(r)
    back = p.inverse(spec)
    torch.cuda.synchronize()
    s2 = torch.empty_like(spec)
    b2 = torch.empty_like(back)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        p.forward(r, out=s2, stream=side)
        p.inverse(s2, out=b2, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        p.forward(r, out=s2)
        p.inverse(s2, out=b2)
    s2.zero_()
    b2.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert p.device_error() == 0
    assert torch.equal(s2, spec) and torch.equal(b2, back)
    assert err("graph-captured r2c", s2.cpu().numpy(), oracle.rfft3(r.cpu().numpy())) < TOL


@pytest.mark.parametrize("kind,shape,tune", [("r2c", (64, 48, 40), False), ("c2c", (30, 20, 16), False),
                                             ("r2c", (512, 48, 24), True), ("c2c", (64, 96, 3), False)],
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_exec_host_chunked(gb, kind, shape, tune):
    """Host buffers in slabs whose copies overlap the first and last stages (contiguous z slabs on the real /
    natural side of x, strided y slabs on the spectrum side of z): the bits of the one-copy path for ops 0-3
    with the same stage kernels, for slab counts that do and do not divide the axes (more slabs than an axis
    has entries included), pinned and pageable buffers; the FP64 oracle."""
    from paper_2601_12209_gb300 import abi
    nx, ny, nz = shape
    p = gb.Plan(nx, ny, nz, kind=kind)
    if tune:
        p.autotune()
    else:
        for pipe in (0, 1):
            abi.gbfft_plan_set_tuning(p.handle, pipe, False, 0)  # staged thread-load launches
    r2c = kind == "r2c"
    src = synth.normal_real((nz, ny, nx), seed=54) if r2c else synth.uniform_complex((nz, ny, nx), seed=54)
    spec = p.forward(src.to(dev())).cpu()
    for op, hin in ((abi.GBFFT_OP_FORWARD, src), (abi.GBFFT_OP_INVERSE, spec), (abi.GBFFT_OP_ADJOINT, spec),
                    (abi.GBFFT_OP_INVERSE_ADJOINT, src)):
        outs = []
        for chunks in (1, 3, 7, 16):
            p.set_host_chunks(chunks)
            for pinned in (True, False):
                h_in = hin.contiguous().pin_memory() if pinned else hin.contiguous().clone()
                shape_out = spec.shape if op in (abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE_ADJOINT) else src.shape
                dt = spec.dtype if op in (abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE_ADJOINT) else src.dtype
                h_out = torch.empty(shape_out, dtype=dt)
                h_out = h_out.pin_memory() if pinned else h_out
                p.exec_host(op, h_in, h_out)
                outs.append(h_out)
        for o in outs[1:]:
            assert torch.equal(o, outs[0]), (kind, shape, op)
    p.set_host_chunks(8)
    h_out = torch.empty(spec.shape, dtype=spec.dtype).pin_memory()
    p.exec_host(abi.GBFFT_OP_FORWARD, src.pin_memory(), h_out)
    ref = oracle.rfft3(src.numpy()) if r2c else oracle.fft3(src.numpy())
    assert err(f"exec_host chunked {kind} {shape}", h_out.numpy(), ref) < TOL
    back = torch.empty(src.shape, dtype=src.dtype).pin_memory()
    p.exec_host(abi.GBFFT_OP_INVERSE, h_out, back)
    assert err(f"exec_host chunked round trip {kind} {shape}", back.numpy(), src.numpy()) < TOL
    with pytest.raises(abi.GbfftError):
        p.set_host_chunks(17)
    assert p.device_error() == 0
