"""The allocation-free entry point, gbfft_exec_c2c_noalloc.

Callers that cannot allocate device memory when they run a transform -- code
whose memory is managed by a pool or framework allocator that forbids side
allocations, or latency-bound loops where a cudaMalloc would stall the device
-- cannot build a gbfft_plan at that point. This entry point serves them with
a static device scratch buffer instead of plan workspace.

The test calls it through the C ABI twice in a row per operation (the second
call reuses the scratch the first call left behind), for all four operations,
and compares each result with the FP64 oracle and with the plan path's output
on the same input, within the parity tolerance used elsewhere. One grid has
exactly the scratch's limit of points. The file is collected last and runs
the same alone or after the rest of the suite (the per-device set-up happens
on the first call either way).
"""
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


def _oracle(op, x):
    from paper_2601_12209_gb300 import abi
    fn = {abi.GBFFT_OP_FORWARD: oracle.fft3, abi.GBFFT_OP_INVERSE: oracle.ifft3,
          abi.GBFFT_OP_ADJOINT: oracle.c2c_adjoint, abi.GBFFT_OP_INVERSE_ADJOINT: oracle.c2c_inverse_adjoint}[op]
    return fn(x)


@pytest.mark.parametrize("shape", [(64, 48, 40), (128, 128, 160), (30, 20, 16), (256, 128, 128)],
                         ids=lambda s: "x".join(map(str, s)))
def test_noalloc_matches_oracle_and_plan_path_twice(gb, shape):
    from paper_2601_12209_gb300 import abi
    nx, ny, nz = shape
    plan = gb.Plan(nx, ny, nz)
    for op in (abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE, abi.GBFFT_OP_ADJOINT, abi.GBFFT_OP_INVERSE_ADJOINT):
        for call in range(2):
            xh = synth.uniform_complex((nz, ny, nx), seed=900 + 10 * op + call)
            x = xh.cuda()
            ref = plan.exec(op, x)
            out = torch.empty_like(x)
            stream = torch.cuda.current_stream().cuda_stream
            abi.gbfft_exec_c2c_noalloc(nx, ny, nz, op, x.data_ptr(), out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            e_plan = oracle.rel_l2(got, ref.cpu().numpy())
            e_oracle = oracle.rel_l2(got, _oracle(op, xh.numpy()))
            print(f"[noalloc] {shape} op {op} call {call}: rel-L2 vs oracle {e_oracle:.3e}, vs plan path {e_plan:.3e}")
            assert e_oracle < TOL and e_plan < TOL
            assert torch.equal(x.cpu(), xh)


def test_noalloc_rejects_oversize_and_bad_args(gb):
    from paper_2601_12209_gb300 import abi
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    y = torch.zeros(16, dtype=torch.complex64, device="cuda")
    assert 256 * 128 * 128 == abi.GBFFT_NOALLOC_MAX_POINTS
    rc = abi.raw_rc("gbfft_exec_c2c_noalloc", 256, 256, 128, 0, x.data_ptr(), y.data_ptr(), None)
    assert rc == abi.GBFFT_ERR_STATIC_LIMIT  # 8 Mi points > the 4 Mi-point scratch; nothing launched
    assert "static scratch" in abi.strerror(rc)
    rc = abi.raw_rc("gbfft_exec_c2c_noalloc", 256, 128, 130, 0, x.data_ptr(), y.data_ptr(), None)
    assert rc == abi.GBFFT_ERR_STATIC_LIMIT  # one plane over the limit
    assert abi.raw_rc("gbfft_exec_c2c_noalloc", 8, 8, 8, 0, x.data_ptr(), x.data_ptr(), None) == abi.GBFFT_ERR_INPLACE
    assert abi.raw_rc("gbfft_exec_c2c_noalloc", 7, 8, 8, 0, x.data_ptr(), y.data_ptr(), None) == \
        abi.GBFFT_ERR_UNSUPPORTED_SIZE
    assert abi.raw_rc("gbfft_exec_c2c_noalloc", 8, 8, 8, 7, x.data_ptr(), y.data_ptr(), None) == \
        abi.GBFFT_ERR_INVALID_ARG
