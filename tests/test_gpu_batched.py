"""Batched grids: 64 C2C grids of uneven sizes (each axis drawn from
{32,48,60,64,80,96,120,128,160,192,256}) in one launch that pulls every grid's
tiles from one ticket queue, checked per grid against the FP64 oracle, replayed
from a CUDA graph, and compared with one plan per grid.
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


def test_batched_small_mixed(gb):
    from paper_2601_12209_gb300 import abi
    shapes = [(32, 48, 60), (60, 32, 48), (64, 64, 64), (80, 96, 32), (120, 32, 48), (48, 160, 32),
              (192, 32, 32), (32, 32, 256)]
    m = gb.ManyPlan(shapes)
    grids = [synth.uniform_complex((nz, ny, nx), seed=300 + i) for i, (nx, ny, nz) in enumerate(shapes)]
    x = m.pack([g.cuda() for g in grids])
    y = m.empty()
    m.exec(abi.GBFFT_OP_FORWARD, x, y)
    z = m.empty()
    m.exec(abi.GBFFT_OP_INVERSE, y, z)
    torch.cuda.synchronize()
    assert m.device_error() == 0
    for i, (g, out, back) in enumerate(zip(grids, m.unpack(y), m.unpack(z))):
        e = oracle.rel_l2(out.cpu().numpy(), oracle.fft3(g.numpy()))
        e2 = oracle.rel_l2(back.cpu().numpy(), g.numpy())
        print(f"[batched] grid {i} {shapes[i]}: fwd rel-L2 {e:.3e}, roundtrip {e2:.3e}")
        assert e < TOL and e2 < TOL
    # the per-stage launches and the one-plan-per-grid path give the same bits (same tile arithmetic)
    y2 = m.empty()
    m.exec_separate(abi.GBFFT_OP_FORWARD, x, y2)
    assert torch.equal(y, y2)
    y3 = m.empty()
    m.exec_staged(abi.GBFFT_OP_FORWARD, x, y3)
    assert torch.equal(y, y3)
    z3 = m.empty()
    m.exec_staged(abi.GBFFT_OP_INVERSE, y3, z3)
    assert torch.equal(z, z3)


def test_config4_64_uneven_grids_graph_replay(gb):
    """Config 4: 64 grids, one persistent launch captured in a CUDA graph and replayed, forward
    and inverse; every grid of both directions against the FP64 oracle."""
    from paper_2601_12209_gb300 import abi
    shapes, grids = synth.batched_grids(64, seed=6)
    m = gb.ManyPlan(shapes)
    x = m.pack([g.cuda() for g in grids])
    y = m.empty()
    z = m.empty()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        m.exec(abi.GBFFT_OP_FORWARD, x, y, stream=s)  # warm-up outside capture
        m.exec(abi.GBFFT_OP_INVERSE, x, z, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graphs = {}
    for op, out in ((abi.GBFFT_OP_FORWARD, y), (abi.GBFFT_OP_INVERSE, z)):
        graphs[op] = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graphs[op]):
            m.exec(op, x, out)
    y.zero_()
    z.zero_()
    graphs[abi.GBFFT_OP_FORWARD].replay()
    graphs[abi.GBFFT_OP_INVERSE].replay()
    torch.cuda.synchronize()
    assert m.device_error() == 0
    fwd, inv = m.unpack(y), m.unpack(z)
    worst = [0.0, 0.0]
    for i in range(64):
        g = grids[i].numpy()
        e = oracle.rel_l2(fwd[i].cpu().numpy(), oracle.fft3(g))
        e2 = oracle.rel_l2(inv[i].cpu().numpy(), oracle.ifft3(g))
        print(f"[batched] cfg4 grid {i} {shapes[i]}: fwd rel-L2 {e:.3e}, inv rel-L2 {e2:.3e}")
        worst = [max(worst[0], e), max(worst[1], e2)]
        assert e < TOL and e2 < TOL
    print(f"[batched] cfg4 worst over 64 grids: fwd {worst[0]:.3e}, inv {worst[1]:.3e}")
    # a second replay after the input changed in place
    grids2 = [torch.conj_physical(g) for g in grids[:4]]
    for g, off, (nx, ny, nz) in zip(grids2, m.offsets, shapes):
        x[off:off + nx * ny * nz].copy_(g.reshape(-1).cuda())
    graphs[abi.GBFFT_OP_FORWARD].replay()
    torch.cuda.synchronize()
    for i in range(4):
        e = oracle.rel_l2(m.unpack(y)[i].cpu().numpy(), oracle.fft3(grids2[i].numpy()))
        assert e < TOL


def test_batched_timeout_reported(gb):
    from paper_2601_12209_gb300 import abi
    m = gb.ManyPlan([(32, 32, 32), (64, 48, 32)], debug_timeout=True)
    x = m.empty()
    y = m.empty()
    m.exec(abi.GBFFT_OP_FORWARD, x, y)
    assert m.device_error() == abi.GBFFT_ERR_TIMEOUT
    assert m.device_error() == 0


def test_batched_tiles_per_ticket_bitwise_and_oracle(gb):
    """Tiles per ticket (teams of 256 / S threads side by side in one block): every allowed S of
    every length gives the same bits as one tile per ticket (same butterflies, other threads),
    in the one launch and the per-stage launches, forward and inverse; ragged last tickets
    (tile counts not a multiple of S) included; the result matches the FP64 oracle."""
    from paper_2601_12209_gb300 import abi
    shapes = [(32, 48, 60), (80, 32, 48), (48, 80, 32), (64, 96, 120), (128, 60, 32), (32, 32, 256),
              (160, 48, 80), (96, 128, 48)]
    m = gb.ManyPlan(shapes)
    grids = [synth.uniform_complex((nz, ny, nx), seed=400 + i) for i, (nx, ny, nz) in enumerate(shapes)]
    x = m.pack([g.cuda() for g in grids])
    ref = {}
    for op in (abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE):
        y = m.empty()
        m.exec(op, x, y)
        ref[op] = y
    lengths = sorted({v for s in shapes for v in s})
    maxs = {L: (4 if L in (32, 48, 80) else 2 if L <= 128 else 1) for L in lengths}
    for S in (2, 4):
        teams = {L: min(S, maxs[L]) for L in lengths}
        for pipe in (0, 1):
            m.set_tuning(pipe, teams)
        assert m.tuning()["forward"]["teams"] == teams
        for op in (abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE):
            y = m.empty()
            m.exec(op, x, y)
            y2 = m.empty()
            m.exec_staged(op, x, y2)
            torch.cuda.synchronize()
            assert torch.equal(y, ref[op]) and torch.equal(y2, ref[op]), (S, op)
    assert m.device_error() == 0
    for i, (g, out) in enumerate(zip(grids, m.unpack(ref[abi.GBFFT_OP_FORWARD]))):
        assert oracle.rel_l2(out.cpu().numpy(), oracle.fft3(g.numpy())) < TOL
    with pytest.raises(abi.GbfftError):
        m.set_tuning(0, {256: 2})  # a length-256 tile already fills the block
    # the queue lag between a grid's stages reorders tickets only: same bits
    for lag in (2, 4, 8):
        for pipe in (0, 1):
            m.set_lag(pipe, lag)
        assert m.tuning()["inverse"]["lag"] == lag
        for op in (abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE):
            y = m.empty()
            m.exec(op, x, y)
            torch.cuda.synchronize()
            assert torch.equal(y, ref[op]), (lag, op)
    assert m.device_error() == 0


def test_batched_autotune_config4(gb):
    """The tile-shape autotuner on the 64 configuration grids: every choice is allowed for its
    length, the tuned one launch (graph-captured) matches the oracle on sampled grids."""
    from paper_2601_12209_gb300 import abi
    shapes, grids = synth.batched_grids(64, seed=6)
    m = gb.ManyPlan(shapes)
    tun = m.autotune()
    print(f"[batched] tuned tiles per ticket: {tun}")
    for name in ("forward", "inverse"):
        assert tun[name]["ms"] > 0 and tun[name]["lag"] in (1, 2, 4)
        for L, S in tun[name]["teams"].items():
            assert S in (1, 2, 4) and (S == 1 or L <= 128)
    x = m.pack([g.cuda() for g in grids])
    y = m.empty()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        m.exec(abi.GBFFT_OP_FORWARD, x, y, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        m.exec(abi.GBFFT_OP_FORWARD, x, y)
    y.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert m.device_error() == 0
    outs = m.unpack(y)
    for i in (0, 7, 21, 42, 63):
        assert oracle.rel_l2(outs[i].cpu().numpy(), oracle.fft3(grids[i].numpy())) < TOL
