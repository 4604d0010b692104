"""Batched form: many grids' measurements in one persistent fused launch.

Every grid of a batch must equal, voxel for voxel and origin for origin, the
same grid driven frame by frame through vg_integrate_depth + vg_shift (which
the parity tests hold equal to the CPU oracle), after every step.
"""
import numpy as np
import pytest

from synth import make

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13169_gb300 import build
    build.build()
    from paper_2112_13169_gb300 import vg as vgmod
    vgmod.load()
    return vgmod


def _grid(vg, w):
    g = w.grid
    return vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)


def _read(grid):
    out = torch.empty(grid.nvox, dtype=torch.uint8, device="cuda")
    o = grid.read(out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), o


def _compare(grids_a, grids_b, what):
    for k, (ga, gb) in enumerate(zip(grids_a, grids_b)):
        a, oa = _read(ga)
        b, ob = _read(gb)
        assert list(oa) == list(ob), (what, k, oa, ob)
        bad = np.flatnonzero(a != b)
        assert bad.size == 0, "%s grid %d: %d voxels differ, first %d: %d vs %d" % (
            what, k, bad.size, bad[0], a[bad[0]], b[bad[0]])


def _workloads():
    ws = [make("robot", robot=i, frames=3) for i in range(6)]
    ws.append(make("paper", frames=3))
    ws.append(make("hires", frames=2))   # u16 depth, 400x400x120 grid
    return ws


def test_batch_equals_plain_frame_by_frame(vg):
    ws = _workloads()
    plain = [_grid(vg, w) for w in ws]
    batched = [_grid(vg, w) for w in ws]
    batch = vg.Batch(16)
    try:
        for step in range(3):
            frames = []
            for w, gp, gb in zip(ws, plain, batched):
                if step >= len(w.frames):
                    continue
                f = w.frames[step]
                d = torch.from_numpy(f.depth).cuda()
                gp.integrate_depth(d, f.T_wc, w.cam.scale)
                gp.shift(f.robot_pos)
                frames.append((gb, d, f.T_wc, f.robot_pos, w.cam.scale))
            batch.step(frames)
            assert batch.status() == vg.VG_OK
            _compare(plain, batched, "step %d" % step)
    finally:
        batch.close()
        for g in plain + batched:
            g.close()


def test_batch_without_recentre_and_single_frame(vg):
    w = make("seq", frames=2)
    gp, gb = _grid(vg, w), _grid(vg, w)
    batch = vg.Batch(1)
    for f in w.frames:
        d = torch.from_numpy(f.depth).cuda()
        gp.integrate_depth(d, f.T_wc)
        batch.step([(gb, d, f.T_wc, None)])
        assert batch.status() == vg.VG_OK
        _compare([gp], [gb], "seq")
    batch.close()
    gp.close()
    gb.close()


def test_batch_applies_a_pending_shift(vg):
    # a re-centre made with vg_shift before the step, and the step's own
    # re-centre left pending after it, read back both ways
    w = make("robot", robot=7, frames=3)
    gp, gb = _grid(vg, w), _grid(vg, w)
    batch = vg.Batch(2)
    f0, f1, f2 = w.frames
    for g in (gp, gb):
        g.shift(f0.robot_pos + np.array([0.3, -0.2, 0.1]))
    d1, d2 = torch.from_numpy(f1.depth).cuda(), torch.from_numpy(f2.depth).cuda()
    gp.integrate_depth(d1, f1.T_wc, w.cam.scale)
    gp.shift(f1.robot_pos)
    batch.step([(gb, d1, f1.T_wc, f1.robot_pos, w.cam.scale)])
    assert batch.status() == vg.VG_OK
    _compare([gp], [gb], "after the step")              # the read applies the pending re-centre
    gp.shift(f2.robot_pos)
    gb.shift(f2.robot_pos)
    gp.integrate_depth(d2, f2.T_wc, w.cam.scale)
    batch.step([(gb, d2, f2.T_wc, None, w.cam.scale)])
    assert batch.status() == vg.VG_OK
    _compare([gp], [gb], "after a step over a vg_shift")
    batch.close()
    gp.close()
    gb.close()


def test_batch_replayed_from_a_cuda_graph(vg):
    ws = [make("robot", robot=i, frames=4) for i in range(10, 14)]
    plain = [_grid(vg, w) for w in ws]
    batched = [_grid(vg, w) for w in ws]
    batch = vg.Batch(8)
    depth = [[torch.from_numpy(f.depth).cuda() for f in w.frames] for w in ws]

    def frames_of(step):
        return [(gb, depth[k][step], w.frames[step].T_wc, w.frames[step].robot_pos)
                for k, (w, gb) in enumerate(zip(ws, batched))]

    # step 0 runs eagerly; it also warms up the launch before capture
    batch.step(frames_of(0))
    for k, (w, gp) in enumerate(zip(ws, plain)):
        gp.integrate_depth(depth[k][0], w.frames[0].T_wc)
        gp.shift(w.frames[0].robot_pos)
    torch.cuda.synchronize()
    batch.prepare(frames_of(1))
    graph = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            batch.enqueue(stream)
    # capture does not run the step: replay it, then prepare and replay the rest
    for step in range(1, 4):
        if step > 1:
            batch.prepare(frames_of(step))
        graph.replay()
        torch.cuda.synchronize()
        assert batch.status() == vg.VG_OK
        for k, (w, gp) in enumerate(zip(ws, plain)):
            gp.integrate_depth(depth[k][step], w.frames[step].T_wc)
            gp.shift(w.frames[step].robot_pos)
        _compare(plain, batched, "graph step %d" % step)
    del graph
    batch.close()
    for g in plain + batched:
        g.close()


def test_autotune_keeps_results(vg):
    ws = [make("robot", robot=i, frames=2) for i in range(20, 24)]
    plain = [_grid(vg, w) for w in ws]
    batched = [_grid(vg, w) for w in ws]
    batch = vg.Batch(4)
    d0 = [torch.from_numpy(w.frames[0].depth).cuda() for w in ws]
    frames = [(gb, d0[k], w.frames[0].T_wc, w.frames[0].robot_pos) for k, (w, gb) in enumerate(zip(ws, batched))]
    ctas, lanes = batch.autotune(frames, reps=2)
    assert ctas >= 1 and lanes in (0, 8, 16, 32)
    # the autotuner merged frame 0 without re-centring; so does the plain side
    for k, (w, gp) in enumerate(zip(ws, plain)):
        gp.integrate_depth(d0[k], w.frames[0].T_wc)
    _compare(plain, batched, "after autotune")
    d1 = [torch.from_numpy(w.frames[1].depth).cuda() for w in ws]
    batch.step([(gb, d1[k], w.frames[1].T_wc, w.frames[1].robot_pos) for k, (w, gb) in enumerate(zip(ws, batched))])
    assert batch.status() == vg.VG_OK
    for k, (w, gp) in enumerate(zip(ws, plain)):
        gp.integrate_depth(d1[k], w.frames[1].T_wc)
        gp.shift(w.frames[1].robot_pos)
    _compare(plain, batched, "after a tuned step")
    batch.close()
    for g in plain + batched:
        g.close()


def test_batch_rejects_bad_frames(vg):
    w = make("room")
    g = _grid(vg, w)
    d = torch.from_numpy(w.frames[0].depth).cuda()
    batch = vg.Batch(2)
    with pytest.raises(vg.VGError) as e:
        batch.step([(g, d, w.frames[0].T_wc, None), (g, d, w.frames[0].T_wc, None)])   # one grid twice
    assert e.value.status == vg.VG_EINVAL
    with pytest.raises(vg.VGError):
        batch.step([(g, d, w.frames[0].T_wc, None)] * 3)   # over capacity
    big = vg.Grid((40, 40, 20), 0.1, 87.0, 58.0, 3.0, 4, (0, 0, 0))   # vox_inf 4: not batched
    with pytest.raises(vg.VGError):
        batch.step([(big, d, w.frames[0].T_wc, None)])
    with pytest.raises(vg.VGError):
        batch.step([(g, d, np.full((4, 4), np.nan), None)])
    with pytest.raises(vg.VGError):
        batch.tune(vg.VG_TUNE_BATCH_LANES, 12)
    batch.close()
    big.close()
    g.close()
