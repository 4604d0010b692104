"""Batched form: many grids' measurements in one persistent fused launch.

Every grid of a batch must equal, voxel for voxel and origin for origin, the
CPU oracle driven with the same frames (integrate, then re-centre), after
every step: eager steps, steps replayed from a CUDA graph and steps after
the autotuner.  The 64-robot mix is the batched configuration as stated:
depth resolutions from {320x240, 640x480, 848x480}, voxels of 0.05, 0.1 or
0.2 m, grids from 80x80x40 to 256x256x96 and vox_inf 1-3, with one robot
pinned at the mix's largest case (848x480, 0.05 m, 256x256x96, vox_inf 3).
"""
import numpy as np
import pytest

from gridcheck import assert_grid, oracle_grid
from synth import make

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the batched configuration's largest robot: every extreme of the stated sets
LARGEST = (848, 480, 0.05, (256, 256, 96), 3)


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


def _check(ws, grids, oracles, what):
    for k, (w, g, og) in enumerate(zip(ws, grids, oracles)):
        got, o = _read(g)
        assert_grid(got, o, og, "%s, robot %d (%dx%d, %s m, grid %s, vox_inf %d)" % (
            what, k, w.cam.W, w.cam.H, w.grid.vox_size, w.grid.n, w.grid.vox_inf))


class Robots:
    """Workloads, their device frames, the library grids and the oracle
    grids, stepped together."""

    def __init__(self, vg, ws):
        self.ws = ws
        self.depth = [[torch.from_numpy(f.depth).cuda() for f in w.frames] for w in ws]
        self.grids = [_grid(vg, w) for w in ws]
        self.oracles = [oracle_grid(w) for w in ws]

    def frames(self, step, recentre=True):
        out = []
        for k, (w, g) in enumerate(zip(self.ws, self.grids)):
            f = w.frames[step]
            out.append((g, self.depth[k][step], f.T_wc, f.robot_pos if recentre else None, w.cam.scale))
        return out

    def oracle_step(self, step, recentre=True):
        for w, og in zip(self.ws, self.oracles):
            f = w.frames[step]
            og.integrate_depth(f.T_wc, f.depth, w.cam.scale)
            if recentre:
                og.shift(f.robot_pos)

    def check(self, what):
        _check(self.ws, self.grids, self.oracles, what)

    def close(self):
        for g in self.grids:
            g.close()


def _mix(n=64, frames=3):
    ws = [make("robot", robot=i, frames=frames) for i in range(n - 1)]
    ws.append(make("robot", robot=n - 1, frames=frames, spec=LARGEST))
    return ws


def test_batched_config_against_the_oracle_eager_and_graph(vg):
    # the 64-robot mix: steps 0 and 1 eager, steps 2 and 3 replayed from a
    # CUDA graph captured once; every grid is compared after every step
    ws = _mix(64, 4)
    kinds = {(w.cam.W, w.cam.H) for w in ws}
    assert kinds == {(320, 240), (640, 480), (848, 480)}
    assert {w.grid.vox_size for w in ws} == {0.05, 0.1, 0.2} and {w.grid.vox_inf for w in ws} == {1, 2, 3}
    R = Robots(vg, ws)
    batch = vg.Batch(64)
    try:
        for step in range(2):
            batch.step(R.frames(step))
            assert batch.status() == vg.VG_OK
            R.oracle_step(step)
            R.check("eager step %d" % step)
        batch.prepare(R.frames(2))
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        with torch.cuda.stream(cap):
            with torch.cuda.graph(graph, stream=cap):
                batch.enqueue(cap)
        for step in (2, 3):
            if step > 2:
                batch.prepare(R.frames(step))
            graph.replay()
            torch.cuda.synchronize()
            assert batch.status() == vg.VG_OK
            R.oracle_step(step)
            R.check("graph step %d" % step)
        del graph
    finally:
        batch.close()
        R.close()


def test_batch_with_full_size_sequences(vg):
    # the plain configurations' grids batched together: 640x480 f32 into
    # 200x200x100 and 1280x720 u16 into 400x400x120, beside two robots
    ws = [make("seq", frames=3), make("hires", frames=3), make("paper", frames=3),
          make("robot", robot=5, frames=3)]
    R = Robots(vg, ws)
    batch = vg.Batch(8)
    try:
        for step in range(3):
            batch.step(R.frames(step))
            assert batch.status() == vg.VG_OK
            R.oracle_step(step)
            R.check("step %d" % step)
    finally:
        batch.close()
        R.close()


def test_batch_without_recentre_and_single_frame(vg):
    w = make("seq", frames=2)
    R = Robots(vg, [w])
    batch = vg.Batch(1)
    for step in range(2):
        batch.step(R.frames(step, recentre=False))
        assert batch.status() == vg.VG_OK
        R.oracle_step(step, recentre=False)
        R.check("seq step %d" % step)
    batch.close()
    R.close()


def test_batch_applies_a_pending_shift(vg):
    # a re-centre made with vg_shift before the step, and the step's own
    # re-centre left pending after it, read back both ways
    w = make("robot", robot=7, frames=3)
    R = Robots(vg, [w])
    gb, og = R.grids[0], R.oracles[0]
    batch = vg.Batch(2)
    f0, f1, f2 = w.frames
    p = f0.robot_pos + np.array([0.3, -0.2, 0.1])
    gb.shift(p)
    og.shift(p)
    batch.step(R.frames(1))
    assert batch.status() == vg.VG_OK
    R.oracle_step(1)
    R.check("after the step")                       # read out with the step's re-centre pending
    gb.shift(f2.robot_pos)
    og.shift(f2.robot_pos)
    batch.step(R.frames(2, recentre=False))
    assert batch.status() == vg.VG_OK
    R.oracle_step(2, recentre=False)
    R.check("after a step over a vg_shift")
    batch.close()
    R.close()


def test_autotune_keeps_results(vg):
    ws = [make("robot", robot=i, frames=2) for i in range(20, 24)]
    R = Robots(vg, ws)
    batch = vg.Batch(4)
    best = batch.autotune(R.frames(0), reps=2)
    assert best["ctas_per_sm"] >= 1 and best["lanes"] in (0, 8, 16, 32)
    assert best["inflate_slices"] in (4, 8) and best["merge_words"] in (256, 512) and best["spread"] in (0, 1, 2)
    # the autotuner merged frame 0 without re-centring; so does the oracle
    R.oracle_step(0, recentre=False)
    R.check("after autotune")
    batch.step(R.frames(1))
    assert batch.status() == vg.VG_OK
    R.oracle_step(1)
    R.check("after a tuned step")
    batch.close()
    R.close()


@pytest.mark.parametrize("slices,words,spread,ctas", [(4, 256, 0, 1), (4, 512, 1, 2), (8, 256, 1, 3),
                                                     (8, 512, 2, 1), (4, 256, 2, 4)])
def test_batch_schedule_knobs_keep_results(vg, slices, words, spread, ctas):
    # every schedule the batch autotuner can pick gives the oracle's grids
    ws = [make("robot", robot=i, frames=2) for i in (0, 7, 12, 23)]   # vox_inf 1-3, 848x480, 640x480
    R = Robots(vg, ws)
    batch = vg.Batch(4)
    batch.tune(vg.VG_TUNE_BATCH_INFLATE_SLICES, slices)
    batch.tune(vg.VG_TUNE_BATCH_MERGE_WORDS, words)
    batch.tune(vg.VG_TUNE_BATCH_SPREAD, spread)
    batch.tune(vg.VG_TUNE_BATCH_CTAS_PER_SM, ctas)
    for step in range(2):
        batch.step(R.frames(step))
        assert batch.status() == vg.VG_OK
        R.oracle_step(step)
        R.check("schedule %s step %d" % ((slices, words, spread, ctas), step))
    batch.close()
    R.close()


def test_barrier_time_limit_ends_a_step_with_a_timeout(vg):
    # fault injection on the device's own wait: every grid barrier of the
    # fused launch waits for one more CTA than the launch has, with a 1 ms
    # limit, so the first barrier gives up, every CTA leaves the kernel and
    # the step reports VG_ETIMEOUT; the context stays usable, and a grid
    # restored with vg_write steps on as the oracle does
    import time
    ws = [make("robot", robot=i, frames=2) for i in (2, 3)]
    R = Robots(vg, ws)
    batch = vg.Batch(2)
    batch.tune(vg.VG_TUNE_BATCH_BARRIER_US, 1000)
    batch.tune(vg.VG_TUNE_BATCH_BARRIER_EXTRA, 1)
    t0 = time.perf_counter()
    batch.step(R.frames(0, recentre=False))
    assert batch.status() == vg.VG_ETIMEOUT
    assert time.perf_counter() - t0 < 2.0
    torch.cuda.synchronize()                  # no fault, no hang
    batch.tune(vg.VG_TUNE_BATCH_BARRIER_EXTRA, 0)
    for g, og in zip(R.grids, R.oracles):
        g.write(np.zeros(g.nvox, np.uint8), og.o)
    batch.step(R.frames(1))
    assert batch.status() == vg.VG_OK
    R.oracle_step(1)
    R.check("after a timed-out step and vg_write")
    with pytest.raises(vg.VGError):
        batch.tune(vg.VG_TUNE_BATCH_BARRIER_EXTRA, 2)
    batch.close()
    R.close()


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
