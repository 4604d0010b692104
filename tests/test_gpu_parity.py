"""CUDA path vs the CPU oracle, voxel by voxel, through the C ABI.

The bar is bit-exact: every voxel state of loc_grid and the grid origin must
equal the oracle's after every frame.  Any mismatch is reported with the
voxel, both states and the count; none is tolerated.
"""
import numpy as np
import pytest

from gridcheck import assert_same
from oracle import OracleGrid, OracleParams
from oracle.oracle import LIT_INFLATE_AFTER_TRACE, LIT_LOC_OCCUPANCY, LIT_SKIP_START
from synth import body_pose, make

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


class Pair:
    """A GPU grid and an oracle grid driven with the same calls."""

    def __init__(self, vg, n, vs, fx, fy, depth, r, pos, lanes=None, flags=0):
        self.vg = vg
        self.g = vg.Grid(n, vs, fx, fy, depth, r, pos, flags=flags)
        if lanes:
            self.g.tune(lanes)
        lit = ((LIT_INFLATE_AFTER_TRACE if flags & vg.VG_FLAG_LIT_INFLATE_AFTER_TRACE else 0) |
               (LIT_SKIP_START if flags & vg.VG_FLAG_LIT_SKIP_START_VOXEL else 0) |
               (LIT_LOC_OCCUPANCY if flags & vg.VG_FLAG_LIT_LOC_OCCUPANCY else 0))
        self.o = OracleGrid(OracleParams(tuple(n), vs, fx, fy, depth, r, lit), pos)
        self.out = torch.empty(self.g.nvox, dtype=torch.uint8, device="cuda")

    def depth(self, d, T, scale=1.0, device=True, check=True):
        dd = torch.from_numpy(np.ascontiguousarray(d)).cuda() if device else np.ascontiguousarray(d)
        self.g.integrate_depth(dd, T, scale)
        self.o.integrate_depth(T, d, scale)
        if check:
            self.check("depth frame")

    def points(self, xyz, T, device=True, check=True):
        xyz = np.ascontiguousarray(xyz, np.float32)
        self.g.integrate_points(torch.from_numpy(xyz).cuda() if device else xyz, T)
        self.o.integrate_points(T, xyz)
        if check:
            self.check("point frame")

    def shift(self, pos, check=True):
        self.g.shift(pos)
        self.o.shift(pos)
        if check:
            self.check("shift")

    def read(self):
        origin = self.g.read(self.out)
        torch.cuda.synchronize()
        return self.out.cpu().numpy().reshape(self.g.shape), origin

    def check(self, what):
        got, origin = self.read()
        assert list(origin) == list(self.o.o), (what, origin, self.o.o)
        assert_same(got, self.o.loc, what)

    def close(self):
        self.g.close()


def run_workload(vg, w, nframes, lanes=None, device=True, shift=True, flags=0):
    """Frames with a re-centre after each.  A grid is read (and compared)
    after every frame but not after its re-centre, so the re-centre is
    still pending when the next frame comes and that frame's merge clears
    what it brought in; the last one is only read out (through the ring)
    by the final read."""
    g = w.grid
    f0 = w.frames[0]
    P = Pair(vg, g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, f0.robot_pos, lanes, flags=flags)
    try:
        for i in range(nframes):
            f = w.frames[i]
            P.depth(f.depth, f.T_wc, w.cam.scale, device=device, check=False)
            P.check("%s frame %d" % (w.name, i))
            if shift:
                P.shift(f.robot_pos, check=False)
        if shift:
            P.check("%s shift after frame %d" % (w.name, nframes - 1))
        got, _ = P.read()
        return got
    finally:
        P.close()


# --------------------------------------------------------------------------
# the measurement configurations
# --------------------------------------------------------------------------
def test_room_single_frame(vg):
    w = make("room")
    got = run_workload(vg, w, 1, shift=False)
    counts = np.bincount(got.ravel(), minlength=4)
    assert counts[1] > 1000 and counts[2] > 1000, counts   # free and occupied voxels exist


def test_paper_shapes_sequence(vg):
    # the paper's standard set-up, all 100 frames
    run_workload(vg, make("paper"), 100)


def test_sequence_full_size(vg):
    # the whole plain sequence: 100 frames of 640x480 f32 into a 200x200x100
    # grid at 0.05 m, vox_inf 2, re-centred after every frame, in the launch
    # configuration the benchmark times; compared after every frame
    run_workload(vg, make("seq"), 100)


def test_hires_u16_full_size(vg):
    # the whole high-resolution sequence: 50 frames of 1280x720 u16 into a
    # 400x400x120 grid
    run_workload(vg, make("hires"), 50)


@pytest.mark.parametrize("tile", [1, 2, 3, 4])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_schedule_knobs_keep_results(vg, tile, r):
    # every schedule the per-grid autotuner can pick: the four inflate tiles
    # at radii 1-3 (on a grid with 8-word rows, so 8-word tiles are used),
    # staged by tensor copies or by the threads, K3 capped at few CTAs per
    # SM, K4's 256- and 512-word units with re-centres, and K2 launched
    # while K1 runs or after it
    w = make("robot", robot=90 + r, frames=3, spec=(640, 480, 0.05, (256, 120, 60), r))
    g = w.grid
    P = Pair(vg, g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    P.g.set(vg.VG_TUNE_INFLATE_TILE, tile)
    P.g.set(vg.VG_TUNE_RT_CTAS_PER_SM, tile)          # 1..4 CTAs per SM
    P.g.set(vg.VG_TUNE_MERGE_WORDS, 512 if tile % 2 else 256)
    P.g.set(vg.VG_TUNE_INFLATE_TMA, 1 if r != 2 else 0)   # tensor-copy staging, and thread staging at r 2
    P.g.set(vg.VG_TUNE_EARLY_INFLATE, tile % 2)
    for f in w.frames:
        P.depth(f.depth, f.T_wc, check=False)
        P.check("tile %d r %d frame" % (tile, r))
        P.shift(f.robot_pos, check=False)
    P.check("after the last re-centre")
    P.close()


def test_autotune_picks_a_schedule_and_keeps_results(vg):
    w = make("seq", frames=3)
    g = w.grid
    P = Pair(vg, g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    d0 = torch.from_numpy(w.frames[0].depth).cuda()
    best = P.g.autotune(d0, w.frames[0].T_wc, reps=2)
    assert best["tile"] in ("auto", "4x8x4", "4x8x8", "8x8x4", "8x8x8") and best["lanes"] in (8, 16, 32)
    assert 0 <= best["ctas_per_sm"] <= 5 and best["merge_words"] in (256, 512)
    assert best["inflate_tma"] in (0, 1) and best["early_inflate"] in (0, 1)
    # the tuner merged frame 0 (over re-centres by zero); so does the oracle
    P.o.integrate_depth(w.frames[0].T_wc, w.frames[0].depth)
    P.check("after autotune")
    for f in w.frames[1:]:
        P.depth(f.depth, f.T_wc, check=False)
        P.shift(f.robot_pos)
    P.close()


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8, 16, 32])
def test_lanes_per_ray_do_not_change_results(vg, lanes):
    # 0 is automatic; 1, 2 and 4 lanes overflow the per-lane visit buffer on
    # most rays and take the two-pass walk
    run_workload(vg, make("paper", frames=2), 2, lanes=lanes)


def test_lanes_on_full_size_sequence(vg):
    for lanes in (4, 32):
        run_workload(vg, make("seq", frames=2), 2, lanes=lanes)


def test_long_rays_take_more_lanes(vg):
    # 0.02 m voxels and a 5 m range: 250 voxels deep, so the automatic
    # choice gives each ray 32 lanes (a slice of 8 or 16 lanes would not fit
    # the visit buffer), and rays cross a 200 x 160 x 90 grid and leave it
    rng = np.random.default_rng(41)
    P = Pair(vg, (200, 160, 90), 0.02, 87.0, 58.0, 5.0, 2, (0.01, -0.02, 0.03))
    for k in range(2):
        d = rng.uniform(0.8, 5.5, size=(48, 64)).astype(np.float32)
        d[rng.random(d.shape) < 0.15] = 0
        P.depth(d, body_pose([0.01, -0.02, 0.03], rng.uniform(-np.pi, np.pi), rng.uniform(-0.3, 0.3)))
    P.close()


def test_huge_plane_takes_the_unbuffered_walk(vg):
    # 1 x 4096 x 4096 voxels: 2^26 plane words, too many for a packed visit,
    # so every lane walks twice instead of buffering
    rng = np.random.default_rng(29)
    P = Pair(vg, (1, 4096, 4096), 0.1, 87.0, 58.0, 1.0, 1, (0.0, 0.0, 0.0))
    d = rng.uniform(0.2, 1.2, size=(24, 32)).astype(np.float32)
    P.depth(d, body_pose([0.0, 0.0, 0.0], np.pi / 2))   # looking along +y, inside the 1-voxel slab
    P.depth(d, body_pose([0.0, 0.0, 0.0], np.pi / 2, 0.3))
    P.close()


@pytest.mark.parametrize("ny", [511, 600])
def test_plane_words_at_the_run_limit(vg, ny):
    # 1 x 1024 x ny voxels at 4 words a row: 2,093,056 plane words (ny 511,
    # just below 2^21: buffered runs, word indices up to bit 20) and
    # 2,457,600 (ny 600: every lane walks twice)
    rng = np.random.default_rng(31 + ny)
    P = Pair(vg, (1, 1024, ny), 0.1, 87.0, 58.0, 1.5, 1, (0.0, 0.0, 0.0))
    d = rng.uniform(0.2, 1.6, size=(24, 32)).astype(np.float32)
    P.depth(d, body_pose([0.0, 0.0, 0.0], np.pi / 2))
    P.depth(d, body_pose([0.0, 0.0, 0.0], -np.pi / 2, 0.2))
    P.close()


def test_host_memory_inputs(vg):
    run_workload(vg, make("room"), 1, device=False, shift=False)


def test_robot_mix_shapes(vg):
    for i in range(3):
        run_workload(vg, make("robot", robot=i, frames=2), 2)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------
def _pair(vg, n=(40, 36, 20), vs=0.1, fx=87.0, fy=58.0, depth=3.0, r=1, pos=(0.01, 0.02, 0.03), **kw):
    return Pair(vg, n, vs, fx, fy, depth, r, pos, **kw)


def test_empty_and_invalid_frames(vg):
    P = _pair(vg)
    T = body_pose([0.01, 0.02, 0.03], 0.3)
    P.depth(np.zeros((24, 32), np.float32), T)
    P.depth(np.full((24, 32), np.nan, np.float32), T)
    d = np.full((24, 32), np.inf, np.float32)
    d[::2] = -1.0
    P.depth(d, T)
    P.depth(np.full((24, 32), 3.0, np.float32), T)          # exactly the range: valid
    P.depth(np.full((24, 32), np.nextafter(np.float32(3.0), np.float32(4.0)), np.float32), T)
    P.close()


@pytest.mark.parametrize("W,H", [(37, 23), (1, 1), (5, 3), (641, 479)])
def test_ragged_images(vg, W, H):
    rng = np.random.default_rng(W * 1000 + H)
    P = _pair(vg)
    d = rng.uniform(0.2, 3.5, size=(H, W)).astype(np.float32)
    d[rng.random(d.shape) < 0.2] = 0
    P.depth(d, body_pose([0.01, 0.02, 0.03], 0.5, 0.1, -0.1))
    P.close()


def test_unaligned_depth_pointer(vg):
    rng = np.random.default_rng(5)
    P = _pair(vg)
    base = torch.from_numpy(rng.uniform(0.2, 3.5, size=24 * 32 + 1).astype(np.float32)).cuda()
    view = base[1:].view(24, 32)                 # 4-byte aligned, not 16-byte aligned
    T = body_pose([0.01, 0.02, 0.03], 0.2)
    P.g.integrate_depth(view, T)
    P.o.integrate_depth(T, view.cpu().numpy())
    P.check("unaligned f32")
    base16 = torch.from_numpy(rng.integers(0, 4000, size=24 * 32 + 1).astype(np.uint16)).cuda()
    v16 = base16[1:].view(24, 32)
    P.g.integrate_depth(v16, T, 0.001)
    P.o.integrate_depth(T, v16.cpu().numpy(), 0.001)
    P.check("unaligned u16")
    P.close()


@pytest.mark.parametrize("r", [0, 1, 2, 3, 7, 15])
def test_inflation_radii(vg, r):
    rng = np.random.default_rng(100 + r)
    P = _pair(vg, n=(70, 50, 33), r=r)
    d = rng.uniform(0.3, 3.0, size=(30, 40)).astype(np.float32)
    P.depth(d, body_pose([0.01, 0.02, 0.03], 1.0, 0.2))
    P.close()


@pytest.mark.parametrize("n,r", [((200, 200, 100), 1), ((200, 200, 100), 3), ((100, 110, 100), 2)])
def test_inflate_tile_heights(vg, n, r):
    # grids with one to four 8-slice inflate tiles per SM take tiles 4 slices
    # high: 200 x 200 x 100 has 325 tiles 8 words wide, 100 x 110 x 100 has
    # 182 tiles 4 words wide; every radius and both widths match the oracle
    rng = np.random.default_rng(sum(n) + r)
    P = _pair(vg, n=n, vs=0.05, depth=3.0, r=r, pos=(0.01, 0.02, 0.03))
    for k in range(2):
        d = rng.uniform(1.5, 3.5, size=(48, 64)).astype(np.float32)
        d[rng.random(d.shape) < 0.1] = 0
        P.depth(d, body_pose([0.01, 0.02, 0.03], rng.uniform(-np.pi, np.pi), rng.uniform(-0.3, 0.3)))
    P.close()


@pytest.mark.parametrize("n", [(1, 1, 1), (1, 17, 1), (33, 1, 2), (45, 31, 7), (31, 9, 5), (64, 64, 8),
                               (129, 3, 4), (8500, 3, 2)])
def test_grid_shapes(vg, n):
    rng = np.random.default_rng(sum(n))
    P = _pair(vg, n=n, vs=0.1, r=1, pos=(0.0, 0.0, 0.0))
    for k in range(3):
        d = rng.uniform(0.05, 3.0, size=(24, 32)).astype(np.float32)
        P.depth(d, body_pose([0.0, 0.0, 0.0], rng.uniform(-3, 3), rng.uniform(-0.5, 0.5)))
        P.shift(rng.uniform(-0.3, 0.3, 3), check=(k == 2))   # else merged by the next frame
    P.close()


def test_camera_outside_grid(vg):
    rng = np.random.default_rng(9)
    P = _pair(vg, n=(30, 30, 10), pos=(0.0, 0.0, 0.0))
    for cam in ([-2.5, 0.1, 0.2], [0.3, 5.0, 0.0], [0.0, 0.0, 3.0]):
        d = rng.uniform(0.5, 3.0, size=(24, 32)).astype(np.float32)
        P.depth(d, body_pose(cam, rng.uniform(-3, 3), rng.uniform(-0.8, 0.8)))
    P.close()


def test_random_attitudes(vg):
    rng = np.random.default_rng(11)
    P = _pair(vg, n=(60, 60, 30), r=2)
    for _ in range(6):
        d = rng.uniform(0.2, 3.0, size=(48, 64)).astype(np.float32)
        d[rng.random(d.shape) < 0.3] = 0
        T = body_pose(rng.uniform(-0.2, 0.2, 3), *rng.uniform(-np.pi, np.pi, 3))
        P.depth(d, T)
    P.close()


def test_axis_aligned_rays(vg):
    # identity attitude with the camera on a voxel corner: rays along grid
    # planes, many exact ties in the traversal
    P = _pair(vg, n=(40, 40, 20), vs=0.25, fx=90.0, fy=90.0, depth=4.0, r=0, pos=(0.0, 0.0, 0.0))
    P.depth(np.full((9, 9), 2.0, np.float32), np.eye(4))
    P.depth(np.full((9, 9), 2.0, np.float32), body_pose([0.0, 0.0, 0.0]))
    P.depth(np.zeros((9, 9), np.float32), body_pose([0.25, 0.5, 0.0], np.pi / 2))
    P.close()


@pytest.mark.parametrize("read_after_shift", [True, False])
def test_shifts(vg, read_after_shift):
    # read_after_shift: each re-centre is read out through the ring (K5)
    # while pending; else only after the next frame's merge has cleared
    # what it brought in
    rng = np.random.default_rng(13)
    P = _pair(vg, n=(30, 20, 10), pos=(0.0, 0.0, 0.0))
    P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose([0, 0, 0]))
    pos = np.zeros(3)
    for step in ([0.1, 0, 0], [0, -0.25, 0.1], [-0.33, 0.47, -0.2], [0, 0, 0], [2.9, 0, 0], [0, 0, 5.0],
                 [-0.05, 0.05, 0.0], [-3.1, 0.0, 0.0], [0.0, 2.1, -1.1]):
        pos = pos + np.array(step)
        P.shift(pos, check=read_after_shift)
        P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose(pos, rng.uniform(-3, 3)))
    P.close()


def test_shifts_in_a_row_do_not_compose(vg):
    # out by 5 voxels and back: the voxels that left are unknown, so the
    # second re-centre cannot be folded into the first
    rng = np.random.default_rng(14)
    P = _pair(vg, n=(30, 20, 10), pos=(0.0, 0.0, 0.0))
    P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose([0, 0, 0]))
    P.shift([0.5, 0.0, 0.0], check=False)
    P.shift([0.0, 0.0, 0.0], check=False)
    P.check("out and back")
    P.shift([0.0, -0.7, 0.3], check=False)
    P.shift([0.4, -0.7, 0.3], check=False)
    P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose([0.4, -0.7, 0.3], 1.0))
    P.shift([40.0, 0.0, 0.0], check=False)             # nothing survives
    P.shift([40.3, 0.0, 0.0], check=False)
    P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose([40.3, 0.0, 0.0], -1.0))
    P.shift([40.3, 0.0, 0.2], check=False)
    P.check("last")
    P.close()


def test_reads_of_a_pending_shift_leave_the_grid_alone(vg):
    # a read with a re-centre pending writes the re-centred grid into dst:
    # straight into device memory or page-locked host memory (aligned), or
    # through the second buffer (unaligned device memory, pageable memory);
    # none of them changes the grid, whose next merge still clears what the
    # re-centre brought in
    rng = np.random.default_rng(16)
    P = _pair(vg, n=(45, 31, 10))
    P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose([0.1, 0.2, 0.3], 0.2))
    P.shift([0.5, -0.3, 0.2], check=False)
    want = P.o.loc.ravel()
    n = P.g.nvox
    dev = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
    pinned = torch.empty(n + 16, dtype=torch.uint8).pin_memory()
    pageable = np.empty(n + 16, np.uint8)
    for off in (0, 1):
        for dst in (dev, pinned):
            view = dst[off:off + n]
            view.fill_(7)
            o = P.g.read(view)
            torch.cuda.synchronize()
            assert list(o) == list(P.o.o)
            assert np.array_equal(view.cpu().numpy(), want), (dst.device, off)
        view = pageable[off:off + n]
        view[:] = 7
        P.g.read(view)
        torch.cuda.synchronize()
        assert np.array_equal(view, want), ("pageable", off)
    P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose([0.5, -0.3, 0.2], -0.4))
    P.close()


def test_page_locked_host_inputs_are_read_in_place(vg):
    w = make("paper", frames=2)
    g = w.grid
    P = Pair(vg, g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    for f in w.frames:
        d = torch.from_numpy(np.ascontiguousarray(f.depth)).pin_memory()
        P.g.integrate_depth(d, f.T_wc, w.cam.scale)
        P.o.integrate_depth(f.T_wc, f.depth, w.cam.scale)
        P.check("pinned depth")
    pts = np.random.default_rng(5).uniform([-2, -1, 0.2], [2, 1, 4], size=(3000, 3)).astype(np.float32)
    T = w.frames[0].T_wc
    P.g.integrate_points(torch.from_numpy(pts).pin_memory(), T)
    P.o.integrate_points(T, pts)
    P.check("pinned points")
    P.close()


def test_write_replaces_a_pending_shift(vg):
    rng = np.random.default_rng(15)
    P = _pair(vg, n=(40, 30, 16))
    P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose([0.1, 0.2, 0.3], 0.2))
    P.shift([0.6, -0.4, 0.2], check=False)
    prior = rng.integers(0, 4, size=P.g.shape).astype(np.uint8)
    origin = np.array([3, -2, 1], np.int32)
    P.g.write(prior.ravel().copy(), origin)
    P.o.loc = prior.copy()
    P.o.o = origin.copy()
    P.check("write over a pending shift")
    P.close()


def test_point_clouds(vg):
    rng = np.random.default_rng(17)
    P = _pair(vg, n=(50, 40, 20), r=2)
    pts = rng.uniform([-2, -1, 0.1], [2, 1, 3.5], size=(5000, 3)).astype(np.float32)
    pts[::97, 0] = np.nan
    pts[::89, 2] = np.inf
    P.points(pts, body_pose([0.01, 0.02, 0.03], 0.4))
    P.points(pts[:1], body_pose([0.01, 0.02, 0.03], -0.4))
    P.points(np.zeros((0, 3), np.float32), body_pose([0.01, 0.02, 0.03], 2.0))
    P.points(pts, body_pose([0.01, 0.02, 0.03], 1.0), device=False)
    P.close()


@pytest.mark.parametrize("npts", [300000, 1000000])
def test_point_clouds_at_scale(vg, npts):
    # dense clouds as in the paper's populate sweep (Fig. 4a: up to 300,000
    # points; here also 1,000,000), uniform in the field of view up to the
    # range, on the paper's standard grid; with a re-centre between frames
    rng = np.random.default_rng(23 + npts)
    P = Pair(vg, (100, 100, 20), 0.15, 85.0, 101.0, 6.5, 2, (7.5, 7.5, 1.4))
    for k in range(2):
        z = rng.uniform(0.3, 6.5, npts)
        tx, ty = np.tan(np.radians(85.0 / 2)), np.tan(np.radians(101.0 / 2))
        pts = np.stack([rng.uniform(-tx, tx, npts) * z, rng.uniform(-ty, ty, npts) * z, z], 1).astype(np.float32)
        pos = np.array([7.5 + 0.3 * k, 7.5 - 0.2 * k, 1.4])
        P.points(pts, body_pose(pos, 0.3 + 0.5 * k, 0.05))
        P.shift(pos + np.array([0.4, 0.1, 0.0]))
    P.close()


@pytest.mark.parametrize("words", [256, 512])
def test_rows_longer_than_a_merge_unit(vg, words):
    # 16,400 voxels a row: 513 plane words, padded to 1024, so a 256- or
    # 512-word K4 unit is one part of a row, and re-centres along x wrap the
    # ring inside the parts
    rng = np.random.default_rng(43 + words)
    P = Pair(vg, (16400, 6, 4), 0.05, 87.0, 58.0, 2.0, 1, (0.0, 0.0, 0.0))
    P.g.set(vg.VG_TUNE_MERGE_WORDS, words)
    pos = np.array([0.0, 0.0, 0.0])
    for k in range(4):
        d = rng.uniform(0.3, 2.2, size=(24, 32)).astype(np.float32)
        P.depth(d, body_pose(pos, 0.05 * k, 0.0))
        pos = pos + np.array([0.37 * (k + 1), 0.0, 0.0])
        P.shift(pos)
    P.close()


def test_bundle_handout_restarts_every_frame(vg):
    # with one K3 CTA per SM the paper's grid has more ray groups (260) than
    # K3 has CTAs (152), so the rest go out one bundle at a time from the
    # grid's counter, which each frame's K1 zeroes (the depth and the point
    # kernel alike): every frame must still trace every ray
    rng = np.random.default_rng(37)
    P = Pair(vg, (100, 100, 20), 0.15, 85.0, 101.0, 6.5, 2, (7.5, 7.5, 1.4))
    P.g.set(vg.VG_TUNE_RT_CTAS_PER_SM, 1)
    for k in range(3):
        pos = np.array([7.5 + 0.2 * k, 7.5 - 0.1 * k, 1.4])
        z = rng.uniform(0.3, 6.5, 20000)
        pts = np.stack([rng.uniform(-0.9, 0.9, 20000) * z, rng.uniform(-1.2, 1.2, 20000) * z, z], 1)
        P.points(pts.astype(np.float32), body_pose(pos, 0.4 * k, 0.05))
        d = rng.uniform(0.4, 6.3, size=(48, 64)).astype(np.float32)
        d[rng.random(d.shape) < 0.1] = 0
        P.depth(d, body_pose(pos, -0.3 * k, -0.05))
        P.shift(pos + np.array([0.3, 0.0, 0.0]))
    P.close()


def test_read_write_roundtrip_and_resume(vg):
    rng = np.random.default_rng(19)
    P = _pair(vg, n=(40, 30, 16))
    prior = rng.integers(0, 4, size=P.g.shape).astype(np.uint8)
    origin = np.array([-17, -11, -9], np.int32)
    P.g.write(torch.from_numpy(prior.ravel().copy()).cuda(), origin)
    P.o.loc = prior.copy()
    P.o.o = origin.copy()
    P.check("after write")
    P.g.write(prior.ravel().copy(), origin)         # host source
    P.check("after host write")
    pos = (origin + np.array([20, 15, 8])) * 0.1 + 0.01
    P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose(pos, 0.7))
    host = np.empty(P.g.nvox, np.uint8)
    o = P.g.read(host)
    torch.cuda.synchronize()
    assert_same(host.reshape(P.g.shape), P.o.loc, "host read")
    assert list(o) == list(P.o.o)
    P.close()


def test_write_after_recentres(vg):
    # re-centres move the grid's ring; a write replaces the grid whole (in
    # its own frame), and frames and re-centres after it go on from there
    rng = np.random.default_rng(47)
    P = _pair(vg, n=(36, 28, 12))
    pos = np.array([0.01, 0.02, 0.03])
    for k in range(3):
        P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose(pos, 0.5 * k))
        pos = pos + np.array([0.23, -0.31, 0.12])
        P.shift(pos, check=False)
    prior = rng.integers(0, 4, size=P.g.shape).astype(np.uint8)
    origin = np.array([5, -7, 2], np.int32)
    P.g.write(torch.from_numpy(prior.ravel().copy()).cuda(), origin)
    P.o.loc = prior.copy()
    P.o.o = origin.copy()
    P.check("after write")
    pos = (origin + np.array([18, 14, 6])) * 0.1 + 0.01
    for k in range(2):
        P.depth(rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32), body_pose(pos, -0.4 * k))
        pos = pos + np.array([-0.17, 0.26, -0.05])
        P.shift(pos)
    P.close()


def test_stats_count_points_and_visits(vg, orc):
    from oracle import OracleParams as OP
    rng = np.random.default_rng(23)
    n, vs, r = (50, 40, 20), 0.1, 1
    P = _pair(vg, n=n, vs=vs, r=r, flags=vg.VG_FLAG_STATS)
    d = rng.uniform(0.2, 3.5, size=(24, 32)).astype(np.float32)
    T = body_pose([0.01, 0.02, 0.03], 0.3)
    P.depth(d, T)
    s = P.g.stats()
    p = OP(n, vs, 87.0, 58.0, 3.0, r)
    pose = orc.pose_vc(p, T, P.o.o)
    raw, kept = orc.voxelize_depth(p, pose, d)
    _, _, visits = orc.raytrace(p, pose, orc.inflate(p, raw))
    assert s["frames"] == 1 and s["points_in_grid"] == kept and s["ray_visits"] == visits, (s, kept, visits)
    P.close()


def test_profile_counts_launches(vg):
    w = make("paper", frames=3)
    g = w.grid
    grid = vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    grid.profile(True)
    for f in w.frames:
        grid.integrate_depth(torch.from_numpy(f.depth).cuda(), f.T_wc)
        grid.shift(f.robot_pos)
    prof = grid.profile_read()
    for k in ("voxelize", "inflate", "raytrace", "merge"):
        ms, timed, total = prof[k]
        assert timed == 3 and total == 3 and ms > 0, (k, prof[k])
    grid.close()


def test_default_stream_is_torchs_current_stream(vg):
    # with no stream given, the binding enqueues on torch's current stream,
    # also inside a stream context and on a side stream's work order
    default = torch.cuda.current_stream().cuda_stream
    assert vg._stream(None) == default
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        assert vg._stream(None) == side.cuda_stream != default
        w = make("room")
        g = w.grid
        grid = vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
        depth = torch.from_numpy(w.frames[0].depth).cuda()
        out = torch.empty(grid.nvox, dtype=torch.uint8, device="cuda")
        grid.integrate_depth(depth, w.frames[0].T_wc)
        grid.read(out)
    side.synchronize()
    o = OracleGrid(OracleParams(tuple(g.n), g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, 0),
                   w.frames[0].robot_pos)
    o.integrate_depth(w.frames[0].T_wc, w.frames[0].depth)
    assert_same(out.cpu().numpy().reshape(grid.shape), o.loc, "room frame on a side stream")
    assert vg._stream(None) == default
    grid.close()


def test_bad_arguments_on_device(vg):
    P = _pair(vg)
    d = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(vg.VGError) as e:
        P.g.integrate_depth(d, np.full((4, 4), np.nan))
    assert e.value.status == vg.VG_EINVAL
    with pytest.raises(vg.VGError):
        P.g.integrate_depth(torch.zeros((4, 4), dtype=torch.uint16, device="cuda"), np.eye(4), depth_scale=0.0)
    with pytest.raises(ValueError):
        P.g.integrate_depth(torch.zeros((4, 4), dtype=torch.float64, device="cuda"), np.eye(4))
    with pytest.raises(vg.VGError):
        P.g.tune(3)
    small = torch.empty(10, dtype=torch.uint8, device="cuda")
    with pytest.raises(vg.VGError):
        P.g.read(small)
    with pytest.raises(vg.VGError):
        P.g.shift((1e12, 0.0, 0.0))     # origin index beyond int32
    P.close()


# --------------------------------------------------------------------------
# literal readings (comparison flags): the same bit-exact bar


LIT = {"inflate_after_trace": "VG_FLAG_LIT_INFLATE_AFTER_TRACE", "skip_start": "VG_FLAG_LIT_SKIP_START_VOXEL",
       "loc_occupancy": "VG_FLAG_LIT_LOC_OCCUPANCY"}


@pytest.mark.parametrize("lit", sorted(LIT))
@pytest.mark.parametrize("name,frames", [("room", 1), ("paper", 3), ("robot", 4)])
def test_literal_readings(vg, lit, name, frames):
    # the robot sequences re-centre every frame, so the loc_grid reading
    # also reads the grid through a pending re-centre
    w = make(name, frames=frames, robot=3) if name == "robot" else make(name, frames=frames)
    run_workload(vg, w, frames, flags=getattr(vg, LIT[lit]))


def test_literal_readings_full_size(vg):
    w = make("seq", frames=3)
    run_workload(vg, w, 3, flags=vg.VG_FLAG_LIT_SKIP_START_VOXEL | vg.VG_FLAG_LIT_LOC_OCCUPANCY)


def test_literal_flags_rejected_where_unsupported(vg):
    bad = vg.VG_FLAG_LIT_INFLATE_AFTER_TRACE | vg.VG_FLAG_LIT_LOC_OCCUPANCY
    with pytest.raises(vg.VGError):
        vg.Grid((20, 20, 10), 0.1, 87.0, 58.0, 3.0, 1, (0, 0, 0), flags=bad)
    with pytest.raises(vg.VGError):
        vg.Grid((20, 20, 10), 0.1, 87.0, 58.0, 3.0, 1, (0, 0, 0), flags=1 << 9)
    g = vg.Grid((20, 20, 10), 0.1, 87.0, 58.0, 3.0, 1, (0, 0, 0), flags=vg.VG_FLAG_LIT_SKIP_START_VOXEL)
    d = torch.ones((8, 8), dtype=torch.float32, device="cuda")
    b = vg.Batch(1)
    with pytest.raises(vg.VGError):
        b.step([(g, d, np.eye(4), None)])     # batches take the default reading only
    b.close()
    g.close()
