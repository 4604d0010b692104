"""The allocation-free entry point against the ordinary one.

vg_integrate_depth_noalloc is for callers that cannot call cudaMalloc: a
real-time loop that must never block in the driver's allocator, or an
integration that hands out all device memory itself.  It keeps its scratch
planes in a fixed array inside the library instead of allocating them.  Its
grids must equal, voxel for voxel, what vg_create + vg_integrate_depth make
from the same frames, on consecutive calls that reuse the shared array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

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


def _same(a, b, what):
    bad = np.flatnonzero(a != b)
    assert bad.size == 0, "%s: %d voxels differ, first at flat index %d: %d vs %d" % (
        what, bad.size, bad[0], a[bad[0]], b[bad[0]])


def _check_calls(vg, w, frames, depth_of=None):
    """vg_integrate_depth_noalloc into a caller-owned grid and vg_create +
    vg_integrate_depth into a library grid, frame after frame (the re-centre
    is left out: the caller of the allocation-free call owns the origin)."""
    g = w.grid
    grid = vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    origin = grid.origin.copy()
    params = vg.make_params(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf)
    loc = torch.zeros(grid.nvox, dtype=torch.uint8, device="cuda")   # the caller's own grid
    ref = torch.empty_like(loc)
    try:
        for i in frames:
            f = w.frames[i]
            d = torch.from_numpy(f.depth).cuda()
            grid.integrate_depth(d, f.T_wc, w.cam.scale)
            dn = depth_of(f) if depth_of else d   # kept alive until the work has ended
            vg.vg_integrate_depth_noalloc(params, origin, loc, dn, f.T_wc, w.cam.scale)
            grid.read(ref)
            torch.cuda.synchronize()
            del dn
            got, want = loc.cpu().numpy(), ref.cpu().numpy()
            _same(got, want, "%s frame %d" % (w.name, i))
        return got
    finally:
        grid.close()


def test_noalloc_matches_vg_integrate_depth_on_consecutive_calls(vg):
    from synth import make
    w = make("seq", frames=2)          # 640x480 frames, 200x200x100 grid, vox_inf 2
    got = _check_calls(vg, w, range(2))
    counts = np.bincount(got, minlength=4)
    assert counts[1] > 0 and counts[2] > 0 and counts[3] > 0, counts


@pytest.mark.parametrize("vox_inf", [0, 1, 3])
@pytest.mark.parametrize("kind", [0, 4], ids=["f32", "u16"])
def test_noalloc_radii_and_pixel_types(vg, vox_inf, kind):
    # vox_inf 0 skips the inflation (the raw plane is the inflated one);
    # u16 frames carry a depth scale
    from synth import make
    from synth.scenes import GridSpec
    w = make("camera", robot=700 + kind, frames=2, spec=kind)   # 320x240 into 80x80x40
    w.grid = GridSpec(w.grid.n, w.grid.vox_size, w.grid.depth, vox_inf)
    _check_calls(vg, w, range(2))


def test_noalloc_alternating_grid_shapes_reuse_the_array(vg):
    # a small grid, then one at the array's limit (400x256x256: 16 words a
    # row x 256 x 256 = 2^20 words a plane), then the small one again: every
    # call finds the last call's planes, at another stride, in the array
    from synth import make
    small = make("robot", robot=710, frames=2, spec=(320, 240, 0.1, (80, 80, 40), 2))
    large = make("robot", robot=711, frames=1, spec=(640, 480, 0.05, (400, 256, 256), 3))
    _check_calls(vg, small, [0])
    _check_calls(vg, large, [0])
    _check_calls(vg, small, [1])


def test_noalloc_reads_page_locked_depth_in_place(vg):
    from synth import make
    w = make("room")
    _check_calls(vg, w, [0], depth_of=lambda f: torch.from_numpy(f.depth).pin_memory())


def test_noalloc_refuses_memory_the_device_cannot_reach(vg):
    # a pageable host loc grid or depth image: refused before any device work
    L = vg.load()
    params = vg.make_params((40, 40, 20), 0.1, 87.0, 58.0, 3.0, 1)
    origin = np.zeros(3, np.int32)
    T = np.eye(4).ravel()
    loc_dev = torch.zeros(40 * 40 * 20 + 16, dtype=torch.uint8, device="cuda")
    depth_dev = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    loc_host = np.zeros(40 * 40 * 20 + 64, np.uint8)
    loc_host_p = loc_host.ctypes.data + (-loc_host.ctypes.data) % 16     # 16-byte aligned
    depth_host = np.zeros((4, 4), np.float32)

    def call(loc_p, depth_p):
        return L.vg_integrate_depth_noalloc(C.byref(params), origin.ctypes.data_as(C.c_void_p), C.c_void_p(loc_p),
                                            C.c_void_p(depth_p), 4, 4, vg.VG_DEPTH_F32, 1.0,
                                            T.ctypes.data_as(C.c_void_p), None)

    assert call(loc_host_p, depth_dev.data_ptr()) == vg.VG_EINVAL
    assert call(loc_dev.data_ptr(), depth_host.ctypes.data) == vg.VG_EINVAL
    torch.cuda.synchronize()
    assert not loc_dev.any()


def test_noalloc_refuses_grids_beyond_its_scratch(vg):
    # 1024 x 512 x 512 voxels need 32 * 512 * 512 words per plane, more than
    # the fixed array holds: refused before any device work
    L = vg.load()
    params = vg.make_params((1024, 512, 512), 0.05, 87.0, 58.0, 5.0, 2)
    loc = torch.zeros(64, dtype=torch.uint8, device="cuda")
    depth = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    origin = np.zeros(3, np.int32)
    T = np.eye(4).ravel()
    rc = L.vg_integrate_depth_noalloc(C.byref(params), origin.ctypes.data_as(C.c_void_p),
                                      C.c_void_p(loc.data_ptr()), C.c_void_p(depth.data_ptr()), 4, 4,
                                      vg.VG_DEPTH_F32, 1.0, T.ctypes.data_as(C.c_void_p), None)
    assert rc == vg.VG_ESCRATCH, rc
    assert vg.strerror(rc) == "grid too large for the fixed scratch array"
