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


def test_noalloc_matches_vg_integrate_depth_on_consecutive_calls(vg):
    from synth import make
    w = make("seq", frames=2)          # 640x480 frames, 200x200x100 grid, vox_inf 2
    g = w.grid
    grid = vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    origin = grid.origin.copy()
    params = vg.make_params(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf)
    loc = torch.zeros(grid.nvox, dtype=torch.uint8, device="cuda")   # the caller's own grid
    ref = torch.empty_like(loc)
    try:
        for i, f in enumerate(w.frames):
            d = torch.from_numpy(f.depth).cuda()
            grid.integrate_depth(d, f.T_wc)
            vg.vg_integrate_depth_noalloc(params, origin, loc, d, f.T_wc)
            grid.read(ref)
            torch.cuda.synchronize()
            got, want = loc.cpu().numpy(), ref.cpu().numpy()
            _same(got, want, "call %d" % i)
            counts = np.bincount(got, minlength=4)
            assert counts[1] > 0 and counts[2] > 0 and counts[3] > 0, counts
    finally:
        grid.close()


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
