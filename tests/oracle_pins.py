"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each check takes an `Oracle` and raises AssertionError on a violation.  The
same checks run against the real oracle (test_oracle_pins.py) and against
builds of it with a planted mistake (test_oracle_mutants.py), which must
each fail at least one of them.

Sources of truth used here, none of them the oracle's own FP32 arithmetic:
  - numbers printed in the paper (tests/golden/);
  - hand-worked single points and hand-listed voxel walks;
  - float64 brute-force segment/voxel-box intersection with a margin above
    FP32 error (bruteforce.py);
  - scipy.ndimage / numpy routines for dilation and shifting;
  - invariants of the free-space rule (Sec. IV-C) and of Alg. 3.
"""
import json
import os

import numpy as np
import scipy.ndimage as ndi

from oracle import OracleParams
from oracle.oracle import FREE, OCC, TRACED, UNK
from oracle.oracle import LIT_INFLATE_AFTER_TRACE, LIT_LOC_OCCUPANCY, LIT_SKIP_START

import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# tau margins: FP32 error of a crossing time is ~1e-7; segments rebuilt in
# double from the geometry differ from the FP32 ones by ~1e-5 voxel.
EPS_EXACT_SEGMENT = 1e-5
EPS_GEOMETRIC = 2e-4


def _p(n, vs, fx=87.0, fy=58.0, depth=4.0, r=1, literal=0):
    return OracleParams(tuple(int(v) for v in n), float(vs), float(fx), float(fy),
                        float(depth), int(r), int(literal))


# --------------------------------------------------------------------------
# Sec. V printed numbers
# --------------------------------------------------------------------------
def check_paper_standard_setup(orc):
    g = json.load(open(os.path.join(GOLDEN, "paper_standard_setup.json")))
    n = tuple(int(round(m / g["vox_size_m"])) for m in g["grid_size_m"])
    assert n[0] * n[1] * n[2] == g["printed_voxels"], n
    p = _p(n, g["vox_size_m"], g["fov_x_deg"], g["fov_y_deg"], g["depth_m"], g["vox_inf"])
    (vd, hw, hh), nrays = orc.ray_bundle(p)
    assert nrays == (2 * hw + 1) * (2 * hh + 1)
    rel = abs(nrays - g["printed_rays_approx"]) / g["printed_rays_approx"]
    assert rel <= g["rays_rel_tolerance"], (nrays, rel)


def check_ray_bundle_rounding(orc):
    # Sec. IV-C: vox_depth = depth / vox_size and the half widths are the
    # nearest integers to tan(fov/2) * vox_depth, so both sizes are odd.
    rng = np.random.default_rng(7)
    for _ in range(200):
        vs = float(rng.choice([0.05, 0.1, 0.15, 0.2]))
        depth = float(np.float32(rng.uniform(1.0, 8.0)))
        fx, fy = float(rng.uniform(40, 110)), float(rng.uniform(30, 110))
        p = _p((8, 8, 8), vs, fx, fy, depth)
        (vd, hw, hh), nrays = orc.ray_bundle(p)
        vdx = float(np.float32(depth)) / float(np.float32(vs))
        assert abs(vd - vdx) <= 0.5 + 1e-9, (vd, vdx)
        for h, fov in ((hw, fx), (hh, fy)):
            exact = np.tan(np.radians(float(np.float32(fov))) / 2.0) * vd
            assert abs(h - exact) <= 0.5 + 1e-9, (h, exact)
        assert nrays == (2 * hw + 1) * (2 * hh + 1)


def check_intrinsics_span_fov(orc):
    # The image edges (pixel -0.5 and W-0.5) sit at exactly +-fov/2.
    for W, H, fx, fy in ((320, 240, 87.0, 58.0), (640, 480, 90.0, 60.0), (5, 7, 85.0, 101.0)):
        p = _p((8, 8, 8), 0.1, fx, fy)
        K = orc.intrinsics(p, W, H).astype(np.float64)
        ang_x = np.degrees(np.arctan((-0.5 - K[2]) / K[0]))
        ang_y = np.degrees(np.arctan((H - 0.5 - K[3]) / K[1]))
        assert abs(ang_x + fx / 2) < 1e-4 and abs(ang_y - fy / 2) < 1e-4, (K, ang_x, ang_y)
        assert K[2] == (W - 1) / 2 and K[3] == (H - 1) / 2


# --------------------------------------------------------------------------
# Sec. IV-A origin, Sec. IV-B pose composition
# --------------------------------------------------------------------------
def check_origin_centres_robot(orc):
    rng = np.random.default_rng(11)
    for _ in range(300):
        n = rng.integers(2, 60, size=3)
        vs = float(np.float32(rng.choice([0.05, 0.1, 0.15, 0.2, 0.25])))
        pos = rng.uniform(-50, 50, size=3)
        o = orc.origin(_p(n, vs), pos)
        g = pos / vs - o           # robot position in voxel units of the grid
        # the robot is in voxel floor(N/2) (Sec. IV-A, Fig. 1)
        assert np.all(np.floor(g + 1e-9) == n // 2) or np.all(np.floor(g - 1e-9) == n // 2), (n, g)


def check_pose_composition(orc):
    # T^v_c = T^v_w T^w_c: mapping a camera point with T^v_c equals mapping it
    # to the world with T^w_c and subtracting the grid corner o*vox_size.
    rng = np.random.default_rng(12)
    for _ in range(100):
        vs = float(np.float32(rng.choice([0.05, 0.1, 0.2])))
        n = rng.integers(10, 100, size=3)
        T = bf.pose_T_wc(rng.uniform(-5, 5, 3), *rng.uniform(-np.pi, np.pi, 3))
        o = rng.integers(-200, 200, size=3)
        P = orc.pose_vc(_p(n, vs), T, o)
        q = rng.uniform(-3, 3, size=3)
        want = T[:3, :3] @ q + T[:3, 3] - o * vs
        got = P.R.astype(np.float64) @ q + P.t.astype(np.float64)
        assert np.allclose(got, want, atol=1e-4), (got, want)


# --------------------------------------------------------------------------
# Alg. 1: transform and voxelize
# --------------------------------------------------------------------------
def check_single_point_voxel(orc):
    # Hand-worked: body at the world origin, identity attitude, so the camera
    # looks along world +x (camera z -> x, camera x -> -y, camera y -> -z).
    # Grid 40 x 36 x 20 at 0.1 m: origin o = (-20, -18, -10).
    p = _p((40, 36, 20), 0.1, 90.0, 90.0, 5.0, 0)
    T = bf.pose_T_wc([0.0, 0.0, 0.0])
    o = orc.origin(p, [0.0, 0.0, 0.0])
    assert list(o) == [-20, -18, -10], o
    pose = orc.pose_vc(p, T, o)
    # camera point (0.23, -0.11, 1.37) -> world (1.37, -0.23, 0.11)
    # -> grid metres (3.37, 1.57, 1.11) -> voxel (33, 15, 11)
    occ, kept = orc.voxelize_points(p, pose, [[0.23, -0.11, 1.37]])
    assert kept == 1 and occ.sum() == 1 and occ[11, 15, 33] == 1, np.argwhere(occ)
    # depth image, 5 x 5, fov 90 deg: cx = cy = 2, fx = fy = 2.5.
    # pixel (2, 2) at 1.37 m -> camera (0, 0, 1.37) -> voxel (33, 18, 10);
    # pixel (4, 2) at 1.37 m -> camera x = 2*1.37/2.5 = 1.096 -> world
    # y = -1.096 -> grid y = 0.704 m -> voxel (33, 7, 10);
    # pixel (2, 0) at 1.37 m -> camera y = -1.096 -> world z = 1.096 ->
    # grid z = 2.096 m -> voxel (33, 18, 20), outside (Nz = 20): dropped.
    depth = np.zeros((5, 5), np.float32)
    depth[2, 2] = depth[2, 4] = depth[0, 2] = 1.37
    occ, kept = orc.voxelize_depth(p, pose, depth)
    got = sorted(map(tuple, np.argwhere(occ)[:, ::-1].tolist()))
    assert kept == 2 and got == [(33, 7, 10), (33, 18, 10)], (kept, got)
    # the same pixels as u16 millimetres with scale 0.001
    raw = (depth * 1000).round().astype(np.uint16)
    occ16, kept16 = orc.voxelize_depth(p, pose, raw, scale=0.001)
    assert kept16 == 2 and np.array_equal(occ16, occ)


def check_lattice_boundaries(orc):
    # vox_size 0.25 is exact in binary; g = k exactly lands in voxel k
    # (voxel k covers [k, k+1)), and g = N is outside.
    p = _p((8, 8, 8), 0.25, r=0)
    T = np.eye(4)                       # camera frame == world frame
    o = orc.origin(p, [0.0, 0.0, 0.0])  # (-4, -4, -4): grid spans [-1, 1) m
    pose = orc.pose_vc(p, T, o)
    # 0.5 - 2^-23: after adding t = 1.0 the sum 1.5 - 2^-23 is still exact
    below = 0.5 - 2.0 ** -23
    cases = [((0.5, 0.0, 0.0), (6, 4, 4)), ((below, 0.0, 0.0), (5, 4, 4)),
             ((-1.0, -1.0, -1.0), (0, 0, 0)), ((0.0, 0.0, 0.999), (4, 4, 7)),
             ((1.0, 0.0, 0.0), None), ((0.0, float(np.nextafter(np.float32(-1), np.float32(-2))), 0.0), None),
             ((np.nan, 0.0, 0.0), None), ((np.inf, 0.0, 0.0), None)]
    for q, want in cases:
        occ, kept = orc.voxelize_points(p, pose, [q])
        if want is None:
            assert kept == 0 and occ.sum() == 0, (q, np.argwhere(occ))
        else:
            assert kept == 1 and occ[want[2], want[1], want[0]] == 1, (q, np.argwhere(occ))


def check_pixel_validity(orc):
    # a pixel is valid iff its depth is finite, > 0 and <= depth (Sec. IV-C)
    p = _p((80, 80, 80), 0.1, 90.0, 90.0, 3.0, 0)   # grid spans [-4, 4) m
    o = orc.origin(p, [0, 0, 0])
    pose = orc.pose_vc(p, bf.pose_T_wc([0, 0, 0]), o)
    for d, ok in ((0.0, False), (-1.0, False), (np.nan, False), (np.inf, False),
                  (3.0, True), (float(np.nextafter(np.float32(3.0), np.float32(4.0))), False),
                  (1e-3, True)):
        depth = np.zeros((3, 3), np.float32)
        depth[1, 1] = d
        _, kept = orc.voxelize_depth(p, pose, depth)
        assert kept == int(ok), (d, kept)


def check_occupied_voxels_hold_points(orc):
    # Every pre-inflation occupied voxel holds a valid point, and every valid
    # in-grid point away from voxel faces lands in an occupied voxel.
    rng = np.random.default_rng(21)
    for trial in range(6):
        n = (30, 26, 14)
        vs = float(np.float32(0.1))
        p = _p(n, vs, 87.0, 58.0, 2.5, 0)
        pos = rng.uniform(-1, 1, 3)
        T = bf.pose_T_wc(pos, rng.uniform(-3, 3), rng.uniform(-0.4, 0.4), rng.uniform(-0.3, 0.3))
        o = orc.origin(p, pos)
        depth = rng.uniform(0.2, 3.0, size=(24, 32)).astype(np.float32)
        depth[rng.random(depth.shape) < 0.1] = 0.0
        occ, _ = orc.voxelize_depth(p, orc.pose_vc(p, T, o), depth)
        pw = bf.depth_points_world(depth, 87.0, 58.0, T, 2.5)
        g = pw / vs - o
        margin = 1e-3
        for v in np.argwhere(occ)[:, ::-1]:
            inside = np.all((g >= v - margin) & (g <= v + 1 + margin), axis=1)
            assert inside.any(), ("occupied voxel with no point", trial, v)
        frac = g - np.floor(g)
        clear = np.all((frac > margin) & (frac < 1 - margin), axis=1)
        ing = np.all((g >= 0) & (g < np.array(n)), axis=1)
        for gi in np.floor(g[clear & ing]).astype(int):
            assert occ[gi[2], gi[1], gi[0]] == 1, ("point voxel not occupied", gi)


# --------------------------------------------------------------------------
# Alg. 1: inflation
# --------------------------------------------------------------------------
def check_inflation(orc):
    rng = np.random.default_rng(31)
    for r in (0, 1, 2, 3):
        n = (17, 13, 9)
        p = _p(n, 0.1, r=r)
        # one voxel in a corner: the clipped cube
        raw = np.zeros(p.shape, np.uint8)
        raw[0, 12, 1] = 1
        inf = orc.inflate(p, raw)
        want = np.zeros(p.shape, np.uint8)
        want[0:r + 1, max(0, 12 - r):13, max(0, 1 - r):1 + r + 1] = 1
        assert np.array_equal(inf, want), r
        # random sparse occupancy vs scipy's binary dilation with a cube
        raw = (rng.random(p.shape) < 0.02).astype(np.uint8)
        want = ndi.binary_dilation(raw.astype(bool), np.ones((2 * r + 1,) * 3, bool)) if r else raw.astype(bool)
        assert np.array_equal(orc.inflate(p, raw).astype(bool), want), r


def check_literal_alg1_equals_dilation(orc):
    # Alg. 1 stamps a cube per point; stamping per occupied voxel after
    # voxelizing gives the same grid.
    rng = np.random.default_rng(41)
    for r in (1, 2):
        p = _p((24, 20, 12), 0.1, 87.0, 58.0, 2.0, r)
        pos = rng.uniform(-0.5, 0.5, 3)
        T = bf.pose_T_wc(pos, rng.uniform(-3, 3), 0.1, 0.0)
        pose = orc.pose_vc(p, T, orc.origin(p, pos))
        depth = rng.uniform(0.3, 2.2, size=(30, 40)).astype(np.float32)
        lit = orc.add_occ_literal_depth(p, pose, depth)
        raw, _ = orc.voxelize_depth(p, pose, depth)
        assert np.array_equal(lit, orc.inflate(p, raw))


# --------------------------------------------------------------------------
# Alg. 2: traversal
# --------------------------------------------------------------------------
def _walk_ok(vis, n, S, D, eps):
    """The walk is face-connected, never repeats a voxel, enters voxels in
    increasing tau, covers every voxel the segment crosses for longer than
    eps and none it misses by more than eps."""
    vis = np.asarray(vis)
    if len(vis) > 1:
        step = np.abs(np.diff(vis, axis=0)).sum(axis=1)
        assert np.all(step == 1), "walk is not face-connected"
    assert len({tuple(v) for v in vis.tolist()}) == len(vis), "voxel visited twice"
    ov = bf.segment_overlap(n, S, [D])
    must = {tuple(v) for v in np.argwhere(ov > eps)[:, ::-1].tolist()}
    may = {tuple(v) for v in np.argwhere(ov > -eps)[:, ::-1].tolist()}
    got = {tuple(v) for v in vis.tolist()}
    assert must <= got, ("missed voxels", sorted(must - got)[:5])
    assert got <= may, ("spurious voxels", sorted(got - may)[:5])
    # entry tau of each visited voxel is non-decreasing
    S64, D64 = np.asarray(S, np.float64), np.asarray(D, np.float64)
    ent = []
    for v in vis:
        lo = 0.0
        for k in range(3):
            if D64[k] != 0:
                a = (v[k] - S64[k]) / D64[k]
                b = (v[k] + 1 - S64[k]) / D64[k]
                lo = max(lo, min(a, b))
        ent.append(lo)
    assert np.all(np.diff(ent) >= -eps), "walk not monotone in tau"


def check_dda_bruteforce(orc):
    rng = np.random.default_rng(51)
    n = (12, 10, 9)
    for _ in range(400):
        S = rng.uniform(-2, 14, 3).astype(np.float32)
        D = rng.uniform(-14, 14, 3).astype(np.float32)
        if rng.random() < 0.2:
            D[rng.integers(3)] = 0.0     # axis-parallel in one axis
        vis = orc.dda(n, S, D)
        _walk_ok(vis, n, S, D, EPS_EXACT_SEGMENT)


def check_dda_hand_walks(orc):
    # Hand-listed walks.  Ties (a crossing of two or three faces at once) go
    # to the lowest axis first; the start voxel is visited; the walk stops
    # when the next crossing is at tau >= 1.
    n = (8, 8, 8)
    cases = [
        ((0.5, 0.5, 0.5), (2, 2, 0), [(0, 0, 0), (1, 0, 0), (1, 1, 0), (2, 1, 0), (2, 2, 0)]),
        ((0.5, 0.5, 0.5), (2, 2, 2), [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1),
                                      (2, 1, 1), (2, 2, 1), (2, 2, 2)]),
        ((2.5, 0.5, 0.5), (-2, 0, 0), [(2, 0, 0), (1, 0, 0), (0, 0, 0)]),
        ((2.0, 0.5, 0.5), (-1, 0, 0), [(2, 0, 0), (1, 0, 0)]),
        ((0.5, 0.5, 0.5), (1.5, 0, 0), [(0, 0, 0), (1, 0, 0)]),
        # z faces at tau 1/6, 1/2, 5/6; y faces at 1/4, 3/4; ends in (0, 1, 3)
        ((0.5, 3.5, 0.5), (0, -2, 3), [(0, 3, 0), (0, 3, 1), (0, 2, 1), (0, 2, 2), (0, 1, 2),
                                       (0, 1, 3)]),
        ((-1.5, 0.5, 0.5), (3, 0, 0), [(0, 0, 0), (1, 0, 0)]),
        ((7.5, 7.5, 7.5), (3, 0, 0), [(7, 7, 7)]),
        ((3.25, 3.25, 3.25), (0, 0, 0), [(3, 3, 3)]),
    ]
    for S, D, want in cases:
        got = [tuple(v) for v in orc.dda(n, np.float32(S), np.float32(D)).tolist()]
        assert got == want, (S, D, got, want)


# --------------------------------------------------------------------------
# Alg. 2 + resolve: the free-space rule on whole frames
# --------------------------------------------------------------------------
def _small_setup(orc, r=0, n=(28, 24, 12), vs=0.2, depth=2.0, pos=(0.03, -0.02, 0.05), yaw=0.0):
    p = _p(n, vs, 87.0, 58.0, depth, r)
    T = bf.pose_T_wc(pos, yaw, 0.0, 0.0)
    o = orc.origin(p, pos)
    return p, T, o, orc.pose_vc(p, T, o)


def _bundle_sets(orc, p, T, o, eps=EPS_GEOMETRIC):
    (vd, hw, hh), _ = orc.ray_bundle(p)
    S, D = bf.bundle_segments(p.vox_size, o, T, vd, hw, hh)
    ov = bf.segment_overlap(p.n, S, D)
    return ov > eps, ov > -eps


def check_empty_frame_all_free(orc):
    # No valid pixel: nothing is occupied and every voxel a ray crosses is
    # free (the paper's stated assumption that obstacles are all detected).
    for yaw in (0.0, 0.7, -2.0):
        p, T, o, _ = _small_setup(orc, yaw=yaw)
        loc = np.zeros(p.shape, np.uint8)
        ms = orc.integrate_depth(p, o, T, np.zeros((24, 32), np.float32), 1.0, loc, want_ms=True)
        must, may = _bundle_sets(orc, p, T, o)
        assert not np.any(ms == OCC) and not np.any(ms == TRACED)
        assert np.all(ms[must] == FREE), "crossed voxel not free"
        assert np.all(ms[~may] == UNK), "free voxel no ray crosses"
        assert np.array_equal(loc, ms)


def _wall_points(x_wall, extent=6.0, step=0.02):
    # points on the world plane x = x_wall, in camera coordinates of the
    # identity-attitude camera at the world origin (camera z = world x,
    # camera x = -world y, camera y = -world z)
    ys, zs = np.meshgrid(np.arange(-extent, extent, step), np.arange(-extent, extent, step))
    return np.stack([-ys.ravel(), -zs.ravel(), np.full(ys.size, x_wall)], axis=1).astype(np.float32)


def check_wall_closed_form(orc):
    # A wall across the whole grid at world x = 1.13 m: voxels in front of the
    # (inflated) wall that rays cross are free, the wall slab is occupied,
    # voxels behind it that rays cross are unknown-and-traced.
    for r in (0, 1, 2):
        p = _p((28, 24, 12), 0.2, 87.0, 58.0, 2.0, r)
        T = bf.pose_T_wc([0.0, 0.0, 0.0])
        o = orc.origin(p, [0.0, 0.0, 0.0])
        loc = np.zeros(p.shape, np.uint8)
        ms = orc.integrate_points(p, o, T, _wall_points(1.13), loc, want_ms=True)
        k = int(np.floor(1.13 / 0.2)) - o[0]        # wall slice: 5 + 14 = 19
        xs = np.arange(p.n[0]).reshape(1, 1, -1)
        slab = (xs >= k - r) & (xs <= k + r)
        slab = np.broadcast_to(slab, p.shape)
        must, may = _bundle_sets(orc, p, T, o)
        assert np.all(ms[slab] == OCC), r
        assert not np.any(ms[~slab] == OCC), r
        front = np.broadcast_to(xs < k - r, p.shape)
        back = np.broadcast_to(xs > k + r, p.shape)
        assert np.all(ms[must & front] == FREE), r
        assert np.all(ms[must & back] == TRACED), r
        assert not np.any(ms[back] == FREE) and not np.any(ms[front] == TRACED), r
        assert np.all(ms[~may & ~slab] == UNK), r


def check_occluder_shadow(orc):
    # A small cube of points in front of the camera: rays through it are
    # unknown-and-traced behind it, rays beside it stay free; a voxel both
    # kinds of ray cross is free (free wins), and no voxel is both written
    # free and occupied.
    p, T, o, pose = _small_setup(orc, r=0, pos=(0.0, 0.0, 0.0))
    g = np.mgrid[0.5:0.7:0.01, -0.1:0.1:0.01, -0.1:0.1:0.01].reshape(3, -1).T
    pts = np.stack([-g[:, 1], -g[:, 2], g[:, 0]], axis=1).astype(np.float32)
    raw, _ = orc.voxelize_points(p, pose, pts)
    inf = orc.inflate(p, raw)
    fr, tr, _ = orc.raytrace(p, pose, inf)
    assert not np.any(fr & inf), "a ray wrote free into an occupied voxel"
    assert np.any(tr), "nothing behind the occluder"
    assert np.any(fr & tr), "no voxel seen both free and behind the occluder"
    ms = orc.resolve(inf, fr, tr)
    assert np.all(ms[(fr == 1) & (inf == 0)] == FREE)
    # every traced-only voxel lies behind the occluder (world x > 0.5)
    xs = (np.argwhere((ms == TRACED))[:, 2] + o[0]) * p.vox_size
    assert np.all(xs >= 0.5 - p.vox_size), xs.min()


def check_rays_stop_at_inflated_voxels(orc):
    # Alg. 1 inflates before Alg. 2 runs, so a ray that only grazes the
    # inflated halo of an obstacle is blocked there too.  One point, r = 2:
    # behind the halo, a voxel that some ray crosses without touching the
    # halo is free; a voxel that only halo-crossing rays reach is
    # unknown-and-traced.
    p = _p((40, 32, 16), 0.1, 87.0, 58.0, 3.0, 2)
    pos = np.array([0.013, 0.027, 0.031])
    T = bf.pose_T_wc(pos)
    o = orc.origin(p, pos)
    w = np.array([1.05, 0.05, 0.05])                      # the obstacle point
    cam = np.array([-(w[1] - pos[1]), -(w[2] - pos[2]), w[0] - pos[0]], np.float32)
    loc = np.zeros(p.shape, np.uint8)
    ms = orc.integrate_points(p, o, T, cam[None, :], loc, want_ms=True)
    c = np.floor(w / p.vox_size).astype(int) - o          # point voxel (30, 16, 8)
    assert ms[c[2], c[1], c[0]] == OCC
    (vd, hw, hh), _ = orc.ray_bundle(p)
    S, D = bf.bundle_segments(p.vox_size, o, T, vd, hw, hh)
    halo_lo, halo_hi = c - 2, c + 3
    hit_may = bf.box_overlap(S, D, halo_lo, halo_hi) > -EPS_GEOMETRIC
    hit_must = bf.box_overlap(S, D, halo_lo, halo_hi) > EPS_GEOMETRIC
    seen_free = seen_traced = 0
    for x in range(c[0] + 3, p.n[0]):
        for y in range(c[1] - 6, c[1] + 7):
            for z in range(c[2] - 6, c[2] + 7):
                v = np.array([x, y, z])
                ov = bf.box_overlap(S, D, v, v + 1)
                must, may = ov > EPS_GEOMETRIC, ov > -EPS_GEOMETRIC
                state = ms[z, y, x]
                if np.any(must & ~hit_may):
                    assert state == FREE, (v, state)
                    seen_free += 1
                elif np.any(must) and np.all(hit_must[may]):
                    assert state == TRACED, (v, state)
                    seen_traced += 1
    assert seen_free > 0 and seen_traced > 0, (seen_free, seen_traced)


# --------------------------------------------------------------------------
# The literal readings (comparison flags): each pinned by brute force or a
# closed form of its own, and against the default where they must agree
# --------------------------------------------------------------------------
def check_skip_start_walks(orc):
    # "move by a voxel" before the first test: the walk is the segment's
    # crossed voxels without the start voxel floor(S)
    rng = np.random.default_rng(52)
    n = (12, 10, 9)
    for _ in range(300):
        S = rng.uniform(-2, 14, 3).astype(np.float32)
        D = rng.uniform(-14, 14, 3).astype(np.float32)
        if rng.random() < 0.2:
            D[rng.integers(3)] = 0.0
        start = tuple(int(v) for v in np.floor(S))
        vis = orc.dda(n, S, D, literal=LIT_SKIP_START)
        got = [tuple(v) for v in vis.tolist()]
        assert start not in got, (S, D)
        inside = all(0 <= start[k] < n[k] for k in range(3))
        _walk_ok(np.array(([start] if inside else []) + got, np.int32).reshape(-1, 3), n, S, D,
                 EPS_EXACT_SEGMENT)
    # hand walk: the first case of the default's hand list without its start
    got = [tuple(v) for v in orc.dda((8, 8, 8), np.float32((0.5, 0.5, 0.5)), np.float32((2, 2, 0)),
                                     literal=LIT_SKIP_START).tolist()]
    assert got == [(1, 0, 0), (1, 1, 0), (2, 1, 0), (2, 2, 0)], got


def check_skip_start_leaves_camera_voxel(orc):
    # every ray starts in the camera's voxel and walks away from it, so with
    # the start skipped no ray visits it: an empty frame leaves it unknown
    # and marks every other crossed voxel free
    p, T, o, pose = _small_setup(orc, yaw=0.4)
    ps = _p(p.n, p.vox_size, p.fov_x_deg, p.fov_y_deg, p.depth, p.vox_inf, LIT_SKIP_START)
    loc = np.zeros(p.shape, np.uint8)
    ms = orc.integrate_depth(ps, o, T, np.zeros((24, 32), np.float32), 1.0, loc, want_ms=True)
    cam = np.floor(np.asarray(pose.t, np.float64) / p.vox_size).astype(int)
    must, may = _bundle_sets(orc, p, T, o)
    must[cam[2], cam[1], cam[0]] = False
    assert ms[cam[2], cam[1], cam[0]] == UNK
    assert np.all(ms[must] == FREE) and np.all(ms[~may] == UNK)
    assert not np.any(ms == OCC) and not np.any(ms == TRACED)


def _point_shadow(orc, p, pos, w, blocker_lo, blocker_hi, ms):
    # behind a single obstacle point w: a voxel some ray crosses without
    # touching the blocker box is free, a voxel only blocker-crossing rays
    # reach is unknown-and-traced (the blocker is what the rays test)
    o = orc.origin(p, pos)
    T = bf.pose_T_wc(pos)
    (vd, hw, hh), _ = orc.ray_bundle(p)
    S, D = bf.bundle_segments(p.vox_size, o, T, vd, hw, hh)
    hit_may = bf.box_overlap(S, D, blocker_lo, blocker_hi) > -EPS_GEOMETRIC
    hit_must = bf.box_overlap(S, D, blocker_lo, blocker_hi) > EPS_GEOMETRIC
    c = np.floor(w / p.vox_size).astype(int) - o
    seen_free = seen_traced = 0
    for x in range(c[0] + 3, p.n[0]):
        for y in range(c[1] - 6, c[1] + 7):
            for z in range(c[2] - 6, c[2] + 7):
                v = np.array([x, y, z])
                ov = bf.box_overlap(S, D, v, v + 1)
                must, may = ov > EPS_GEOMETRIC, ov > -EPS_GEOMETRIC
                if np.any(must & ~hit_may):
                    assert ms[z, y, x] == FREE, (v, ms[z, y, x])
                    seen_free += 1
                elif np.any(must) and np.all(hit_must[may]):
                    assert ms[z, y, x] == TRACED, (v, ms[z, y, x])
                    seen_traced += 1
    return seen_free, seen_traced


def check_inflate_after_trace_rays_see_points(orc):
    # tracing before inflating: rays stop only at the point's own voxel, yet
    # the inflated halo is still marked occupied.  Same scene as
    # check_rays_stop_at_inflated_voxels, where the halo blocks.
    pos = np.array([0.013, 0.027, 0.031])
    w = np.array([1.05, 0.05, 0.05])
    p = _p((40, 32, 16), 0.1, 87.0, 58.0, 3.0, 2, LIT_INFLATE_AFTER_TRACE)
    o = orc.origin(p, pos)
    T = bf.pose_T_wc(pos)
    cam = np.array([-(w[1] - pos[1]), -(w[2] - pos[2]), w[0] - pos[0]], np.float32)
    loc = np.zeros(p.shape, np.uint8)
    ms = orc.integrate_points(p, o, T, cam[None, :], loc, want_ms=True)
    c = np.floor(w / p.vox_size).astype(int) - o
    assert np.all(ms[c[2] - 2:c[2] + 3, c[1] - 2:c[1] + 3, c[0] - 2:c[0] + 3] == OCC)
    f, t = _point_shadow(orc, p, pos, w, c, c + 1, ms)
    assert f > 0 and t > 0, (f, t)
    # some voxel the halo shadows in the default reading is free here
    pd = _p((40, 32, 16), 0.1, 87.0, 58.0, 3.0, 2)
    msd = orc.integrate_points(pd, o, T, cam[None, :], np.zeros(p.shape, np.uint8), want_ms=True)
    assert np.any((msd == TRACED) & (ms == FREE))
    assert not np.any((msd == FREE) & (ms == TRACED))


def check_loc_reading(orc):
    # Alg. 2 testing loc_grid: rays stop at an obstacle the grid held before
    # this measurement (kept occupied, as no ray writes it), and pass through
    # the measurement's own obstacle, whose voxel they overwrite with free.
    pos = np.array([0.013, 0.027, 0.031])
    T = bf.pose_T_wc(pos)
    p = _p((40, 32, 16), 0.1, 87.0, 58.0, 3.0, 0, LIT_LOC_OCCUPANCY)
    o = orc.origin(p, pos)
    old = np.array([1.05, 0.05, 0.05])                    # obstacle in loc only
    c = np.floor(old / p.vox_size).astype(int) - o
    prior = np.zeros(p.shape, np.uint8)
    prior[c[2], c[1], c[0]] = OCC
    new = np.array([0.55, -0.35, 0.05])                   # obstacle in the frame only, off the old one's line
    cn = np.floor(new / p.vox_size).astype(int) - o
    cam = np.array([-(new[1] - pos[1]), -(new[2] - pos[2]), new[0] - pos[0]], np.float32)
    loc = prior.copy()
    ms = orc.integrate_points(p, o, T, cam[None, :], loc, want_ms=True)
    assert ms[cn[2], cn[1], cn[0]] == FREE and loc[cn[2], cn[1], cn[0]] == FREE
    assert ms[c[2], c[1], c[0]] == UNK and loc[c[2], c[1], c[0]] == OCC
    f, t = _point_shadow(orc, p, pos, old, c, c + 1, ms)
    assert f > 0 and t > 0, (f, t)
    # the default reading: the frame's obstacle is occupied and blocks, the
    # stale one is crossed and freed
    pd = _p((40, 32, 16), 0.1, 87.0, 58.0, 3.0, 0)
    locd = prior.copy()
    msd = orc.integrate_points(pd, o, T, cam[None, :], locd, want_ms=True)
    assert msd[cn[2], cn[1], cn[0]] == OCC and locd[c[2], c[1], c[0]] == FREE
    # the resolve table of this reading: free > traced > occupied > unknown
    combos = np.array([[a, b, d] for a in (0, 1) for b in (0, 1) for d in (0, 1)], np.uint8)
    got = orc.resolve(combos[:, 0], combos[:, 1], combos[:, 2], literal=LIT_LOC_OCCUPANCY)
    assert got.tolist() == [FREE if b else TRACED if d else OCC if a else UNK for a, b, d in combos]


def check_resolve_and_merge_tables(orc):
    # resolve: precedence occupied > free > traced > unknown
    combos = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], np.uint8)
    ms = orc.resolve(combos[:, 0], combos[:, 1], combos[:, 2])
    want = [OCC if a else FREE if b else TRACED if c else UNK for a, b, c in combos]
    assert ms.tolist() == want
    # Alg. 3: loc takes ms wherever ms is not unknown, for all 16 pairs
    old = np.repeat(np.arange(4, dtype=np.uint8), 4)
    new = np.tile(np.arange(4, dtype=np.uint8), 4)
    loc = old.copy()
    orc.merge(new, loc)
    assert loc.tolist() == [o if m == UNK else m for o, m in zip(old, new)]


def check_untouched_voxels_keep_prior(orc):
    rng = np.random.default_rng(61)
    for trial in range(3):
        p, T, o, pose = _small_setup(orc, r=1, yaw=rng.uniform(-3, 3), pos=rng.uniform(-0.2, 0.2, 3))
        prior = rng.integers(0, 4, size=p.shape).astype(np.uint8)
        loc = prior.copy()
        depth = rng.uniform(0.3, 2.5, size=(24, 32)).astype(np.float32)
        depth[rng.random(depth.shape) < 0.3] = 0.0
        ms = orc.integrate_depth(p, o, T, depth, 1.0, loc, want_ms=True)
        must, may = _bundle_sets(orc, p, T, o)
        occ = ms == OCC
        assert np.array_equal(loc[~may & ~occ], prior[~may & ~occ]), trial
        assert np.all(ms[must] != UNK), trial
        assert np.array_equal(loc[ms != UNK], ms[ms != UNK])


def check_order_independence(orc):
    rng = np.random.default_rng(71)
    p, T, o, pose = _small_setup(orc, r=1, yaw=0.4)
    pts = rng.uniform([-1, -1, 0.3], [1, 1, 2.2], size=(400, 3)).astype(np.float32)
    raw, _ = orc.voxelize_points(p, pose, pts)
    raw2, _ = orc.voxelize_points(p, pose, pts[rng.permutation(len(pts))])
    assert np.array_equal(raw, raw2)
    inf = orc.inflate(p, raw)
    fr, tr, _ = orc.raytrace(p, pose, inf)
    _, nrays = orc.ray_bundle(p)
    for _ in range(3):
        fr2, tr2, _ = orc.raytrace(p, pose, inf, ray_order=rng.permutation(nrays))
        assert np.array_equal(fr, fr2) and np.array_equal(tr, tr2)


# --------------------------------------------------------------------------
# Sec. IV-E: shift
# --------------------------------------------------------------------------
def _np_shift(a, delta):
    out = np.zeros_like(a)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    for k in range(3):
        ax = 2 - k
        d = int(delta[k])
        m = a.shape[ax]
        if abs(d) >= m:
            return out
        src[ax] = slice(max(d, 0), m + min(d, 0))
        dst[ax] = slice(max(-d, 0), m - max(d, 0))
    out[tuple(dst)] = a[tuple(src)]
    return out


def check_shift(orc):
    rng = np.random.default_rng(81)
    n = (11, 7, 5)
    a = rng.integers(0, 4, size=(5, 7, 11)).astype(np.uint8)
    assert np.array_equal(orc.shift(n, (0, 0, 0), a), a)
    for d in ((11, 0, 0), (0, -7, 0), (0, 0, 9), (-20, 3, 1)):
        assert not np.any(orc.shift(n, d, a)), d
    for _ in range(50):
        d = rng.integers(-4, 5, size=3)
        got = orc.shift(n, d, a)
        assert np.array_equal(got, _np_shift(a, d)), d
        back = orc.shift(n, -d, got)
        # shifting back restores the voxels that stayed inside the grid
        keep = _np_shift(_np_shift(np.ones_like(a), d), -d).astype(bool)
        assert np.array_equal(back[keep], a[keep]) and not np.any(back[~keep]), d


def check_grid_follows_robot(orc):
    # Sec. IV-E: after the robot moves, each world voxel keeps its state and
    # the voxels that entered the grid are unknown.
    from oracle import OracleGrid
    p = _p((20, 16, 8), 0.1, 87.0, 58.0, 1.5, 0)
    g = OracleGrid(p, [0.0, 0.0, 0.0], orc)
    rng = np.random.default_rng(91)
    g.loc[:] = rng.integers(0, 4, size=p.shape)
    before = {tuple(int(c) for c in (np.array(v[::-1]) + g.o)): int(g.loc[tuple(v)])
              for v in np.argwhere(np.ones(p.shape, bool))}
    g.shift([0.33, -0.21, 0.12])
    assert list(g.o) == [3 - 10, -3 - 8, 1 - 4], g.o
    for v in np.argwhere(np.ones(p.shape, bool)):
        w = tuple(int(c) for c in (np.array(v[::-1]) + g.o))
        assert int(g.loc[tuple(v)]) == before.get(w, UNK), (v, w)


ALL_CHECKS = [
    check_paper_standard_setup, check_ray_bundle_rounding, check_intrinsics_span_fov,
    check_origin_centres_robot, check_pose_composition, check_single_point_voxel,
    check_lattice_boundaries, check_pixel_validity, check_occupied_voxels_hold_points,
    check_inflation, check_literal_alg1_equals_dilation, check_dda_bruteforce,
    check_dda_hand_walks, check_empty_frame_all_free, check_wall_closed_form,
    check_occluder_shadow, check_rays_stop_at_inflated_voxels, check_resolve_and_merge_tables, check_untouched_voxels_keep_prior,
    check_skip_start_walks, check_skip_start_leaves_camera_voxel, check_inflate_after_trace_rays_see_points,
    check_loc_reading,
    check_order_independence, check_shift, check_grid_follows_robot,
]
