"""Independent float64 geometry used to pin the oracle.

Nothing here restates the oracle's FP32 operation order: segments and points
are computed from the geometric definitions in double precision with numpy,
and comparisons carry a margin above FP32 rounding error.
"""
import numpy as np

# Camera optical frame (x right, y down, z forward) mounted on a FLU body:
# columns are the camera axes written in body coordinates.
R_BODY_CAM = np.array([[0.0, 0.0, 1.0],
                       [-1.0, 0.0, 0.0],
                       [0.0, -1.0, 0.0]])


def pose_T_wc(pos, yaw=0.0, pitch=0.0, roll=0.0):
    """Camera-to-world 4x4 for a body at pos with Z-Y-X Euler angles."""
    cy, sy = np.cos(yaw), np.sin(yaw)
    cp, sp = np.cos(pitch), np.sin(pitch)
    cr, sr = np.cos(roll), np.sin(roll)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1.0]])
    Ry = np.array([[cp, 0, sp], [0, 1.0, 0], [-sp, 0, cp]])
    Rx = np.array([[1.0, 0, 0], [0, cr, -sr], [0, sr, cr]])
    T = np.eye(4)
    T[:3, :3] = Rz @ Ry @ Rx @ R_BODY_CAM
    T[:3, 3] = pos
    return T


def segment_overlap(n, S, D):
    """For every voxel of an (nx, ny, nz) grid, the length in tau of the
    overlap between the closed voxel box and the segment S + tau*D,
    tau in [0, 1]; negative where they are apart (by that much, roughly).

    S: (3,), D: (R, 3).  Returns the max over the R segments, shape (nz, ny, nx).
    """
    n = [int(v) for v in n]
    S = np.asarray(S, np.float64)
    D = np.atleast_2d(np.asarray(D, np.float64))
    best = np.full((n[2], n[1], n[0]), -np.inf)
    coords = [np.arange(n[k], dtype=np.float64) for k in range(3)]
    for r0 in range(0, D.shape[0], 64):
        Dc = D[r0:r0 + 64]
        lo = np.zeros((Dc.shape[0], n[2], n[1], n[0]))
        hi = np.ones((Dc.shape[0], n[2], n[1], n[0]))
        for k in range(3):
            shape = [1, 1, 1, 1]
            shape[3 - k] = n[k]
            c = coords[k].reshape(shape)
            d = Dc[:, k].reshape(-1, 1, 1, 1)
            with np.errstate(divide="ignore", invalid="ignore"):
                t0 = (c - S[k]) / d
                t1 = (c + 1.0 - S[k]) / d
            a = np.minimum(t0, t1)
            b = np.maximum(t0, t1)
            inside = (S[k] >= c) & (S[k] <= c + 1.0)
            zero = (d == 0.0)
            a = np.where(zero, np.where(inside, -np.inf, np.inf), a)
            b = np.where(zero, np.where(inside, np.inf, -np.inf), b)
            lo = np.maximum(lo, a)
            hi = np.minimum(hi, b)
        best = np.maximum(best, (hi - lo).max(axis=0))
    return best


def bundle_segments(vox_size, o, T_wc, vd, hw, hh):
    """The ray bundle of Sec. IV-C in double: camera centre in voxel units
    and one direction per far-plane voxel (a, b, vd), rotated to the grid."""
    T = np.asarray(T_wc, np.float64)
    S = (T[:3, 3] - np.asarray(o, np.float64) * vox_size) / vox_size
    a, b = np.meshgrid(np.arange(-hw, hw + 1), np.arange(-hh, hh + 1))
    cam = np.stack([a.ravel(), b.ravel(), np.full(a.size, vd)], axis=1).astype(np.float64)
    D = cam @ T[:3, :3].T
    return S, D


def depth_points_world(depth, fov_x_deg, fov_y_deg, T_wc, max_depth, scale=1.0):
    """Back-project a depth image in double (pinhole, principal point at the
    image centre, focal lengths from the field of view); valid pixels only."""
    depth = np.asarray(depth)
    H, W = depth.shape
    if depth.dtype == np.uint16:
        # the depth a u16 pixel stands for, (float)raw * scale, as the method reads it
        d = (depth.astype(np.float32) * np.float32(scale)).astype(np.float64)
    else:
        d = depth.astype(np.float32).astype(np.float64)
    valid = np.isfinite(d) & (d > 0) & (d <= np.float64(np.float32(max_depth)))
    fx = (W / 2.0) / np.tan(np.radians(fov_x_deg) / 2.0)
    fy = (H / 2.0) / np.tan(np.radians(fov_y_deg) / 2.0)
    v, u = np.nonzero(valid)
    z = d[v, u]
    x = (u - (W - 1) / 2.0) * z / fx
    y = (v - (H - 1) / 2.0) * z / fy
    pc = np.stack([x, y, z], axis=1)
    T = np.asarray(T_wc, np.float64)
    return pc @ T[:3, :3].T + T[:3, 3]


def box_overlap(S, D, lo, hi):
    """Per segment S + tau*D (D: (R, 3)), the tau-length of its overlap with
    the closed box [lo, hi]; negative where they are apart."""
    S = np.asarray(S, np.float64)
    D = np.atleast_2d(np.asarray(D, np.float64))
    a = np.zeros(D.shape[0])
    b = np.ones(D.shape[0])
    for k in range(3):
        d = D[:, k]
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = (lo[k] - S[k]) / d
            t1 = (hi[k] - S[k]) / d
        inside = (S[k] >= lo[k]) & (S[k] <= hi[k])
        t_lo = np.where(d == 0, np.where(inside, -np.inf, np.inf), np.minimum(t0, t1))
        t_hi = np.where(d == 0, np.where(inside, np.inf, -np.inf), np.maximum(t0, t1))
        a = np.maximum(a, t_lo)
        b = np.minimum(b, t_hi)
    return b - a
