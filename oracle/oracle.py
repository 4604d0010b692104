"""ctypes/numpy wrapper of the C oracle (test infrastructure only).

Arrays follow the paper's layout (Sec. IV-D): a grid of size (Nx, Ny, Nz) is
a C-contiguous numpy array of shape (Nz, Ny, Nx), so that the flat index is
x + y*Nx + z*Nx*Ny.  Every function forwards to the C routine of the same
name in vg_oracle.c; no arithmetic of the method happens in Python.
"""
import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

UNK, FREE, OCC, TRACED = 0, 1, 2, 3
DEPTH_F32, DEPTH_U16 = 0, 1
LIT_INFLATE_AFTER_TRACE, LIT_SKIP_START, LIT_LOC_OCCUPANCY = 1, 2, 4


@dataclasses.dataclass(frozen=True)
class OracleParams:
    """Table I parameters; n is the grid size in voxels (x, y, z)."""
    n: tuple
    vox_size: float
    fov_x_deg: float
    fov_y_deg: float
    depth: float
    vox_inf: int
    literal: int = 0   # LIT_* flags; 0 is the default reading

    @property
    def shape(self):
        return (int(self.n[2]), int(self.n[1]), int(self.n[0]))

    @property
    def nvox(self):
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


class _CParams(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("vox_size", C.c_float), ("fov_x_deg", C.c_float),
                ("fov_y_deg", C.c_float), ("depth", C.c_float), ("vox_inf", C.c_int32),
                ("literal", C.c_uint32)]


class _CPose(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3)]


def _cparams(p):
    c = _CParams()
    for k in range(3):
        c.n[k] = int(p.n[k])
    c.vox_size = p.vox_size
    c.fov_x_deg = p.fov_x_deg
    c.fov_y_deg = p.fov_y_deg
    c.depth = p.depth
    c.vox_inf = int(p.vox_inf)
    c.literal = int(p.literal)
    return c


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _i32(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32))


def _f64(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64))


class Pose:
    """T^v_c rounded to float (R row-major 3x3, t)."""

    def __init__(self, cpose):
        self._c = cpose

    @property
    def R(self):
        return np.array(self._c.R[:], dtype=np.float32).reshape(3, 3)

    @property
    def t(self):
        return np.array(self._c.t[:], dtype=np.float32)


class Oracle:
    """One loaded build of the C oracle (the default build, or a variant)."""

    def __init__(self, lib_path=None):
        path = lib_path or _build.build()
        self.path = path
        L = C.CDLL(path)
        vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
        sig = {
            "or_origin": (None, [vp, vp, vp]),
            "or_pose_vc": (None, [vp, vp, vp, vp]),
            "or_intrinsics": (None, [vp, i32, i32, vp]),
            "or_ray_bundle": (i64, [vp, vp]),
            "or_voxelize_depth": (i64, [vp, vp, vp, i32, i32, i32, f32, vp]),
            "or_voxelize_points": (i64, [vp, vp, vp, i64, vp]),
            "or_inflate": (None, [vp, vp, vp]),
            "or_add_occ_literal_depth": (i64, [vp, vp, vp, i32, i32, i32, f32, vp]),
            "or_dda": (i64, [vp, vp, vp, C.c_uint32, vp, i64]),
            "or_raytrace": (i64, [vp, vp, vp, vp, vp, vp]),
            "or_resolve": (None, [i64, C.c_uint32, vp, vp, vp, vp]),
            "or_merge": (None, [i64, vp, vp]),
            "or_shift": (None, [vp, vp, vp, vp]),
            "or_integrate_depth": (C.c_int, [vp, vp, vp, vp, i32, i32, i32, f32, vp, vp]),
            "or_integrate_points": (C.c_int, [vp, vp, vp, vp, i64, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        self._L = L

    # --- set-up quantities -------------------------------------------------
    def origin(self, p, robot_pos_w):
        o = np.zeros(3, np.int32)
        cp = _cparams(p)
        self._L.or_origin(C.byref(cp), _ptr(_f64(robot_pos_w)), _ptr(o))
        return o

    def pose_vc(self, p, T_wc, o):
        cp, out = _cparams(p), _CPose()
        T = _f64(T_wc).reshape(16)
        self._L.or_pose_vc(C.byref(cp), _ptr(T), _ptr(_i32(o)), C.byref(out))
        return Pose(out)

    def intrinsics(self, p, W, H):
        K = np.zeros(4, np.float32)
        cp = _cparams(p)
        self._L.or_intrinsics(C.byref(cp), int(W), int(H), _ptr(K))
        return K

    def ray_bundle(self, p):
        out = np.zeros(3, np.int32)
        cp = _cparams(p)
        nrays = self._L.or_ray_bundle(C.byref(cp), _ptr(out))
        return tuple(int(v) for v in out), int(nrays)

    # --- Alg. 1 -------------------------------------------------------------
    def voxelize_depth(self, p, pose, depth, scale=1.0, occ_raw=None):
        depth = np.ascontiguousarray(depth)
        H, W = depth.shape
        dt = DEPTH_U16 if depth.dtype == np.uint16 else DEPTH_F32
        if dt == DEPTH_F32:
            depth = depth.astype(np.float32, copy=False)
        if occ_raw is None:
            occ_raw = np.zeros(p.shape, np.uint8)
        cp = _cparams(p)
        kept = self._L.or_voxelize_depth(C.byref(cp), C.byref(pose._c), _ptr(depth), W, H,
                                         dt, float(scale), _ptr(occ_raw))
        return occ_raw, int(kept)

    def voxelize_points(self, p, pose, xyz, occ_raw=None):
        xyz = np.ascontiguousarray(np.asarray(xyz, np.float32).reshape(-1, 3))
        if occ_raw is None:
            occ_raw = np.zeros(p.shape, np.uint8)
        cp = _cparams(p)
        kept = self._L.or_voxelize_points(C.byref(cp), C.byref(pose._c), _ptr(xyz),
                                          xyz.shape[0], _ptr(occ_raw))
        return occ_raw, int(kept)

    def inflate(self, p, occ_raw):
        occ_raw = np.ascontiguousarray(occ_raw, np.uint8)
        occ_inf = np.zeros(p.shape, np.uint8)
        cp = _cparams(p)
        self._L.or_inflate(C.byref(cp), _ptr(occ_raw), _ptr(occ_inf))
        return occ_inf

    def add_occ_literal_depth(self, p, pose, depth, scale=1.0):
        depth = np.ascontiguousarray(depth)
        H, W = depth.shape
        dt = DEPTH_U16 if depth.dtype == np.uint16 else DEPTH_F32
        occ_inf = np.zeros(p.shape, np.uint8)
        cp = _cparams(p)
        self._L.or_add_occ_literal_depth(C.byref(cp), C.byref(pose._c), _ptr(depth), W, H,
                                         dt, float(scale), _ptr(occ_inf))
        return occ_inf

    # --- Alg. 2 -------------------------------------------------------------
    def dda(self, n, S, D, cap=1 << 16, literal=0):
        out = np.zeros((cap, 3), np.int32)
        S = np.ascontiguousarray(np.asarray(S, np.float32))
        D = np.ascontiguousarray(np.asarray(D, np.float32))
        cnt = self._L.or_dda(_ptr(_i32(n)), _ptr(S), _ptr(D), int(literal), _ptr(out), cap)
        if cnt > cap:
            return self.dda(n, S, D, cap=int(cnt), literal=literal)
        return out[:cnt].copy()

    def raytrace(self, p, pose, occ_inf, ray_order=None):
        occ_inf = np.ascontiguousarray(occ_inf, np.uint8)
        fr = np.zeros(p.shape, np.uint8)
        tr = np.zeros(p.shape, np.uint8)
        order = None
        if ray_order is not None:
            order = np.ascontiguousarray(np.asarray(ray_order, np.int64))
        cp = _cparams(p)
        visits = self._L.or_raytrace(C.byref(cp), C.byref(pose._c), _ptr(occ_inf),
                                     _ptr(order) if order is not None else None,
                                     _ptr(fr), _ptr(tr))
        return fr, tr, int(visits)

    # --- resolve / Alg. 3 / shift ---------------------------------------------
    def resolve(self, occ_inf, fr, tr, literal=0):
        occ_inf, fr, tr = (np.ascontiguousarray(a, np.uint8) for a in (occ_inf, fr, tr))
        ms = np.zeros_like(occ_inf)
        self._L.or_resolve(occ_inf.size, int(literal), _ptr(occ_inf), _ptr(fr), _ptr(tr), _ptr(ms))
        return ms

    def merge(self, ms, loc):
        ms = np.ascontiguousarray(ms, np.uint8)
        assert loc.flags.c_contiguous and loc.dtype == np.uint8 and loc.size == ms.size
        self._L.or_merge(ms.size, _ptr(ms), _ptr(loc))
        return loc

    def shift(self, n, delta, src):
        src = np.ascontiguousarray(src, np.uint8)
        dst = np.empty_like(src)
        self._L.or_shift(_ptr(_i32(n)), _ptr(_i32(delta)), _ptr(src), _ptr(dst))
        return dst

    # --- whole measurement ----------------------------------------------------
    def integrate_depth(self, p, o, T_wc, depth, scale, loc, want_ms=False):
        depth = np.ascontiguousarray(depth)
        H, W = depth.shape
        dt = DEPTH_U16 if depth.dtype == np.uint16 else DEPTH_F32
        assert loc.flags.c_contiguous and loc.dtype == np.uint8 and loc.shape == p.shape
        ms = np.zeros(p.shape, np.uint8) if want_ms else None
        cp = _cparams(p)
        rc = self._L.or_integrate_depth(C.byref(cp), _ptr(_i32(o)), _ptr(_f64(T_wc).reshape(16)),
                                        _ptr(depth), W, H, dt, float(scale), _ptr(loc),
                                        _ptr(ms) if ms is not None else None)
        if rc != 0:
            raise MemoryError("oracle could not allocate its scratch grids")
        return ms

    def integrate_points(self, p, o, T_wc, xyz, loc, want_ms=False):
        xyz = np.ascontiguousarray(np.asarray(xyz, np.float32).reshape(-1, 3))
        assert loc.flags.c_contiguous and loc.dtype == np.uint8 and loc.shape == p.shape
        ms = np.zeros(p.shape, np.uint8) if want_ms else None
        cp = _cparams(p)
        rc = self._L.or_integrate_points(C.byref(cp), _ptr(_i32(o)),
                                         _ptr(_f64(T_wc).reshape(16)), _ptr(xyz),
                                         xyz.shape[0], _ptr(loc),
                                         _ptr(ms) if ms is not None else None)
        if rc != 0:
            raise MemoryError("oracle could not allocate its scratch grids")
        return ms


class OracleGrid:
    """A local grid driven through the paper's per-measurement sequence:
    set-up (Sec. IV-A), integrate (Sec. IV-B..D) and shift (Sec. IV-E)."""

    def __init__(self, params, robot_pos_w, oracle=None):
        self.orc = oracle or default()
        self.p = params
        self.o = self.orc.origin(params, robot_pos_w)
        self.loc = np.zeros(params.shape, np.uint8)

    def integrate_depth(self, T_wc, depth, scale=1.0, want_ms=False):
        return self.orc.integrate_depth(self.p, self.o, T_wc, depth, scale, self.loc, want_ms)

    def integrate_points(self, T_wc, xyz, want_ms=False):
        return self.orc.integrate_points(self.p, self.o, T_wc, xyz, self.loc, want_ms)

    def shift(self, robot_pos_w):
        o2 = self.orc.origin(self.p, robot_pos_w)
        delta = o2 - self.o
        if np.any(delta != 0):
            self.loc = self.orc.shift(self.p.n, delta, self.loc)
            self.o = o2
        return delta


_DEFAULT = None


def default():
    """The oracle built from oracle/vg_oracle.c (built on first use)."""
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle()
    return _DEFAULT
