"""Seeded synthetic workloads for the voxel-grid path.

Each workload is a scene of analytic primitives, a camera, a local-grid
specification and a sequence of frames (camera pose, robot position and a
depth image rendered by render.c).  The recipes follow the measurement
configurations of the project:

  paper  -- the paper's standard shapes (Sec. V): 320x240, fov 85x101 deg,
            depth 6.5 m, 100x100x20 grid at 0.15 m, vox_inf 2, room-like scene
  room   -- one 320x240 f32 frame, fov 87x58, depth 4 m, 6x6x3 m room with 20
            boxes and 10 spheres, 5% invalid pixels, identity pose;
            80x80x40 grid at 0.1 m, vox_inf 1
  seq    -- 640x480 f32 frames along a smooth trajectory through a 20x20x5 m
            scene of 200 boxes/cylinders, depth 5 m, 10% invalid pixels,
            depth noise sigma = 1% of the depth; 200x200x100 at 0.05 m, vox_inf 2
  hires  -- 1280x720 u16 millimetre frames, fov 90x60, depth 6 m, 1000
            primitives, 15% invalid; 400x400x120 at 0.05 m, vox_inf 2
  robot  -- one robot of the batched mix: resolution, voxel size, grid and
            vox_inf drawn from the stated sets (or given, to pin the mix's
            extremes)
  camera -- one camera of the served mix: 320x240 f32 or u16, 640x480 f32
            or u16, or 1280x720 u16 or f32, with a grid of 80x80x40 at
            0.1 m, 200x200x100 at 0.05 m or 400x400x120 at 0.05 m

Seeds are recipe_id * 1000 + robot index.  Nothing here computes any step
of the voxel-grid method; the same frames feed the CPU oracle and the CUDA
library.
"""
import concurrent.futures as cf
import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

BOX, SPHERE, CYL, ROOM = 0, 1, 2, 3

# kinds of simulated camera in the served mix ("camera"; spec picks one)
CAMERA_KINDS = 6

# Optical camera (x right, y down, z forward) on a FLU body: columns are the
# camera axes in body coordinates.
R_BODY_CAM = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])


class _Prim(C.Structure):
    _fields_ = [("type", C.c_int32), ("pad", C.c_int32), ("p", C.c_double * 6)]


def build(force=False):
    out_dir = os.path.join(HERE, "_build")
    lib = os.path.join(out_dir, "librender.so")
    src = os.path.join(HERE, "render.c")
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        os.makedirs(out_dir, exist_ok=True)
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, src, "-lm"],
                       check=True)
        os.replace(tmp, lib)
    return lib


def _lib():
    global _LIB
    if _LIB is None:
        L = C.CDLL(build())
        L.sy_render.restype = C.c_int
        L.sy_render.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.c_void_p]
        _LIB = L
    return _LIB


@dataclasses.dataclass
class Camera:
    W: int
    H: int
    fov_x: float
    fov_y: float
    dtype: str = "f32"        # "f32" (metres) or "u16" (raw units times scale)
    scale: float = 1.0


@dataclasses.dataclass
class GridSpec:
    n: tuple
    vox_size: float
    depth: float
    vox_inf: int


@dataclasses.dataclass
class Frame:
    T_wc: np.ndarray          # 4x4 camera optical -> world
    robot_pos: np.ndarray     # body position in the world (grid centre)
    depth: np.ndarray         # H x W float32 metres or uint16


@dataclasses.dataclass
class Workload:
    name: str
    cam: Camera
    grid: GridSpec
    frames: list
    prims: np.ndarray = None

    @property
    def nvox(self):
        return int(self.grid.n[0]) * int(self.grid.n[1]) * int(self.grid.n[2])


def body_pose(pos, yaw=0.0, pitch=0.0, roll=0.0):
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


def render(prims, T_wc, cam, max_t):
    """z-depth image (float32 metres, 0 = no return within max_t)."""
    fx = (cam.W / 2.0) / np.tan(np.radians(cam.fov_x) / 2.0)
    fy = (cam.H / 2.0) / np.tan(np.radians(cam.fov_y) / 2.0)
    out = np.zeros((cam.H, cam.W), np.float32)
    T = np.ascontiguousarray(T_wc, np.float64)
    rc = _lib().sy_render(prims.ctypes.data, len(prims), T.ctypes.data, cam.W, cam.H, fx, fy,
                          (cam.W - 1) / 2.0, (cam.H - 1) / 2.0, float(max_t), out.ctypes.data)
    if rc != 0:
        raise MemoryError("render scratch allocation failed")
    return out


def _prims_array(items):
    a = (_Prim * len(items))()
    for i, (t, p) in enumerate(items):
        a[i].type = t
        for k, v in enumerate(p):
            a[i].p[k] = float(v)
    return np.frombuffer(a, dtype=np.dtype([("type", "<i4"), ("pad", "<i4"), ("p", "<f8", (6,))])).copy()


def _random_prims(rng, count, lo, hi, kinds, keep_clear=None, clear_r=0.6):
    """count primitives inside [lo, hi]; none within clear_r of keep_clear points."""
    items = []
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    tries = 0
    while len(items) < count and tries < count * 50:
        tries += 1
        kind = kinds[rng.integers(len(kinds))]
        c = rng.uniform(lo, hi)
        if kind == BOX:
            half = rng.uniform(0.1, 0.8, 3)
            blo, bhi = c - half, c + half
            blo[2] = max(blo[2], lo[2])
            p = list(blo) + list(bhi)
        elif kind == SPHERE:
            r = rng.uniform(0.1, 0.6)
            blo, bhi = c - r, c + r
            p = list(c) + [r]
        else:
            r = rng.uniform(0.08, 0.5)
            z0 = lo[2]
            z1 = min(hi[2], z0 + rng.uniform(0.5, hi[2] - lo[2]))
            blo, bhi = np.array([c[0] - r, c[1] - r, z0]), np.array([c[0] + r, c[1] + r, z1])
            p = [c[0], c[1], z0, z1, r]
        if keep_clear is not None:
            q = np.clip(keep_clear, blo, bhi)
            if np.min(np.linalg.norm(q - keep_clear, axis=1)) < clear_r:
                continue
        items.append((kind, p))
    return items


def _trajectory(rng, nframes, centre, amp_xy, z0, dt=1.0 / 30.0):
    """Smooth seeded trajectory: a sum of random sinusoids per axis, yaw
    following the velocity, small pitch and roll."""
    t = np.arange(nframes) * dt
    pos = np.zeros((nframes, 3))
    vel = np.zeros((nframes, 3))
    for k in range(3):
        a = amp_xy if k < 2 else 0.15
        for _ in range(3):
            A = rng.uniform(0.3, 1.0) * a / 3.0
            w = rng.uniform(0.3, 0.9)
            ph = rng.uniform(0, 2 * np.pi)
            pos[:, k] += A * np.sin(w * t + ph)
            vel[:, k] += A * w * np.cos(w * t + ph)
    pos += np.array([centre[0], centre[1], z0])
    # guarantee motion of about 1.5 m/s along x on top of the wander
    pos[:, 0] += 1.5 * t
    vel[:, 0] += 1.5
    yaw = np.arctan2(vel[:, 1], vel[:, 0])
    pitch = 0.05 * np.sin(1.3 * t + rng.uniform(0, 6))
    roll = 0.04 * np.sin(1.7 * t + rng.uniform(0, 6))
    return pos, yaw, pitch, roll


def _postprocess(rng, depth, cam, invalid_frac, noise_rel):
    d = depth.astype(np.float64)
    hit = d > 0
    if noise_rel > 0:
        d = np.where(hit, d + rng.normal(0.0, 1.0, d.shape) * noise_rel * d, 0.0)
        d = np.where(d > 0, d, 0.0)
    if invalid_frac > 0:
        d[rng.random(d.shape) < invalid_frac] = 0.0
    if cam.dtype == "u16":
        return np.clip(np.round(d / cam.scale), 0, 65535).astype(np.uint16)
    return d.astype(np.float32)


def _render_frames(prims, cam, poses, max_t, rng, invalid_frac, noise_rel):
    workers = max(1, min(len(poses), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        raw = list(ex.map(lambda T: render(prims, T, cam, max_t), poses))
    return [_postprocess(rng, r, cam, invalid_frac, noise_rel) for r in raw]


def _sequence(name, seed, cam, grid, scene_lo, scene_hi, nprims, kinds, nframes, invalid,
              noise, room=True):
    rng = np.random.default_rng(seed)
    centre = (np.asarray(scene_lo) + np.asarray(scene_hi)) / 2.0
    span = min(scene_hi[0] - scene_lo[0], scene_hi[1] - scene_lo[1])
    pos, yaw, pitch, roll = _trajectory(rng, nframes, centre - np.array([0.35 * span, 0, 0]),
                                        0.15 * span, scene_lo[2] + 1.4)
    items = _random_prims(rng, nprims, scene_lo, scene_hi, kinds, keep_clear=pos)
    if room:
        items.append((ROOM, list(scene_lo) + list(scene_hi)))
    prims = _prims_array(items)
    poses = [body_pose(pos[i], yaw[i], pitch[i], roll[i]) for i in range(nframes)]
    depths = _render_frames(prims, cam, poses, 2.0 * grid.depth, rng, invalid, noise)
    frames = [Frame(poses[i], pos[i].copy(), depths[i]) for i in range(nframes)]
    return Workload(name, cam, grid, frames, prims)


def make(name, frames=None, seed=None, robot=0, spec=None):
    """Build a named workload.  frames overrides the frame count.  For
    "robot", spec = (W, H, vox_size, (nx, ny, nz), vox_inf) replaces the
    drawn resolution, voxel size, grid and radius (the scene and the
    trajectory are still drawn from the seed); for "camera", spec is the
    kind of camera, 0 .. CAMERA_KINDS - 1, instead of a drawn one."""
    if name == "room":
        rng = np.random.default_rng(1000 if seed is None else seed)
        cam = Camera(320, 240, 87.0, 58.0)
        grid = GridSpec((80, 80, 40), 0.1, 4.0, 1)
        lo, hi = np.array([-3.0, -3.0, -1.5]), np.array([3.0, 3.0, 1.5])
        keep = np.zeros((1, 3))
        items = _random_prims(rng, 20, lo, hi, [BOX], keep_clear=keep, clear_r=0.5)
        items += _random_prims(rng, 10, lo, hi, [SPHERE], keep_clear=keep, clear_r=0.5)
        items.append((ROOM, list(lo) + list(hi)))
        prims = _prims_array(items)
        nf = frames or 1
        poses = [body_pose([0.0, 0.0, 0.0])] * nf
        depths = _render_frames(prims, cam, poses, 2.0 * grid.depth, rng, 0.05, 0.0)
        return Workload(name, cam, grid, [Frame(poses[i], np.zeros(3), depths[i]) for i in range(nf)],
                        prims)
    if name == "paper":
        cam = Camera(320, 240, 85.0, 101.0)
        grid = GridSpec((100, 100, 20), 0.15, 6.5, 2)
        return _sequence(name, 0 if seed is None else seed, cam, grid, [0, 0, 0], [15, 15, 3], 40,
                         [BOX, CYL], frames or 100, 0.02, 0.0)
    if name == "seq":
        cam = Camera(640, 480, 87.0, 58.0)
        grid = GridSpec((200, 200, 100), 0.05, 5.0, 2)
        return _sequence(name, 2000 if seed is None else seed, cam, grid, [0, 0, 0], [20, 20, 5], 200,
                         [BOX, CYL], frames or 100, 0.10, 0.01)
    if name == "hires":
        cam = Camera(1280, 720, 90.0, 60.0, "u16", 0.001)
        grid = GridSpec((400, 400, 120), 0.05, 6.0, 2)
        return _sequence(name, 3000 if seed is None else seed, cam, grid, [0, 0, 0], [30, 30, 6], 1000,
                         [BOX, SPHERE, CYL], frames or 50, 0.15, 0.0)
    if name == "robot":
        s = 4000 + robot if seed is None else seed
        rng = np.random.default_rng(s)
        W, H = [(320, 240), (640, 480), (848, 480)][rng.integers(3)]
        vs = float([0.05, 0.1, 0.2][rng.integers(3)])
        n = (int(rng.integers(80, 257)), int(rng.integers(80, 257)), int(rng.integers(40, 97)))
        r = int(rng.integers(1, 4))
        if spec is not None:
            W, H, vs, n, r = spec
        cam = Camera(W, H, 87.0, 58.0)
        grid = GridSpec(tuple(n), float(vs), 5.0, int(r))
        return _sequence(name, s, cam, grid, [0, 0, 0], [16, 16, 4], 120, [BOX, SPHERE, CYL],
                         frames or 8, 0.05, 0.005)
    if name == "camera":
        # one simulated camera of the served mix: resolution and pixel type
        # from the stated set, the grid sized to the camera's range
        s = 5000 + robot if seed is None else seed
        rng = np.random.default_rng(s)
        kind = int(rng.integers(CAMERA_KINDS)) if spec is None else int(spec)
        if kind == 0:
            cam, grid = Camera(320, 240, 87.0, 58.0), GridSpec((80, 80, 40), 0.1, 4.0, 1)
        elif kind == 1:
            cam, grid = Camera(640, 480, 87.0, 58.0), GridSpec((200, 200, 100), 0.05, 5.0, 2)
        elif kind == 2:
            cam, grid = Camera(640, 480, 87.0, 58.0, "u16", 0.001), GridSpec((200, 200, 100), 0.05, 5.0, 2)
        elif kind == 3:
            cam, grid = Camera(1280, 720, 90.0, 60.0, "u16", 0.001), GridSpec((400, 400, 120), 0.05, 6.0, 2)
        elif kind == 4:
            cam, grid = Camera(320, 240, 87.0, 58.0, "u16", 0.001), GridSpec((80, 80, 40), 0.1, 4.0, 1)
        else:
            cam, grid = Camera(1280, 720, 90.0, 60.0), GridSpec((400, 400, 120), 0.05, 6.0, 2)
        return _sequence(name, s, cam, grid, [0, 0, 0], [20, 20, 5], 150, [BOX, SPHERE, CYL], frames or 4,
                         0.08, 0.005)
    raise ValueError("unknown workload " + name)
