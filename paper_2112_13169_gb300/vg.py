"""Python binding of libvg.so, the C-ABI voxel-grid library (include/vg.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Functions carry the C names; `Grid` is a small owning wrapper.
Buffers may be torch tensors (CUDA tensors are passed as device pointers,
CPU tensors as host pointers) or numpy arrays (host).  `stream` may be a
torch.cuda.Stream, a raw cudaStream_t integer or None (torch's current
stream).  There is no CPU fallback: if the library cannot be loaded every
call raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvg.so")

VG_OK, VG_EINVAL, VG_ENOMEM, VG_ECUDA, VG_ETIMEOUT, VG_EBUSY, VG_ESCRATCH = range(7)
VG_UNK, VG_FREE, VG_OCC, VG_TRACED = range(4)
VG_DEPTH_F32, VG_DEPTH_U16 = 0, 1
VG_MEM_DEVICE, VG_MEM_HOST = 0, 1
VG_FLAG_STATS = 1
VG_FLAG_LIT_INFLATE_AFTER_TRACE = 2
VG_FLAG_LIT_SKIP_START_VOXEL = 4
VG_FLAG_LIT_LOC_OCCUPANCY = 8

# every symbol include/vg.h declares
EXPORTS = ("vg_create", "vg_destroy", "vg_integrate_depth", "vg_integrate_points", "vg_shift",
           "vg_read", "vg_write", "vg_get_origin", "vg_grid_bytes", "vg_ray_bundle", "vg_stats",
           "vg_profile_enable", "vg_profile_read", "vg_tune", "vg_strerror", "vg_integrate_depth_noalloc",
           "vg_batch_create", "vg_batch_destroy", "vg_batch_prepare", "vg_batch_enqueue", "vg_batch_step",
           "vg_batch_status", "vg_batch_tune", "vg_batch_autotune", "vg_server_create", "vg_server_destroy",
           "vg_server_add_camera", "vg_server_remove_camera", "vg_server_submit", "vg_server_wait",
           "vg_server_read", "vg_server_stats", "vg_server_ticket_times", "vg_autotune")
VG_TUNE_BATCH_CTAS_PER_SM, VG_TUNE_BATCH_LANES, VG_TUNE_BATCH_BARRIER_US, VG_TUNE_BATCH_BARRIER_EXTRA = 100, 101, 102, 103
VG_TUNE_BATCH_INFLATE_SLICES, VG_TUNE_BATCH_MERGE_WORDS, VG_TUNE_BATCH_SPREAD = 104, 105, 106
KERNELS = ("voxelize", "inflate", "raytrace", "merge", "shift", "loc_occupancy")
(VG_TUNE_RT_LANES, VG_TUNE_INFLATE_TILE, VG_TUNE_RT_CTAS_PER_SM, VG_TUNE_MERGE_WORDS, VG_TUNE_INFLATE_TMA,
 VG_TUNE_EARLY_INFLATE) = range(6)
VG_TILE_AUTO, VG_TILE_4x8x4, VG_TILE_4x8x8, VG_TILE_8x8x4, VG_TILE_8x8x8 = range(5)
TILE_NAMES = {VG_TILE_AUTO: "auto", VG_TILE_4x8x4: "4x8x4", VG_TILE_4x8x8: "4x8x8", VG_TILE_8x8x4: "8x8x4",
              VG_TILE_8x8x8: "8x8x8"}


class vg_params(C.Structure):
    _fields_ = [("grid_size", C.c_int32 * 3), ("vox_size", C.c_float), ("fov_x_deg", C.c_float),
                ("fov_y_deg", C.c_float), ("depth", C.c_float), ("vox_inf", C.c_int32),
                ("flags", C.c_uint32)]


class vg_stats_t(C.Structure):
    _fields_ = [("frames", C.c_uint64), ("points_in_grid", C.c_uint64), ("ray_visits", C.c_uint64),
                ("wait_timeouts", C.c_uint64)]


class vg_frame(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("depth", C.c_void_p), ("width", C.c_int32), ("height", C.c_int32),
                ("dtype", C.c_int32), ("depth_scale", C.c_float), ("T_wc", C.c_double * 16),
                ("recentre", C.c_int32), ("pad", C.c_int32), ("robot_pos_w", C.c_double * 3)]


class vg_server_params(C.Structure):
    _fields_ = [("memory_budget", C.c_int64), ("max_batch", C.c_int32), ("max_width", C.c_int32),
                ("max_height", C.c_int32), ("queue_depth", C.c_int32), ("pending_frames", C.c_int32),
                ("plain_max", C.c_int32)]


class vg_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("batches", C.c_uint64), ("mean_batch", C.c_double), ("latency_p50_us", C.c_double),
                ("latency_p99_us", C.c_double), ("latency_max_us", C.c_double), ("bytes_in_use", C.c_int64),
                ("cameras", C.c_int32)]


class VGError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, strerror(status), status))


_LIB = None


def load(path=None):
    """Load libvg.so (built by paper_2112_13169_gb300.build); raise if absent."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libvg.so not found at %s: build it with paper_2112_13169_gb300.build.build()" % p)
    L = C.CDLL(p)
    vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    sig = {
        "vg_create": (C.c_int, [vp, vp, vp, C.POINTER(vp)]),
        "vg_destroy": (None, [vp]),
        "vg_integrate_depth": (C.c_int, [vp, vp, i32, i32, i32, i32, f32, vp, vp]),
        "vg_integrate_points": (C.c_int, [vp, vp, i32, i64, vp, vp]),
        "vg_shift": (C.c_int, [vp, vp, vp]),
        "vg_read": (C.c_int, [vp, vp, i32, i64, vp, vp]),
        "vg_write": (C.c_int, [vp, vp, i32, i64, vp, vp]),
        "vg_get_origin": (C.c_int, [vp, vp]),
        "vg_grid_bytes": (i64, [vp]),
        "vg_ray_bundle": (i64, [vp, vp]),
        "vg_stats": (C.c_int, [vp, vp]),
        "vg_profile_enable": (C.c_int, [vp, i32]),
        "vg_profile_read": (C.c_int, [vp, vp, vp, vp, i32]),
        "vg_tune": (C.c_int, [vp, i32, i32]),
        "vg_autotune": (C.c_int, [vp, vp, i32, i32, i32, i32, f32, vp, i32, vp, vp]),
        "vg_strerror": (C.c_char_p, [C.c_int]),
        "vg_integrate_depth_noalloc": (C.c_int, [vp, vp, vp, vp, i32, i32, i32, f32, vp, vp]),
        "vg_batch_create": (C.c_int, [i32, C.POINTER(vp)]),
        "vg_batch_destroy": (None, [vp]),
        "vg_batch_prepare": (C.c_int, [vp, vp, i32]),
        "vg_batch_enqueue": (C.c_int, [vp, vp]),
        "vg_batch_step": (C.c_int, [vp, vp, i32, vp]),
        "vg_batch_status": (C.c_int, [vp]),
        "vg_batch_tune": (C.c_int, [vp, i32, i32]),
        "vg_batch_autotune": (C.c_int, [vp, vp, i32, i32, vp, vp]),
        "vg_server_create": (C.c_int, [vp, C.POINTER(vp)]),
        "vg_server_destroy": (None, [vp]),
        "vg_server_add_camera": (C.c_int, [vp, vp, vp, vp]),
        "vg_server_remove_camera": (C.c_int, [vp, i32]),
        "vg_server_submit": (C.c_int, [vp, i32, vp, i32, i32, i32, f32, vp, i32, vp, vp]),
        "vg_server_wait": (C.c_int, [vp, C.c_uint64, i64]),
        "vg_server_read": (C.c_int, [vp, i32, vp, i32, i64, vp]),
        "vg_server_stats": (C.c_int, [vp, vp, i32]),
        "vg_server_ticket_times": (C.c_int, [vp, C.c_uint64, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = L
    return L


def strerror(status):
    try:
        return load().vg_strerror(int(status)).decode()
    except RuntimeError:
        return "status %d" % status


def _check(status, what):
    if status != VG_OK:
        raise VGError(status, what)


def make_params(n, vox_size, fov_x_deg, fov_y_deg, depth, vox_inf, flags=0):
    p = vg_params()
    for k in range(3):
        p.grid_size[k] = int(n[k])
    p.vox_size = float(vox_size)
    p.fov_x_deg = float(fov_x_deg)
    p.fov_y_deg = float(fov_y_deg)
    p.depth = float(depth)
    p.vox_inf = int(vox_inf)
    p.flags = int(flags)
    return p


# torch is optional (numpy buffers work without it); looked up once
_TORCH = None
_TORCH_DTYPES = None
_CUDA = None
_CURRENT_STREAM = None   # () -> torch's current cudaStream_t on the current device, as an int


def _torch():
    global _TORCH, _TORCH_DTYPES
    if _TORCH is None:
        try:
            import torch
        except ImportError:
            _TORCH = False
            return None
        _TORCH = torch
        _TORCH_DTYPES = {torch.float32: "float32", torch.uint16: "uint16", torch.uint8: "uint8",
                         torch.float64: "float64", torch.int32: "int32", torch.int16: "int16"}
    return _TORCH or None


def _current_stream_getter(t):
    """torch's current stream as an int.  torch.cuda.current_stream() builds a
    Stream object on every call (about 3 us on a Grace core); the raw getter
    that torch's own generated code uses returns the handle directly, and the
    public call is the fallback where it is missing."""
    raw = getattr(t._C, "_cuda_getCurrentRawStream", None)
    if raw is None:
        return lambda: t.cuda.current_stream().cuda_stream
    device = t.cuda.current_device
    return lambda: raw(device())


def _stream(stream):
    """The cudaStream_t (an integer) to pass for `stream`."""
    global _CUDA, _CURRENT_STREAM
    if stream is None:
        if _CUDA is None:
            t = _torch()
            _CUDA = bool(t is not None and t.cuda.is_available())
            if _CUDA:
                _CURRENT_STREAM = _current_stream_getter(t)
        return _CURRENT_STREAM() if _CUDA else 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _buffer(x):
    """(pointer, mem kind, nbytes, dtype string) of a tensor or array."""
    t = _torch()
    if t is not None and isinstance(x, t.Tensor):
        if not x.is_contiguous():
            raise ValueError("buffer must be contiguous")
        dt = _TORCH_DTYPES.get(x.dtype) or str(x.dtype).replace("torch.", "")
        return x.data_ptr(), (VG_MEM_DEVICE if x.is_cuda else VG_MEM_HOST), x.numel() * x.element_size(), dt
    a = x
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
        raise ValueError("buffer must be a contiguous numpy array or torch tensor")
    return a.ctypes.data, VG_MEM_HOST, a.nbytes, a.dtype.name


def _f64(v, n):
    """(array, pointer) of v as n contiguous float64 values; the array must
    outlive the call that uses the pointer."""
    if type(v) is np.ndarray and v.dtype is _F64 and v.size == n and v.flags.c_contiguous:
        a = v
    else:
        a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(n))
    return a, a.__array_interface__["data"][0]


_F64 = np.dtype(np.float64)
_DEPTH_DTYPES = {"float32": VG_DEPTH_F32, "uint16": VG_DEPTH_U16}


def _depth_dtype(dt):
    d = _DEPTH_DTYPES.get(dt)
    if d is None:
        raise ValueError("depth must be float32 or uint16, got " + dt)
    return d


def vg_grid_bytes(params):
    return int(load().vg_grid_bytes(C.byref(params)))


def vg_ray_bundle(params):
    out = (C.c_int32 * 3)()
    n = load().vg_ray_bundle(C.byref(params), out)
    return (out[0], out[1], out[2]), int(n)


def vg_create(params, robot_pos_w, stream=None):
    h = C.c_void_p()
    pos, pp = _f64(robot_pos_w, 3)
    _check(load().vg_create(C.byref(params), pp, _stream(stream), C.byref(h)), "vg_create")
    return h


def vg_destroy(h):
    if h:
        load().vg_destroy(h)


def vg_integrate_depth(h, depth, T_wc, depth_scale=1.0, stream=None):
    ptr, mem, nbytes, dt = _buffer(depth)
    dtype = _depth_dtype(dt)
    H, W = depth.shape
    T, tp = _f64(T_wc, 16)
    _check((_LIB or load()).vg_integrate_depth(h, ptr, mem, W, H, dtype, depth_scale, tp, _stream(stream)),
           "vg_integrate_depth")


def vg_integrate_depth_noalloc(params, origin, loc, depth, T_wc, depth_scale=1.0, stream=None):
    """One measurement into a caller-owned loc grid (a CUDA uint8 tensor of
    Nx*Ny*Nz bytes, updated in place) without any device allocation: for
    callers that cannot allocate device memory.  The library keeps the
    measurement planes in a fixed 16 MiB array shared by all calls, so calls
    whose device work overlaps race; see include/vg.h."""
    lptr, lmem, lbytes, ldt = _buffer(loc)
    dptr, dmem, dbytes, dt = _buffer(depth)
    if lmem != VG_MEM_DEVICE:
        raise ValueError("loc must be a device buffer")
    if dmem == VG_MEM_DEVICE and depth.device != loc.device:
        raise ValueError("loc and depth must be on the same device")
    n = params.grid_size
    if ldt != "uint8" or lbytes != n[0] * n[1] * n[2]:
        raise ValueError("loc must hold Nx*Ny*Nz uint8 voxels")
    dtype = _depth_dtype(dt)
    H, W = depth.shape
    o = np.ascontiguousarray(np.asarray(origin, np.int32).reshape(3))
    T, tp = _f64(T_wc, 16)
    t = _torch()
    # the library runs on the current device: make it loc's
    with t.cuda.device(loc.device):
        _check(load().vg_integrate_depth_noalloc(C.byref(params), o.ctypes.data, lptr, dptr, int(W), int(H),
                                                 dtype, float(depth_scale), tp, _stream(stream)),
               "vg_integrate_depth_noalloc")


def vg_integrate_points(h, xyz, T_wc, stream=None):
    ptr, mem, nbytes, dt = _buffer(xyz)
    if dt != "float32":
        raise ValueError("points must be float32 xyz triples")
    T, tp = _f64(T_wc, 16)
    _check(load().vg_integrate_points(h, ptr, mem, nbytes // 12, tp, _stream(stream)), "vg_integrate_points")


def vg_shift(h, robot_pos_w, stream=None):
    pos, pp = _f64(robot_pos_w, 3)
    _check((_LIB or load()).vg_shift(h, pp, _stream(stream)), "vg_shift")


def vg_read(h, dst, stream=None):
    """Enqueue a copy of loc_grid into dst; returns the origin (int32[3])."""
    ptr, mem, nbytes, _ = _buffer(dst)
    o = np.zeros(3, np.int32)
    _check((_LIB or load()).vg_read(h, ptr, mem, nbytes, o.ctypes.data, _stream(stream)), "vg_read")
    return o


def vg_write(h, src, origin, stream=None):
    ptr, mem, nbytes, _ = _buffer(src)
    o = np.ascontiguousarray(np.asarray(origin, np.int32).reshape(3))
    _check(load().vg_write(h, ptr, mem, nbytes, o.ctypes.data, _stream(stream)), "vg_write")


def vg_get_origin(h):
    o = np.zeros(3, np.int32)
    _check(load().vg_get_origin(h, o.ctypes.data), "vg_get_origin")
    return o


def vg_stats(h):
    s = vg_stats_t()
    _check(load().vg_stats(h, C.byref(s)), "vg_stats")
    return {"frames": s.frames, "points_in_grid": s.points_in_grid, "ray_visits": s.ray_visits,
            "wait_timeouts": s.wait_timeouts}


def vg_profile_enable(h, enable=True):
    _check(load().vg_profile_enable(h, 1 if enable else 0), "vg_profile_enable")


def vg_profile_read(h, reset=True):
    """{kernel: (summed ms, timed launches, total launches)}; synchronises."""
    nk = len(KERNELS)   # VG_NKERNELS
    ms = (C.c_double * nk)()
    timed = (C.c_int64 * nk)()
    total = (C.c_int64 * nk)()
    _check(load().vg_profile_read(h, ms, timed, total, 1 if reset else 0), "vg_profile_read")
    return {k: (ms[i], timed[i], total[i]) for i, k in enumerate(KERNELS)}


def vg_tune(h, knob, value):
    _check(load().vg_tune(h, int(knob), int(value)), "vg_tune")


class Grid:
    """One local grid on the current CUDA device (owns its vg_grid)."""

    def __init__(self, n, vox_size, fov_x_deg, fov_y_deg, depth, vox_inf, robot_pos_w=(0, 0, 0),
                 flags=0, stream=None):
        self.params = make_params(n, vox_size, fov_x_deg, fov_y_deg, depth, vox_inf, flags)
        self.n = tuple(int(v) for v in n)
        self.shape = (self.n[2], self.n[1], self.n[0])
        self.nvox = self.n[0] * self.n[1] * self.n[2]
        self.h = vg_create(self.params, robot_pos_w, stream)

    def integrate_depth(self, depth, T_wc, depth_scale=1.0, stream=None):
        vg_integrate_depth(self.h, depth, T_wc, depth_scale, stream)

    def integrate_points(self, xyz, T_wc, stream=None):
        vg_integrate_points(self.h, xyz, T_wc, stream)

    def shift(self, robot_pos_w, stream=None):
        vg_shift(self.h, robot_pos_w, stream)

    def read(self, dst, stream=None):
        return vg_read(self.h, dst, stream)

    def write(self, src, origin, stream=None):
        vg_write(self.h, src, origin, stream)

    @property
    def origin(self):
        return vg_get_origin(self.h)

    def stats(self):
        return vg_stats(self.h)

    def profile(self, enable=True):
        vg_profile_enable(self.h, enable)

    def profile_read(self, reset=True):
        return vg_profile_read(self.h, reset)

    def tune(self, lanes_per_ray):
        vg_tune(self.h, VG_TUNE_RT_LANES, lanes_per_ray)

    def set(self, knob, value):
        vg_tune(self.h, knob, value)

    def autotune(self, depth, T_wc, depth_scale=1.0, reps=5, stream=None):
        """Times the schedule knobs on this frame and keeps the fastest;
        returns {"tile", "lanes", "ctas_per_sm", "merge_words", "inflate_tma", "early_inflate"}."""
        ptr, mem, nbytes, dt = _buffer(depth)
        dtype = _depth_dtype(dt)
        H, W = depth.shape
        T, tp = _f64(T_wc, 16)
        best = (C.c_int32 * 6)()
        _check(load().vg_autotune(self.h, ptr, mem, W, H, dtype, float(depth_scale), tp, int(reps), _stream(stream),
                                  best), "vg_autotune")
        return {"tile": TILE_NAMES[best[0]], "lanes": best[1], "ctas_per_sm": best[2], "merge_words": best[3],
                "inflate_tma": best[4], "early_inflate": best[5]}

    def close(self):
        if self.h:
            vg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_frames(frames):
    """ctypes array of vg_frame from (grid, depth, T_wc, recentre_pos_or_None[, depth_scale])
    tuples; grid is a Grid, depth a CUDA tensor."""
    arr = (vg_frame * len(frames))()
    for i, f in enumerate(frames):
        grid, depth, T_wc, pos = f[0], f[1], f[2], f[3]
        scale = f[4] if len(f) > 4 else 1.0
        ptr, mem, nbytes, dt = _buffer(depth)
        if mem != VG_MEM_DEVICE:
            raise ValueError("batched depth frames must be device buffers")
        if dt not in ("float32", "uint16"):
            raise ValueError("depth must be float32 or uint16, got " + dt)
        H, W = depth.shape
        fr = arr[i]
        fr.grid = grid.h.value if isinstance(grid.h, C.c_void_p) else grid.h
        fr.depth = ptr
        fr.width, fr.height = int(W), int(H)
        fr.dtype = VG_DEPTH_F32 if dt == "float32" else VG_DEPTH_U16
        fr.depth_scale = float(scale)
        T, tp = _f64(T_wc, 16)
        C.memmove(fr.T_wc, tp, 128)
        if pos is not None:
            fr.recentre = 1
            P, pp = _f64(pos, 3)
            C.memmove(fr.robot_pos_w, pp, 24)
    return arr


class Batch:
    """Many grids' measurements in one persistent fused launch (vg_batch_*)."""

    def __init__(self, capacity):
        self.h = C.c_void_p()
        _check(load().vg_batch_create(int(capacity), C.byref(self.h)), "vg_batch_create")
        self.capacity = int(capacity)

    def prepare(self, frames):
        arr = make_frames(frames)
        _check(load().vg_batch_prepare(self.h, arr, len(frames)), "vg_batch_prepare")

    def enqueue(self, stream=None):
        _check(load().vg_batch_enqueue(self.h, _stream(stream)), "vg_batch_enqueue")

    def step(self, frames, stream=None):
        arr = make_frames(frames)
        _check(load().vg_batch_step(self.h, arr, len(frames), _stream(stream)), "vg_batch_step")

    def status(self):
        return load().vg_batch_status(self.h)

    def tune(self, knob, value):
        _check(load().vg_batch_tune(self.h, int(knob), int(value)), "vg_batch_tune")

    def autotune(self, frames, reps=3, stream=None):
        """The batch autotuner; returns {"ctas_per_sm", "lanes", "inflate_slices",
        "merge_words", "spread"} (lanes 0: each grid's own)."""
        arr = make_frames(frames)
        best = (C.c_int32 * 5)()
        _check(load().vg_batch_autotune(self.h, arr, len(frames), int(reps), _stream(stream), best),
               "vg_batch_autotune")
        return dict(zip(("ctas_per_sm", "lanes", "inflate_slices", "merge_words", "spread"), (int(v) for v in best)))

    def close(self):
        if self.h:
            load().vg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over many cameras (vg_server_*)."""

    def __init__(self, memory_budget, max_batch=64, max_width=1280, max_height=720, queue_depth=2,
                 pending_frames=None, plain_max=0):
        p = vg_server_params()
        p.plain_max = int(plain_max)
        p.memory_budget = int(memory_budget)
        p.max_batch = int(max_batch)
        p.max_width = int(max_width)
        p.max_height = int(max_height)
        p.queue_depth = int(queue_depth)
        p.pending_frames = int(pending_frames or 4 * max_batch)
        self.h = C.c_void_p()
        _check(load().vg_server_create(C.byref(p), C.byref(self.h)), "vg_server_create")

    def add_camera(self, n, vox_size, fov_x_deg, fov_y_deg, depth, vox_inf, robot_pos_w=(0, 0, 0)):
        params = make_params(n, vox_size, fov_x_deg, fov_y_deg, depth, vox_inf)
        cam = C.c_int32()
        pos, pp = _f64(robot_pos_w, 3)
        _check(load().vg_server_add_camera(self.h, C.byref(params), pp, C.byref(cam)), "vg_server_add_camera")
        return int(cam.value)

    def remove_camera(self, camera):
        _check(load().vg_server_remove_camera(self.h, int(camera)), "vg_server_remove_camera")

    def submit(self, camera, depth, T_wc, robot_pos_w=None, depth_scale=1.0):
        """Queue a host depth frame; returns its ticket, or None when the
        server's pool is full (VG_EBUSY)."""
        ptr, mem, nbytes, dt = _buffer(depth)
        if mem != VG_MEM_HOST:
            raise ValueError("served frames come from host memory")
        dtype = _depth_dtype(dt)
        H, W = depth.shape
        T, tp = _f64(T_wc, 16)
        pos, pp = _f64(robot_pos_w if robot_pos_w is not None else (0.0, 0.0, 0.0), 3)
        t = C.c_uint64()
        rc = load().vg_server_submit(self.h, int(camera), ptr, int(W), int(H), dtype, float(depth_scale), tp,
                                     1 if robot_pos_w is not None else 0, pp, C.byref(t))
        if rc == VG_EBUSY:
            return None
        _check(rc, "vg_server_submit")
        return int(t.value)

    def wait(self, ticket, timeout_us=-1):
        return load().vg_server_wait(self.h, C.c_uint64(ticket), int(timeout_us))

    def ticket_times(self, ticket):
        """(status, submitted, completed): monotonic-clock seconds, the same
        clock as time.monotonic() and time.perf_counter() on Linux;
        completed is None unless the status is VG_OK."""
        a, b = C.c_double(), C.c_double()
        rc = load().vg_server_ticket_times(self.h, C.c_uint64(ticket), C.byref(a), C.byref(b))
        if rc == VG_EINVAL:
            _check(rc, "vg_server_ticket_times")
        return rc, a.value, (b.value if rc == VG_OK else None)

    def read(self, camera, dst):
        ptr, mem, nbytes, _ = _buffer(dst)
        o = np.zeros(3, np.int32)
        _check(load().vg_server_read(self.h, int(camera), ptr, mem, nbytes, o.ctypes.data), "vg_server_read")
        return o

    def stats(self, reset=False):
        st = vg_server_stats_t()
        _check(load().vg_server_stats(self.h, C.byref(st), 1 if reset else 0), "vg_server_stats")
        return {f[0]: getattr(st, f[0]) for f in st._fields_}

    def close(self):
        if self.h:
            load().vg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
