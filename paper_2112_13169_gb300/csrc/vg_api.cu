// vg_api.cu -- host side of the C ABI declared in include/vg.h.
//
// Per-frame host work is argument checking and the set-up arithmetic the
// paper assigns to the CPU (Sec. IV-B: T^v_c = T^v_w T^w_c is composed on the
// host and passed to the kernels), plus the pinhole intrinsics and the ray
// bundle size, all in double and rounded once to float / integer (the
// helpers of vg_host.h).  Everything else runs in the kernels K1..K5,
// enqueued on the caller's stream without host sync.
#include "vg.h"
#include "vg_host.h"
#include "vg_internal.cuh"

#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

using vg::FrameArgs;
using vg::PlaneGeom;

struct vg_grid {
    vg_params p;
    PlaneGeom g;
    int32_t origin[3];
    int32_t vd, hw, hh;
    int lanes_per_ray;
    vg::Sched sched;      // tile and launch shapes of K2..K4 (vg_tune, vg_autotune)
    int device;
    uint8_t *base;        // the one device allocation
    uint8_t *loc;         // ring-addressed by ring (vg::Ring)
    uint8_t *loc_alt;     // staging for reads into memory the device cannot store to
    // A re-centre by d (o' = o + d) moves the ring by d at once; the voxels
    // it brings in still hold stale bytes until the next merge sets them to
    // unknown (a read treats them as unknown meanwhile): pend = d while that
    // is pending.  origin already holds o'.
    int32_t ring[3];
    bool pend_on;
    int32_t pend[3];
    vg::Planes pl;
    uint32_t *loc_occ;    // VG_FLAG_LIT_LOC_OCCUPANCY: the plane its rays test
    unsigned long long *stats;
    void *staging;        // device copy of host inputs
    size_t staging_bytes;
    uint64_t frames;
    int64_t launches[VG_NKERNELS];
    // profiling: event pairs recorded around launches
    bool prof_on;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    size_t prof_used;
};

struct vg_batch {
    int32_t capacity;
    int device;
    int ctas_per_sm;    // 0: occupancy limit
    int lanes;          // 0: each grid's own
    int inflate_tz;     // inflate tile height in slices: 8 or 4
    int merge_words;    // plane words per merge unit with a re-centre: 512 or 256
    int spread;         // spread each frame's rays over proportionally more phase-3 units
    int64_t bar_ns;     // grid barrier time limit
    uint32_t bar_extra; // 1: the barrier waits for one CTA too many (tests its time limit)
    uint8_t *dev;       // BatchCtl followed by capacity BatchItems
    uint8_t *host;      // pinned copy
    size_t bytes;       // bytes of the table to copy (set by prepare)
    cudaEvent_t copied; // the table copy of the last enqueue
    cudaEvent_t done;   // the kernel of the last enqueue
    bool enqueued;
    bool prepared;
    uint64_t launches;
};

namespace {

using vg::host::bundle_of;
using vg::host::geom_of;
using vg::host::origin_of;
using vg::host::status_of;

bool finite3(const double v[3]) {
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

// A robot position whose origin index fits int32 with room to spare.
bool position_ok(const vg_params *p, const double pos[3]) {
    if (!finite3(pos)) return false;
    for (int k = 0; k < 3; ++k)
        if (std::fabs(pos[k] / (double)p->vox_size) >= 1073741824.0) return false;
    return true;
}

constexpr uint32_t kLitFlags =
    VG_FLAG_LIT_INFLATE_AFTER_TRACE | VG_FLAG_LIT_SKIP_START_VOXEL | VG_FLAG_LIT_LOC_OCCUPANCY;

bool params_ok(const vg_params *p) {
    if (!vg::host::shape_ok(p)) return false;
    if (p->flags & ~(VG_FLAG_STATS | kLitFlags)) return false;
    if ((p->flags & VG_FLAG_LIT_INFLATE_AFTER_TRACE) && (p->flags & VG_FLAG_LIT_LOC_OCCUPANCY)) return false;
    return true;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    size_t loc, loc_alt, occ_raw, occ_inf, fr, tr, loc_occ, stats, total;
};

Layout layout_of(const PlaneGeom &g, uint32_t flags) {
    Layout L;
    size_t off = 0;
    // 16 bytes of slack after each loc buffer: K5's vector path may read up
    // to 4 bytes past the last voxel (and discards them)
    const size_t locb = align256((size_t)g.nvox + 16), planeb = align256((size_t)g.words * 4);
    L.loc = off; off += locb;
    L.loc_alt = off; off += locb;
    L.occ_raw = off; off += planeb;
    L.occ_inf = off; off += planeb;
    L.fr = off; off += planeb;
    L.tr = off; off += planeb;
    L.loc_occ = off;   // only for the literal loc_grid reading
    if (flags & VG_FLAG_LIT_LOC_OCCUPANCY) off += planeb;
    L.stats = off; off += 256;
    L.total = off;
    return L;
}

// delta = o2 - o1, with an axis whose offset is the grid's size or more
// (nothing survives the shift) set to the size, so that index sums in the
// kernels stay small.
void shift_delta(const vg_params *p, const int32_t o1[3], const int32_t o2[3], int32_t d[3]) {
    for (int k = 0; k < 3; ++k) {
        const int64_t v = (int64_t)o2[k] - o1[k];
        const int64_t n = p->grid_size[k];
        d[k] = (int32_t)(v >= n ? n : (v <= -n ? -n : v));
    }
}

// Composes T^v_c for the grid's current origin (vg::host::pose_vc).
bool pose_of(const vg_grid *G, const double T_wc[16], vg::Pose32 &T) {
    return vg::host::pose_vc(T_wc, G->origin, G->p.vox_size, T);
}

// Keeps the caller's current device and switches to the grid's for the call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

std::once_flag g_configured[64];
cudaError_t g_config_err[64];

cudaError_t configure_device(int dev) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(g_configured[dev], [dev] {
        cudaError_t e = vg::configure_inflate();
        if (e == cudaSuccess) e = vg::configure_raytrace(dev);
        if (e == cudaSuccess) e = vg::configure_batch(dev);
        g_config_err[dev] = e;
    });
    return g_config_err[dev];
}

// The address at which the device reads or writes host memory directly:
// page-locked allocations (cudaMallocHost / cudaHostAlloc / registered),
// which the GPU reaches in place over the host link.  NULL for other
// memory, which must be copied through the DMA engines instead.
void *mapped_host(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // not a CUDA-known pointer: clear the error
        return nullptr;
    }
    return (at.type == cudaMemoryTypeHost) ? at.devicePointer : nullptr;
}

int stage_input(vg_grid *G, const void *src, size_t bytes, cudaStream_t s, const void **dev_ptr) {
    // page-locked input is read in place by K1 (no staging copy)
    if (const void *m = mapped_host(src)) {
        *dev_ptr = m;
        return VG_OK;
    }
    if (bytes > G->staging_bytes) {
        // grow-only staging buffer; the old one may still be read by queued work
        if (G->staging) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return status_of(e);
            cudaFree(G->staging);
            G->staging = nullptr;
            G->staging_bytes = 0;
        }
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VG_ENOMEM : VG_ECUDA;
        G->staging = p;
        G->staging_bytes = bytes;
    }
    cudaError_t e = cudaMemcpyAsync(G->staging, src, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return status_of(e);
    *dev_ptr = G->staging;
    return VG_OK;
}

FrameArgs frame_args(vg_grid *G, const vg::Pose32 &T) {
    FrameArgs a = vg::host::frame_args(&G->p, G->g, T);
    a.pl = G->pl;
    a.loc = G->loc;
    a.stats = (G->p.flags & VG_FLAG_STATS) ? G->stats : nullptr;
    a.rt_next = reinterpret_cast<uint32_t *>(G->stats + 31);   // the last 8 of the 256 stats bytes
    a.lit = ((G->p.flags & VG_FLAG_LIT_SKIP_START_VOXEL) ? vg::kLitSkipStart : 0) |
            ((G->p.flags & VG_FLAG_LIT_LOC_OCCUPANCY) ? vg::kLitRaysLast : 0);
    return a;
}

// FrameArgs of a depth frame: the pinhole intrinsics from the field of view.
FrameArgs depth_frame_args(vg_grid *G, const vg::Pose32 &T, const void *depth, int32_t width, int32_t height,
                           int32_t dtype, float depth_scale) {
    FrameArgs a = frame_args(G, T);
    vg::host::set_depth_frame(a, &G->p, depth, width, height, dtype, depth_scale);
    return a;
}

constexpr size_t kProfPairs = 65536;

// Runs one kernel launcher, counting it and, when profiling, bracketing it
// with events on its stream.
template <typename F>
cudaError_t launch(vg_grid *G, int kind, cudaStream_t s, F &&fn) {
    ++G->launches[kind];
    if (!G->prof_on || G->prof_used >= kProfPairs) return fn();
    const size_t i = G->prof_used++;
    cudaError_t e = cudaEventRecord(G->prof_ev[2 * i], s);
    if (e != cudaSuccess) return e;
    e = fn();
    if (e != cudaSuccess) return e;
    G->prof_kind[i] = kind;
    return cudaEventRecord(G->prof_ev[2 * i + 1], s);
}

// The grid's ring, with the voxels a pending re-centre by d brought in:
// along each axis, x in [n - d, n) for d > 0, [0, -d) for d < 0, every x
// for |d| >= n.
vg::Ring ring_of(const vg_grid *G) {
    vg::Ring R;
    const int32_t n[3] = {G->g.nx, G->g.ny, G->g.nz};
    for (int k = 0; k < 3; ++k) {
        R.r[k] = G->ring[k];
        const int64_t d = G->pend_on ? G->pend[k] : 0;
        int64_t lo = 0, hi = 0;
        if (d > 0) lo = std::max<int64_t>(0, n[k] - d), hi = n[k];
        if (d < 0) lo = 0, hi = std::min<int64_t>(n[k], -d);
        R.elo[k] = (int32_t)lo;
        R.ehi[k] = (int32_t)hi;
    }
    return R;
}

// The ring moved by d: ((r + d) mod n) per axis.
void move_ring(vg_grid *G, const int32_t d[3]) {
    const int64_t n[3] = {G->g.nx, G->g.ny, G->g.nz};
    for (int k = 0; k < 3; ++k) G->ring[k] = (int32_t)((((int64_t)G->ring[k] + d[k]) % n[k] + n[k]) % n[k]);
}

// Applies a pending re-centre on its own: K4 over the (empty, between
// frames) planes sets the voxels it brought in to unknown.
cudaError_t apply_pending(vg_grid *G, cudaStream_t s) {
    if (!G->pend_on) return cudaSuccess;
    FrameArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = G->g;
    a.pl = G->pl;
    a.loc = G->loc;
    a.ring = ring_of(G);
    cudaError_t e = launch(G, VG_K_SHIFT, s, [&] { return vg::launch_merge(a, s, G->sched); });
    if (e != cudaSuccess) return e;
    G->pend_on = false;
    return cudaSuccess;
}

// K2..K4 after K1 has filled occ_raw.

cudaError_t finish_frame(vg_grid *G, FrameArgs &a, cudaStream_t s) {
    cudaError_t e;
    if (a.r > 0) {
        e = launch(G, VG_K_INFLATE, s, [&] { return vg::launch_inflate(a, s, G->sched); });
        if (e != cudaSuccess) return e;
    } else {
        a.pl.occ_inf = a.pl.occ_raw;   // no inflation: the raw plane is the inflated one
    }
    // the plane the rays test: the inflated one (Alg. 1's order), or a
    // literal reading's
    a.occ_test = a.pl.occ_inf;
    if (G->p.flags & VG_FLAG_LIT_INFLATE_AFTER_TRACE) a.occ_test = a.pl.occ_raw;
    if (G->p.flags & VG_FLAG_LIT_LOC_OCCUPANCY) {
        const vg::Ring R = ring_of(G);
        e = launch(G, VG_K_LOC_OCCUPANCY, s,
                   [&] { return vg::launch_loc_occupancy(G->g, G->loc, R, G->loc_occ, s); });
        if (e != cudaSuccess) return e;
        a.occ_test = G->loc_occ;
    }
    const int lpr = G->lanes_per_ray ? G->lanes_per_ray : vg::auto_lanes_per_ray(G->vd, G->hw, G->hh);
    e = launch(G, VG_K_RAYTRACE, s, [&] { return vg::launch_raytrace(a, lpr, s, G->sched); });
    if (e != cudaSuccess) return e;
    // the measurement is in the grid's current frame: the merge writes it
    // through the ring, and sets what a pending re-centre brought in (and
    // the measurement does not mark) to unknown
    a.ring = ring_of(G);
    e = launch(G, VG_K_MERGE, s, [&] { return vg::launch_merge(a, s, G->sched); });
    if (e != cudaSuccess) return e;
    G->pend_on = false;
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char *vg_strerror(int status) {
    switch (status) {
    case VG_OK: return "ok";
    case VG_EINVAL: return "invalid argument";
    case VG_ENOMEM: return "out of memory";
    case VG_ECUDA: return "CUDA error";
    case VG_ETIMEOUT: return "device wait timed out";
    case VG_EBUSY: return "busy";
    case VG_ESCRATCH: return "grid too large for the fixed scratch array";
    default: return "unknown status";
    }
}

int64_t vg_grid_bytes(const vg_params *params) {
    if (!params_ok(params)) return 0;
    return (int64_t)layout_of(geom_of(params), params->flags).total;
}

int64_t vg_ray_bundle(const vg_params *params, int32_t out[3]) {
    if (!params_ok(params) || !out) return 0;
    bundle_of(params, out[0], out[1], out[2]);
    return (2 * (int64_t)out[1] + 1) * (2 * (int64_t)out[2] + 1);
}

int vg_create(const vg_params *params, const double robot_pos_w[3], void *stream, vg_grid **out) {
    if (!out) return VG_EINVAL;
    *out = nullptr;
    if (!params_ok(params) || !robot_pos_w || !position_ok(params, robot_pos_w)) return VG_EINVAL;
    vg_grid *G = new (std::nothrow) vg_grid();
    if (!G) return VG_ENOMEM;
    G->p = *params;
    G->g = geom_of(params);
    origin_of(params, robot_pos_w, G->origin);
    bundle_of(params, G->vd, G->hw, G->hh);
    G->lanes_per_ray = 0;   // automatic
    cudaError_t e = cudaGetDevice(&G->device);
    if (e == cudaSuccess) e = configure_device(G->device);
    const Layout L = layout_of(G->g, params->flags);
    if (e == cudaSuccess) e = cudaMalloc((void **)&G->base, L.total);
    if (e != cudaSuccess) {
        delete G;
        return status_of(e);
    }
    G->loc = G->base + L.loc;
    G->loc_alt = G->base + L.loc_alt;
    G->pl.occ_raw = reinterpret_cast<uint32_t *>(G->base + L.occ_raw);
    G->pl.occ_inf = reinterpret_cast<uint32_t *>(G->base + L.occ_inf);
    G->pl.fr = reinterpret_cast<uint32_t *>(G->base + L.fr);
    G->pl.tr = reinterpret_cast<uint32_t *>(G->base + L.tr);
    G->loc_occ = (params->flags & VG_FLAG_LIT_LOC_OCCUPANCY) ? reinterpret_cast<uint32_t *>(G->base + L.loc_occ)
                                                              : nullptr;
    G->stats = reinterpret_cast<unsigned long long *>(G->base + L.stats);
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(G->base, 0, L.total, s);   // VG_UNK == 0, planes empty
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(G->base);
        delete G;
        return status_of(e);
    }
    *out = G;
    return VG_OK;
}

void vg_destroy(vg_grid *G) {
    if (!G) return;
    DeviceGuard dg(G->device);
    cudaDeviceSynchronize();
    for (cudaEvent_t ev : G->prof_ev) cudaEventDestroy(ev);
    cudaFree(G->staging);
    cudaFree(G->base);
    delete G;
}

int vg_profile_enable(vg_grid *G, int32_t enable) {
    if (!G) return VG_EINVAL;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    if (enable && G->prof_ev.empty()) {
        try {
            G->prof_ev.resize(2 * kProfPairs, nullptr);
            G->prof_kind.resize(kProfPairs, 0);
        } catch (...) {
            G->prof_ev.clear();
            return VG_ENOMEM;
        }
        for (auto &ev : G->prof_ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return status_of(e);
        }
    }
    G->prof_on = enable != 0;
    return VG_OK;
}

int vg_profile_read(vg_grid *G, double ms[VG_NKERNELS], int64_t timed[VG_NKERNELS],
                    int64_t launches_total[VG_NKERNELS], int32_t reset) {
    if (!G) return VG_EINVAL;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    double acc[VG_NKERNELS] = {};
    int64_t cnt[VG_NKERNELS] = {};
    if (G->prof_used) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return status_of(e);
        for (size_t i = 0; i < G->prof_used; ++i) {
            float t = 0.0f;
            e = cudaEventElapsedTime(&t, G->prof_ev[2 * i], G->prof_ev[2 * i + 1]);
            if (e != cudaSuccess) return status_of(e);
            acc[G->prof_kind[i]] += t;
            cnt[G->prof_kind[i]] += 1;
        }
    }
    for (int k = 0; k < VG_NKERNELS; ++k) {
        if (ms) ms[k] = acc[k];
        if (timed) timed[k] = cnt[k];
        if (launches_total) launches_total[k] = G->launches[k];
    }
    if (reset) G->prof_used = 0;
    return VG_OK;
}

int vg_tune(vg_grid *G, int32_t knob, int32_t value) {
    if (!G) return VG_EINVAL;
    if (knob == VG_TUNE_RT_LANES) {
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16 && value != 32)
            return VG_EINVAL;
        G->lanes_per_ray = value;
        return VG_OK;
    }
    if (knob == VG_TUNE_INFLATE_TILE) {
        if (value < VG_TILE_AUTO || value > VG_TILE_8x8x8) return VG_EINVAL;
        G->sched.inflate_tile = value;
        return VG_OK;
    }
    if (knob == VG_TUNE_RT_CTAS_PER_SM) {
        if (value < 0 || value > 64) return VG_EINVAL;
        G->sched.rt_ctas = value;
        return VG_OK;
    }
    if (knob == VG_TUNE_MERGE_WORDS) {
        if (value != 256 && value != 512) return VG_EINVAL;
        G->sched.merge_words = value;
        return VG_OK;
    }
    if (knob == VG_TUNE_INFLATE_TMA) {
        if (value != 0 && value != 1) return VG_EINVAL;
        G->sched.inflate_tma = value;
        return VG_OK;
    }
    if (knob == VG_TUNE_EARLY_INFLATE) {
        if (value != 0 && value != 1) return VG_EINVAL;
        G->sched.early_inflate = value;
        return VG_OK;
    }
    return VG_EINVAL;
}

int vg_autotune(vg_grid *G, const void *depth, int32_t mem, int32_t width, int32_t height, int32_t dtype,
                float depth_scale, const double T_wc[16], int32_t reps, void *stream, int32_t best[6]) {
    if (!G || reps < 1 || reps > 1000) return VG_EINVAL;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // a re-centre pending at the start is applied first, so that every timed
    // frame starts from the same grid
    cudaError_t e = apply_pending(G, s);
    if (e != cudaSuccess) return status_of(e);
    // every timed frame starts with a cold L2: a write of twice its size
    int l2 = 0;
    e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, G->device);
    if (e != cudaSuccess) return status_of(e);
    const size_t flush_bytes = 2 * (size_t)std::max(l2, 1 << 20);
    void *flush = nullptr;
    e = cudaMalloc(&flush, flush_bytes);
    if (e != cudaSuccess) return status_of(e);
    std::vector<cudaEvent_t> ev(4 * (size_t)reps, nullptr);
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    int rc = status_of(e);
    // One measurement under a schedule, events e0/e1 around it (none when
    // NULL), after the L2 flush.
    auto frame = [&](const vg::Sched &sc, int lp, cudaEvent_t e0, cudaEvent_t e1) -> int {
        G->sched = sc;
        G->lanes_per_ray = lp;
        if (cudaMemsetAsync(flush, 0, flush_bytes, s) != cudaSuccess) return VG_ECUDA;
        if (e0 && cudaEventRecord(e0, s) != cudaSuccess) return VG_ECUDA;
        const int c = vg_integrate_depth(G, depth, mem, width, height, dtype, depth_scale, T_wc, stream);
        if (c != VG_OK) return c;
        if (e1 && cudaEventRecord(e1, s) != cudaSuccess) return VG_ECUDA;
        return VG_OK;
    };
    auto median = [&](size_t first) -> float {
        std::vector<float> ms((size_t)reps);
        for (int r = 0; r < reps; ++r)
            if (cudaEventElapsedTime(&ms[r], ev[first + 4 * r], ev[first + 4 * r + 1]) != cudaSuccess) return -1.0f;
        std::sort(ms.begin(), ms.end());
        return ms[(size_t)reps / 2];
    };
    // Whether candidate (sc, lp) is at least 2 % faster than the incumbent
    // (bs, bl): their frames alternate, the incumbent first in even pairs
    // and the candidate first in odd ones (a frame right after another
    // one's timed 4 % slower on `seq` even with identical schedules), so
    // that drifts and order hit both alike, and their median event times
    // are compared.
    auto better = [&](const vg::Sched &bs, int bl, const vg::Sched &sc, int lp, bool &win) -> int {
        for (int r = -1; r < reps; ++r) {   // r = -1: untimed warm-up of both
            const size_t k = 4 * (size_t)(r < 0 ? 0 : r);
            cudaEvent_t i0 = r < 0 ? nullptr : ev[k], i1 = r < 0 ? nullptr : ev[k + 1];
            cudaEvent_t c0 = r < 0 ? nullptr : ev[k + 2], c1 = r < 0 ? nullptr : ev[k + 3];
            int c;
            if (r & 1) {
                c = frame(sc, lp, c0, c1);
                if (c == VG_OK) c = frame(bs, bl, i0, i1);
            } else {
                c = frame(bs, bl, i0, i1);
                if (c == VG_OK) c = frame(sc, lp, c0, c1);
            }
            if (c != VG_OK) return c;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return VG_ECUDA;
        const float mi = median(0), mc = median(2);
        if (mi < 0.0f || mc < 0.0f) return VG_ECUDA;
        win = mc < 0.98f * mi;
        return VG_OK;
    };
    // the schedule as it stands is the incumbent; coordinate descent then
    // takes each knob in turn over its candidates, the others held at the
    // best values so far, and a candidate replaces the incumbent only if it
    // is at least 2 % faster in an alternating comparison
    const int tiles[4] = {VG_TILE_4x8x4, VG_TILE_4x8x8, VG_TILE_8x8x4, VG_TILE_8x8x8};
    const int lanes[3] = {8, 16, 32};
    const int ctas[5] = {1, 2, 3, 4, 5};
    const int words[2] = {256, 512};
    const int tma[2] = {1, 0};
    const int early[2] = {1, 0};
    vg::Sched bs = G->sched;
    int bl = G->lanes_per_ray ? G->lanes_per_ray : vg::auto_lanes_per_ray(G->vd, G->hw, G->hh);
    for (int pass = 0; pass < 6 && rc == VG_OK; ++pass) {
        const int n = pass == 0 ? 4 : (pass == 1 ? 3 : (pass == 2 ? 5 : 2));
        if ((pass == 0 || pass == 4) && G->p.vox_inf == 0) continue;   // no K2 to tune
        for (int i = 0; i < n && rc == VG_OK; ++i) {
            vg::Sched sc = bs;
            int lp = bl;
            if (pass == 0) sc.inflate_tile = tiles[i];
            if (pass == 1) lp = lanes[i];
            if (pass == 2) sc.rt_ctas = ctas[i];
            if (pass == 3) sc.merge_words = words[i];
            if (pass == 4) sc.inflate_tma = tma[i];
            if (pass == 5) sc.early_inflate = early[i];
            if (std::memcmp(&sc, &bs, sizeof(sc)) == 0 && lp == bl) continue;   // the incumbent itself
            bool win = false;
            rc = better(bs, bl, sc, lp, win);
            if (rc == VG_OK && win) {
                bs = sc;
                bl = lp;
            }
        }
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    cudaStreamSynchronize(s);
    cudaFree(flush);
    G->sched = bs;
    G->lanes_per_ray = bl;
    if (best) {
        best[0] = bs.inflate_tile;
        best[1] = bl;
        best[2] = bs.rt_ctas;
        best[3] = bs.merge_words;
        best[4] = bs.inflate_tma;
        best[5] = bs.early_inflate;
    }
    return rc;
}

int vg_integrate_depth(vg_grid *G, const void *depth, int32_t mem, int32_t width, int32_t height,
                       int32_t dtype, float depth_scale, const double T_wc[16], void *stream) {
    if (!G || !depth || width < 1 || height < 1) return VG_EINVAL;
    if ((int64_t)width * height >= (int64_t(1) << 31)) return VG_EINVAL;
    if (dtype != VG_DEPTH_F32 && dtype != VG_DEPTH_U16) return VG_EINVAL;
    if (mem != VG_MEM_DEVICE && mem != VG_MEM_HOST) return VG_EINVAL;
    if (dtype == VG_DEPTH_U16 && !(std::isfinite(depth_scale) && depth_scale > 0.0f)) return VG_EINVAL;
    vg::Pose32 T;
    if (!pose_of(G, T_wc, T)) return VG_EINVAL;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const void *dptr = depth;
    if (mem == VG_MEM_HOST) {
        const size_t bytes = (size_t)width * height * (dtype == VG_DEPTH_F32 ? 4 : 2);
        int rc = stage_input(G, depth, bytes, s, &dptr);
        if (rc != VG_OK) return rc;
    }
    FrameArgs a = depth_frame_args(G, T, dptr, width, height, dtype, depth_scale);
    cudaError_t e = launch(G, VG_K_VOXELIZE, s, [&] { return vg::launch_voxelize_depth(a, dtype, s, G->sched); });
    if (e == cudaSuccess) e = finish_frame(G, a, s);
    if (e != cudaSuccess) return status_of(e);
    ++G->frames;
    return VG_OK;
}

int vg_integrate_points(vg_grid *G, const float *xyz, int32_t mem, int64_t n, const double T_wc[16],
                        void *stream) {
    if (!G || n < 0 || (n > 0 && !xyz) || n >= (int64_t(1) << 31)) return VG_EINVAL;
    if (mem != VG_MEM_DEVICE && mem != VG_MEM_HOST) return VG_EINVAL;
    vg::Pose32 T;
    if (!pose_of(G, T_wc, T)) return VG_EINVAL;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const void *dptr = xyz;
    if (mem == VG_MEM_HOST && n > 0) {
        int rc = stage_input(G, xyz, (size_t)n * 12, s, &dptr);
        if (rc != VG_OK) return rc;
    }
    FrameArgs a = frame_args(G, T);
    a.xyz = static_cast<const float *>(dptr);
    a.npts = n;
    cudaError_t e = launch(G, VG_K_VOXELIZE, s, [&] { return vg::launch_voxelize_points(a, s, G->sched); });
    if (e == cudaSuccess) e = finish_frame(G, a, s);
    if (e != cudaSuccess) return status_of(e);
    ++G->frames;
    return VG_OK;
}

int vg_shift(vg_grid *G, const double robot_pos_w[3], void *stream) {
    if (!G || !robot_pos_w || !position_ok(&G->p, robot_pos_w)) return VG_EINVAL;
    int32_t o2[3], delta[3];
    origin_of(&G->p, robot_pos_w, o2);
    shift_delta(&G->p, G->origin, o2, delta);
    if (delta[0] == 0 && delta[1] == 0 && delta[2] == 0) return VG_OK;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    // two re-centres do not compose into one (a voxel shifted out and back
    // is unknown), so an earlier one is applied first
    cudaError_t e = apply_pending(G, (cudaStream_t)stream);
    if (e != cudaSuccess) return status_of(e);
    move_ring(G, delta);
    std::memcpy(G->pend, delta, sizeof(delta));
    G->pend_on = true;
    std::memcpy(G->origin, o2, sizeof(o2));
    return VG_OK;
}

int vg_read(vg_grid *G, uint8_t *dst, int32_t dst_mem, int64_t dst_bytes, int32_t origin[3],
            void *stream) {
    if (!G || !dst || dst_bytes < G->g.nvox) return VG_EINVAL;
    if (dst_mem != VG_MEM_DEVICE && dst_mem != VG_MEM_HOST) return VG_EINVAL;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    const cudaMemcpyKind kind = dst_mem == VG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (G->pend_on || G->ring[0] || G->ring[1] || G->ring[2]) {
        // the grid in its own frame, out of the ring (voxels a pending
        // re-centre brought in read as unknown; the grid is left as it is):
        // K5 writes it straight into dst where the device can store there
        // (device memory or page-locked host memory, 16-byte aligned), else
        // into loc_alt and then copies
        const vg::Ring R = ring_of(G);
        uint8_t *ddst = dst_mem == VG_MEM_DEVICE ? dst : static_cast<uint8_t *>(mapped_host(dst));
        if (ddst && reinterpret_cast<uintptr_t>(ddst) % 16 == 0) {
            e = launch(G, VG_K_SHIFT, s, [&] { return vg::launch_shift(G->g, R, G->loc, ddst, s); });
        } else {
            e = launch(G, VG_K_SHIFT, s, [&] { return vg::launch_shift(G->g, R, G->loc, G->loc_alt, s); });
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, G->loc_alt, (size_t)G->g.nvox, kind, s);
        }
    } else {
        e = cudaMemcpyAsync(dst, G->loc, (size_t)G->g.nvox, kind, s);
    }
    if (e != cudaSuccess) return status_of(e);
    if (origin) std::memcpy(origin, G->origin, sizeof(G->origin));
    return VG_OK;
}

int vg_write(vg_grid *G, const uint8_t *src, int32_t src_mem, int64_t src_bytes, const int32_t origin[3],
             void *stream) {
    if (!G || !src || !origin || src_bytes != G->g.nvox) return VG_EINVAL;
    if (src_mem != VG_MEM_DEVICE && src_mem != VG_MEM_HOST) return VG_EINVAL;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    const cudaMemcpyKind kind = src_mem == VG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaMemcpyAsync(G->loc, src, (size_t)G->g.nvox, kind, (cudaStream_t)stream);
    // the measurement planes start empty again (after a failed batch step
    // they may hold a partial measurement)
    if (e == cudaSuccess)
        e = cudaMemsetAsync(G->pl.occ_raw, 0, (size_t)G->g.words * 4, (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(G->pl.occ_inf, 0, (size_t)G->g.words * 4, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(G->pl.fr, 0, (size_t)G->g.words * 4, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(G->pl.tr, 0, (size_t)G->g.words * 4, (cudaStream_t)stream);
    if (e != cudaSuccess) return status_of(e);
    G->pend_on = false;   // replaced whole, in the grid's own frame
    G->ring[0] = G->ring[1] = G->ring[2] = 0;
    std::memcpy(G->origin, origin, sizeof(G->origin));
    return VG_OK;
}

int vg_get_origin(const vg_grid *G, int32_t origin[3]) {
    if (!G || !origin) return VG_EINVAL;
    std::memcpy(origin, G->origin, sizeof(G->origin));
    return VG_OK;
}

int vg_stats(vg_grid *G, vg_stats_t *out) {
    if (!G || !out) return VG_EINVAL;
    DeviceGuard dg(G->device);
    if (!dg.ok) return VG_ECUDA;
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, G->stats, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status_of(e);
    unsigned waits = 0;
    e = vg::wait_timeouts(&waits);
    if (e != cudaSuccess) return status_of(e);
    out->frames = G->frames;
    out->points_in_grid = h[1];
    out->ray_visits = h[2];
    out->wait_timeouts = waits;
    return VG_OK;
}

int vg_batch_create(int32_t capacity, vg_batch **out) {
    if (!out) return VG_EINVAL;
    *out = nullptr;
    if (capacity < 1 || capacity > 65536) return VG_EINVAL;
    vg_batch *B = new (std::nothrow) vg_batch();
    if (!B) return VG_ENOMEM;
    B->capacity = capacity;
    B->inflate_tz = 8;
    B->merge_words = vg::kBatchMergeWords;
    B->spread = 1;
    B->bar_ns = vg::kBarrierNs;
    B->bytes = sizeof(vg::BatchCtl) + (size_t)capacity * sizeof(vg::BatchItem);
    cudaError_t e = cudaGetDevice(&B->device);
    if (e == cudaSuccess) e = configure_device(B->device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&B->dev, B->bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&B->host, B->bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        vg_batch_destroy(B);
        return status_of(e);
    }
    std::memset(B->host, 0, B->bytes);
    *out = B;
    return VG_OK;
}

void vg_batch_destroy(vg_batch *B) {
    if (!B) return;
    DeviceGuard dg(B->device);
    cudaDeviceSynchronize();
    if (B->copied) cudaEventDestroy(B->copied);
    if (B->done) cudaEventDestroy(B->done);
    cudaFreeHost(B->host);
    cudaFree(B->dev);
    delete B;
}

int vg_batch_tune(vg_batch *B, int32_t knob, int32_t value) {
    if (!B) return VG_EINVAL;
    if (knob == VG_TUNE_BATCH_CTAS_PER_SM) {
        if (value < 0 || value > 64) return VG_EINVAL;
        B->ctas_per_sm = value;
        return VG_OK;
    }
    if (knob == VG_TUNE_BATCH_LANES) {
        if (value != 0 && value != 8 && value != 16 && value != 32) return VG_EINVAL;
        B->lanes = value;
        return VG_OK;
    }
    if (knob == VG_TUNE_BATCH_INFLATE_SLICES) {
        if (value != 0 && value != 4 && value != 8) return VG_EINVAL;
        B->inflate_tz = value ? value : 8;
        return VG_OK;
    }
    if (knob == VG_TUNE_BATCH_MERGE_WORDS) {
        if (value != 0 && value != 256 && value != 512) return VG_EINVAL;
        B->merge_words = value ? value : vg::kBatchMergeWords;
        return VG_OK;
    }
    if (knob == VG_TUNE_BATCH_SPREAD) {
        if (value < 0 || value > 2) return VG_EINVAL;
        B->spread = value;
        return VG_OK;
    }
    if (knob == VG_TUNE_BATCH_BARRIER_US) {
        if (value < 0 || value > 60000000) return VG_EINVAL;
        B->bar_ns = value ? (int64_t)value * 1000 : vg::kBarrierNs;
        return VG_OK;
    }
    if (knob == VG_TUNE_BATCH_BARRIER_EXTRA) {
        if (value != 0 && value != 1) return VG_EINVAL;
        B->bar_extra = (uint32_t)value;
        return VG_OK;
    }
    return VG_EINVAL;
}

namespace {

// CTAs of the batch's cooperative launch: the occupancy limit, or the
// ctas_per_sm knob when it is lower.  0 on error.
int batch_blocks(const vg_batch *B) {
    const int max_blocks = vg::batch_max_blocks(B->device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess) return 0;
    int blocks = max_blocks;
    if (B->ctas_per_sm > 0 && B->ctas_per_sm * sms < max_blocks) blocks = B->ctas_per_sm * sms;
    return blocks;
}

// The relative cost of one phase-3 unit of a frame (a group of 256 / lpr
// rays): a lane's ray-trace work is its set-up, worth about five visits,
// plus its share of a ray's in-grid visits.  The visits are estimated from
// 5 x 5 of the bundle's rays: a ray from the camera S along D visits about
// |D|_1 * t_end + 1 voxels, t_end the parameter (at most 1) where it leaves
// the grid.  Scaled by 16 and clamped to [1, 4096].
int64_t ray_unit_weight(const FrameArgs &a, int lpr) {
    const float S[3] = {a.T.t[0] / a.vs, a.T.t[1] / a.vs, a.T.t[2] / a.vs};
    const double n[3] = {(double)a.g.nx, (double)a.g.ny, (double)a.g.nz};
    double sum = 0.0;
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            const double ra = a.hw * (i - 2) / 2.0, rb = a.hh * (j - 2) / 2.0;
            double D[3], l1 = 0.0, t_end = 1.0;
            for (int k = 0; k < 3; ++k) {
                D[k] = a.T.R[3 * k] * ra + a.T.R[3 * k + 1] * rb + a.T.R[3 * k + 2] * (double)a.vd;
                l1 += std::fabs(D[k]);
                if (D[k] > 0.0) t_end = std::min(t_end, (n[k] - S[k]) / D[k]);
                if (D[k] < 0.0) t_end = std::min(t_end, -S[k] / D[k]);
            }
            sum += l1 * std::max(t_end, 0.0) + 1.0;
        }
    const double w = 16.0 * (5.0 + sum / 25.0 / lpr);
    return (int64_t)std::min(4096.0, std::max(1.0, std::round(w)));
}

}  // namespace

int vg_batch_prepare(vg_batch *B, const vg_frame *frames, int32_t n) {
    if (!B || !frames || n < 1 || n > B->capacity) return VG_EINVAL;
    // every frame's grid is distinct and usable, before any state changes
    std::vector<const vg_grid *> seen;
    seen.reserve((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        const vg_frame &f = frames[i];
        const vg_grid *G = f.grid;
        if (!G || !f.depth || f.width < 1 || f.height < 1) return VG_EINVAL;
        if ((int64_t)f.width * f.height >= (int64_t(1) << 31)) return VG_EINVAL;
        if (f.dtype != VG_DEPTH_F32 && f.dtype != VG_DEPTH_U16) return VG_EINVAL;
        if (f.dtype == VG_DEPTH_U16 && !(std::isfinite(f.depth_scale) && f.depth_scale > 0.0f)) return VG_EINVAL;
        if (G->device != B->device || G->p.vox_inf > 3 || (G->p.flags & kLitFlags)) return VG_EINVAL;
        if (f.recentre && !position_ok(&G->p, f.robot_pos_w)) return VG_EINVAL;
        vg::Pose32 T;
        if (!pose_of(G, f.T_wc, T)) return VG_EINVAL;
        seen.push_back(G);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return VG_EINVAL;

    DeviceGuard dg(B->device);
    if (!dg.ok) return VG_ECUDA;
    if (B->enqueued) {
        cudaError_t e = cudaEventSynchronize(B->copied);   // the table is free again
        if (e != cudaSuccess) return status_of(e);
    }
    vg::BatchCtl *ctl = reinterpret_cast<vg::BatchCtl *>(B->host);
    vg::BatchItem *items = reinterpret_cast<vg::BatchItem *>(B->host + sizeof(vg::BatchCtl));
    int64_t total[4] = {0, 0, 0, 0};
    for (int32_t i = 0; i < n; ++i) {
        const vg_frame &f = frames[i];
        vg_grid *G = f.grid;
        vg::Pose32 T;
        pose_of(G, f.T_wc, T);
        vg::BatchItem &it = items[i];
        std::memset(&it, 0, sizeof(it));
        it.a = depth_frame_args(G, T, f.depth, f.width, f.height, f.dtype, f.depth_scale);
        if (G->p.vox_inf == 0) it.a.pl.occ_inf = it.a.pl.occ_raw;
        it.a.occ_test = it.a.pl.occ_inf;
        it.dtype = f.dtype;
        it.vec = (reinterpret_cast<uintptr_t>(f.depth) % (f.dtype == VG_DEPTH_F32 ? 16 : 8)) == 0;
        int lpr = B->lanes ? B->lanes : (G->lanes_per_ray ? G->lanes_per_ray : vg::auto_lanes_per_ray(G->vd, G->hw, G->hh));
        it.lpr = lpr < 8 ? 8 : lpr;
        it.txw = G->g.wx % 8 == 0 ? 8 : 4;
        it.tz = B->inflate_tz;
        it.mwpu = B->merge_words;
        it.tiles[0] = (G->g.wx + it.txw - 1) / it.txw;
        it.tiles[1] = (G->g.ny + 7) / 8;
        it.tiles[2] = (G->g.nz + it.tz - 1) / it.tz;
        it.buffered = G->g.words < vg::kRunWords ? 1 : 0;
        const int64_t npix = (int64_t)f.width * f.height;
        const int64_t nrays = (2 * (int64_t)G->hw + 1) * (2 * (int64_t)G->hh + 1);
        int64_t units[4] = {
            ((npix + 3) / 4 + 255) / 256,
            G->p.vox_inf > 0 ? (int64_t)it.tiles[0] * it.tiles[1] * it.tiles[2] : 0,
            (nrays + (256 / it.lpr) - 1) / (256 / it.lpr),
            (G->g.words + it.mwpu - 1) / it.mwpu};
        // the merge writes through the grid's ring and sets what a pending
        // re-centre brought in to unknown
        it.a.ring = ring_of(G);
        G->pend_on = false;
        if (f.recentre) {
            // the ring moves now; what the re-centre brings in is left
            // pending, for the grid's next merge (or read)
            int32_t o2[3], d[3];
            origin_of(&G->p, f.robot_pos_w, o2);
            shift_delta(&G->p, G->origin, o2, d);
            if (d[0] || d[1] || d[2]) {
                move_ring(G, d);
                std::memcpy(G->pend, d, sizeof(d));
                G->pend_on = true;
                std::memcpy(G->origin, o2, sizeof(o2));
            }
        }
        for (int p = 0; p < 4; ++p) {
            it.off[p] = total[p];
            total[p] += units[p];
        }
        ++G->frames;
    }
    // Phase 3 hands each CTA a contiguous run of units.  Unless the units
    // fill whole rounds of the grid, some CTAs would take one more unit
    // than others, so each frame's rays are spread over proportionally more
    // (partly filled) units: G_i = ceil(groups_i * rounds * blocks / T)
    // (unless the spread is tuned off).
    if (B->spread == 1) {
        const int64_t T = total[2];
        const int64_t nb = batch_blocks(B);
        if (nb < 1) return VG_ECUDA;
        const int64_t slots = (T + nb - 1) / nb * nb;
        int64_t off = 0;
        for (int32_t i = 0; i < n; ++i) {
            const int64_t groups = (i + 1 < n ? items[i + 1].off[2] : T) - items[i].off[2];
            items[i].off[2] = off;
            off += (groups * slots + T - 1) / T;
        }
        total[2] = off;
    }
    // Phase 3's runs split the units' total weight evenly: with spread 2
    // each frame's units weigh its estimated ray cost, otherwise 1 each.
    int64_t wtotal = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int64_t units3 = (i + 1 < n ? items[i + 1].off[2] : total[2]) - items[i].off[2];
        items[i].w3 = B->spread == 2 ? ray_unit_weight(items[i].a, items[i].lpr) : 1;
        items[i].woff3 = wtotal;
        wtotal += units3 * items[i].w3;
    }
    std::memset(ctl, 0, sizeof(*ctl));
    ctl->n = n;
    ctl->wtotal3 = wtotal;
    ctl->bar_ns = B->bar_ns;
    ctl->bar_extra = B->bar_extra;
    for (int p = 0; p < 4; ++p) ctl->total[p] = total[p];
    B->bytes = sizeof(vg::BatchCtl) + (size_t)n * sizeof(vg::BatchItem);
    B->prepared = true;
    return VG_OK;
}

int vg_batch_enqueue(vg_batch *B, void *stream) {
    if (!B || !B->prepared) return VG_EINVAL;
    DeviceGuard dg(B->device);
    if (!dg.ok) return VG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = batch_blocks(B);
    if (blocks < 1) return VG_ECUDA;
    cudaError_t e;
    // under stream capture the events must become record nodes of the graph,
    // so that every replay records them
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return status_of(e);
    const unsigned rec = (cs == cudaStreamCaptureStatusActive) ? cudaEventRecordExternal : cudaEventRecordDefault;
    e = cudaMemcpyAsync(B->dev, B->host, B->bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(B->copied, s, rec);
    if (e == cudaSuccess)
        e = vg::launch_batch(reinterpret_cast<const vg::BatchItem *>(B->dev + sizeof(vg::BatchCtl)),
                             reinterpret_cast<vg::BatchCtl *>(B->dev), blocks, s);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(B->done, s, rec);
    if (e != cudaSuccess) return status_of(e);
    B->enqueued = true;
    ++B->launches;
    return VG_OK;
}

int vg_batch_step(vg_batch *B, const vg_frame *frames, int32_t n, void *stream) {
    int rc = vg_batch_prepare(B, frames, n);
    return rc == VG_OK ? vg_batch_enqueue(B, stream) : rc;
}

int vg_batch_status(vg_batch *B) {
    if (!B) return VG_EINVAL;
    if (!B->enqueued) return VG_OK;
    DeviceGuard dg(B->device);
    if (!dg.ok) return VG_ECUDA;
    cudaError_t e = cudaEventSynchronize(B->done);
    unsigned err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&err, B->dev + offsetof(vg::BatchCtl, error), sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status_of(e);
    return err ? VG_ETIMEOUT : VG_OK;
}

int vg_batch_autotune(vg_batch *B, const vg_frame *frames, int32_t n, int32_t reps, void *stream,
                      int32_t best[5]) {
    if (!B || !frames || n < 1 || n > B->capacity || reps < 1) return VG_EINVAL;
    std::vector<vg_frame> fr(frames, frames + n);
    for (auto &f : fr) f.recentre = 0;
    DeviceGuard dg(B->device);
    if (!dg.ok) return VG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int max_blocks = vg::batch_max_blocks(B->device);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device);
    const int max_per_sm = std::max(1, max_blocks / std::max(1, sms));
    cudaEvent_t t0, t1;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) return status_of(e);
    // the knobs: CTAs per SM, lanes per ray, inflate tile slices, merge
    // words per unit, phase-3 spread; coordinate descent, one knob at a time
    // over its candidates with the others at the best values so far
    int cur[5] = {B->ctas_per_sm ? B->ctas_per_sm : max_per_sm, B->lanes, B->inflate_tz, B->merge_words, B->spread};
    std::vector<int> cand[5];
    for (int c = 1; c <= max_per_sm; ++c) cand[0].push_back(c);
    cand[1] = {0, 8, 16, 32};
    cand[2] = {8, 4};
    cand[3] = {512, 256};
    cand[4] = {2, 1, 0};
    auto apply = [&](const int v[5]) {
        B->ctas_per_sm = v[0];
        B->lanes = v[1];
        B->inflate_tz = v[2];
        B->merge_words = v[3];
        B->spread = v[4];
    };
    float best_ms = 1e30f;
    int rc = VG_OK;
    for (int k = 0; k < 5 && rc == VG_OK; ++k) {
        int pick[5];
        std::memcpy(pick, cur, sizeof(pick));
        for (size_t i = 0; i < cand[k].size() && rc == VG_OK; ++i) {
            int v[5];
            std::memcpy(v, cur, sizeof(v));
            v[k] = cand[k][i];
            apply(v);
            rc = vg_batch_step(B, fr.data(), n, stream);   // warm-up
            if (rc != VG_OK) break;
            e = cudaEventRecord(t0, s);
            for (int r = 0; r < reps && rc == VG_OK && e == cudaSuccess; ++r) rc = vg_batch_step(B, fr.data(), n, stream);
            if (e == cudaSuccess) e = cudaEventRecord(t1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e != cudaSuccess) rc = status_of(e);
            if (rc == VG_OK) rc = vg_batch_status(B);
            if (rc == VG_OK && ms < best_ms) {
                best_ms = ms;
                std::memcpy(pick, v, sizeof(pick));
            }
        }
        std::memcpy(cur, pick, sizeof(cur));
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    apply(cur);
    if (best)
        for (int k = 0; k < 5; ++k) best[k] = cur[k];
    return rc;
}

}  // extern "C"
