// vg_noalloc.cu -- one measurement without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is
// off limits (a real-time control loop that must not block in the driver's
// allocator, firmware-style integrations that own all device memory up
// front, or hosts where the CUDA allocator is reserved by another runtime).
// vg_create allocates the grid and its measurement planes; this entry point
// instead takes the caller's loc grid and depth image as plain device
// pointers and keeps the four measurement bit planes in a fixed array
// compiled into the library.  It calls no cudaMalloc, cudaFree or any other
// allocating routine.
//
// The array is a file-scope __device__ object, so host code only holds a
// host-side stand-in for it under its name; its device address is looked up
// with cudaGetSymbolAddress, once per device, with that device current, the
// first time the entry point runs there.  Every call shares the array and
// finds the previous call's contents in it; the part a call uses is cleared
// on its stream before the kernels run.  Calls that overlap on the GPU (on
// different streams, or from several host threads) race on the array.
#include "vg.h"
#include "vg_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace {

constexpr double kPi = 3.14159265358979323846;

// Four planes of up to kPlaneWords 32-bit words each: 16 MiB in total, held
// by every GPU that loads the library until the process exits.
constexpr int64_t kPlaneWords = int64_t(1) << 20;
static __device__ __align__(256) uint32_t g_scratch[4 * kPlaneWords];

std::once_flag g_once[64];
uint32_t *g_scratch_dev[64];
cudaError_t g_setup_err[64];

// Looks up the array's device address and configures the kernels for the
// current device (first call on that device only).
cudaError_t setup_device(int dev) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(g_once[dev], [dev] {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e == cudaSuccess) e = vg::configure_inflate();
        if (e == cudaSuccess) e = vg::configure_raytrace(dev);
        g_scratch_dev[dev] = static_cast<uint32_t *>(p);
        g_setup_err[dev] = e;
    });
    return g_setup_err[dev];
}

double half_fov(float deg) { return (double)deg * kPi / 360.0; }

bool params_ok(const vg_params *p) {
    if (!p) return false;
    int64_t nv = 1;
    for (int k = 0; k < 3; ++k) {
        if (p->grid_size[k] < 1) return false;
        nv *= p->grid_size[k];
        if (nv >= (int64_t(1) << 31)) return false;
    }
    if (!(std::isfinite(p->vox_size) && p->vox_size > 0.0f)) return false;
    if (!(p->fov_x_deg > 0.0f && p->fov_x_deg < 180.0f)) return false;
    if (!(p->fov_y_deg > 0.0f && p->fov_y_deg < 180.0f)) return false;
    if (!(std::isfinite(p->depth) && p->depth > 0.0f)) return false;
    if (p->vox_inf < 0 || p->vox_inf > vg::kMaxInflate) return false;
    return (double)p->depth / (double)p->vox_size < 1.0e6;
}

}  // namespace

extern "C" VG_API int vg_integrate_depth_noalloc(const vg_params *params, const int32_t origin[3],
                                                 uint8_t *loc, const void *depth, int32_t width,
                                                 int32_t height, int32_t dtype, float depth_scale,
                                                 const double T_wc[16], void *stream) {
    if (!params_ok(params) || !origin || !loc || !depth || !T_wc) return VG_EINVAL;
    if (width < 1 || height < 1 || (int64_t)width * height >= (int64_t(1) << 31)) return VG_EINVAL;
    if (dtype != VG_DEPTH_F32 && dtype != VG_DEPTH_U16) return VG_EINVAL;
    if (dtype == VG_DEPTH_U16 && !(std::isfinite(depth_scale) && depth_scale > 0.0f)) return VG_EINVAL;
    if (reinterpret_cast<uintptr_t>(loc) % 16 != 0) return VG_EINVAL;

    // plane geometry, as for a grid made by vg_create
    vg::PlaneGeom g;
    g.nx = params->grid_size[0];
    g.ny = params->grid_size[1];
    g.nz = params->grid_size[2];
    const int32_t w = (g.nx + 31) / 32;
    g.wx = 4;
    while (g.wx < w) g.wx *= 2;
    g.words = (int64_t)g.wx * g.ny * g.nz;
    g.nvox = (int64_t)g.nx * g.ny * g.nz;
    if (g.words > kPlaneWords) return VG_ESCRATCH;

    // T^v_c from T^w_c and the caller's origin (Sec. IV-B), as vg_integrate_depth does
    vg::Pose32 T;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T_wc[i])) return VG_EINVAL;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            if (!(std::fabs(T_wc[r * 4 + c]) <= 1.5)) return VG_EINVAL;
            T.R[r * 3 + c] = (float)T_wc[r * 4 + c];
        }
        const double t = T_wc[r * 4 + 3] - (double)origin[r] * (double)params->vox_size;
        if (!(std::fabs(t / (double)params->vox_size) < 4194304.0)) return VG_EINVAL;
        T.t[r] = (float)t;
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = setup_device(dev);
    if (e != cudaSuccess) return VG_ECUDA;
    uint32_t *scratch = g_scratch_dev[dev];
    cudaStream_t s = (cudaStream_t)stream;

    vg::FrameArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.T = T;
    a.vs = params->vox_size;
    a.depth_max = params->depth;
    a.depth = depth;
    a.W = width;
    a.H = height;
    a.scale = (dtype == VG_DEPTH_U16) ? depth_scale : 1.0f;
    a.fx = (float)(((double)width / 2.0) / tan(half_fov(params->fov_x_deg)));
    a.fy = (float)(((double)height / 2.0) / tan(half_fov(params->fov_y_deg)));
    a.cx = (float)(((double)width - 1.0) / 2.0);
    a.cy = (float)(((double)height - 1.0) / 2.0);
    const long vd = lround((double)params->depth / (double)params->vox_size);
    a.vd = (int32_t)vd;
    a.hw = (int32_t)lround(tan(half_fov(params->fov_x_deg)) * (double)vd);
    a.hh = (int32_t)lround(tan(half_fov(params->fov_y_deg)) * (double)vd);
    a.r = params->vox_inf;
    a.pl.occ_raw = scratch;
    a.pl.occ_inf = scratch + g.words;
    a.pl.fr = scratch + 2 * g.words;
    a.pl.tr = scratch + 3 * g.words;
    a.loc = loc;
    a.stats = nullptr;

    // the planes must start empty; the array holds whatever the last call left
    e = cudaMemsetAsync(scratch, 0, (size_t)(4 * g.words) * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = vg::launch_voxelize_depth(a, dtype, s);
    if (e == cudaSuccess && a.r > 0) e = vg::launch_inflate(a, s);
    if (e == cudaSuccess && a.r == 0) a.pl.occ_inf = a.pl.occ_raw;
    if (e == cudaSuccess)
        e = vg::launch_raytrace(a, vg::auto_lanes_per_ray(a.vd, a.hw, a.hh), s);
    if (e == cudaSuccess) e = vg::launch_merge(a, s);
    return e == cudaSuccess ? VG_OK : VG_ECUDA;
}
