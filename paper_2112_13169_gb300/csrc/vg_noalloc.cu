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
#include "vg_host.h"
#include "vg_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace {

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

// The address at which the kernels on device `dev` reach p: p itself for
// device (or managed) memory of that device, the mapped device address for
// page-locked host memory when host_ok, else NULL (memory of another device,
// pageable host memory, or a pointer CUDA does not know).  Allocates nothing.
const void *reachable(const void *p, int dev, bool host_ok) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // not a CUDA-known pointer: clear the error
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return at.device == dev ? p : nullptr;
    if (at.type == cudaMemoryTypeHost && host_ok) return at.devicePointer;
    return nullptr;
}

}  // namespace

extern "C" VG_API int vg_integrate_depth_noalloc(const vg_params *params, const int32_t origin[3],
                                                 uint8_t *loc, const void *depth, int32_t width,
                                                 int32_t height, int32_t dtype, float depth_scale,
                                                 const double T_wc[16], void *stream) {
    if (!vg::host::shape_ok(params) || !origin || !loc || !depth || !T_wc) return VG_EINVAL;
    if (!vg::host::depth_frame_ok(width, height, dtype, depth_scale)) return VG_EINVAL;
    if (reinterpret_cast<uintptr_t>(loc) % 16 != 0) return VG_EINVAL;

    // plane geometry, as for a grid made by vg_create
    const vg::PlaneGeom g = vg::host::geom_of(params);
    if (g.words > kPlaneWords) return VG_ESCRATCH;

    // T^v_c from T^w_c and the caller's origin (Sec. IV-B), as vg_integrate_depth does
    vg::Pose32 T;
    if (!vg::host::pose_vc(T_wc, origin, params->vox_size, T)) return VG_EINVAL;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return vg::host::status_of(e);
    // the kernels run on the current device: loc must be its memory, and
    // depth its memory or page-locked host memory it reads in place
    uint8_t *dloc = static_cast<uint8_t *>(const_cast<void *>(reachable(loc, dev, false)));
    const void *ddepth = reachable(depth, dev, true);
    if (!dloc || !ddepth) return VG_EINVAL;
    e = setup_device(dev);
    if (e != cudaSuccess) return vg::host::status_of(e);
    uint32_t *scratch = g_scratch_dev[dev];
    cudaStream_t s = (cudaStream_t)stream;

    vg::FrameArgs a = vg::host::frame_args(params, g, T);
    vg::host::set_depth_frame(a, params, ddepth, width, height, dtype, depth_scale);
    a.pl.occ_raw = scratch;
    a.pl.occ_inf = scratch + g.words;
    a.pl.fr = scratch + 2 * g.words;
    a.pl.tr = scratch + 3 * g.words;
    a.loc = dloc;
    a.stats = nullptr;

    // the planes must start empty; the array holds whatever the last call left
    e = cudaMemsetAsync(scratch, 0, (size_t)(4 * g.words) * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = vg::launch_voxelize_depth(a, dtype, s);
    if (e == cudaSuccess && a.r > 0) e = vg::launch_inflate(a, s);
    if (e == cudaSuccess && a.r == 0) a.pl.occ_inf = a.pl.occ_raw;
    if (e == cudaSuccess)
        e = vg::launch_raytrace(a, vg::auto_lanes_per_ray(a.vd, a.hw, a.hh), s);
    if (e == cudaSuccess) e = vg::launch_merge(a, s);
    return vg::host::status_of(e);
}
