// K1 as its own launch: one thread per four pixels (or per point); the work
// itself is in vg_units.cuh.
#include "vg_units.cuh"

namespace vg {
namespace {

// K1 lets the frame's later kernels launch only once the work before the
// frame has completed: with `early` right after its own wait, so that K2's
// launch overlaps K1; without, when K1 completes, which leaves K1's SM
// slots to K3's CTAs, whose walk runs before they wait for K2.
template <int DT, bool VEC>
__global__ void __launch_bounds__(256) k_voxelize_depth(const FrameArgs a, const int early) {
    pdl_wait();   // the depth image and the planes belong to earlier work
    if (early) pdl_trigger();
    if (a.rt_next && blockIdx.x == 0 && threadIdx.x == 0) *a.rt_next = 0u;   // K3 of this frame counts from 0
    units::voxelize_depth_thread<DT, VEC>(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256) k_voxelize_points(const FrameArgs a, const int early) {
    pdl_wait();
    if (early) pdl_trigger();
    if (a.rt_next && blockIdx.x == 0 && threadIdx.x == 0) *a.rt_next = 0u;
    units::voxelize_points_thread(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

}  // namespace

cudaError_t launch_voxelize_depth(const FrameArgs &a, int32_t dtype, cudaStream_t s, const Sched &sc) {
    const int early = sc.early_inflate;
    const int64_t npix = (int64_t)a.W * a.H;
    const int64_t threads = (npix + 3) / 4;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    const uintptr_t base = reinterpret_cast<uintptr_t>(a.depth);
    if (dtype == 0) {
        if (base % 16 == 0) return launch_pdl(k_voxelize_depth<0, true>, blocks, 256, 0, s, a, early);
        return launch_pdl(k_voxelize_depth<0, false>, blocks, 256, 0, s, a, early);
    }
    if (base % 8 == 0) return launch_pdl(k_voxelize_depth<1, true>, blocks, 256, 0, s, a, early);
    return launch_pdl(k_voxelize_depth<1, false>, blocks, 256, 0, s, a, early);
}

cudaError_t launch_voxelize_points(const FrameArgs &a, cudaStream_t s, const Sched &sc) {
    const unsigned blocks = (unsigned)((a.npts + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(k_voxelize_points, blocks, 256, 0, s, a, (int)sc.early_inflate);
}

}  // namespace vg
