// K2 as its own launch: one CTA per 8-word x 8-row x 8-slice tile of the
// occupancy plane; the work itself is in vg_units.cuh.  For r = 1, 2, 3 the
// radius is a compile-time constant; other radii use a runtime radius.
#include "vg_units.cuh"

namespace vg {
namespace {

template <int R, int TXW, int TY, int TZ>
__global__ void __launch_bounds__(256) k_inflate(const PlaneGeom g, const uint32_t *__restrict__ raw,
                                                 uint32_t *__restrict__ out, const int r_rt) {
    extern __shared__ uint32_t sm[];
    pdl_trigger();
    pdl_wait();
    units::inflate_tile<R, TXW, TY, TZ, units::LoadRO>(g, raw, out, r_rt, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

template <int R, int TXW, int TY, int TZ>
cudaError_t run(const FrameArgs &a, cudaStream_t s) {
    dim3 grid((a.g.wx + TXW - 1) / TXW, (a.g.ny + TY - 1) / TY, (a.g.nz + TZ - 1) / TZ);
    const size_t bytes = sizeof(uint32_t) * units::inflate_smem_words<R, TXW, TY, TZ>(a.r);
    return launch_pdl(k_inflate<R, TXW, TY, TZ>, grid, 256, bytes, s, a.g, (const uint32_t *)a.pl.occ_raw,
                      a.pl.occ_inf, a.r);
}

template <int TXW>
cudaError_t run_r(const FrameArgs &a, cudaStream_t s) {
    switch (a.r) {
    case 1: return run<1, TXW, 8, 8>(a, s);
    case 2: return run<2, TXW, 8, 8>(a, s);
    case 3: return run<3, TXW, 8, 8>(a, s);
    default: return run<0, TXW, 8, 8>(a, s);
    }
}

}  // namespace

cudaError_t configure_inflate() {
    // the runtime-radius tile at vox_inf 15 needs about 104 KB of shared memory
    cudaError_t e = cudaFuncSetAttribute(k_inflate<0, 4, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         160 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_inflate<0, 8, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 160 * 1024);
    return e;
}

cudaError_t launch_inflate(const FrameArgs &a, cudaStream_t s) {
    // rows are a power of two of words, at least 4: 4-word tiles for narrow rows
    return a.g.wx % 8 == 0 ? run_r<8>(a, s) : run_r<4>(a, s);
}

}  // namespace vg
