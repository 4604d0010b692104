// K4 (merge), K4 with a pending re-centre, and K5 (shift) as their own
// launches: one thread per plane word, one CTA per 256 plane words, or one
// thread per 16 bytes of the new grid; the work itself is in vg_units.cuh.
#include "vg_units.cuh"

namespace vg {
namespace {

template <bool ALIGN8, bool RL>
__global__ void __launch_bounds__(256) k_merge(const PlaneGeom g, Planes pl, uint8_t *__restrict__ loc) {
    pdl_trigger();
    pdl_wait();
    units::merge_word<ALIGN8, units::LoadPlain, RL>(g, pl, loc, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <bool RL, int WPU>
__global__ void __launch_bounds__(256) k_merge_shift(const PlaneGeom g, Planes pl, const uint8_t *__restrict__ src,
                                                     uint8_t *__restrict__ dst, const int32_t dx, const int32_t dy,
                                                     const int32_t dz) {
    __shared__ __align__(16) uint8_t sm[units::merge_shift_smem(WPU)];
    pdl_trigger();
    // the source grid is staged before the wait for K3 (see merge_shift_unit)
    units::merge_shift_unit<WPU, units::LoadRO, units::LoadPlain, RL, true>(g, pl, src, dst, dx, dy, dz, blockIdx.x,
                                                                            sm);
}

// The literal loc_grid reading of Alg. 2: the occupied voxels of loc_grid,
// after a pending re-centre by (dx, dy, dz), as a bit plane (one thread per
// plane word, every word written).
__global__ void __launch_bounds__(256) k_loc_occupancy(const PlaneGeom g, const uint8_t *__restrict__ loc,
                                                       const int32_t dx, const int32_t dy, const int32_t dz,
                                                       uint32_t *__restrict__ out) {
    pdl_trigger();
    pdl_wait();
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= g.words) return;
    const int32_t x0 = (int32_t)(w % g.wx) * 32;
    const int64_t row = w / g.wx;
    const int32_t sy = (int32_t)(row % g.ny) + dy, sz = (int32_t)(row / g.ny) + dz;
    uint32_t bits = 0;
    if (x0 < g.nx && (unsigned)sy < (unsigned)g.ny && (unsigned)sz < (unsigned)g.nz) {
        const uint8_t *src = loc + ((int64_t)sz * g.ny + sy) * g.nx;
        const int nbits = min(32, g.nx - x0);
        for (int k = 0; k < nbits; ++k) {
            const int32_t sx = x0 + k + dx;
            if ((unsigned)sx < (unsigned)g.nx && __ldg(src + sx) == 2) bits |= 1u << k;   // VG_OCC
        }
    }
    out[w] = bits;
}

__global__ void __launch_bounds__(256) k_shift(const PlaneGeom g, const int32_t dx, const int32_t dy,
                                               const int32_t dz, const uint8_t *__restrict__ src,
                                               uint8_t *__restrict__ dst) {
    pdl_trigger();
    pdl_wait();
    units::shift_chunk<units::LoadRO>(g, dx, dy, dz, src, dst, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

}  // namespace

cudaError_t launch_merge(const FrameArgs &a, cudaStream_t s) {
    const unsigned blocks = (unsigned)((a.g.words + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    // 8-byte loc stores need 8-byte aligned rows and buffer
    const bool a8 = a.g.nx % 8 == 0 && reinterpret_cast<uintptr_t>(a.loc) % 8 == 0;
    if (a.lit & kLitRaysLast) {
        if (a8) return launch_pdl(k_merge<true, true>, blocks, 256, 0, s, a.g, a.pl, a.loc);
        return launch_pdl(k_merge<false, true>, blocks, 256, 0, s, a.g, a.pl, a.loc);
    }
    if (a8) return launch_pdl(k_merge<true, false>, blocks, 256, 0, s, a.g, a.pl, a.loc);
    return launch_pdl(k_merge<false, false>, blocks, 256, 0, s, a.g, a.pl, a.loc);
}

template <int WPU>
cudaError_t run_merge_shift(const FrameArgs &a, const int32_t delta[3], uint8_t *dst, cudaStream_t s) {
    const unsigned blocks = (unsigned)units::merge_shift_units<WPU>(a.g);
    if (blocks == 0) return cudaSuccess;
    if (a.lit & kLitRaysLast)
        return launch_pdl(k_merge_shift<true, WPU>, blocks, 256, 0, s, a.g, a.pl, (const uint8_t *)a.loc, dst,
                          delta[0], delta[1], delta[2]);
    return launch_pdl(k_merge_shift<false, WPU>, blocks, 256, 0, s, a.g, a.pl, (const uint8_t *)a.loc, dst,
                      delta[0], delta[1], delta[2]);
}

// One CTA per 256 plane words (8 KB of loc at most), or per 512
// (sc.merge_words): a larger unit keeps more loads in flight per CTA, and
// fewer CTAs share the device.
cudaError_t launch_merge_shift(const FrameArgs &a, const int32_t delta[3], uint8_t *dst, cudaStream_t s,
                               const Sched &sc) {
    if (sc.merge_words == 512) return run_merge_shift<512>(a, delta, dst, s);
    return run_merge_shift<256>(a, delta, dst, s);
}

cudaError_t launch_loc_occupancy(const PlaneGeom &g, const uint8_t *loc, const int32_t delta[3], uint32_t *out,
                                 cudaStream_t s) {
    const unsigned blocks = (unsigned)((g.words + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(k_loc_occupancy, blocks, 256, 0, s, g, loc, delta[0], delta[1], delta[2], out);
}

cudaError_t launch_shift(const PlaneGeom &g, const int32_t delta[3], const uint8_t *src, uint8_t *dst,
                         cudaStream_t s) {
    const int64_t threads = (g.nvox + 15) / 16;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(k_shift, blocks, 256, 0, s, g, delta[0], delta[1], delta[2], src, dst);
}

}  // namespace vg
