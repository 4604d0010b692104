// K4 (merge) and K5 (the grid read out in its own frame) as their own
// launches over the ring-addressed loc_grid: one thread per plane word (two
// with 512-word CTAs), or one thread per 16 bytes of the output; the work
// itself is in vg_units.cuh.
#include "vg_units.cuh"

namespace vg {
namespace {

template <bool RL, int WPU>
__global__ void __launch_bounds__(256) k_merge(const PlaneGeom g, Planes pl, uint8_t *__restrict__ loc,
                                               const Ring ring) {
    pdl_trigger();
    pdl_wait();
#pragma unroll
    for (int k = 0; k < WPU / 256; ++k)
        units::merge_word<units::LoadPlain, RL>(g, pl, loc, ring, (int64_t)blockIdx.x * WPU + k * 256 + threadIdx.x);
}

// The literal loc_grid reading of Alg. 2: the occupied voxels of loc_grid
// in the grid's own frame (voxels a re-centre brought in are unknown), as a
// bit plane (one thread per plane word, every word written).
__global__ void __launch_bounds__(256) k_loc_occupancy(const PlaneGeom g, const uint8_t *__restrict__ loc,
                                                       const Ring R, uint32_t *__restrict__ out) {
    pdl_trigger();
    pdl_wait();
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= g.words) return;
    const int32_t x0 = (int32_t)(w % g.wx) * 32;
    const int64_t row = w / g.wx;
    const int32_t y = (int32_t)(row % g.ny), z = (int32_t)(row / g.ny);
    uint32_t bits = 0;
    if (x0 < g.nx) {
        const int nbits = min(32, g.nx - x0);
        const uint32_t ent = units::entering_bits(R, x0, y, z, nbits);
        const uint8_t *rowp =
            loc + ((int64_t)units::ring_at(z, R.r[2], g.nz) * g.ny + units::ring_at(y, R.r[1], g.ny)) * g.nx;
        for (int k = 0; k < nbits; ++k)
            if (!((ent >> k) & 1u) && __ldg(rowp + units::ring_at(x0 + k, R.r[0], g.nx)) == 2)   // VG_OCC
                bits |= 1u << k;
    }
    out[w] = bits;
}

__global__ void __launch_bounds__(256) k_shift(const PlaneGeom g, const Ring ring, const uint8_t *__restrict__ src,
                                               uint8_t *__restrict__ dst) {
    pdl_trigger();
    pdl_wait();
    units::shift_chunk<units::LoadRO>(g, ring, src, dst, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <int WPU>
cudaError_t run_merge(const FrameArgs &a, cudaStream_t s) {
    const unsigned blocks = (unsigned)((a.g.words + WPU - 1) / WPU);
    if (blocks == 0) return cudaSuccess;
    if (a.lit & kLitRaysLast) return launch_pdl(k_merge<true, WPU>, blocks, 256, 0, s, a.g, a.pl, a.loc, a.ring);
    return launch_pdl(k_merge<false, WPU>, blocks, 256, 0, s, a.g, a.pl, a.loc, a.ring);
}

}  // namespace

// One thread per plane word, 256 to a CTA, or two per thread (sc.merge_words
// 512): fewer CTAs share the device.
cudaError_t launch_merge(const FrameArgs &a, cudaStream_t s, const Sched &sc) {
    if (sc.merge_words == 512) return run_merge<512>(a, s);
    return run_merge<256>(a, s);
}

cudaError_t launch_loc_occupancy(const PlaneGeom &g, const uint8_t *loc, const Ring &ring, uint32_t *out,
                                 cudaStream_t s) {
    const unsigned blocks = (unsigned)((g.words + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(k_loc_occupancy, blocks, 256, 0, s, g, loc, ring, out);
}

cudaError_t launch_shift(const PlaneGeom &g, const Ring &ring, const uint8_t *src, uint8_t *dst, cudaStream_t s) {
    const int64_t threads = (g.nvox + 15) / 16;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(k_shift, blocks, 256, 0, s, g, ring, src, dst);
}

}  // namespace vg
