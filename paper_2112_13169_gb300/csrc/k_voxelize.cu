// K1: transform and voxelize (Sec. IV-B, Alg. 1 before the inflation loops).
//
// Each thread reads four consecutive pixels of the row-major depth image
// (one 16-byte float4 or 8-byte ushort4 load when aligned), back-projects
// the valid ones with the pinhole model, transforms them by T^v_c and sets
// their voxel's bit in the occ_raw plane.  Neighbouring pixels mostly land
// in the same 32-voxel word, so each warp de-duplicates its words with
// a segmented OR-scan across lanes before one atomicOr per run of lanes
// that share a word: the plane is bit-packed, so concurrent sets need an
// atomic, but only about one per distinct word per warp.
//
// Arithmetic follows the oracle's order with one IEEE rounding per operation
// (explicit __f*_rn intrinsics; this file is also built with -fmad=false):
//   xc = ((u - cx) * d) / fx,  yc = ((v - cy) * d) / fy,  zc = d
//   g_k = (((R_k0 xc + R_k1 yc) + R_k2 zc) + t_k) / vox_size
//   kept iff 0 <= g_k < N_k on every axis; voxel = floor(g).
#include "vg_internal.cuh"

namespace vg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNoWord = 0xffffffffu;

// Returns the plane word of the point's voxel and its bit, or kNoWord.
__device__ __forceinline__ uint32_t point_word(const FrameArgs &a, float x, float y, float z,
                                               uint32_t &bit) {
    int32_t v[3];
    const int32_t n[3] = {a.g.nx, a.g.ny, a.g.nz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float g = __fadd_rn(__fmul_rn(a.T.R[k * 3 + 0], x), __fmul_rn(a.T.R[k * 3 + 1], y));
        g = __fadd_rn(g, __fmul_rn(a.T.R[k * 3 + 2], z));
        g = __fadd_rn(g, a.T.t[k]);
        g = __fdiv_rn(g, a.vs);
        if (!(g >= 0.0f && g < (float)n[k])) return kNoWord;
        v[k] = (int32_t)floorf(g);
    }
    bit = 1u << (v[0] & 31);
    return (uint32_t)plane_word(a.g, v[0], v[1], v[2]);
}

__device__ __forceinline__ uint32_t pixel_word(const FrameArgs &a, float d, int32_t u, int32_t v,
                                               uint32_t &bit) {
    if (!(isfinite(d) && d > 0.0f && d <= a.depth_max)) return kNoWord;
    float xc = __fdiv_rn(__fmul_rn(__fsub_rn((float)u, a.cx), d), a.fx);
    float yc = __fdiv_rn(__fmul_rn(__fsub_rn((float)v, a.cy), d), a.fy);
    return point_word(a, xc, yc, d, bit);
}

// ORs `bit` into plane[key] for every lane, with one atomicOr per run of
// consecutive lanes that share a word (neighbouring pixels usually do): an
// inclusive OR-scan over lanes that only pulls from lanes with the same key,
// after which the last lane of each run holds the run's bits.  Lanes whose
// keys match but are not adjacent may fold bits into each other; that is
// harmless, they name the same word.  Every lane of the warp must call this
// (keys of idle lanes are kNoWord).
__device__ __forceinline__ void warp_set_bits(uint32_t *plane, uint32_t key, uint32_t bit) {
    const int lane = threadIdx.x & 31;
    uint32_t v = bit;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t kd = __shfl_up_sync(kFull, key, d);
        const uint32_t vd = __shfl_up_sync(kFull, v, d);
        if (lane >= d && kd == key) v |= vd;
    }
    const uint32_t knext = __shfl_down_sync(kFull, key, 1);
    if (key != kNoWord && (lane == 31 || knext != key)) atomicOr(plane + key, v);
}

// Adds the warp's number of in-grid points to the stats counter.  Every lane
// of the warp must call this.
__device__ __forceinline__ void count(const FrameArgs &a, unsigned kept) {
    if (!a.stats) return;
    const unsigned total = __reduce_add_sync(kFull, kept);
    if ((threadIdx.x & 31) == 0 && total) atomicAdd(a.stats + 1, (unsigned long long)total);
}

// DT: 0 = f32, 1 = u16.  VEC: the image base is aligned for a 4-pixel load.
template <int DT, bool VEC>
__global__ void __launch_bounds__(256) k_voxelize_depth(const FrameArgs a) {
    const int64_t npix = (int64_t)a.W * a.H;
    const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    float d[4];
    if (VEC && p0 + 3 < npix) {
        if (DT == 0) {
            const float4 q = __ldg(reinterpret_cast<const float4 *>(a.depth) + (p0 >> 2));
            d[0] = q.x; d[1] = q.y; d[2] = q.z; d[3] = q.w;
        } else {
            const ushort4 q = __ldg(reinterpret_cast<const ushort4 *>(a.depth) + (p0 >> 2));
            d[0] = __fmul_rn((float)q.x, a.scale);
            d[1] = __fmul_rn((float)q.y, a.scale);
            d[2] = __fmul_rn((float)q.z, a.scale);
            d[3] = __fmul_rn((float)q.w, a.scale);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            d[j] = 0.0f;
            if (p0 + j < npix) {
                if (DT == 0) d[j] = __ldg(reinterpret_cast<const float *>(a.depth) + p0 + j);
                else d[j] = __fmul_rn((float)__ldg(reinterpret_cast<const uint16_t *>(a.depth) + p0 + j), a.scale);
            }
        }
    }
    uint32_t key[4], bit[4];
    int32_t v = (int32_t)(p0 / a.W), u = (int32_t)(p0 - (int64_t)v * a.W);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        key[j] = kNoWord;
        bit[j] = 0;
        if (p0 + j < npix) key[j] = pixel_word(a, d[j], u, v, bit[j]);
        if (++u == a.W) { u = 0; ++v; }
    }
    unsigned kept = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) kept += (key[j] != kNoWord);
    // merge equal words inside the thread first (neighbouring pixels)
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        if (key[j] != kNoWord && key[j] == key[j - 1]) {
            bit[j] |= bit[j - 1];
            key[j - 1] = kNoWord;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) warp_set_bits(a.pl.occ_raw, key[j], bit[j]);
    count(a, kept);
}

__global__ void __launch_bounds__(256) k_voxelize_points(const FrameArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t key = kNoWord, bit = 0;
    if (i < a.npts) {
        const float x = __ldg(a.xyz + 3 * i + 0);
        const float y = __ldg(a.xyz + 3 * i + 1);
        const float z = __ldg(a.xyz + 3 * i + 2);
        if (isfinite(x) && isfinite(y) && isfinite(z)) key = point_word(a, x, y, z, bit);
    }
    warp_set_bits(a.pl.occ_raw, key, bit);
    count(a, key != kNoWord);
}

}  // namespace

cudaError_t launch_voxelize_depth(const FrameArgs &a, int32_t dtype, cudaStream_t s) {
    const int64_t npix = (int64_t)a.W * a.H;
    const int64_t threads = (npix + 3) / 4;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    const uintptr_t base = reinterpret_cast<uintptr_t>(a.depth);
    if (dtype == 0) {
        if (base % 16 == 0) k_voxelize_depth<0, true><<<blocks, 256, 0, s>>>(a);
        else k_voxelize_depth<0, false><<<blocks, 256, 0, s>>>(a);
    } else {
        if (base % 8 == 0) k_voxelize_depth<1, true><<<blocks, 256, 0, s>>>(a);
        else k_voxelize_depth<1, false><<<blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_voxelize_points(const FrameArgs &a, cudaStream_t s) {
    const unsigned blocks = (unsigned)((a.npts + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    k_voxelize_points<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vg
