// K3: free-space ray-trace (Sec. IV-C, Alg. 2).
//
// Ray bundle: one ray per far-plane voxel (a, b, vox_depth) of the camera,
// a in [-hw, hw], b in [-hh, hh]; ray id = (b + hh) * (2hw + 1) + (a + hw).
// In voxel units the ray is the segment S + tau * D, tau in [0, 1], with
//   S_k = t_k / vox_size,
//   D_k = (R_k0 * a + R_k1 * b) + R_k2 * vox_depth.
// The walk is Amanatides & Woo's: per active axis (D_k != 0 and 1/D_k
// finite) the m-th face crossing happens at
//   t_k(m) = ((float)(b0_k + step_k * m) - S_k) * (1 / D_k),
//   b0_k = floor(S_k) + (D_k > 0),
// always recomputed from the integer face; the next crossing is the smallest
// t, the lowest axis on a tie; the walk ends at the first crossing >= 1.
// The start voxel floor(S) is visited.  Voxels outside the grid are skipped.
//
// Free-space rule (Alg. 2): voxels before the ray's first occupied voxel
// (of the inflated plane) are marked free, voxels after it
// unknown-and-traced; occupied voxels are never marked free.  The paper's
// racy single-grid writes are replaced by two bit planes, fr and tr, merged
// by K4 with precedence occupied > free > traced, so the result does not
// depend on the order rays run in.
//
// Parallel walk.  LPR lanes of a warp share one ray.  Lane j owns the face
// crossings with tau in [c_j, c_{j+1}), c_0 = -inf, c_LPR = 1, c_j = j/LPR
// otherwise.  Because each axis's crossing times are non-decreasing in m,
// the serial walk performs exactly the crossings with t < c_j before any
// other, so lane j starts from voxel floor(S) + step * n(c_j), with
// n_k(c) = #{m : t_k(m) < c} found by an estimate and an exact fix-up on
// the same float expression, and then merges the three axes exactly as the
// serial walk does.  The lanes' visit lists concatenate to the serial list.
//
// Pass 1: each lane walks its slice and stops at its first occupied voxel.
// A ballot over the ray's lanes gives the first lane F that met one.
// Pass 2: each lane walks again and marks: lanes before F all free; lane F
// free before its occupied voxel and traced after it; lanes after F traced.
// Marks after the first occupied voxel are written without re-reading the
// occupancy: a traced mark on an occupied voxel is overridden by K4.  Marks
// that fall in the same 32-voxel word are OR-ed in a register and flushed
// with one atomicOr.
#include "vg_internal.cuh"

#include <cfloat>

namespace vg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Axis {
    float S;       // start, voxel units
    float inv;     // 1 / D, 0 when inactive
    int32_t b0;    // first face crossed
    int32_t step;  // -1, 0, +1
};

__device__ __forceinline__ float cross_t(const Axis &ax, int32_t m) {
    return __fmul_rn(__fsub_rn((float)(ax.b0 + ax.step * m), ax.S), ax.inv);
}

// Number of crossings of this axis with t < c (c finite, > 0).
__device__ __forceinline__ int32_t crossings_before(const Axis &ax, float D, float c) {
    if (ax.step == 0) return 0;
    const float t0 = cross_t(ax, 0);
    if (!(t0 < c)) return 0;
    float est = __fmul_rn(__fsub_rn(c, t0), fabsf(D));
    int32_t m = est < 1.0e7f ? (int32_t)est + 1 : 10000000;
    while (m > 1 && !(cross_t(ax, m - 1) < c)) --m;
    while (cross_t(ax, m) < c) ++m;
    return m;
}

struct Walker {
    int32_t i[3];
    float tmax[3];
};

__device__ __forceinline__ void walker_init(Walker &w, const Axis ax[3], const int32_t n0[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        w.i[k] = (int32_t)floorf(ax[k].S) + ax[k].step * n0[k];
        w.tmax[k] = ax[k].step ? cross_t(ax[k], n0[k]) : INFINITY;
    }
}

__device__ __forceinline__ void advance_axis(Walker &w, const Axis ax[3], int k) {
    w.i[k] += ax[k].step;
    const int32_t b = w.i[k] + (ax[k].step > 0 ? 1 : 0);
    w.tmax[k] = __fmul_rn(__fsub_rn((float)b, ax[k].S), ax[k].inv);
}

// Advances to the next voxel if the next crossing is before c_hi.  The axis
// with the smallest tMax moves, the lowest axis on a tie: x iff
// t0 <= t1 and t0 <= t2, else y iff t1 <= t2, else z.  (Written with
// constant indices so the walker stays in registers.)
__device__ __forceinline__ bool walker_next(Walker &w, const Axis ax[3], float c_hi) {
    const float t0 = w.tmax[0], t1 = w.tmax[1], t2 = w.tmax[2];
    const bool mx = (t0 <= t1) && (t0 <= t2);
    const bool my = !mx && (t1 <= t2);
    const float tm = mx ? t0 : (my ? t1 : t2);
    if (!(tm < c_hi)) return false;
    if (mx) advance_axis(w, ax, 0);
    else if (my) advance_axis(w, ax, 1);
    else advance_axis(w, ax, 2);
    return true;
}

__device__ __forceinline__ bool in_grid(const PlaneGeom &g, const int32_t i[3]) {
    return (unsigned)i[0] < (unsigned)g.nx && (unsigned)i[1] < (unsigned)g.ny &&
           (unsigned)i[2] < (unsigned)g.nz;
}

// True when an out-of-grid axis can no longer come back.
__device__ __forceinline__ bool gone(const PlaneGeom &g, const int32_t i[3], const Axis ax[3]) {
    const int32_t n[3] = {g.nx, g.ny, g.nz};
    bool out = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        out |= (i[k] < 0 && ax[k].step <= 0);
        out |= (i[k] >= n[k] && ax[k].step >= 0);
    }
    return out;
}

template <int LPR>
__global__ void __launch_bounds__(256) k_raytrace(const FrameArgs a) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int j = lane & (LPR - 1);
    const int64_t width = 2 * (int64_t)a.hw + 1;
    const int64_t nrays = width * (2 * (int64_t)a.hh + 1);
    const int64_t ray = gtid / LPR;
    const bool active = ray < nrays;

    Axis ax[3];
    float D[3];
    {
        const int32_t ra = active ? (int32_t)(ray % width) - a.hw : 0;
        const int32_t rb = active ? (int32_t)(ray / width) - a.hh : 0;
        const float fa = (float)ra, fb = (float)rb, fvd = (float)a.vd;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float S = __fdiv_rn(a.T.t[k], a.vs);
            const float d = __fadd_rn(__fadd_rn(__fmul_rn(a.T.R[k * 3 + 0], fa),
                                                __fmul_rn(a.T.R[k * 3 + 1], fb)),
                                      __fmul_rn(a.T.R[k * 3 + 2], fvd));
            D[k] = d;
            ax[k].S = S;
            ax[k].inv = 0.0f;
            ax[k].step = 0;
            if (d != 0.0f) {
                const float r = __fdiv_rn(1.0f, d);
                if (isfinite(r)) {
                    ax[k].inv = r;
                    ax[k].step = d > 0.0f ? 1 : -1;
                }
            }
            ax[k].b0 = (int32_t)floorf(S) + (ax[k].step > 0 ? 1 : 0);
        }
    }

    // this lane's slice of tau
    const float c_lo = (float)j / (float)LPR;   // exact: LPR is a power of two
    const float c_hi = (j == LPR - 1) ? 1.0f : (float)(j + 1) / (float)LPR;
    int32_t n0[3] = {0, 0, 0};
    if (j > 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) n0[k] = crossings_before(ax[k], D[k], c_lo);
    }

    // ---- pass 1: first occupied voxel of the slice -----------------------
    int32_t hit_at = -1;  // visit index of the first occupied voxel
    if (active) {
        Walker w;
        walker_init(w, ax, n0);
        int32_t q = 0;
        int64_t cw_idx = -1;
        uint32_t cw = 0;
        bool more = (j == 0) ? true : walker_next(w, ax, c_hi);
        while (more) {
            if (in_grid(a.g, w.i)) {
                const int64_t widx = plane_word(a.g, w.i[0], w.i[1], w.i[2]);
                if (widx != cw_idx) {
                    cw = __ldg(a.pl.occ_inf + widx);
                    cw_idx = widx;
                }
                if ((cw >> (w.i[0] & 31)) & 1u) {
                    hit_at = q;
                    break;
                }
            } else if (gone(a.g, w.i, ax)) {
                break;
            }
            ++q;
            more = walker_next(w, ax, c_hi);
        }
    }

    // ---- first lane of this ray with an occupied voxel -------------------
    const unsigned hits = __ballot_sync(kFull, hit_at >= 0);
    const int base = lane & ~(LPR - 1);
    const unsigned gmask = (LPR == 32) ? kFull : (((1u << LPR) - 1u) << base);
    const unsigned gh = hits & gmask;
    const int F = gh ? (__ffs(gh) - 1 - base) : LPR;

    // ---- pass 2: mark free / traced ---------------------------------------
    unsigned long long visits = 0;
    if (active) {
        Walker w;
        walker_init(w, ax, n0);
        int32_t q = 0;
        int64_t pend_idx = -1;
        uint32_t pend_bits = 0;
        uint32_t *pend_plane = nullptr;
        bool more = (j == 0) ? true : walker_next(w, ax, c_hi);
        while (more) {
            if (in_grid(a.g, w.i)) {
                ++visits;
                const bool traced = (j > F) || (j == F && q > hit_at);
                const bool skip = (j == F && q == hit_at);
                if (!skip) {
                    uint32_t *plane = traced ? a.pl.tr : a.pl.fr;
                    const int64_t widx = plane_word(a.g, w.i[0], w.i[1], w.i[2]);
                    if (widx != pend_idx || plane != pend_plane) {
                        if (pend_bits) atomicOr(pend_plane + pend_idx, pend_bits);
                        pend_idx = widx;
                        pend_plane = plane;
                        pend_bits = 0;
                    }
                    pend_bits |= 1u << (w.i[0] & 31);
                }
            } else if (gone(a.g, w.i, ax)) {
                break;
            }
            ++q;
            more = walker_next(w, ax, c_hi);
        }
        if (pend_bits) atomicOr(pend_plane + pend_idx, pend_bits);
    }

    if (a.stats) {
        const unsigned long long total = __reduce_add_sync(kFull, (unsigned)visits);
        if (lane == 0 && total) atomicAdd(a.stats + 2, total);
    }
}

template <int LPR>
cudaError_t launch_lpr(const FrameArgs &a, cudaStream_t s) {
    const int64_t nrays = (2 * (int64_t)a.hw + 1) * (2 * (int64_t)a.hh + 1);
    const int64_t threads = nrays * LPR;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    k_raytrace<LPR><<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raytrace(const FrameArgs &a, int lanes_per_ray, cudaStream_t s) {
    switch (lanes_per_ray) {
    case 1: return launch_lpr<1>(a, s);
    case 2: return launch_lpr<2>(a, s);
    case 4: return launch_lpr<4>(a, s);
    case 8: return launch_lpr<8>(a, s);
    case 16: return launch_lpr<16>(a, s);
    case 32: return launch_lpr<32>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vg
