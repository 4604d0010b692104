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
// with one atomicOr; near the camera, where all rays overlap, they go to a
// per-CTA shared-memory box first (see kBoxW).
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

// Walker state of one lane: voxel (i0, i1, i2), next crossing times
// (t0, t1, t2), and the voxel's plane word and bit, kept up to date
// incrementally (w = (i2*ny + i1)*wx + (i0 >> 5), xb = i0 & 31).
struct Walker {
    int32_t i0, i1, i2;
    float t0, t1, t2;
    uint32_t w;   // modulo 2^32 while outside the grid; exact inside it
    int32_t xb;
};

struct Ray {
    Axis ax[3];
    int32_t dw1, dw2;   // word-index change of one y / z step
    int32_t nx, ny, nz;
};

__device__ __forceinline__ void walker_init(Walker &w, const Ray &r, const int32_t n0[3], int32_t wx) {
    w.i0 = (int32_t)floorf(r.ax[0].S) + r.ax[0].step * n0[0];
    w.i1 = (int32_t)floorf(r.ax[1].S) + r.ax[1].step * n0[1];
    w.i2 = (int32_t)floorf(r.ax[2].S) + r.ax[2].step * n0[2];
    w.t0 = r.ax[0].step ? cross_t(r.ax[0], n0[0]) : INFINITY;
    w.t1 = r.ax[1].step ? cross_t(r.ax[1], n0[1]) : INFINITY;
    w.t2 = r.ax[2].step ? cross_t(r.ax[2], n0[2]) : INFINITY;
    w.w = ((uint32_t)w.i2 * (uint32_t)r.ny + (uint32_t)w.i1) * (uint32_t)wx + (uint32_t)(w.i0 >> 5);
    w.xb = w.i0 & 31;
}

// Advances to the next voxel if the next crossing is before c_hi.  The axis
// with the smallest tMax moves, the lowest axis on a tie: x iff
// t0 <= t1 and t0 <= t2, else y iff t1 <= t2, else z.  Branch-free, so the
// lanes of a warp stepping different axes do not diverge.
__device__ __forceinline__ bool walker_next(Walker &w, const Ray &r, float c_hi) {
    const bool mx = (w.t0 <= w.t1) && (w.t0 <= w.t2);
    const bool my = !mx && (w.t1 <= w.t2);
    const bool mz = !mx && !my;
    const float tm = mx ? w.t0 : (my ? w.t1 : w.t2);
    if (!(tm < c_hi)) return false;
    const int32_t s0 = mx ? r.ax[0].step : 0;
    w.i0 += s0;
    w.i1 += my ? r.ax[1].step : 0;
    w.i2 += mz ? r.ax[2].step : 0;
    int32_t xb = w.xb + s0;
    const int32_t carry = (xb >> 5);          // +1 when xb reached 32, -1 when it went below 0
    w.xb = xb & 31;
    w.w += (uint32_t)(carry + (my ? r.dw1 : 0) + (mz ? r.dw2 : 0));
    const int32_t ik = mx ? w.i0 : (my ? w.i1 : w.i2);
    const int32_t sk = mx ? r.ax[0].step : (my ? r.ax[1].step : r.ax[2].step);
    const float Sk = mx ? r.ax[0].S : (my ? r.ax[1].S : r.ax[2].S);
    const float ik_inv = mx ? r.ax[0].inv : (my ? r.ax[1].inv : r.ax[2].inv);
    const float nt = __fmul_rn(__fsub_rn((float)(ik + (sk > 0 ? 1 : 0)), Sk), ik_inv);
    w.t0 = mx ? nt : w.t0;
    w.t1 = my ? nt : w.t1;
    w.t2 = mz ? nt : w.t2;
    return true;
}

__device__ __forceinline__ bool in_grid(const Walker &w, const Ray &r) {
    return (unsigned)w.i0 < (unsigned)r.nx && (unsigned)w.i1 < (unsigned)r.ny &&
           (unsigned)w.i2 < (unsigned)r.nz;
}

// True when an out-of-grid axis can no longer come back.
__device__ __forceinline__ bool gone(const Walker &w, const Ray &r) {
    return (w.i0 < 0 && r.ax[0].step <= 0) || (w.i0 >= r.nx && r.ax[0].step >= 0) ||
           (w.i1 < 0 && r.ax[1].step <= 0) || (w.i1 >= r.ny && r.ax[1].step >= 0) ||
           (w.i2 < 0 && r.ax[2].step <= 0) || (w.i2 >= r.nz && r.ax[2].step >= 0);
}

constexpr int kChunk = 4;   // occupancy words loaded together
constexpr int kThreads = 256;

// Near the camera every ray of the bundle crosses the same few voxels.  A
// box of kBoxW plane words (x) by kBoxY rows by kBoxZ slices around the
// camera voxel is kept in shared memory by every CTA: the occupancy words
// are staged there once, and free/traced marks inside the box are OR-ed
// there and flushed to the planes once per CTA.
constexpr int kBoxW = 2, kBoxY = 32, kBoxZ = 32;
constexpr int kBoxWords = kBoxW * kBoxY * kBoxZ;

// A visit packed in 32 bits: bit 31 set -> shared-box word (index in bits
// 5..15), else plane word w (< 2^26) in bits 5..30; bits 0..4 are x & 31.
constexpr uint32_t kBoxFlag = 0x80000000u;

struct Box {
    int32_t bw0, by0, bz0;
};

__device__ __forceinline__ uint32_t pack_visit(const Walker &w, const Box &b) {
    const uint32_t dw = (uint32_t)((w.i0 >> 5) - b.bw0), dy = (uint32_t)(w.i1 - b.by0),
                   dz = (uint32_t)(w.i2 - b.bz0);
    if (dw < kBoxW && dy < kBoxY && dz < kBoxZ)
        return kBoxFlag | (((dz * kBoxY + dy) * kBoxW + dw) << 5) | (uint32_t)w.xb;
    return (w.w << 5) | (uint32_t)w.xb;
}

__device__ __forceinline__ uint32_t occ_word(const FrameArgs &a, const uint32_t *occ_box, uint32_t p) {
    return (p & kBoxFlag) ? occ_box[(p >> 5) & 0x7ffu] : __ldg(a.pl.occ_inf + (p >> 5));
}

// Pending marks of one lane: consecutive marks of the same word and kind
// are OR-ed in a register; a change of word or kind flushes them, to the
// shared box or to the plane.
struct Marks {
    uint32_t key = 0xffffffffu;   // p >> 5 of the pending word
    uint32_t bits = 0;
    bool traced = false;
};

__device__ __forceinline__ void marks_flush(const FrameArgs &a, uint32_t *box_fr, uint32_t *box_tr,
                                            const Marks &m) {
    if (!m.bits) return;
    if (m.key & (kBoxFlag >> 5)) atomicOr((m.traced ? box_tr : box_fr) + (m.key & 0x7ffu), m.bits);
    else atomicOr((m.traced ? a.pl.tr : a.pl.fr) + m.key, m.bits);
}

__device__ __forceinline__ void marks_add(const FrameArgs &a, uint32_t *box_fr, uint32_t *box_tr, Marks &m,
                                          uint32_t p, bool traced) {
    const uint32_t key = p >> 5;
    if (key != m.key || traced != m.traced) {
        marks_flush(a, box_fr, box_tr, m);
        m.key = key;
        m.traced = traced;
        m.bits = 0;
    }
    m.bits |= 1u << (p & 31u);
}

// Two-pass walk for a lane whose slice does not fit its buffer: pass 1
// returns the index (among the slice's in-grid visits) of the first
// occupied voxel, or -1.
__device__ int walk_first_hit(const FrameArgs &a, const Ray &r, const int32_t n0[3], bool visit_start,
                              float c_hi, const Box &b, const uint32_t *occ_box) {
    Walker w;
    walker_init(w, r, n0, a.g.wx);
    bool more = visit_start ? true : walker_next(w, r, c_hi);
    int32_t q = 0;
    while (more) {
        uint32_t p[kChunk];
        int n = 0;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
            p[c] = 0;
            while (more && n == c) {
                if (in_grid(w, r)) {
                    p[c] = pack_visit(w, b);
                    ++n;
                } else if (gone(w, r)) {
                    more = false;
                    break;
                }
                more = walker_next(w, r, c_hi);
            }
        }
        uint32_t v[kChunk];
#pragma unroll
        for (int c = 0; c < kChunk; ++c) v[c] = c < n ? occ_word(a, occ_box, p[c]) : 0u;
        int hit = -1;
#pragma unroll
        for (int c = kChunk - 1; c >= 0; --c)
            if (c < n && ((v[c] >> (p[c] & 31u)) & 1u)) hit = c;
        if (hit >= 0) return q + hit;
        q += n;
    }
    return -1;
}

// Pass 2 of the two-pass walk: marks the slice's in-grid visits.
__device__ unsigned walk_marks(const FrameArgs &a, const Ray &r, const int32_t n0[3], bool visit_start,
                               float c_hi, const Box &b, int mode, int32_t hit_at, uint32_t *box_fr,
                               uint32_t *box_tr) {
    Walker w;
    walker_init(w, r, n0, a.g.wx);
    bool more = visit_start ? true : walker_next(w, r, c_hi);
    int32_t q = 0;
    Marks m;
    while (more) {
        if (in_grid(w, r)) {
            // mode: 0 all free, 1 free before hit_at and traced after, 2 all traced
            if (!(mode == 1 && q == hit_at))
                marks_add(a, box_fr, box_tr, m, pack_visit(w, b), mode == 2 || (mode == 1 && q > hit_at));
            ++q;
        } else if (gone(w, r)) {
            break;
        }
        more = walker_next(w, r, c_hi);
    }
    marks_flush(a, box_fr, box_tr, m);
    return (unsigned)q;
}

// kBuf visits per lane are kept in dynamic shared memory (column-major,
// one column per thread) when `buffered` is set; lanes whose slice holds
// more use the two-pass walk.  Persistent: each CTA loops over groups of
// kThreads / LPR rays.
template <int LPR>
__global__ void __launch_bounds__(kThreads) k_raytrace(const FrameArgs a, const int buffered) {
    __shared__ uint32_t box_fr[kBoxWords], box_tr[kBoxWords], occ_box[kBoxWords];
    extern __shared__ uint32_t buf[];   // kRtBuf * kThreads

    const int lane = threadIdx.x & 31;
    const int j = lane & (LPR - 1);
    const int32_t width = 2 * a.hw + 1;
    const int64_t nrays = (int64_t)width * (2 * a.hh + 1);
    float S[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) S[k] = __fdiv_rn(a.T.t[k], a.vs);

    // the box around the camera voxel, the same for every ray
    Box b;
    {
        const int32_t cx0 = (int32_t)floorf(S[0]);
        b.bw0 = (cx0 >> 5) - ((cx0 & 31) < 16 ? 1 : 0);   // x words bw0, bw0+1
        b.by0 = (int32_t)floorf(S[1]) - kBoxY / 2;
        b.bz0 = (int32_t)floorf(S[2]) - kBoxZ / 2;
    }
    for (int i = threadIdx.x; i < kBoxWords; i += kThreads) {
        box_fr[i] = 0;
        box_tr[i] = 0;
        const int32_t dw = i % kBoxW, dy = (i / kBoxW) % kBoxY, dz = i / (kBoxW * kBoxY);
        const int32_t wx = b.bw0 + dw, y = b.by0 + dy, z = b.bz0 + dz;
        uint32_t v = 0;
        if (wx >= 0 && wx < a.g.wx && y >= 0 && y < a.g.ny && z >= 0 && z < a.g.nz)
            v = __ldg(a.pl.occ_inf + ((uint32_t)z * (uint32_t)a.g.ny + (uint32_t)y) * (uint32_t)a.g.wx + wx);
        occ_box[i] = v;
    }
    __syncthreads();

    unsigned visits = 0;
    const int rays_per_cta = kThreads / LPR;
    for (int64_t base = (int64_t)blockIdx.x * rays_per_cta; base < nrays;
         base += (int64_t)gridDim.x * rays_per_cta) {
        const int64_t ray = base + threadIdx.x / LPR;
        const bool active = ray < nrays;

        Ray r;
        r.nx = a.g.nx;
        r.ny = a.g.ny;
        r.nz = a.g.nz;
        float D[3];
        {
            const int32_t ra = active ? (int32_t)(ray % width) - a.hw : 0;
            const int32_t rb = active ? (int32_t)(ray / width) - a.hh : 0;
            const float fa = (float)ra, fb = (float)rb, fvd = (float)a.vd;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float d = __fadd_rn(__fadd_rn(__fmul_rn(a.T.R[k * 3 + 0], fa),
                                                    __fmul_rn(a.T.R[k * 3 + 1], fb)),
                                          __fmul_rn(a.T.R[k * 3 + 2], fvd));
                D[k] = d;
                r.ax[k].S = S[k];
                r.ax[k].inv = 0.0f;
                r.ax[k].step = 0;
                if (d != 0.0f) {
                    const float q = __fdiv_rn(1.0f, d);
                    if (isfinite(q)) {
                        r.ax[k].inv = q;
                        r.ax[k].step = d > 0.0f ? 1 : -1;
                    }
                }
                r.ax[k].b0 = (int32_t)floorf(S[k]) + (r.ax[k].step > 0 ? 1 : 0);
            }
        }
        r.dw1 = r.ax[1].step * a.g.wx;
        r.dw2 = r.ax[2].step * a.g.wx * a.g.ny;

        // this lane's slice of tau
        const float c_lo = (float)j / (float)LPR;   // exact: LPR is a power of two
        const float c_hi = (j == LPR - 1) ? 1.0f : (float)(j + 1) / (float)LPR;
        int32_t n0[3] = {0, 0, 0};
        if (j > 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) n0[k] = crossings_before(r.ax[k], D[k], c_lo);
        }

        // ---- pass 1: walk the slice once, keep its in-grid visits --------
        int32_t nvis = 0, hit_at = -1;
        bool ovf = !buffered;
        if (active && !ovf) {
            Walker w;
            walker_init(w, r, n0, a.g.wx);
            bool more = (j == 0) ? true : walker_next(w, r, c_hi);
            while (more) {
                if (in_grid(w, r)) {
                    if (nvis == kRtBuf) {
                        ovf = true;
                        break;
                    }
                    buf[nvis * kThreads + threadIdx.x] = pack_visit(w, b);
                    ++nvis;
                } else if (gone(w, r)) {
                    break;
                }
                more = walker_next(w, r, c_hi);
            }
            // first occupied visit, kChunk occupancy words in flight at a time
            for (int q0 = 0; !ovf && q0 < nvis && hit_at < 0; q0 += kChunk) {
                uint32_t p[kChunk], v[kChunk];
#pragma unroll
                for (int c = 0; c < kChunk; ++c) p[c] = q0 + c < nvis ? buf[(q0 + c) * kThreads + threadIdx.x] : 0u;
#pragma unroll
                for (int c = 0; c < kChunk; ++c) v[c] = q0 + c < nvis ? occ_word(a, occ_box, p[c]) : 0u;
#pragma unroll
                for (int c = kChunk - 1; c >= 0; --c)
                    if (q0 + c < nvis && ((v[c] >> (p[c] & 31u)) & 1u)) hit_at = q0 + c;
            }
        }
        if (active && ovf) hit_at = walk_first_hit(a, r, n0, j == 0, c_hi, b, occ_box);

        // ---- first lane of this ray with an occupied voxel ---------------
        const unsigned hits = __ballot_sync(kFull, hit_at >= 0);
        const int gbase = lane & ~(LPR - 1);
        const unsigned gmask = (LPR == 32) ? kFull : (((1u << LPR) - 1u) << gbase);
        const unsigned gh = hits & gmask;
        const int F = gh ? (__ffs(gh) - 1 - gbase) : LPR;
        const int mode = j < F ? 0 : (j == F ? 1 : 2);

        // ---- pass 2: mark free / traced -----------------------------------
        if (active && !ovf) {
            Marks m;
            for (int q = 0; q < nvis; ++q) {
                if (mode == 1 && q == hit_at) continue;
                marks_add(a, box_fr, box_tr, m, buf[q * kThreads + threadIdx.x],
                          mode == 2 || (mode == 1 && q > hit_at));
            }
            marks_flush(a, box_fr, box_tr, m);
            visits += (unsigned)nvis;
        } else if (active) {
            visits += walk_marks(a, r, n0, j == 0, c_hi, b, mode, hit_at, box_fr, box_tr);
        }
    }

    // ---- flush the shared box once per CTA --------------------------------
    __syncthreads();
    for (int i = threadIdx.x; i < kBoxWords; i += kThreads) {
        const uint32_t f = box_fr[i], t = box_tr[i];
        if ((f | t) == 0) continue;
        const int32_t dw = i % kBoxW, dy = (i / kBoxW) % kBoxY, dz = i / (kBoxW * kBoxY);
        // only in-grid voxels are ever marked, so the word exists
        const uint32_t gw = ((uint32_t)(b.bz0 + dz) * (uint32_t)a.g.ny + (uint32_t)(b.by0 + dy)) *
                                (uint32_t)a.g.wx + (uint32_t)(b.bw0 + dw);
        if (f) atomicOr(a.pl.fr + gw, f);
        if (t) atomicOr(a.pl.tr + gw, t);
    }

    if (a.stats) {
        const unsigned total = __reduce_add_sync(kFull, visits);
        if (lane == 0 && total) atomicAdd(a.stats + 2, (unsigned long long)total);
    }
}

int g_sms[64];
int g_blocks_per_sm[64][6];

template <int LPR>
cudaError_t configure_lpr(int dev, int idx) {
    const size_t dyn = sizeof(uint32_t) * kRtBuf * kThreads;
    cudaError_t e = cudaFuncSetAttribute(k_raytrace<LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_blocks_per_sm[dev][idx], k_raytrace<LPR>, kThreads,
                                                         dyn);
}

template <int LPR>
cudaError_t launch_lpr(const FrameArgs &a, int idx, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int64_t nrays = (2 * (int64_t)a.hw + 1) * (2 * (int64_t)a.hh + 1);
    const int64_t need = (nrays * LPR + kThreads - 1) / kThreads;
    const int64_t resident = (int64_t)g_sms[dev] * (g_blocks_per_sm[dev][idx] > 0 ? g_blocks_per_sm[dev][idx] : 1);
    const unsigned blocks = (unsigned)(need < resident ? need : resident);
    if (blocks == 0) return cudaSuccess;
    // packed visits hold a plane word in 26 bits
    const int buffered = a.g.words < (int64_t(1) << 26) ? 1 : 0;
    k_raytrace<LPR><<<blocks, kThreads, sizeof(uint32_t) * kRtBuf * kThreads, s>>>(a, buffered);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_raytrace(int dev) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaError_t e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = configure_lpr<1>(dev, 0);
    if (e == cudaSuccess) e = configure_lpr<2>(dev, 1);
    if (e == cudaSuccess) e = configure_lpr<4>(dev, 2);
    if (e == cudaSuccess) e = configure_lpr<8>(dev, 3);
    if (e == cudaSuccess) e = configure_lpr<16>(dev, 4);
    if (e == cudaSuccess) e = configure_lpr<32>(dev, 5);
    return e;
}

int auto_lanes_per_ray(int32_t vd, int32_t hw, int32_t hh) {
    // a slice of 1/LPR of a ray crosses about L1/LPR faces, plus up to three
    // more at its ends; pick the fewest lanes whose slices fit the buffer
    const int64_t l1 = (int64_t)vd + hw + hh + 4;
    for (int lpr = 8; lpr < 32; lpr *= 2)
        if ((l1 + lpr - 1) / lpr + 3 <= kRtBuf) return lpr;
    return 32;
}

cudaError_t launch_raytrace(const FrameArgs &a, int lanes_per_ray, cudaStream_t s) {
    switch (lanes_per_ray) {
    case 1: return launch_lpr<1>(a, 0, s);
    case 2: return launch_lpr<2>(a, 1, s);
    case 4: return launch_lpr<4>(a, 2, s);
    case 8: return launch_lpr<8>(a, 3, s);
    case 16: return launch_lpr<16>(a, 4, s);
    case 32: return launch_lpr<32>(a, 5, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vg
