// vg_rt.cuh -- K3, the free-space ray trace, as device functions over one
// group of rays, shared by the one-kernel-per-step launch (k_raytrace.cu)
// and the fused persistent launch (k_batch.cu).
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
// 1/D_k is taken with the correctly rounded reciprocal, which is the IEEE
// quotient 1/D_k; the face coordinate is kept as an exact float.
//
// Free-space rule (Alg. 2): voxels before the ray's first occupied voxel
// (of the inflated plane; a.occ_test, which a literal reading may point
// elsewhere) are marked free, voxels after it unknown-and-traced; occupied
// voxels are never marked free.  With kLitSkipStart the walk moves before
// its first visit, so the start voxel is left out.  The paper's
// racy single-grid writes are replaced by two bit planes, fr and tr, merged
// by K4 with precedence occupied > free > traced, so the result does not
// depend on the order rays run in.
//
// Parallel walk.  LPR lanes of a warp share one ray.  Lane j owns the face
// crossings with tau in [c_j, c_{j+1}), c_0 = -inf, c_LPR = 1, and the
// other cuts split the part of the segment inside the grid evenly.  Because
// each axis's crossing times are non-decreasing in m, the serial walk
// performs exactly the crossings with t < c_j before any other, so lane j
// starts from voxel floor(S) + step * n(c_j), with n_k(c) = #{m : t_k(m) < c}
// found by an estimate and an exact fix-up on the same float expression,
// and then merges the three axes exactly as the serial walk does.  The
// lanes' visit lists concatenate to the serial list.
//
// Fast walk.  A crossing of axis k's face F happens at exactly the float
// time ((float)F - S_k) * (1/D_k), because the walker keeps F as an exact
// float and evaluates that expression.  So while the next crossing is
// earlier than the ray's first outward grid-face crossing t_out (computed
// once with the same expression), a voxel inside the grid stays inside, and
// likewise for the camera box and t_box: the walk needs no per-step bounds
// or box tests.  Exact steps (with tests) lead to a lane's first in-grid
// voxel and finish a slice in which the ray leaves the grid.
//
// Pass 1: each lane walks its slice once and keeps its in-grid visits in
// its own shared-memory column (kRtBuf entries) as runs: consecutive visits
// in one 32-voxel word, which can only be x-steps of one sign, share an
// entry.  It then finds the first occupied visit, one occupancy word per
// run and kChunk runs in flight at a time.  A ballot over the ray's lanes
// gives the first lane F that met one.
// Pass 2: each lane replays its runs and marks: free before the ray's
// first occupied voxel, traced from it on (lanes before F all free, lanes
// after F all traced), one atomicOr per run and kind.  Traced marks are
// written without re-reading the occupancy: a traced mark on an occupied
// voxel, the first one included, is overridden by K4.  Near the camera,
// where all rays overlap, marks go to a per-CTA shared-memory box first
// (see kBoxW).  A lane whose slice holds more than kRtBuf runs, or a grid
// whose planes are too large for a packed run, walks twice instead.
//
// Work mapping: warp w of group g takes a bundle of 32 / LPR neighbouring
// rays, bundle w * G + g of the frame's G groups, so every group samples
// rows across the whole image (rows near the top and bottom leave the grid
// early).  The CTAs are persistent: each loops over groups, so the box is
// staged and flushed once per CTA.
#pragma once

#include "vg_units.cuh"

namespace vg {
namespace rt {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kChunk = 4;   // occupancy words loaded together
constexpr int kThreads = 256;

// The box around the camera voxel: kBoxW plane words (x) by kBoxY rows by
// kBoxZ slices.  Its occupancy words are staged in shared memory once per
// CTA and its free/traced marks are OR-ed there, then flushed once per CTA.
constexpr int kBoxW = 2, kBoxY = 16, kBoxZ = 16;
constexpr int kBoxWords = kBoxW * kBoxY * kBoxZ;

// A visit packed in 32 bits: bit 31 set -> box word (index in bits 5..),
// else the plane bit index P = ((z*ny + y) * 32*wx + x) < 2^31; bits 0..4
// are x & 31 either way, so p >> 5 is the word.
constexpr uint32_t kBoxFlag = 0x80000000u;

// A run of visits packed in 32 bits: its first visit, packed as above, with
// the number of further visits (n - 1 <= 31) in bits 26..30, which a plane
// visit leaves free when plane bit indices are below 2^26 (plane words
// below kRunWords) and a box visit always.  The run's bits are lo, lo + sx,
// ..., lo + (n - 1) sx of its word, lo = bits 0..4, sx the ray's x step.
constexpr uint32_t kRunOne = 1u << 26;                  // one more visit
constexpr uint32_t kRunKey = kBoxFlag | 0x03ffffe0u;    // the word, box flag included

__device__ __forceinline__ uint32_t run_mask(uint32_t e, int32_t sx) {
    const uint32_t n = ((e >> 26) & 31u) + 1u, lo = e & 31u;
    return (0xffffffffu >> (32u - n)) << (sx < 0 ? lo + 1u - n : lo);
}

// The bits of a run's word that its walk visits before bit b.
__device__ __forceinline__ uint32_t bits_before(uint32_t b, int32_t sx) {
    return sx < 0 ? ~((2u << b) - 1u) : (1u << b) - 1u;
}

// Appends visit v to a lane's runs, without a branch: the pending run
// `cur` (in slot `last` of the column) grows if v is in its word, else v
// starts the next one in the next slot; the pending run is stored every
// time.  False when the column is full.
__device__ __forceinline__ bool run_add(uint32_t *col, int32_t &last, uint32_t &cur, uint32_t v) {
    const bool same = ((v ^ cur) & kRunKey) == 0;
    cur = same ? cur + kRunOne : v;
    last += same ? 0 : 1;
    if (last == kRtBuf) return false;
    col[last * kThreads] = cur;
    return true;
}

struct Box {
    int32_t bw0, by0, bz0;
};

// Per-ray constants of one lane.
struct Ray {
    float S[3];      // start, voxel units
    float inv[3];    // 1/D, 0 for an inactive axis
    float fs[3];     // step as float
    int32_t s[3];    // step: -1, 0, +1
    int32_t dP[3];   // change of the plane bit index per step
    int32_t dPb[3];  // change of the packed box index per step
    int32_t nx, ny, nz;
};

struct Walker {
    float t0, t1, t2;     // next crossing time per axis
    float nb0, nb1, nb2;  // coordinate of the next face per axis (exact)
    int32_t i0, i1, i2;   // voxel
    uint32_t P;           // plane bit index, modulo 2^32 outside the grid
};

__device__ __forceinline__ float cross_at(float b, float S, float inv) {
    return __fmul_rn(__fsub_rn(b, S), inv);
}

// Number of crossings of axis k with t < c (c finite, > 0).
__device__ __forceinline__ int32_t crossings_before(const Ray &r, int k, float absD, float c) {
    if (r.s[k] == 0) return 0;
    const int32_t b0 = (int32_t)floorf(r.S[k]) + (r.s[k] > 0 ? 1 : 0);
    const float t0 = cross_at((float)b0, r.S[k], r.inv[k]);
    if (!(t0 < c)) return 0;
    const float est = __fmul_rn(__fsub_rn(c, t0), absD);
    int32_t m = est < 1.0e7f ? (int32_t)est + 1 : 10000000;
    while (m > 1 && !(cross_at((float)(b0 + r.s[k] * (m - 1)), r.S[k], r.inv[k]) < c)) --m;
    while (cross_at((float)(b0 + r.s[k] * m), r.S[k], r.inv[k]) < c) ++m;
    return m;
}

__device__ __forceinline__ void walker_init(Walker &w, const Ray &r, const int32_t n0[3], uint32_t R) {
    w.i0 = (int32_t)floorf(r.S[0]) + r.s[0] * n0[0];
    w.i1 = (int32_t)floorf(r.S[1]) + r.s[1] * n0[1];
    w.i2 = (int32_t)floorf(r.S[2]) + r.s[2] * n0[2];
    w.nb0 = (float)(w.i0 + (r.s[0] > 0 ? 1 : 0));
    w.nb1 = (float)(w.i1 + (r.s[1] > 0 ? 1 : 0));
    w.nb2 = (float)(w.i2 + (r.s[2] > 0 ? 1 : 0));
    w.t0 = r.s[0] ? cross_at(w.nb0, r.S[0], r.inv[0]) : INFINITY;
    w.t1 = r.s[1] ? cross_at(w.nb1, r.S[1], r.inv[1]) : INFINITY;
    w.t2 = r.s[2] ? cross_at(w.nb2, r.S[2], r.inv[2]) : INFINITY;
    w.P = ((uint32_t)w.i2 * (uint32_t)r.ny + (uint32_t)w.i1) * R + (uint32_t)w.i0;
}

// Advances to the next voxel if the next crossing is before c_hi.  The axis
// with the smallest tMax moves, the lowest axis on a tie: x iff t0 is the
// minimum, else y iff t1 is, else z.  The three updates are short, mutually
// exclusive blocks, so lanes stepping different axes do not diverge.
__device__ __forceinline__ bool walker_next(Walker &w, const Ray &r, float c_hi) {
    const float tm = fminf(w.t0, fminf(w.t1, w.t2));
    if (!(tm < c_hi)) return false;
    const bool mx = (w.t0 == tm);
    const bool my = !mx && (w.t1 == tm);
    const bool mz = !mx && !my;
    if (mx) {
        w.i0 += r.s[0];
        w.P += (uint32_t)r.dP[0];
        w.nb0 = __fadd_rn(w.nb0, r.fs[0]);
        w.t0 = cross_at(w.nb0, r.S[0], r.inv[0]);
    }
    if (my) {
        w.i1 += r.s[1];
        w.P += (uint32_t)r.dP[1];
        w.nb1 = __fadd_rn(w.nb1, r.fs[1]);
        w.t1 = cross_at(w.nb1, r.S[1], r.inv[1]);
    }
    if (mz) {
        w.i2 += r.s[2];
        w.P += (uint32_t)r.dP[2];
        w.nb2 = __fadd_rn(w.nb2, r.fs[2]);
        w.t2 = cross_at(w.nb2, r.S[2], r.inv[2]);
    }
    return true;
}

__device__ __forceinline__ bool in_grid(const Walker &w, const Ray &r) {
    return (unsigned)w.i0 < (unsigned)r.nx && (unsigned)w.i1 < (unsigned)r.ny &&
           (unsigned)w.i2 < (unsigned)r.nz;
}

// True when an out-of-grid axis can no longer come back.
__device__ __forceinline__ bool gone(const Walker &w, const Ray &r) {
    return (w.i0 < 0 && r.s[0] <= 0) || (w.i0 >= r.nx && r.s[0] >= 0) || (w.i1 < 0 && r.s[1] <= 0) ||
           (w.i1 >= r.ny && r.s[1] >= 0) || (w.i2 < 0 && r.s[2] <= 0) || (w.i2 >= r.nz && r.s[2] >= 0);
}

__device__ __forceinline__ uint32_t pack_visit(const Walker &w, const Box &b) {
    const uint32_t dw = (uint32_t)((w.i0 >> 5) - b.bw0), dy = (uint32_t)(w.i1 - b.by0),
                   dz = (uint32_t)(w.i2 - b.bz0);
    if (dw < kBoxW && dy < kBoxY && dz < kBoxZ)
        return kBoxFlag | (((dz * kBoxY + dy) * kBoxW + dw) << 5) | ((uint32_t)w.i0 & 31u);
    return w.P;
}

template <class L>
__device__ __forceinline__ uint32_t occ_word(const FrameArgs &a, const uint32_t *occ_box, uint32_t p) {
    return (p & kBoxFlag) ? occ_box[(p >> 5) & (kBoxWords - 1)] : L::ld(a.occ_test + (p >> 5));
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
    if (m.key & (kBoxFlag >> 5)) atomicOr((m.traced ? box_tr : box_fr) + (m.key & (kBoxWords - 1)), m.bits);
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

// Two-pass walk for a lane whose slice does not fit its buffer: returns the
// index (among the slice's in-grid visits) of the first occupied voxel, or -1.
template <class L>
__device__ int walk_first_hit(const FrameArgs &a, const Ray &r, const int32_t n0[3], bool visit_start,
                              float c_hi, const Box &b, const uint32_t *occ_box, uint32_t R) {
    Walker w;
    walker_init(w, r, n0, R);
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
        for (int c = 0; c < kChunk; ++c) v[c] = c < n ? occ_word<L>(a, occ_box, p[c]) : 0u;
        int hit = -1;
#pragma unroll
        for (int c = kChunk - 1; c >= 0; --c)
            if (c < n && ((v[c] >> (p[c] & 31u)) & 1u)) hit = c;
        if (hit >= 0) return q + hit;
        q += n;
    }
    return -1;
}

// Pass 2 of the two-pass walk: marks the slice's in-grid visits.  EXACT:
// traced marks skip voxels the rays test as occupied (see rt_resolve).
template <bool EXACT, class L>
__device__ inline unsigned walk_marks(const FrameArgs &a, const Ray &r, const int32_t n0[3], bool visit_start,
                               float c_hi, const Box &b, int mode, int32_t hit_at, uint32_t *box_fr,
                               uint32_t *box_tr, const uint32_t *occ_box, uint32_t R) {
    Walker w;
    walker_init(w, r, n0, R);
    bool more = visit_start ? true : walker_next(w, r, c_hi);
    int32_t q = 0;
    Marks m;
    while (more) {
        if (in_grid(w, r)) {
            // mode: 0 all free, 1 free before hit_at and traced after, 2 all traced
            const bool traced = mode == 2 || (mode == 1 && q > hit_at);
            const uint32_t p = pack_visit(w, b);
            bool skip = mode == 1 && q == hit_at;
            if (EXACT && traced && !skip) skip = (occ_word<L>(a, occ_box, p) >> (p & 31u)) & 1u;
            if (!skip) marks_add(a, box_fr, box_tr, m, p, traced);
            ++q;
        } else if (gone(w, r)) {
            break;
        }
        more = walker_next(w, r, c_hi);
    }
    marks_flush(a, box_fr, box_tr, m);
    return (unsigned)q;
}

// The camera box of this frame: its origin, then staging of its occupancy
// words (zero outside the grid) and clearing of its marks.  CTA-cooperative;
// ends with a barrier.
__device__ __forceinline__ Box box_of(const float S[3]) {
    Box b;
    const int32_t cx0 = (int32_t)floorf(S[0]);
    b.bw0 = (cx0 >> 5) - ((cx0 & 31) < 16 ? 1 : 0);   // x words bw0, bw0+1
    b.by0 = (int32_t)floorf(S[1]) - kBoxY / 2;
    b.bz0 = (int32_t)floorf(S[2]) - kBoxZ / 2;
    return b;
}

// CLEAR: also clear the box's marks (without it, box_clear has done so
// earlier in the same CTA).
template <class L, bool CLEAR = true>
__device__ __forceinline__ void box_stage(const FrameArgs &a, const Box &b, uint32_t *box_fr, uint32_t *box_tr,
                                          uint32_t *occ_box) {
    for (int i = threadIdx.x; i < kBoxWords; i += kThreads) {
        if (CLEAR) {
            box_fr[i] = 0;
            box_tr[i] = 0;
        }
        const int32_t dw = i % kBoxW, dy = (i / kBoxW) % kBoxY, dz = i / (kBoxW * kBoxY);
        const int32_t wx = b.bw0 + dw, y = b.by0 + dy, z = b.bz0 + dz;
        uint32_t v = 0;
        if (wx >= 0 && wx < a.g.wx && y >= 0 && y < a.g.ny && z >= 0 && z < a.g.nz)
            v = L::ld(a.occ_test + ((uint32_t)z * (uint32_t)a.g.ny + (uint32_t)y) * (uint32_t)a.g.wx + wx);
        occ_box[i] = v;
    }
    __syncthreads();
}

// Clears the box's marks only; the next box_stage<L, false> ends with the
// barrier that makes the zeros visible to the CTA.
__device__ __forceinline__ void box_clear(uint32_t *box_fr, uint32_t *box_tr) {
    for (int i = threadIdx.x; i < kBoxWords; i += kThreads) {
        box_fr[i] = 0;
        box_tr[i] = 0;
    }
}

// ORs the box's marks into the planes.  CTA-cooperative; starts with a
// barrier so every lane's marks are in.
__device__ __forceinline__ void box_flush(const FrameArgs &a, const Box &b, const uint32_t *box_fr,
                                          const uint32_t *box_tr) {
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
    __syncthreads();
}

__device__ __forceinline__ void frame_start(const FrameArgs &a, float S[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) S[k] = __fdiv_rn(a.T.t[k], a.vs);
}

// One lane's share of one ray: the ray's constants, the lane's tau slice
// and its first voxel.  Depends on the pose and the grid's shape only.
struct Lane {
    Ray r;
    float c_hi;
    float t_out;   // the ray's first crossing of a grid face on its way out
    float t_box;   // the ray's first crossing of a camera-box face on its way out
    int32_t n0[3];
    int j;         // lane within the ray
    bool active;   // the lane has a ray
};

// Number of groups of kThreads / LPR rays a frame's bundle needs.
template <int LPR>
__device__ __forceinline__ int64_t rt_groups(const FrameArgs &a) {
    const int64_t nrays = (2 * (int64_t)a.hw + 1) * (2 * (int64_t)a.hh + 1);
    return (nrays + kThreads / LPR - 1) / (kThreads / LPR);
}

// Set-up of this thread's lane for bundle `bundle` of 32 / LPR neighbouring
// rays (ray ids bundle * 32 / LPR ..), taken by this thread's warp; lanes
// past the last ray are idle.  Reads no memory but its arguments.
template <int LPR>
__device__ __forceinline__ void rt_setup_bundle(const FrameArgs &a, const float S[3], const Box &bx, int64_t bundle,
                                                Lane &ln) {
    const int lane = threadIdx.x & 31;
    const int j = lane & (LPR - 1);
    const int32_t width = 2 * a.hw + 1;
    const int64_t nrays = (int64_t)width * (2 * a.hh + 1);
    const uint32_t R = 32u * (uint32_t)a.g.wx;   // plane bits per row
    constexpr int kRaysPerWarp = 32 / LPR;
    const int64_t ray = bundle * kRaysPerWarp + (lane / LPR);
    ln.active = ray < nrays;
    ln.j = j;
    Ray &r = ln.r;
    r.nx = a.g.nx;
    r.ny = a.g.ny;
    r.nz = a.g.nz;
    float absD[3];
    {
        int32_t ra = 0, rb = 0;
        if (ln.active) {
            if (nrays <= INT32_MAX) {   // 32-bit division where the ids allow it
                ra = (int32_t)((uint32_t)ray % (uint32_t)width) - a.hw;
                rb = (int32_t)((uint32_t)ray / (uint32_t)width) - a.hh;
            } else {
                ra = (int32_t)(ray % width) - a.hw;
                rb = (int32_t)(ray / width) - a.hh;
            }
        }
        const float fa = (float)ra, fb = (float)rb, fvd = (float)a.vd;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float d = __fadd_rn(__fadd_rn(__fmul_rn(a.T.R[k * 3 + 0], fa),
                                                __fmul_rn(a.T.R[k * 3 + 1], fb)),
                                      __fmul_rn(a.T.R[k * 3 + 2], fvd));
            absD[k] = fabsf(d);
            r.S[k] = S[k];
            r.inv[k] = 0.0f;
            r.s[k] = 0;
            if (d != 0.0f) {
                const float q = __frcp_rn(d);
                if (isfinite(q)) {
                    r.inv[k] = q;
                    r.s[k] = d > 0.0f ? 1 : -1;
                }
            }
            r.fs[k] = (float)r.s[k];
        }
        r.dP[0] = r.s[0];
        r.dP[1] = r.s[1] * (int32_t)R;
        r.dP[2] = r.s[2] * (int32_t)R * a.g.ny;
        r.dPb[0] = r.s[0];
        r.dPb[1] = r.s[1] * (32 * kBoxW);
        r.dPb[2] = r.s[2] * (32 * kBoxW * kBoxY);
    }

    // Exit times.  A crossing of axis k's face F happens at exactly
    // cross_at((float)F, S_k, 1/D_k): the walker keeps F as an exact float
    // and evaluates the same expression.  So a crossing with t below the
    // first outward grid (box) face crossing keeps a voxel that is inside
    // the grid (box) inside it.
    {
        const float glo[3] = {0.0f, 0.0f, 0.0f};
        const float ghi[3] = {(float)a.g.nx, (float)a.g.ny, (float)a.g.nz};
        const float blo[3] = {(float)(32 * bx.bw0), (float)bx.by0, (float)bx.bz0};
        const float bhi[3] = {(float)(32 * (bx.bw0 + kBoxW)), (float)(bx.by0 + kBoxY), (float)(bx.bz0 + kBoxZ)};
        float to = INFINITY, tb = INFINITY;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (r.s[k] != 0) {
                to = fminf(to, cross_at(r.s[k] > 0 ? ghi[k] : glo[k], S[k], r.inv[k]));
                tb = fminf(tb, cross_at(r.s[k] > 0 ? bhi[k] : blo[k], S[k], r.inv[k]));
            }
        }
        ln.t_out = to;
        ln.t_box = tb;
    }

    // this lane's slice of tau: the in-grid part of the segment is cut
    // into LPR equal pieces (any cuts give the same visits as long as
    // neighbouring lanes agree on them and the last lane ends at 1)
    float c_lo;
    {
        float ts = 0.0f, te = 1.0f;
        const float nk[3] = {(float)a.g.nx, (float)a.g.ny, (float)a.g.nz};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (r.s[k] != 0) {
                const float t_lo = __fmul_rn(__fsub_rn(r.s[k] > 0 ? 0.0f : nk[k], S[k]), r.inv[k]);
                const float t_hi = __fmul_rn(__fsub_rn(r.s[k] > 0 ? nk[k] : 0.0f, S[k]), r.inv[k]);
                ts = fmaxf(ts, t_lo);
                te = fminf(te, t_hi);
            }
        }
        if (!(te > ts)) {
            ts = 0.0f;
            te = 1.0f;
        }
        const float span = __fsub_rn(te, ts);
        c_lo = __fadd_rn(ts, __fmul_rn(span, (float)j / (float)LPR));
        ln.c_hi = (j == LPR - 1) ? 1.0f : __fadd_rn(ts, __fmul_rn(span, (float)(j + 1) / (float)LPR));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) ln.n0[k] = j > 0 ? crossings_before(r, k, absD[k], c_lo) : 0;
}

// Set-up of this thread's lane for group `group` of the G >= rt_groups
// groups the frame's rays are spread over.  Warp w of group g takes bundle
// w * G + g, so the warps of one group sample rows spread over the whole
// image and groups get similar amounts of work (rays of rows near the
// image's top and bottom leave the grid early).  With G above the frame's
// own group count the idle bundles spread evenly too.
template <int LPR>
__device__ __forceinline__ void rt_setup(const FrameArgs &a, const float S[3], const Box &bx, int64_t group,
                                         int64_t G, Lane &ln) {
    rt_setup_bundle<LPR>(a, S, bx, (int64_t)(threadIdx.x >> 5) * G + group, ln);
}

// One crossing of the fast walker (the caller has checked that tm, the
// smallest of t0..t2, is below its limit): the axis with the smallest time
// moves, the lowest axis on a tie, as in walker_next.  PB: also step the
// packed box index.
template <bool PB>
__device__ __forceinline__ void fast_step(const Ray &r, float tm, float &t0, float &t1, float &t2, float &nb0,
                                          float &nb1, float &nb2, uint32_t &P, uint32_t &Pb) {
    const bool mx = (t0 == tm);
    const bool my = !mx && (t1 == tm);
    const bool mz = !mx && !my;
    if (mx) {
        nb0 = __fadd_rn(nb0, r.fs[0]);
        t0 = cross_at(nb0, r.S[0], r.inv[0]);
        P += (uint32_t)r.dP[0];
        if (PB) Pb += (uint32_t)r.dPb[0];
    }
    if (my) {
        nb1 = __fadd_rn(nb1, r.fs[1]);
        t1 = cross_at(nb1, r.S[1], r.inv[1]);
        P += (uint32_t)r.dP[1];
        if (PB) Pb += (uint32_t)r.dPb[1];
    }
    if (mz) {
        nb2 = __fadd_rn(nb2, r.fs[2]);
        t2 = cross_at(nb2, r.S[2], r.inv[2]);
        P += (uint32_t)r.dP[2];
        if (PB) Pb += (uint32_t)r.dPb[2];
    }
}

// Pass 1 of a lane: its in-grid visits in walk order, as runs, into its
// buffer column col[q * kThreads], box-packed while the walk is inside the
// camera box, plane bit indices after that.  Returns false when the column
// overflows.
//
// Exact steps (walker_next, with in-grid tests) lead to the first in-grid
// voxel.  From there the walk runs without tests while its next crossing is
// before t_lim = min(c_hi, t_out): such a crossing keeps the voxel in the
// grid, and one before t_box keeps a voxel that is in the box in it (the
// box may be left early on a tie, which only means that later box voxels
// are marked in the planes directly).  All lanes run the same loop, so a
// warp stays converged.  If the walk leaves the grid within the slice,
// exact steps finish it.
__device__ __forceinline__ bool walk_record(const Ray &r, const Lane &ln, const int32_t n0[3], bool visit_start,
                                            const Box &b, uint32_t R, uint32_t *col, int32_t &nent,
                                            int32_t &nvis) {
    const float c_hi = ln.c_hi;
    Walker w;
    walker_init(w, r, n0, R);
    bool more = visit_start ? true : walker_next(w, r, c_hi);
    while (more && !in_grid(w, r)) {
        if (gone(w, r)) return true;
        more = walker_next(w, r, c_hi);
    }
    if (!more) return true;

    float t0 = w.t0, t1 = w.t1, t2 = w.t2, nb0 = w.nb0, nb1 = w.nb1, nb2 = w.nb2;
    uint32_t P = w.P;
    const uint32_t dw = (uint32_t)((w.i0 >> 5) - b.bw0), dy = (uint32_t)(w.i1 - b.by0), dz = (uint32_t)(w.i2 - b.bz0);
    bool inb = dw < kBoxW && dy < kBoxY && dz < kBoxZ;
    uint32_t Pb = kBoxFlag | (((dz * kBoxY + dy) * kBoxW + dw) << 5) | ((uint32_t)w.i0 & 31u);
    const float t_lim = fminf(c_hi, ln.t_out), t_b = ln.t_box;
    uint32_t cur = inb ? Pb : P;   // the pending run, in slot `last`
    int32_t last = 0;
    col[0] = cur;
    nvis = 1;
    float tm;
    for (;;) {
        tm = fminf(t0, fminf(t1, t2));
        if (!(tm < t_lim)) break;
        inb = inb && tm < t_b;
        fast_step<true>(r, tm, t0, t1, t2, nb0, nb1, nb2, P, Pb);
        if (!run_add(col, last, cur, inb ? Pb : P)) return false;
        ++nvis;
    }
    nent = last + 1;
    if (!(tm < c_hi)) return true;   // the next crossing is the next lane's

    // the walk leaves the grid within this slice: exact steps from here
    w.t0 = t0;
    w.t1 = t1;
    w.t2 = t2;
    w.nb0 = nb0;
    w.nb1 = nb1;
    w.nb2 = nb2;
    w.i0 = (int32_t)nb0 - (r.s[0] > 0 ? 1 : 0);
    w.i1 = (int32_t)nb1 - (r.s[1] > 0 ? 1 : 0);
    w.i2 = (int32_t)nb2 - (r.s[2] > 0 ? 1 : 0);
    w.P = P;
    more = walker_next(w, r, c_hi);
    while (more) {
        if (in_grid(w, r)) {
            if (!run_add(col, last, cur, w.P)) return false;
            ++nvis;
        } else if (gone(w, r)) {
            break;
        }
        more = walker_next(w, r, c_hi);
    }
    nent = last + 1;
    return true;
}

// Index of the first recorded run that holds a voxel the rays see
// occupied, or -1, and in hit_bit that voxel's bit; kChunk occupancy words
// in flight at a time (box runs read the staged box).
template <class L>
__device__ __forceinline__ int32_t first_hit(const FrameArgs &a, const uint32_t *occ_box, const uint32_t *col,
                                             int32_t nent, int32_t sx, uint32_t &hit_bit) {
    for (int32_t q0 = 0; q0 < nent; q0 += kChunk) {
        uint32_t e[kChunk], v[kChunk];
#pragma unroll
        for (int c = 0; c < kChunk; ++c) e[c] = q0 + c < nent ? col[(q0 + c) * kThreads] : 0u;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
            // both sources without a branch: the box word (any index is in
            // range) and, for a plane run, the plane word
            const bool isb = (e[c] & kBoxFlag) != 0;
            const uint32_t vb = occ_box[(e[c] >> 5) & (kBoxWords - 1)];
            uint32_t vg = 0;
            if (!isb && q0 + c < nent) vg = L::ld(a.occ_test + ((e[c] >> 5) & (uint32_t)(kRunWords - 1)));
            v[c] = (isb ? vb : vg) & run_mask(e[c], sx);
        }
        int32_t hit = -1;
        uint32_t h = 0;
#pragma unroll
        for (int c = kChunk - 1; c >= 0; --c)
            if (q0 + c < nent && v[c]) {
                hit = q0 + c;
                h = v[c];
            }
        if (hit >= 0) {
            hit_bit = sx < 0 ? 31u - (uint32_t)__clz(h) : (uint32_t)(__ffs(h) - 1);
            return hit;
        }
    }
    return -1;
}

// Marks the recorded runs: runs before f_q free, run f_q free before bit
// f_bit (in walk order) and traced from it on, later runs traced.  One
// atomicOr per run and kind, to the box arrays or the planes.  EXACT:
// traced marks leave out voxels the rays test as occupied (see rt_resolve).
template <bool EXACT, class L>
__device__ __forceinline__ void mark_runs(const FrameArgs &a, uint32_t *box_fr, uint32_t *box_tr,
                                          const uint32_t *occ_box, const uint32_t *col, int32_t nent, int32_t f_q,
                                          uint32_t f_bit, int32_t sx) {
    for (int32_t q = 0; q < nent; ++q) {
        const uint32_t e = col[q * kThreads];
        const uint32_t m = run_mask(e, sx);
        uint32_t fr = q < f_q ? m : 0u;
        if (q == f_q) fr = m & bits_before(f_bit, sx);
        uint32_t tr = m & ~fr;
        if (e & kBoxFlag) {
            const uint32_t i = (e >> 5) & (kBoxWords - 1);
            if (EXACT && tr) tr &= ~occ_box[i];
            if (fr) atomicOr(box_fr + i, fr);
            if (tr) atomicOr(box_tr + i, tr);
        } else {
            const uint32_t wi = (e >> 5) & (uint32_t)(kRunWords - 1);
            if (EXACT && tr) tr &= ~L::ld(a.occ_test + wi);
            if (fr) atomicOr(a.pl.fr + wi, fr);
            if (tr) atomicOr(a.pl.tr + wi, tr);
        }
    }
}

// What pass 1 leaves for the rest of a lane's walk.
struct Pass1 {
    int32_t nent;   // runs recorded in the lane's buffer column
    int32_t nvis;   // visits they hold
    bool ovf;       // the slice does not fit the column: walk twice instead
};

// Pass 1 of a group's walk, by all threads of the CTA: each lane walks its
// slice once and keeps its in-grid visits in its column of `buf` as runs
// (box-packed runs first, then plane bit indices).  Reads no global memory, so it may
// run before the occupancy the visits are tested against is ready.
// Warp-synchronous, like rt_walk.
__device__ __forceinline__ Pass1 rt_record(const FrameArgs &a, const Lane &ln, const Box &b, int buffered,
                                           uint32_t *buf) {
    Pass1 p1{0, 0, !buffered};
    const bool visit_start = ln.j == 0 && !(a.lit & kLitSkipStart);
    // (each phase starts with the warp reconverged, so that its lanes run
    // the phase's loop together rather than in groups)
    __syncwarp();
    if (ln.active && !p1.ovf)
        p1.ovf = !walk_record(ln.r, ln, ln.n0, visit_start, b, 32u * (uint32_t)a.g.wx, buf + threadIdx.x, p1.nent,
                              p1.nvis);
    __syncwarp();
    return p1;
}

// The rest of a group's walk after rt_record: the first occupied visit of
// each lane, the ray's first lane that met one, then the marks.  Returns
// this thread's in-grid visits.  Warp-synchronous (every lane of every warp
// must call it; the CTA need not be in step).
// Traced marks after a ray's first occupied voxel are written without
// re-reading the occupancy; a traced mark on an occupied voxel is then
// overridden by K4's precedence.  That holds whenever the tested plane is a
// subset of occ_inf; for a tested plane that is not (the literal loc_grid
// reading, whose resolve also puts traced above occupied) EXACT re-reads it
// and leaves tested-occupied voxels unmarked, as Alg. 2 does.
template <int LPR, class L, bool EXACT = false>
__device__ __forceinline__ unsigned rt_resolve(const FrameArgs &a, const Lane &ln, const Box &b, const Pass1 &p1,
                                               uint32_t *box_fr, uint32_t *box_tr, const uint32_t *occ_box,
                                               uint32_t *buf) {
    const int lane = threadIdx.x & 31;
    const int j = ln.j;
    const bool active = ln.active;
    const Ray &r = ln.r;
    const float c_hi = ln.c_hi;
    const int32_t *n0 = ln.n0;
    const uint32_t R = 32u * (uint32_t)a.g.wx;
    const uint32_t *col = buf + threadIdx.x;
    const int32_t nent = p1.nent;
    const bool ovf = p1.ovf;
    const bool visit_start = j == 0 && !(a.lit & kLitSkipStart);
    unsigned visits = 0;

    // ---- first occupied visit of this lane -----------------------------
    // (a run index with its bit for a buffered lane, a visit index for one
    // that walks twice)
    int32_t hit_at = -1;
    uint32_t hit_bit = 0;
    if (active && !ovf) hit_at = first_hit<L>(a, occ_box, col, nent, r.s[0], hit_bit);
    if (active && ovf) hit_at = walk_first_hit<L>(a, r, n0, visit_start, c_hi, b, occ_box, R);

    // ---- first lane of this ray with an occupied voxel ---------------
    const unsigned hits = __ballot_sync(kFull, hit_at >= 0);
    const int gbase = lane & ~(LPR - 1);
    const unsigned gmask = (LPR == 32) ? kFull : (((1u << LPR) - 1u) << gbase);
    const unsigned gh = hits & gmask;
    const int F = gh ? (__ffs(gh) - 1 - gbase) : LPR;
    const int mode = j < F ? 0 : (j == F ? 1 : 2);

    // ---- pass 2: mark free / traced -----------------------------------
    if (active && !ovf) {
        // free before the ray's first occupied voxel, traced from it on
        // (its own traced mark is overridden by K4: it is in occ_inf)
        mark_runs<EXACT, L>(a, box_fr, box_tr, occ_box, col, nent, mode == 0 ? nent : (mode == 1 ? hit_at : -1),
                            hit_bit, r.s[0]);
        visits += (unsigned)p1.nvis;
    } else if (active) {
        visits += walk_marks<EXACT, L>(a, r, n0, visit_start, c_hi, b, mode, hit_at, box_fr, box_tr, occ_box, R);
    }
    return visits;
}

// The walk of one group of rays set up by rt_setup, by all threads of the
// CTA; `buf` is this CTA's visit buffer (kRtBuf columns of kThreads words).
// Returns this thread's in-grid visits.  Warp-synchronous.
template <int LPR, class L, bool EXACT = false>
__device__ __forceinline__ unsigned rt_walk(const FrameArgs &a, const Lane &ln, const Box &b, int buffered,
                                            uint32_t *box_fr, uint32_t *box_tr, const uint32_t *occ_box,
                                            uint32_t *buf) {
    const Pass1 p1 = rt_record(a, ln, b, buffered, buf);
    return rt_resolve<LPR, L, EXACT>(a, ln, b, p1, box_fr, box_tr, occ_box, buf);
}

// One bundle of rays, by one warp: rt_setup_bundle then rt_walk.
template <int LPR, class L, bool EXACT = false>
__device__ __forceinline__ unsigned rt_bundle(const FrameArgs &a, const float S[3], const Box &b, int64_t bundle,
                                              int buffered, uint32_t *box_fr, uint32_t *box_tr,
                                              const uint32_t *occ_box, uint32_t *buf) {
    Lane ln;
    rt_setup_bundle<LPR>(a, S, b, bundle, ln);
    return rt_walk<LPR, L, EXACT>(a, ln, b, buffered, box_fr, box_tr, occ_box, buf);
}

// One group of rays: rt_setup then rt_walk.
template <int LPR, class L, bool EXACT = false>
__device__ __forceinline__ unsigned rt_group(const FrameArgs &a, const float S[3], const Box &b, int64_t group,
                                             int64_t G, int buffered, uint32_t *box_fr, uint32_t *box_tr,
                                             const uint32_t *occ_box, uint32_t *buf) {
    Lane ln;
    rt_setup<LPR>(a, S, b, group, G, ln);
    return rt_walk<LPR, L, EXACT>(a, ln, b, buffered, box_fr, box_tr, occ_box, buf);
}

}  // namespace rt
}  // namespace vg
