// vg_units.cuh -- the work of K1, K2, K4 and K5 as device functions over one
// unit of work, shared by the one-kernel-per-step launches (k_*.cu) and the
// fused persistent launch (k_batch.cu).
//
// Loads of data that an earlier phase of the same launch may have written go
// through a load policy: LoadRO (the read-only path, for one-step kernels
// whose inputs were written by earlier launches and are not written by the
// kernel), LoadPlain (ordinary loads, for data the kernel itself updates)
// or LoadL2 (loads that skip the SM's L1, for phases of a fused launch that
// read what other SMs wrote before a grid barrier).
#pragma once

#include "vg_internal.cuh"

namespace vg {
namespace units {

constexpr unsigned kFull = 0xffffffffu;

struct LoadRO {
    template <class T>
    static __device__ __forceinline__ T ld(const T *p) { return __ldg(p); }
};

struct LoadPlain {
    template <class T>
    static __device__ __forceinline__ T ld(const T *p) { return *p; }
};

struct LoadL2 {
    template <class T>
    static __device__ __forceinline__ T ld(const T *p) { return __ldcg(p); }
};

// ---------------------------------------------------------------------------
// K1: transform and voxelize (Sec. IV-B, Alg. 1 before the inflation loops).
//
// Each thread reads four consecutive pixels of the row-major depth image
// (one 16-byte float4 or 8-byte ushort4 load when aligned), back-projects
// the valid ones with the pinhole model, transforms them by T^v_c and sets
// their voxel's bit in the occ_raw plane.  Neighbouring pixels often land in
// the same 32-voxel word, so each warp de-duplicates its words with a
// segmented OR-scan across lanes before one atomicOr per run of lanes that
// share a word: the plane is bit-packed, so concurrent sets need an atomic,
// but only about one per distinct word per warp.
//
// Arithmetic follows the oracle's order with one IEEE rounding per operation
// (explicit __f*_rn intrinsics; the translation units are also built with
// -fmad=false):
//   xc = ((u - cx) * d) / fx,  yc = ((v - cy) * d) / fy,  zc = d
//   g_k = (((R_k0 xc + R_k1 yc) + R_k2 zc) + t_k) / vox_size
//   kept iff 0 <= g_k < N_k on every axis; voxel = floor(g).
// ---------------------------------------------------------------------------
constexpr uint32_t kNoWord = 0xffffffffu;

// Returns the plane word of the point's voxel and its bit, or kNoWord.
__device__ __forceinline__ uint32_t point_word(const FrameArgs &a, float x, float y, float z, uint32_t &bit) {
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

__device__ __forceinline__ uint32_t pixel_word(const FrameArgs &a, float d, int32_t u, int32_t v, uint32_t &bit) {
    if (!(isfinite(d) && d > 0.0f && d <= a.depth_max)) return kNoWord;
    float xc = __fdiv_rn(__fmul_rn(__fsub_rn((float)u, a.cx), d), a.fx);
    float yc = __fdiv_rn(__fmul_rn(__fsub_rn((float)v, a.cy), d), a.fy);
    return point_word(a, xc, yc, d, bit);
}

// ORs `bit` into plane[key] for every lane, with one atomicOr per run of
// consecutive lanes that share a word: an inclusive OR-scan over lanes that
// only pulls from lanes with the same key, after which the last lane of each
// run holds the run's bits.  Lanes whose keys match but are not adjacent may
// fold bits into each other; that is harmless, they name the same word.
// Every lane of the warp must call this (keys of idle lanes are kNoWord).
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
__device__ __forceinline__ void count_points(const FrameArgs &a, unsigned kept) {
    if (!a.stats) return;
    const unsigned total = __reduce_add_sync(kFull, kept);
    if ((threadIdx.x & 31) == 0 && total) atomicAdd(a.stats + 1, (unsigned long long)total);
}

// Pixels 4t .. 4t+3 of the image.  DT: 0 = f32, 1 = u16.  VEC: the image
// base is aligned for a 4-pixel load.  Warp-synchronous: every lane of the
// warp must call this (threads past the image do nothing).
template <int DT, bool VEC>
__device__ __forceinline__ void voxelize_depth_thread(const FrameArgs &a, int64_t t) {
    const int64_t npix = (int64_t)a.W * a.H;
    const int64_t p0 = t * 4;
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
    // images hold fewer than 2^31 pixels, so p0 (at most 1023 past the last
    // one) fits 32 bits
    const uint32_t q0 = (uint32_t)p0;
    int32_t v = (int32_t)(q0 / (uint32_t)a.W), u = (int32_t)(q0 - (uint32_t)v * (uint32_t)a.W);
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
    count_points(a, kept);
}

// Point i of the cloud.  Warp-synchronous like voxelize_depth_thread.
__device__ __forceinline__ void voxelize_points_thread(const FrameArgs &a, int64_t i) {
    uint32_t key = kNoWord, bit = 0;
    if (i < a.npts) {
        const float x = __ldg(a.xyz + 3 * i + 0);
        const float y = __ldg(a.xyz + 3 * i + 1);
        const float z = __ldg(a.xyz + 3 * i + 2);
        if (isfinite(x) && isfinite(y) && isfinite(z)) key = point_word(a, x, y, z, bit);
    }
    warp_set_bits(a.pl.occ_raw, key, bit);
    count_points(a, key != kNoWord);
}

// ---------------------------------------------------------------------------
// K2: inflation (Sec. IV-B, Alg. 1, the three nested loops around each
// point).  Stamping the cube of half side r around every occupied voxel is
// the Chebyshev dilation of occ_raw, which separates into three 1-D OR
// filters of width 2r+1 along x, y and z.  Clipping at the grid faces falls
// out of the zero fill outside the grid.
//
// One CTA produces a TXW x TY x TZ tile of 32-bit plane words.  It stages
// the tile plus its halo (one word each side in x, r rows in y, r slices in
// z) in shared memory, then runs the x pass (funnel shifts across word
// boundaries), the y pass and the z pass in shared memory and writes the
// tile of occ_inf once.  Bits beyond Nx are cleared so the plane's padding
// stays zero.  R > 0 is a compile-time radius (all index arithmetic folds);
// R == 0 takes the radius r_rt at run time.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t dilate_x(uint32_t prev, uint32_t cur, uint32_t next, int r) {
    uint32_t acc = cur;
#pragma unroll 4
    for (int d = 1; d <= r; ++d) {
        acc |= __funnelshift_r(cur, next, d);   // voxel x+d -> x
        acc |= __funnelshift_l(prev, cur, d);   // voxel x-d -> x
    }
    return acc;
}

template <int R, int TXW, int TY, int TZ>
__host__ __device__ constexpr size_t inflate_smem_words(int r) {
    return (size_t)(TZ + 2 * r) * (TY + 2 * r) * (TXW + 2) + (size_t)(TZ + 2 * r) * (TY + 2 * r) * TXW;
}

// The x, y and z passes of a tile whose raw words are staged in shared
// memory: word w0 - 1 + lx of row y0 - r + ly, slice z0 - r + lz at
// st[(lz * hy + ly) * sx + ox + lx], lx in [0, TXW + 2), with zeros outside
// the grid.  buf1 (hz * hy * TXW words) must not overlap the staged words;
// the y pass reuses the staged words' memory.  CTA-cooperative (256
// threads); ends with a barrier.
template <int R, int TXW, int TY, int TZ>
__device__ __forceinline__ void inflate_passes(const PlaneGeom &g, uint32_t *out, const int r_rt, int tile_x,
                                               int tile_y, int tile_z, uint32_t *st, int sx, int ox, uint32_t *buf1) {
    const int r = R > 0 ? R : r_rt;
    const int hy = TY + 2 * r, hz = TZ + 2 * r;
    const int w0 = tile_x * TXW, y0 = tile_y * TY, z0 = tile_z * TZ;

    // x pass, clearing bits past the end of the row
    const int n1 = hz * hy * TXW;
    for (int i = threadIdx.x; i < n1; i += 256) {
        const int lx = i % TXW, row = i / TXW;
        const uint32_t *b = st + row * sx + ox + lx;
        uint32_t v = dilate_x(b[0], b[1], b[2], r);
        const int valid = g.nx - 32 * (w0 + lx);
        if (valid < 32) v &= valid > 0 ? ((1u << valid) - 1u) : 0u;
        buf1[i] = v;
    }
    __syncthreads();

    // y pass into the staged words' memory (now free): hz * TY * TXW
    uint32_t *buf2 = st;
    const int n2 = hz * TY * TXW;
    for (int i = threadIdx.x; i < n2; i += 256) {
        const int lx = i % TXW, rest = i / TXW, ly = rest % TY, lz = rest / TY;
        const uint32_t *b = buf1 + (lz * hy + ly) * TXW + lx;
        uint32_t v = 0;
        for (int d = 0; d <= 2 * r; ++d) v |= b[d * TXW];
        buf2[i] = v;
    }
    __syncthreads();

    // z pass to global
    constexpr int n3 = TZ * TY * TXW;
    for (int i = threadIdx.x; i < n3; i += 256) {
        const int lx = i % TXW, rest = i / TXW, ly = rest % TY, lz = rest / TY;
        const int w = w0 + lx, y = y0 + ly, z = z0 + lz;
        if (w >= g.wx || y >= g.ny || z >= g.nz) continue;
        const uint32_t *b = buf2 + (lz * TY + ly) * TXW + lx;
        uint32_t v = 0;
        for (int d = 0; d <= 2 * r; ++d) v |= b[d * TY * TXW];
        out[((int64_t)z * g.ny + y) * g.wx + w] = v;
    }
    __syncthreads();   // the tile's shared memory may be reused right away
}

// CTA-cooperative: every thread of the (256-thread) CTA must call this.
// The threads stage the tile's raw words with halo themselves.
template <int R, int TXW, int TY, int TZ, class L, int STAGE_UNROLL = 8>
__device__ __forceinline__ void inflate_tile(const PlaneGeom &g, const uint32_t *raw, uint32_t *out, const int r_rt,
                                             int tile_x, int tile_y, int tile_z, uint32_t *sm) {
    const int r = R > 0 ? R : r_rt;
    const int hx = TXW + 2, hy = TY + 2 * r, hz = TZ + 2 * r;
    uint32_t *buf0 = sm;                          // hz * hy * hx: raw with halo
    uint32_t *buf1 = sm + hz * hy * hx;           // hz * hy * TXW: x-dilated
    const int w0 = tile_x * TXW, y0 = tile_y * TY, z0 = tile_z * TZ;

    // stage raw words (zero outside the grid)
    const int n0 = hz * hy * hx;
#pragma unroll STAGE_UNROLL
    for (int i = threadIdx.x; i < n0; i += 256) {
        const int lx = i % hx, rest = i / hx, ly = rest % hy, lz = rest / hy;
        const int w = w0 + lx - 1, y = y0 + ly - r, z = z0 + lz - r;
        uint32_t v = 0;
        if (w >= 0 && w < g.wx && y >= 0 && y < g.ny && z >= 0 && z < g.nz)
            v = L::ld(raw + ((int64_t)z * g.ny + y) * g.wx + w);
        buf0[i] = v;
    }
    __syncthreads();
    inflate_passes<R, TXW, TY, TZ>(g, out, r_rt, tile_x, tile_y, tile_z, buf0, hx, 0, buf1);
}

// ---------------------------------------------------------------------------
// K4: merge the measurement grid into loc_grid (Sec. IV-D, Alg. 3).
//
// One 32-voxel plane word per thread.  The voxel's measurement state is
// resolved from the three planes with precedence
//   occupied (occ_inf) > free (fr) > unknown-and-traced (tr) > unknown,
// and Alg. 3 writes it to loc_grid wherever it is not unknown.  loc_grid is
// ring-addressed (Ring): a re-centre only moves the ring, and the voxels it
// brings into the grid are set to unknown by the next merge.  A word with no
// bit set in any plane and no voxel brought in touches neither loc_grid nor
// the planes, so the pass reads the bit planes everywhere but writes
// loc_grid only inside the measured frustum and the slabs a re-centre
// brought in, and never reads it.  Every plane word read non-zero is
// cleared, which leaves all planes zero for the next frame (occ_raw is a
// subset of occ_inf, so its non-zero words are cleared too).
// ---------------------------------------------------------------------------
// RAYS_LAST: the literal loc_grid reading, in which the rays' marks replace
// the measurement's occupied marks (free > traced > occupied).
//
// The resolve works on four voxels at once.  With the state codes
// OCC = 2, FREE = 1, TRACED = 3, a word's codes are two bit masks, hi (bit
// 1 of each code: occupied or traced) and lo (bit 0: free or traced), and
// known marks the voxels that are not unknown.  expand4 spreads a nibble
// into one 0/1 byte per bit (bit i times 2^(7i) lands on bit 8i; no other
// product of the multiply lands on a byte's low bit).  merge4 then writes
// the codes of voxels 4m..4m+3 over the four old bytes where known.
__device__ __forceinline__ uint32_t expand4(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

template <bool RAYS_LAST = false>
__device__ __forceinline__ void code_masks(uint32_t oc, uint32_t f, uint32_t t, uint32_t &hi, uint32_t &lo,
                                           uint32_t &known) {
    uint32_t occ, fr, tr;
    if (!RAYS_LAST) {
        occ = oc;
        fr = f & ~oc;
        tr = t & ~(f | oc);
    } else {
        fr = f;
        tr = t & ~f;
        occ = oc & ~(f | t);
    }
    hi = occ | tr;
    lo = fr | tr;
    known = occ | fr | tr;
}

__device__ __forceinline__ uint32_t merge4(uint32_t hi, uint32_t lo, uint32_t known, int m, uint32_t old) {
    const int s = 4 * m;
    const uint32_t kb = expand4((known >> s) & 15u);
    const uint32_t code = (expand4((hi >> s) & 15u) << 1) | expand4((lo >> s) & 15u);
    return (old & ~(kb * 0xffu)) | code;
}

// The ring position of coordinate c (0 <= c < n) moved by r (0 <= r < n).
__device__ __forceinline__ int32_t ring_at(int32_t c, int32_t r, int32_t n) {
    const int32_t v = c + r;
    return v >= n ? v - n : v;
}

// Bits of the voxels of a row word (x0 .. x0 + nbits - 1, row (y, z)) that a
// re-centre brought into the grid: the whole word if its row did, else the
// part of it inside [elo[0], ehi[0]).
__device__ __forceinline__ uint32_t entering_bits(const Ring &R, int32_t x0, int32_t y, int32_t z, int nbits) {
    const uint32_t all = nbits >= 32 ? 0xffffffffu : ((1u << nbits) - 1u);
    if ((y >= R.elo[1] && y < R.ehi[1]) || (z >= R.elo[2] && z < R.ehi[2])) return all;
    const int32_t lo = max(R.elo[0] - x0, 0), hi = min(R.ehi[0] - x0, nbits);
    if (hi <= lo) return 0u;
    const uint32_t below_hi = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
    return below_hi & ~((1u << lo) - 1u);
}

// Writes codes[v] (byte v of the 8 words codes[0..7], codes[8] = 0) to
// p[v - v0] for the voxels v in [v0, v1) whose bit is set in touch: aligned
// 4-byte stores where all four bytes are this word's and touched, byte
// stores elsewhere, so that no store reaches a byte of another word.
__device__ __forceinline__ void store_codes(uint8_t *p, int v0, int v1, const uint32_t codes[9], uint32_t touch) {
    int v = v0;
    // head: bytes up to the first 4-byte boundary of the buffer
    while (v < v1 && (reinterpret_cast<uintptr_t>(p + (v - v0)) & 3u) != 0) {
        if ((touch >> v) & 1u) p[v - v0] = (uint8_t)(codes[v >> 2] >> (8 * (v & 3)));
        ++v;
    }
    for (; v + 4 <= v1; v += 4) {
        const uint32_t t4 = (touch >> v) & 15u;
        if (t4 == 0) continue;
        const uint32_t w = __funnelshift_r(codes[v >> 2], codes[(v >> 2) + 1], 8 * (v & 3));
        if (t4 == 15u) {
            *reinterpret_cast<uint32_t *>(p + (v - v0)) = w;
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if ((t4 >> b) & 1u) p[v - v0 + b] = (uint8_t)(w >> (8 * b));
        }
    }
    for (; v < v1; ++v)
        if ((touch >> v) & 1u) p[v - v0] = (uint8_t)(codes[v >> 2] >> (8 * (v & 3)));
}

// K4 of one plane word w (the 32 voxels x0 .. x0 + 31 of one row of the
// grid in its own frame) into the ring-addressed loc: the measurement's
// codes where a plane marks a voxel, unknown where a re-centre brought the
// voxel in and no plane marks it, nothing elsewhere.  loc is only written,
// never read.  The row's voxels from x0 on sit at buffer x ring_at(x0, r[0])
// up to the row's end, the rest (when the ring wraps inside the word) from
// buffer x 0.  Clears the plane words it reads non-zero.
template <class L, bool RAYS_LAST = false>
__device__ __forceinline__ void merge_word(const PlaneGeom &g, const Planes &pl, uint8_t *loc, const Ring &R,
                                           int64_t w) {
    if (w >= g.words) return;
    // rows are a power of two of words; grids hold fewer than 2^31 voxels
    const int32_t wxi = (int32_t)(w & (g.wx - 1));
    const uint32_t row = (uint32_t)(w >> (__ffs(g.wx) - 1));
    const int32_t x0 = wxi * 32;
    if (x0 >= g.nx) return;   // padding word, always zero
    const uint32_t oc = L::ld(pl.occ_inf + w), f = L::ld(pl.fr + w), t = L::ld(pl.tr + w);
    const uint32_t any = oc | f | t;
    const int32_t y = (int32_t)(row % (uint32_t)g.ny), z = (int32_t)(row / (uint32_t)g.ny);
    const int nbits = min(32, g.nx - x0);
    const uint32_t ent = entering_bits(R, x0, y, z, nbits);
    if ((any | ent) == 0) return;
    uint32_t codes[9];
    codes[8] = 0;
    uint32_t touch = ent;
    if (any) {
        uint32_t hi, lo, known;
        code_masks<RAYS_LAST>(oc, f, t, hi, lo, known);
#pragma unroll
        for (int m = 0; m < 8; ++m) codes[m] = merge4(hi, lo, known, m, 0u);
        touch |= known;
    } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) codes[m] = 0u;
    }
    uint8_t *rowp = loc + ((int64_t)ring_at(z, R.r[2], g.nz) * g.ny + ring_at(y, R.r[1], g.ny)) * g.nx;
    const int32_t xb = ring_at(x0, R.r[0], g.nx);
    const int n1 = min(nbits, g.nx - xb);
    store_codes(rowp + xb, 0, n1, codes, touch);
    if (n1 < nbits) store_codes(rowp, n1, nbits, codes, touch);   // voxel v at rowp[v - n1]
    if (oc) {
        pl.occ_inf[w] = 0;
        pl.occ_raw[w] = 0;
    }
    if (f) pl.fr[w] = 0;
    if (t) pl.tr[w] = 0;
}

// ---------------------------------------------------------------------------
// K5: loc_grid in its own frame (Sec. IV-E), out of the ring-addressed
// buffer: voxel (x, y, z) is the buffer's byte at the ring position of
// (x, y, z), or unknown where a re-centre brought the voxel in.  One
// 16-byte chunk of the output per call; dst is 16-byte aligned.
// ---------------------------------------------------------------------------
template <class L>
__device__ __forceinline__ void shift_chunk(const PlaneGeom &g, const Ring &R, const uint8_t *src, uint8_t *dst,
                                            int64_t chunk) {
    const int64_t i0 = chunk * 16;
    if (i0 >= g.nvox) return;
    // grids hold fewer than 2^31 voxels: 32-bit division
    const uint32_t yz = (uint32_t)i0 / (uint32_t)g.nx;
    int32_t x = (int32_t)((uint32_t)i0 - yz * (uint32_t)g.nx);
    int32_t y = (int32_t)(yz % (uint32_t)g.ny), z = (int32_t)(yz / (uint32_t)g.ny);
    uint32_t o[4];
    const int32_t xb = ring_at(x, R.r[0], g.nx);
    const bool row_in = !((y >= R.elo[1] && y < R.ehi[1]) || (z >= R.elo[2] && z < R.ehi[2]));
    if (i0 + 16 <= g.nvox && x + 16 <= g.nx && xb + 16 <= g.nx && row_in && (x + 16 <= R.elo[0] || x >= R.ehi[0])) {
        // 16 voxels of one row, all old, contiguous in the buffer: bytes
        // [sb, sb + 16), read as five aligned words; the last may reach up
        // to 3 bytes past nvox, into the slack the host leaves after every
        // loc buffer, and those bytes are shifted out
        const int64_t sb = ((int64_t)ring_at(z, R.r[2], g.nz) * g.ny + ring_at(y, R.r[1], g.ny)) * g.nx + xb;
        const uint32_t *wsrc = reinterpret_cast<const uint32_t *>(src + (sb & ~int64_t(3)));
        const int sh = (int)(sb & 3) * 8;
        uint32_t wv[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) wv[m] = L::ld(wsrc + m);
#pragma unroll
        for (int m = 0; m < 4; ++m) o[m] = __funnelshift_r(wv[m], wv[m + 1], sh);
    } else {
        // byte by byte, through at most two rows: each row's ring position
        // and whether a re-centre brought it in are found once, and the
        // buffer x advances with the voxel (wrapping at the row's end)
        uint8_t ob[16];
        const uint8_t *rowp =
            src + ((int64_t)ring_at(z, R.r[2], g.nz) * g.ny + ring_at(y, R.r[1], g.ny)) * g.nx;
        bool rin = row_in;
        int32_t xr = xb;
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            ob[b] = 0;
            if (i0 + b < g.nvox && rin && !(x >= R.elo[0] && x < R.ehi[0])) ob[b] = L::ld(rowp + xr);
            if (++x == g.nx) {
                x = 0;
                if (++y == g.ny) { y = 0; ++z; }
                // the next row (past the grid's end only where no voxel is read)
                const int32_t zr = z < g.nz ? z : 0;
                rowp = src + ((int64_t)ring_at(zr, R.r[2], g.nz) * g.ny + ring_at(y, R.r[1], g.ny)) * g.nx;
                rin = !((y >= R.elo[1] && y < R.ehi[1]) || (z >= R.elo[2] && z < R.ehi[2]));
                xr = R.r[0];
            } else if (++xr == g.nx) {
                xr = 0;
            }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m)
            o[m] = ob[4 * m] | (ob[4 * m + 1] << 8) | (ob[4 * m + 2] << 16) | ((uint32_t)ob[4 * m + 3] << 24);
    }
    if (i0 + 16 <= g.nvox) {
        *reinterpret_cast<uint4 *>(dst + i0) = make_uint4(o[0], o[1], o[2], o[3]);
    } else {
        for (int b = 0; b < 16 && i0 + b < g.nvox; ++b) dst[i0 + b] = (uint8_t)(o[b >> 2] >> (8 * (b & 3)));
    }
}

}  // namespace units
}  // namespace vg
