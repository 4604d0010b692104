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
// and Alg. 3 writes it to loc_grid wherever it is not unknown.  A word with
// no bit set in any plane touches neither loc_grid nor the planes, so the
// pass reads the bit planes everywhere but loc_grid only inside the
// measured frustum.  Loc bytes move as 8-byte words when the row layout and
// the buffer allow.  Every plane word read non-zero is cleared, which
// leaves all planes zero for the next frame (occ_raw is a subset of occ_inf,
// so its non-zero words are cleared too).
// ---------------------------------------------------------------------------
// RAYS_LAST: the literal loc_grid reading, in which the rays' marks replace
// the measurement's occupied marks (free > traced > occupied).
template <bool RAYS_LAST = false>
__device__ __forceinline__ uint8_t resolve(uint32_t oc, uint32_t f, uint32_t t, int b, uint8_t old) {
    if (!RAYS_LAST && ((oc >> b) & 1u)) return 2;   // VG_OCC
    if ((f >> b) & 1u) return 1;                    // VG_FREE
    if ((t >> b) & 1u) return 3;                    // VG_TRACED
    if (RAYS_LAST && ((oc >> b) & 1u)) return 2;
    return old;
}

// The same resolve for four voxels at once.  With the state codes
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

template <bool ALIGN8, class L, bool RAYS_LAST = false>
__device__ __forceinline__ void merge_word(const PlaneGeom &g, const Planes &pl, uint8_t *loc, int64_t w) {
    if (w >= g.words) return;
    // rows are a power of two of words
    const int32_t wxi = (int32_t)(w & (g.wx - 1));
    const int64_t row = w >> (__ffs(g.wx) - 1);
    const int32_t x0 = wxi * 32;
    if (x0 >= g.nx) return;   // padding word, always zero
    const uint32_t oc = L::ld(pl.occ_inf + w), f = L::ld(pl.fr + w), t = L::ld(pl.tr + w);
    const uint32_t any = oc | f | t;
    if (any == 0) return;
    const int nbits = min(32, g.nx - x0);
    uint8_t *Lp = loc + row * g.nx + x0;
    uint32_t hi, lo, known;
    code_masks<RAYS_LAST>(oc, f, t, hi, lo, known);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (8 * c >= nbits) break;
        const uint32_t m = (any >> (8 * c)) & 0xffu;
        if (m == 0) continue;
        if (ALIGN8 && 8 * c + 8 <= nbits) {
            uint64_t *p = reinterpret_cast<uint64_t *>(Lp + 8 * c);
            const uint64_t old = (m == 0xffu) ? 0ull : *p;
            const uint32_t v0 = merge4(hi, lo, known, 2 * c, (uint32_t)old);
            const uint32_t v1 = merge4(hi, lo, known, 2 * c + 1, (uint32_t)(old >> 32));
            *p = ((uint64_t)v1 << 32) | v0;
        } else {
            for (int b = 8 * c; b < 8 * c + 8 && b < nbits; ++b)
                if ((any >> b) & 1u) Lp[b] = resolve<RAYS_LAST>(oc, f, t, b, 0);
        }
    }
    if (oc) {
        pl.occ_inf[w] = 0;
        pl.occ_raw[w] = 0;
    }
    if (f) pl.fr[w] = 0;
    if (t) pl.tr[w] = 0;
}

// K4 with a pending re-centre (Sec. IV-E followed by Alg. 3): unit u is the
// WPU plane words u*WPU .. u*WPU+WPU-1 (WPU a multiple of 256), and writes
// every voxel of the new grid they cover, dst[i] = the merge of the
// measurement (whose planes are in the new grid's frame) over src[i + delta],
// delta = dx + dy*Nx + dz*Nx*Ny, or over unknown where that voxel of the old
// grid does not exist.  Clears the plane words it reads, as merge_word does.
//
// Because the plane row pitch wx is a power of two, the WPU words are whole
// rows (wx <= WPU) or one part of a row (wx > WPU), so the unit's voxels are
// one contiguous range [b0, b1) of at most 32*WPU bytes of dst, and their
// sources one contiguous range of src.  The CTA stages the sources in shared
// memory with aligned 16-byte loads (all issued before the first wait, so a
// larger unit keeps more bytes in flight), each thread resolves the 32
// voxels of each of its WPU/256 words into a second shared buffer, and the
// results go out as aligned 16-byte stores.
// sm: 16-byte aligned, merge_shift_smem(WPU) bytes.  Called by all threads
// of a 256-thread CTA with the same u.  LS loads src (never written by the
// launch), LP the planes (cleared by the launch).
__host__ __device__ constexpr int merge_shift_smem(int wpu) { return 2 * (32 * wpu + 32); }
constexpr int kMergeShiftSmem = merge_shift_smem(256);

// PDL_WAIT: the unit is a chained launch's only one (k_merge_shift); its
// sources (the grid before this measurement, which K1-K3 do not write) are
// staged before the launch waits for its predecessor (pdl_wait), so that
// their DRAM latency overlaps the end of K3; the planes are read after it.
template <int WPU, class LS, class LP, bool RAYS_LAST = false, bool PDL_WAIT = false>
__device__ __forceinline__ void merge_shift_unit(const PlaneGeom &g, const Planes &pl, const uint8_t *src,
                                                 uint8_t *dst, int32_t dx, int32_t dy, int32_t dz, int64_t u,
                                                 uint8_t *sm) {
    static_assert(WPU % 256 == 0, "whole CTAs of words");
    constexpr int kVox = 32 * WPU;
    uint8_t *sm_src = sm;                 // staged sources, kVox + 16 bytes
    uint8_t *sm_out = sm + kVox + 32;     // results, 16-byte aligned
    const int tid = threadIdx.x;
    const int64_t rows = (int64_t)g.ny * g.nz;
    // rows are a power of two of words, and so is WPU; grids have fewer
    // than 2^31 voxels, so rows and voxel indices fit 32 bits
    const int lw = __ffs(g.wx) - 1;
    int64_t b0, b1;
    if (g.wx <= WPU) {
        const int64_t R = WPU >> lw;
        const int64_t r0 = u * R, r1 = min(r0 + R, rows);
        b0 = r0 * g.nx;
        b1 = r1 * g.nx;
    } else {
        const int lp = lw - (__ffs(WPU) - 1);   // log2 of the units per row
        const int64_t row = u >> lp, xa = (u & ((int64_t(1) << lp) - 1)) * kVox;
        b0 = row * g.nx + min(xa, (int64_t)g.nx);
        b1 = row * g.nx + min(xa + kVox, (int64_t)g.nx);
    }
    if (b0 >= b1) {   // uniform over the CTA
        if (PDL_WAIT) pdl_wait();
        return;
    }
    const int64_t off = (int64_t)dx + (int64_t)dy * g.nx + (int64_t)dz * g.nx * g.ny;

    // stage src[s0, s1): bytes [A, A + 16*n16) land at sm_src[0 ..); the
    // last chunk may reach 15 bytes past nvox, into the buffer's slack
    const int64_t s0 = max(b0 + off, (int64_t)0), s1 = min(b1 + off, g.nvox);
    const int64_t A = s0 & ~int64_t(15);
    __syncthreads();   // sm may still be read by the CTA's previous unit
    if (s0 < s1) {
        const int n16 = (int)((s1 - A + 15) >> 4);
        for (int i = tid; i < n16; i += 256)
            reinterpret_cast<uint4 *>(sm_src)[i] = LS::ld(reinterpret_cast<const uint4 *>(src + A) + i);
    }
    if (PDL_WAIT) pdl_wait();
    __syncthreads();

    // results at sm_out[q0 + (i - b0)], q0 = b0 mod 16, so that sm_out and
    // dst agree on 16-byte alignment
    const int q0 = (int)(b0 & 15);
#pragma unroll 1
    for (int k = 0; k < WPU / 256; ++k) {
        // this thread's plane word and its 32 voxels
        const int64_t w = u * WPU + k * 256 + tid;
        const int32_t x0 = (int32_t)(w & (g.wx - 1)) * 32;
        if (!(w < g.words && x0 < g.nx)) continue;
        const uint32_t row = (uint32_t)(w >> lw);
        const int32_t y = (int32_t)(row % (uint32_t)g.ny), z = (int32_t)(row / (uint32_t)g.ny);
        const int nbits = min(32, g.nx - x0);
        const int64_t d = (int64_t)row * g.nx + x0;
        const uint32_t oc = LP::ld(pl.occ_inf + w), f = LP::ld(pl.fr + w), t = LP::ld(pl.tr + w);
        const int32_t sy = y + dy, sz = z + dz, sx0 = x0 + dx;
        const bool row_ok = (unsigned)sy < (unsigned)g.ny && (unsigned)sz < (unsigned)g.nz;
        const int p = (int)(d + off - A);   // sm_src index of the first source voxel
        uint32_t old[8];
        if (row_ok && sx0 >= 0 && sx0 + nbits <= g.nx) {
            // all present: aligned shared words and a funnel shift (bytes
            // past nbits are garbage and discarded)
            const uint32_t *ws = reinterpret_cast<const uint32_t *>(sm_src + (p & ~3));
            const int sh = (p & 3) * 8;
            uint32_t wv[9];
#pragma unroll
            for (int m = 0; m < 9; ++m) wv[m] = ws[m];
#pragma unroll
            for (int m = 0; m < 8; ++m) old[m] = __funnelshift_r(wv[m], wv[m + 1], sh);
        } else {
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                uint32_t v = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int kk = 4 * m + b;
                    if (row_ok && kk < nbits && (unsigned)(sx0 + kk) < (unsigned)g.nx)
                        v |= (uint32_t)sm_src[p + kk] << (8 * b);
                }
                old[m] = v;
            }
        }
        uint32_t nv[8];
        if ((oc | f | t) == 0) {
#pragma unroll
            for (int m = 0; m < 8; ++m) nv[m] = old[m];
        } else {
            uint32_t hi, lo, known;
            code_masks<RAYS_LAST>(oc, f, t, hi, lo, known);
#pragma unroll
            for (int m = 0; m < 8; ++m) nv[m] = merge4(hi, lo, known, m, old[m]);
            if (oc) {
                pl.occ_inf[w] = 0;
                pl.occ_raw[w] = 0;
            }
            if (f) pl.fr[w] = 0;
            if (t) pl.tr[w] = 0;
        }
        const int q = q0 + (int)(d - b0);
        const bool words = (q & 3) == 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if (words && 4 * m + 4 <= nbits) {
                *reinterpret_cast<uint32_t *>(sm_out + q + 4 * m) = nv[m];
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (4 * m + b < nbits) sm_out[q + 4 * m + b] = (uint8_t)(nv[m] >> (8 * b));
            }
        }
    }
    __syncthreads();
    // [b0, h) and [t1, b1) bytewise, [h, t1) in aligned 16-byte chunks
    const int64_t h = min(b1, (b0 + 15) & ~int64_t(15));
    const int64_t t1 = max(h, b1 & ~int64_t(15));
    const int64_t base = b0 - q0;   // dst address of sm_out[0]; a multiple of 16
    if (tid < 16) {
        const int64_t i = b0 + tid;
        if (i < h) dst[i] = sm_out[i - base];
    } else if (tid < 32) {
        const int64_t i = t1 + (tid - 16);
        if (i < b1) dst[i] = sm_out[i - base];
    }
    const int n16o = (int)((t1 - h) >> 4);
    for (int i = tid; i < n16o; i += 256) {
        const int64_t at = h + 16 * (int64_t)i;
        *reinterpret_cast<uint4 *>(dst + at) = *reinterpret_cast<const uint4 *>(sm_out + (at - base));
    }
}

// Units of merge_shift_unit<WPU> for a grid.
template <int WPU>
__host__ __device__ __forceinline__ int64_t merge_shift_units(const PlaneGeom &g) {
    return (g.words + WPU - 1) / WPU;
}

// ---------------------------------------------------------------------------
// K5: shift loc_grid to re-centre it on the robot (Sec. IV-E).
//
// An out-of-place copy with a constant flat offset: voxel (x, y, z) of the
// new grid is voxel (x+dx, y+dy, z+dz) of the old one, i.e. flat index
// i + dx + dy*Nx + dz*Nx*Ny, or unknown when that voxel does not exist.
// One 16-byte chunk of the new grid per call.
// ---------------------------------------------------------------------------
template <class L>
__device__ __forceinline__ void shift_chunk(const PlaneGeom &g, int32_t dx, int32_t dy, int32_t dz,
                                            const uint8_t *src, uint8_t *dst, int64_t chunk) {
    const int64_t i0 = chunk * 16;
    if (i0 >= g.nvox) return;
    const int64_t off = (int64_t)dx + (int64_t)dy * g.nx + (int64_t)dz * g.nx * g.ny;
    // grids hold fewer than 2^31 voxels: 32-bit division
    const uint32_t yz = (uint32_t)i0 / (uint32_t)g.nx;
    int32_t x = (int32_t)((uint32_t)i0 - yz * (uint32_t)g.nx);
    int32_t y = (int32_t)(yz % (uint32_t)g.ny), z = (int32_t)(yz / (uint32_t)g.ny);
    // which of the 16 voxels have a source voxel
    uint32_t valid = 0;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        const int32_t sx = x + dx, sy = y + dy, sz = z + dz;
        if (i0 + b < g.nvox && (unsigned)sx < (unsigned)g.nx && (unsigned)sy < (unsigned)g.ny &&
            (unsigned)sz < (unsigned)g.nz)
            valid |= 1u << b;
        if (++x == g.nx) {
            x = 0;
            if (++y == g.ny) { y = 0; ++z; }
        }
    }
    uint32_t o[4];
    if (valid == 0xffffu) {
        // all sources exist: bytes [sb, sb+16) of src, 0 <= sb and sb+15 < nvox,
        // read as five aligned words; the last may reach up to 4 bytes past
        // nvox, into the slack the host leaves after every loc buffer, and
        // those bytes are shifted out
        const int64_t sb = i0 + off;
        const uint32_t *wsrc = reinterpret_cast<const uint32_t *>(src + (sb & ~int64_t(3)));
        const int sh = (int)(sb & 3) * 8;
        uint32_t wv[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) wv[m] = L::ld(wsrc + m);
#pragma unroll
        for (int m = 0; m < 4; ++m) o[m] = __funnelshift_r(wv[m], wv[m + 1], sh);
    } else {
        uint8_t ob[16];
#pragma unroll
        for (int b = 0; b < 16; ++b) ob[b] = ((valid >> b) & 1u) ? L::ld(src + i0 + b + off) : (uint8_t)0;
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
