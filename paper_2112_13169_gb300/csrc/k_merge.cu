// K4: merge the measurement grid into loc_grid (Sec. IV-D, Alg. 3) and
// K5: shift loc_grid to re-centre it on the robot (Sec. IV-E).
//
// K4 takes one 32-voxel plane word per thread.  The voxel's measurement
// state is resolved from the three planes with precedence
//   occupied (occ_inf) > free (fr) > unknown-and-traced (tr) > unknown,
// and Alg. 3 writes it to loc_grid wherever it is not unknown.  A word with
// no bit set in any plane touches neither loc_grid nor the planes, so the
// pass reads the bit planes everywhere but loc_grid only inside the
// measured frustum.  Loc bytes move as 8-byte words when the row layout
// allows.  Every plane word read non-zero is cleared, which leaves all
// planes zero for the next frame (occ_raw is a subset of occ_inf, so its
// non-zero words are cleared too).
//
// K5 is an out-of-place copy with a constant flat offset: voxel (x, y, z)
// of the new grid is voxel (x+dx, y+dy, z+dz) of the old one, i.e. flat
// index i + dx + dy*Nx + dz*Nx*Ny, or unknown when that voxel does not
// exist.  Each thread writes 16 bytes.
#include "vg_internal.cuh"

namespace vg {
namespace {

__device__ __forceinline__ uint8_t resolve(uint32_t oc, uint32_t f, uint32_t t, int b, uint8_t old) {
    if ((oc >> b) & 1u) return 2;   // VG_OCC
    if ((f >> b) & 1u) return 1;    // VG_FREE
    if ((t >> b) & 1u) return 3;    // VG_TRACED
    return old;
}

template <bool ALIGN8>
__global__ void __launch_bounds__(256) k_merge(const PlaneGeom g, Planes pl, uint8_t *__restrict__ loc) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= g.words) return;
    const int32_t wxi = (int32_t)(w % g.wx);
    const int64_t row = w / g.wx;
    const int32_t x0 = wxi * 32;
    if (x0 >= g.nx) return;   // padding word, always zero
    const uint32_t oc = pl.occ_inf[w], f = pl.fr[w], t = pl.tr[w];
    const uint32_t any = oc | f | t;
    if (any == 0) return;
    const int nbits = min(32, g.nx - x0);
    uint8_t *L = loc + row * g.nx + x0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (8 * c >= nbits) break;
        const uint32_t m = (any >> (8 * c)) & 0xffu;
        if (m == 0) continue;
        if (ALIGN8 && 8 * c + 8 <= nbits) {
            uint64_t *p = reinterpret_cast<uint64_t *>(L + 8 * c);
            const uint64_t old = (m == 0xffu) ? 0ull : *p;
            uint64_t v = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint8_t ob = (uint8_t)(old >> (8 * b));
                v |= (uint64_t)resolve(oc, f, t, 8 * c + b, ob) << (8 * b);
            }
            *p = v;
        } else {
            for (int b = 8 * c; b < 8 * c + 8 && b < nbits; ++b)
                if ((any >> b) & 1u) L[b] = resolve(oc, f, t, b, 0);
        }
    }
    if (oc) {
        pl.occ_inf[w] = 0;
        pl.occ_raw[w] = 0;
    }
    if (f) pl.fr[w] = 0;
    if (t) pl.tr[w] = 0;
}

__global__ void __launch_bounds__(256) k_shift(const PlaneGeom g, const int32_t dx, const int32_t dy,
                                               const int32_t dz, const uint8_t *__restrict__ src,
                                               uint8_t *__restrict__ dst) {
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16;
    if (i0 >= g.nvox) return;
    const int64_t off = (int64_t)dx + (int64_t)dy * g.nx + (int64_t)dz * g.nx * g.ny;
    int32_t x = (int32_t)(i0 % g.nx);
    int64_t yz = i0 / g.nx;
    int32_t y = (int32_t)(yz % g.ny), z = (int32_t)(yz / g.ny);
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
        for (int m = 0; m < 5; ++m) wv[m] = __ldg(wsrc + m);
#pragma unroll
        for (int m = 0; m < 4; ++m) o[m] = __funnelshift_r(wv[m], wv[m + 1], sh);
    } else {
        uint8_t ob[16];
#pragma unroll
        for (int b = 0; b < 16; ++b) ob[b] = ((valid >> b) & 1u) ? __ldg(src + i0 + b + off) : (uint8_t)0;
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

}  // namespace

cudaError_t launch_merge(const FrameArgs &a, cudaStream_t s) {
    const unsigned blocks = (unsigned)((a.g.words + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    if (a.g.nx % 8 == 0) k_merge<true><<<blocks, 256, 0, s>>>(a.g, a.pl, a.loc);
    else k_merge<false><<<blocks, 256, 0, s>>>(a.g, a.pl, a.loc);
    return cudaGetLastError();
}

cudaError_t launch_shift(const PlaneGeom &g, const int32_t delta[3], const uint8_t *src, uint8_t *dst,
                         cudaStream_t s) {
    const int64_t threads = (g.nvox + 15) / 16;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    k_shift<<<blocks, 256, 0, s>>>(g, delta[0], delta[1], delta[2], src, dst);
    return cudaGetLastError();
}

}  // namespace vg
