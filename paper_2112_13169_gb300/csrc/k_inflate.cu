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
// stays zero.
#include "vg_internal.cuh"

namespace vg {
namespace {

struct TileShape {
    int txw, ty, tz;
};

__device__ __forceinline__ uint32_t dilate_x(uint32_t prev, uint32_t cur, uint32_t next, int r) {
    uint32_t acc = cur;
    for (int d = 1; d <= r; ++d) {
        acc |= __funnelshift_r(cur, next, d);   // voxel x+d -> x
        acc |= __funnelshift_l(prev, cur, d);   // voxel x-d -> x
    }
    return acc;
}

__global__ void __launch_bounds__(256) k_inflate(const PlaneGeom g, const uint32_t *__restrict__ raw,
                                                 uint32_t *__restrict__ out, const int r,
                                                 const TileShape ts) {
    extern __shared__ uint32_t sm[];
    const int hx = ts.txw + 2, hy = ts.ty + 2 * r, hz = ts.tz + 2 * r;
    uint32_t *buf0 = sm;                          // hz * hy * hx: raw with halo
    uint32_t *buf1 = sm + (size_t)hz * hy * hx;   // hz * hy * txw: x-dilated
    const int w0 = blockIdx.x * ts.txw, y0 = blockIdx.y * ts.ty, z0 = blockIdx.z * ts.tz;

    // 1. stage raw words (zero outside the grid)
    const int n0 = hz * hy * hx;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const int lx = i % hx, rest = i / hx, ly = rest % hy, lz = rest / hy;
        const int w = w0 + lx - 1, y = y0 + ly - r, z = z0 + lz - r;
        uint32_t v = 0;
        if (w >= 0 && w < g.wx && y >= 0 && y < g.ny && z >= 0 && z < g.nz)
            v = __ldg(raw + ((int64_t)z * g.ny + y) * g.wx + w);
        buf0[i] = v;
    }
    __syncthreads();

    // 2. x pass, clearing bits past the end of the row
    const int n1 = hz * hy * ts.txw;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        const int lx = i % ts.txw, row = i / ts.txw;
        const uint32_t *b = buf0 + (size_t)row * hx + lx;
        uint32_t v = dilate_x(b[0], b[1], b[2], r);
        const int valid = g.nx - 32 * (w0 + lx);
        if (valid < 32) v &= valid > 0 ? ((1u << valid) - 1u) : 0u;
        buf1[i] = v;
    }
    __syncthreads();

    // 3. y pass into buf0 (now free): hz * ty * txw
    const int n2 = hz * ts.ty * ts.txw;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int lx = i % ts.txw, rest = i / ts.txw, ly = rest % ts.ty, lz = rest / ts.ty;
        const uint32_t *b = buf1 + ((size_t)lz * hy + ly) * ts.txw + lx;
        uint32_t v = 0;
        for (int d = 0; d <= 2 * r; ++d) v |= b[(size_t)d * ts.txw];
        buf0[i] = v;
    }
    __syncthreads();

    // 4. z pass to global
    const int n3 = ts.tz * ts.ty * ts.txw;
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int lx = i % ts.txw, rest = i / ts.txw, ly = rest % ts.ty, lz = rest / ts.ty;
        const int w = w0 + lx, y = y0 + ly, z = z0 + lz;
        if (w >= g.wx || y >= g.ny || z >= g.nz) continue;
        const uint32_t *b = buf0 + ((size_t)lz * ts.ty + ly) * ts.txw + lx;
        uint32_t v = 0;
        for (int d = 0; d <= 2 * r; ++d) v |= b[(size_t)d * ts.ty * ts.txw];
        out[((int64_t)z * g.ny + y) * g.wx + w] = v;
    }
}

size_t smem_bytes(const TileShape &ts, int r) {
    const size_t hx = ts.txw + 2, hy = ts.ty + 2 * r, hz = ts.tz + 2 * r;
    return sizeof(uint32_t) * (hz * hy * hx + hz * hy * ts.txw);
}

}  // namespace

cudaError_t configure_inflate() {
    // the largest tile (vox_inf 15) needs about 104 KB of shared memory
    return cudaFuncSetAttribute(k_inflate, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
}

cudaError_t launch_inflate(const FrameArgs &a, cudaStream_t s) {
    const int r = a.r;
    TileShape ts{a.g.wx < 8 ? a.g.wx : 8, 16, 8};
    if (r > 4) ts = TileShape{ts.txw, 8, 8};
    const size_t bytes = smem_bytes(ts, r);
    dim3 grid((a.g.wx + ts.txw - 1) / ts.txw, (a.g.ny + ts.ty - 1) / ts.ty,
              (a.g.nz + ts.tz - 1) / ts.tz);
    k_inflate<<<grid, 256, bytes, s>>>(a.g, a.pl.occ_raw, a.pl.occ_inf, r, ts);
    return cudaGetLastError();
}

}  // namespace vg
