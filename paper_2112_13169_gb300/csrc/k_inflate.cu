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
// stays zero.  For r = 1, 2, 3 the radius and tile are compile-time
// constants (all index arithmetic folds, the halo loads issue back to
// back); other radii use the same kernel with a runtime radius.
#include "vg_internal.cuh"

namespace vg {
namespace {

__device__ __forceinline__ uint32_t dilate_x(uint32_t prev, uint32_t cur, uint32_t next, int r) {
    uint32_t acc = cur;
#pragma unroll 4
    for (int d = 1; d <= r; ++d) {
        acc |= __funnelshift_r(cur, next, d);   // voxel x+d -> x
        acc |= __funnelshift_l(prev, cur, d);   // voxel x-d -> x
    }
    return acc;
}

// R > 0: compile-time radius; R == 0: radius r_rt at run time.
template <int R, int TXW, int TY, int TZ>
__global__ void __launch_bounds__(256) k_inflate(const PlaneGeom g, const uint32_t *__restrict__ raw,
                                                 uint32_t *__restrict__ out, const int r_rt) {
    extern __shared__ uint32_t sm[];
    const int r = R > 0 ? R : r_rt;
    const int hx = TXW + 2, hy = TY + 2 * r, hz = TZ + 2 * r;
    uint32_t *buf0 = sm;                          // hz * hy * hx: raw with halo
    uint32_t *buf1 = sm + hz * hy * hx;           // hz * hy * TXW: x-dilated
    const int w0 = blockIdx.x * TXW, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;

    // 1. stage raw words (zero outside the grid)
    const int n0 = hz * hy * hx;
#pragma unroll 8
    for (int i = threadIdx.x; i < n0; i += 256) {
        const int lx = i % hx, rest = i / hx, ly = rest % hy, lz = rest / hy;
        const int w = w0 + lx - 1, y = y0 + ly - r, z = z0 + lz - r;
        uint32_t v = 0;
        if (w >= 0 && w < g.wx && y >= 0 && y < g.ny && z >= 0 && z < g.nz)
            v = __ldg(raw + ((int64_t)z * g.ny + y) * g.wx + w);
        buf0[i] = v;
    }
    __syncthreads();

    // 2. x pass, clearing bits past the end of the row
    const int n1 = hz * hy * TXW;
    for (int i = threadIdx.x; i < n1; i += 256) {
        const int lx = i % TXW, row = i / TXW;
        const uint32_t *b = buf0 + row * hx + lx;
        uint32_t v = dilate_x(b[0], b[1], b[2], r);
        const int valid = g.nx - 32 * (w0 + lx);
        if (valid < 32) v &= valid > 0 ? ((1u << valid) - 1u) : 0u;
        buf1[i] = v;
    }
    __syncthreads();

    // 3. y pass into buf0 (now free): hz * TY * TXW
    const int n2 = hz * TY * TXW;
    for (int i = threadIdx.x; i < n2; i += 256) {
        const int lx = i % TXW, rest = i / TXW, ly = rest % TY, lz = rest / TY;
        const uint32_t *b = buf1 + (lz * hy + ly) * TXW + lx;
        uint32_t v = 0;
        for (int d = 0; d <= 2 * r; ++d) v |= b[d * TXW];
        buf0[i] = v;
    }
    __syncthreads();

    // 4. z pass to global
    constexpr int n3 = TZ * TY * TXW;
    for (int i = threadIdx.x; i < n3; i += 256) {
        const int lx = i % TXW, rest = i / TXW, ly = rest % TY, lz = rest / TY;
        const int w = w0 + lx, y = y0 + ly, z = z0 + lz;
        if (w >= g.wx || y >= g.ny || z >= g.nz) continue;
        const uint32_t *b = buf0 + (lz * TY + ly) * TXW + lx;
        uint32_t v = 0;
        for (int d = 0; d <= 2 * r; ++d) v |= b[d * TY * TXW];
        out[((int64_t)z * g.ny + y) * g.wx + w] = v;
    }
}

template <int R, int TXW, int TY, int TZ>
size_t smem_bytes(int r) {
    const size_t hx = TXW + 2, hy = TY + 2 * r, hz = TZ + 2 * r;
    return sizeof(uint32_t) * (hz * hy * hx + hz * hy * TXW);
}

template <int R, int TXW, int TY, int TZ>
cudaError_t run(const FrameArgs &a, cudaStream_t s) {
    dim3 grid((a.g.wx + TXW - 1) / TXW, (a.g.ny + TY - 1) / TY, (a.g.nz + TZ - 1) / TZ);
    k_inflate<R, TXW, TY, TZ><<<grid, 256, smem_bytes<R, TXW, TY, TZ>(a.r), s>>>(a.g, a.pl.occ_raw,
                                                                               a.pl.occ_inf, a.r);
    return cudaGetLastError();
}

template <int TXW>
cudaError_t run_r(const FrameArgs &a, cudaStream_t s) {
    switch (a.r) {
    case 1: return run<1, TXW, 8, 8>(a, s);
    case 2: return run<2, TXW, 8, 8>(a, s);
    case 3: return run<3, TXW, 8, 8>(a, s);
    default: return run<0, TXW, 8, 8>(a, s);
    }
}

}  // namespace

cudaError_t configure_inflate() {
    // the runtime-radius tile at vox_inf 15 needs about 140 KB of shared memory
    cudaError_t e = cudaFuncSetAttribute(k_inflate<0, 4, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         160 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_inflate<0, 8, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 160 * 1024);
    return e;
}

cudaError_t launch_inflate(const FrameArgs &a, cudaStream_t s) {
    // rows are a multiple of 4 words: 4-word tiles when a row is that narrow
    return a.g.wx % 8 == 0 ? run_r<8>(a, s) : run_r<4>(a, s);
}

}  // namespace vg
