// K2 as its own launch: one CTA per 8-word x 8-row x 8-slice tile of the
// occupancy plane (4 slices for grids of one to four such tiles per SM);
// the work itself is in vg_units.cuh.  For r = 1, 2, 3 the
// radius is a compile-time constant; other radii use a runtime radius.
#include "vg_units.cuh"

#include <atomic>

namespace vg {
namespace {

template <int R, int TXW, int TY, int TZ>
__global__ void __launch_bounds__(256) k_inflate(const PlaneGeom g, const uint32_t *__restrict__ raw,
                                                 uint32_t *__restrict__ out, const int r_rt) {
    extern __shared__ uint32_t sm[];
    pdl_trigger();
    pdl_wait();
    units::inflate_tile<R, TXW, TY, TZ, units::LoadRO>(g, raw, out, r_rt, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

template <int R, int TXW, int TY, int TZ>
cudaError_t run(const FrameArgs &a, cudaStream_t s) {
    dim3 grid((a.g.wx + TXW - 1) / TXW, (a.g.ny + TY - 1) / TY, (a.g.nz + TZ - 1) / TZ);
    const size_t bytes = sizeof(uint32_t) * units::inflate_smem_words<R, TXW, TY, TZ>(a.r);
    return launch_pdl(k_inflate<R, TXW, TY, TZ>, grid, 256, bytes, s, a.g, (const uint32_t *)a.pl.occ_raw,
                      a.pl.occ_inf, a.r);
}

template <int TXW, int TZ>
cudaError_t run_r(const FrameArgs &a, cudaStream_t s) {
    switch (a.r) {
    case 1: return run<1, TXW, 8, TZ>(a, s);
    case 2: return run<2, TXW, 8, TZ>(a, s);
    case 3: return run<3, TXW, 8, TZ>(a, s);
    default: return run<0, TXW, 8, 8>(a, s);   // other radii: 8-slice tiles, the radius at run time
    }
}

std::atomic<int> g_sms[64];   // SMs per device, read on first use (any thread)

int sms_of_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int n = g_sms[dev].load(std::memory_order_relaxed);
    if (!n) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        g_sms[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

}  // namespace

cudaError_t configure_inflate() {
    // the runtime-radius tile at vox_inf 15 needs about 104 KB of shared memory
    cudaError_t e = cudaFuncSetAttribute(k_inflate<0, 4, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         160 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_inflate<0, 8, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 160 * 1024);
    return e;
}

// Tiles of 8 words (4 for rows of 4 words) by 8 rows by 8 slices, or 4
// slices when a grid has between one and four 8-slice tiles per SM: the
// shorter tiles stage more halo per word, but twice as many CTAs share the
// device and the launch ends sooner.  Measured frame times: a 200x200x100
// grid (325 tiles of 8 slices) fell by about 2.3 us with 650 of 4; an
// 80x80x40 grid (50 tiles, fewer than the SMs) rose by 1.3 us, and a
// 400x400x120 grid (1500 tiles) did better with 8 slices.  sc.inflate_tile
// picks a shape instead (8-word tiles only where rows have a multiple of 8
// words).
cudaError_t launch_inflate(const FrameArgs &a, cudaStream_t s, const Sched &sc) {
    // rows are a power of two of words, at least 4
    const bool wide_ok = a.g.wx % 8 == 0;
    int tile = sc.inflate_tile;
    if (tile == kTileAuto) {
        const int txw = wide_ok ? 8 : 4;
        const int64_t tiles8 = (int64_t)((a.g.wx + txw - 1) / txw) * ((a.g.ny + 7) / 8) * ((a.g.nz + 7) / 8);
        const int64_t sms = sms_of_current_device();
        const bool short_tiles = tiles8 >= sms && tiles8 < 4 * sms;
        tile = wide_ok ? (short_tiles ? kTile8x8x4 : kTile8x8x8) : (short_tiles ? kTile4x8x4 : kTile4x8x8);
    }
    if (!wide_ok && tile == kTile8x8x4) tile = kTile4x8x4;
    if (!wide_ok && tile == kTile8x8x8) tile = kTile4x8x8;
    switch (tile) {
    case kTile4x8x4: return run_r<4, 4>(a, s);
    case kTile4x8x8: return run_r<4, 8>(a, s);
    case kTile8x8x4: return run_r<8, 4>(a, s);
    default: return run_r<8, 8>(a, s);
    }
}

}  // namespace vg
