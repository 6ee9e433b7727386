// K2: relaxed tip scan (Sec. 5.1.1 step 2) with an optional fused df epilogue.
//
// One thread owns one pixel column and walks its heights from the top down:
// the PP starts at anchor + d0 for the first height and at p*(k-1) - dz z_hat
// (the tip moved down by dz, the deflection kept) for the others, and is
// relaxed by FIRE on G(p) = F_T(p) + F_S(p) (Eq. F_PP), with the tip springs
// of Eq. F_tip and F_S trilinearly interpolated from the force grid.  The tip
// force is read out as Fz = -F^T_{R,z} = kR (|d| - R0) d_z / |d| (Sec. 2.1).
//
// The FIRE state is e = d - d0, the deflection from the spring's rest
// displacement.  Then |d|^2 - R0^2 = (2 d0 + e).e + (|d0|^2 - R0^2) is formed
// without cancellation, so the radial extension and Fz keep full FP32
// relative precision however stiff the spring (with d itself the extension
// would be quantised at ulp(R0) ~ 5e-7 A, i.e. 3e-4 eV/A at 1e4 N/m).
//
// Lanes of a warp cover an 8x4 pixel tile, so the 32 PPs sit in neighbouring
// grid cells and their corner loads share L1 lines.  Each lane advances to its
// next height as soon as it has converged; the warp only waits for its
// slowest lane once, at the end of the columns, not at every height.
// Interpolation is done by hand in FP32 from eight float4 corner loads on the
// read-only path (hardware texture filtering carries only 8 fractional bits
// in its weights, which would cost the 1e-3 A position parity).
#include "relax_core.cuh"

namespace pp {
namespace {

constexpr int kThreads = 32;  // one warp per CTA: an 8x4 pixel tile (evens out warps per SM)
constexpr int kTileX = 8;
constexpr int kTileY = 4;

// Node range [lo, hi] (clamped to the grid) covering coordinates a..b along one axis.
__device__ __forceinline__ int2 node_range(float a, float b, float inv_d, float g0s, int n) {
    const float fa = fmaf(fminf(a, b), inv_d, g0s), fb = fmaf(fmaxf(a, b), inv_d, g0s);
    const int lo = min(max(__float2int_rd(fa), 0), n - 1);
    const int hi = min(max(__float2int_rd(fb) + 1, 0), n - 1);
    return make_int2(lo, hi);
}

// Linear layout: ask L2 for the grid rows under this warp's 8x4 tile over the
// z-range its PPs will visit (anchor heights + d0, 0.5 A margin), so that the
// scan's first touches of the slab are served in parallel at the start instead
// of one demand miss at a time inside the FIRE loops.  Rows are contiguous in
// x; each lane issues a bulk prefetch (a hint: it never faults and changes no
// result) for every 32nd row.  Lateral deflections reach the neighbouring
// tiles' rows, which those warps prefetch.
__device__ __forceinline__ void prefetch_tile_slab(const RelaxLaunch& P, int tx, int ty, int lane) {
    const int ia = tx * kTileX, ib = min(ia + kTileX, P.snx) - 1;
    const int ja = ty * kTileY, jb = min(ja + kTileY, P.sny) - 1;
    const int2 ri = node_range(fmaf((float)ia, P.spx, P.sx0) + P.d0x, fmaf((float)ib, P.spx, P.sx0) + P.d0x,
                               P.inv_dx, P.gx0s, P.map.nx);
    const int2 rj = node_range(fmaf((float)ja, P.spy, P.sy0) + P.d0y, fmaf((float)jb, P.spy, P.sy0) + P.d0y,
                               P.inv_dy, P.gy0s, P.map.ny);
    const float ztop = P.z_top + P.d0z, zbot = P.z_top - (P.snz - 1) * P.sdz + P.d0z;
    const int2 rk = node_range(fminf(ztop, zbot) - 0.5f, fmaxf(ztop, zbot) + 0.5f, P.inv_dz, P.gz0s, P.map.nz);
    const int nj = rj.y - rj.x + 1, rows = nj * (rk.y - rk.x + 1);
    for (int r = lane; r < rows; r += kThreads) {
        const int j = rj.x + r % nj, k = rk.x + r / nj;
        const int first = node_index(P.map, ri.x, j, k);
        if (P.map.interp == 0) {
            const unsigned bytes = (unsigned)(ri.y - ri.x + 1) * 16u;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(P.ff + first), "r"(bytes) : "memory");
        } else {
            // one float per node: the whole 16-byte groups inside the row (one node wider
            // on the left for the tricubic stencil); up to 3 nodes at the right end are left out
            const int lo = max(first - 1, 0) & ~3, hi = (first + (ri.y - ri.x) + 1) & ~3;
            if (hi > lo)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(P.ffE + lo), "r"((unsigned)(hi - lo) * 4u)
                             : "memory");
        }
    }
}

// The warp's lowest and highest node layer read, folded into P.zspan by lane 0 (all 32 lanes call).
__device__ __forceinline__ void record_zspan(const RelaxLaunch& P, int2 span) {
    const int lo = __reduce_min_sync(0xffffffffu, span.x);
    const int hi = __reduce_max_sync(0xffffffffu, span.y);
    if (threadIdx.x == 0) {
        atomicMin(P.zspan, lo);
        atomicMax(P.zspan + 1, hi);
    }
}

// This warp's pixel (i, j); i = snx marks an idle lane.  Without a plan: lane l of the 8x4 tile
// (blockIdx.x, blockIdx.y).  With one (a 1-D grid): the first plan_hblocks warps take the plan's
// listed pixels, plan_lanes lanes each (-1 or anything outside the scan: idle), and warp
// plan_hblocks + t takes tile t less the listed pixels.  *tx < 0: no tile (no slab prefetch).
__device__ __forceinline__ void scan_pixel(const RelaxLaunch& P, int& i, int& j, int& tx, int& ty) {
    const int lane = threadIdx.x;
    if (!P.plan_list) {
        tx = blockIdx.x;
        ty = blockIdx.y;
        i = tx * kTileX + (lane & 7);
        j = ty * kTileY + (lane >> 3);
        return;
    }
    const int npix = P.snx * P.sny;
    const int b = blockIdx.x;
    if (b < P.plan_hblocks) {
        tx = ty = -1;
        int p = -1;
        if (lane < P.plan_lanes) p = P.plan_list[b * P.plan_lanes + lane];
        const bool ok = p >= 0 && p < npix;
        i = ok ? p % P.snx : P.snx;
        j = ok ? p / P.snx : P.sny;
        return;
    }
    const int ntx = (P.snx + kTileX - 1) / kTileX, t = b - P.plan_hblocks;
    tx = t % ntx;
    ty = t / ntx;
    i = tx * kTileX + (lane & 7);
    j = ty * kTileY + (lane >> 3);
    if (i < P.snx && j < P.sny) {
        const int p = j * P.snx + i;
        if ((P.plan_mask[p >> 5] >> (p & 31)) & 1u) i = P.snx;  // run by a plan warp
    }
}

// kSpan: P.zspan is set and receives the node layers the lookups read.
template <int LAYOUT, bool kPolish, bool kSpan>
__global__ void __launch_bounds__(kThreads) relax_scan_kernel(const RelaxLaunch P) {
    int i, j, tx, ty;
    scan_pixel(P, i, j, tx, ty);
    if (LAYOUT == 0 && tx >= 0) prefetch_tile_slab(P, tx, ty, threadIdx.x);
    const int2 span = relax_pixel<LAYOUT, false, false, false, kPolish, kSpan>(P, P, i, j);
    if constexpr (kSpan) record_zspan(P, span);
}

// Tricubic energy grid (linear layout).
template <bool kPolish, bool kSpan>
__global__ void __launch_bounds__(kThreads) relax_scan_tricubic_kernel(const RelaxLaunch P) {
    int i, j, tx, ty;
    scan_pixel(P, i, j, tx, ty);
    if (tx >= 0) prefetch_tile_slab(P, tx, ty, threadIdx.x);
    const int2 span = relax_pixel<0, false, true, false, kPolish, kSpan>(P, P, i, j);
    if constexpr (kSpan) record_zspan(P, span);
}

template <bool kPolish, bool kSpan>
void launch_relax_scan_t(const RelaxLaunch& L, dim3 grid, cudaStream_t s) {
    if (L.map.interp == 1) relax_scan_tricubic_kernel<kPolish, kSpan><<<grid, kThreads, 0, s>>>(L);
    else if (L.layout == 0) relax_scan_kernel<0, kPolish, kSpan><<<grid, kThreads, 0, s>>>(L);
    else relax_scan_kernel<1, kPolish, kSpan><<<grid, kThreads, 0, s>>>(L);
}

}  // namespace

cudaError_t launch_relax_scan(const RelaxLaunch& L, cudaStream_t s) {
    dim3 grid((L.snx + kTileX - 1) / kTileX, (L.sny + kTileY - 1) / kTileY, 1);
    if (L.plan_list) grid = dim3(L.plan_hblocks + grid.x * grid.y, 1, 1);
    const bool span = L.zspan != nullptr;
    if (L.polish > 0) span ? launch_relax_scan_t<true, true>(L, grid, s) : launch_relax_scan_t<true, false>(L, grid, s);
    else span ? launch_relax_scan_t<false, true>(L, grid, s) : launch_relax_scan_t<false, false>(L, grid, s);
    return cudaGetLastError();
}

PP_CHECK_READER(check_flags_relax_scan)

}  // namespace pp
