// K3: Fz(z) -> df (Eq. df), and K8: force-field layout conversion.
//
// df at the centre height c is a (2m+1)-tap stencil over the Fz column,
//   df[c - m] = sum_{s=-m..m} coef[s+m] Fz[c+s],
// whose weights come from integrating a piecewise-linear Fz exactly against
// the Giessibl kernel u / sqrt(a^2 - u^2) over one peak-to-peak amplitude.
// The stencil is HBM-bound streaming work: lanes run along the pixel axis
// (contiguous loads and stores).  For half-widths m <= 8 (A_pp up to 16 dz)
// each thread owns kRows consecutive outputs of one pixel: it loads the
// kRows + 2m Fz values they need once into registers and forms the kRows sums
// there, so every Fz value is read about (kRows + 2m) / kRows times instead of
// 2m + 1.  Wider stencils take the generic kernel, one output per thread with
// the taps re-read from L1/L2.  Both sum the taps in the same order, so the
// results are identical.
#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kThreads = 256;
constexpr int kRows = 32;      // consecutive df heights per thread (register path)
constexpr int kMaxRegM = 8;    // largest half-width with a register path

template <int M>
__global__ void __launch_bounds__(kThreads) fz_to_df_rows_kernel(const DfLaunch P) {
    constexpr int W = kRows + 2 * M;  // Fz heights behind kRows outputs
    const int64_t px = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (px >= P.npix) return;
    const int nout = P.nz - 2 * M;
    const int o0 = blockIdx.y * kRows;  // first output height; it reads Fz heights o0 .. o0 + W - 1
    float v[W];
#pragma unroll
    for (int t = 0; t < W; ++t) {
        const int z = o0 + t;
        v[t] = z < P.nz ? __ldg(P.fz + checked((int64_t)z * P.npix + px, (long long)P.nz * P.npix, kChkScanRead))
                        : 0.f;
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        if (o0 + r < nout) {
            float s = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * M; ++t) s = fmaf(P.coef[t], v[r + t], s);
            P.df[checked((int64_t)(o0 + r) * P.npix + px, (long long)nout * P.npix, kChkScanWrite)] = s;
        }
    }
}

__global__ void __launch_bounds__(kThreads) fz_to_df_kernel(const DfLaunch P) {
    const int nout = P.nz - 2 * P.m;
    const int64_t total = (int64_t)nout * P.npix;
    for (int64_t o = blockIdx.x * (int64_t)kThreads + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * kThreads) {
        const int c = (int)(o / P.npix) + P.m;
        const int64_t px = o - (int64_t)(c - P.m) * P.npix;
        float s = 0.f;
        for (int t = -P.m; t <= P.m; ++t)
            s = fmaf(P.coef[t + P.m],
                     __ldg(P.fz + checked((int64_t)(c + t) * P.npix + px, (long long)P.nz * P.npix, kChkScanRead)), s);
        P.df[checked(o, total, kChkScanWrite)] = s;
    }
}

__global__ void ff_convert_kernel(const float4* __restrict__ src, const GridMap sm, float4* __restrict__ dst,
                                  const GridMap dm) {
    const int64_t n = (int64_t)dm.nx * dm.ny * dm.nz;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(g % dm.nx);
        const int64_t r = g / dm.nx;
        const int j = (int)(r % dm.ny);
        const int k = (int)(r / dm.ny);
        dst[checked(node_index(dm, i, j, k), dm.stored_nodes, kChkGridWrite)] =
            __ldg(src + checked(node_index(sm, i, j, k), sm.stored_nodes, kChkGridRead));
    }
}

int grid_blocks(int64_t work, int threads) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * 16;
    return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

}  // namespace

template <int M>
static void launch_rows(const DfLaunch& L, cudaStream_t s) {
    const int nout = L.nz - 2 * M;
    const dim3 grid((unsigned)(((int64_t)L.npix + kThreads - 1) / kThreads), (unsigned)((nout + kRows - 1) / kRows));
    fz_to_df_rows_kernel<M><<<grid, kThreads, 0, s>>>(L);
}

cudaError_t launch_fz_to_df(const DfLaunch& L, cudaStream_t s) {
    const int64_t total = (int64_t)(L.nz - 2 * L.m) * L.npix;
    if (total <= 0) return cudaSuccess;
    const int64_t row_blocks = ((int64_t)(L.nz - 2 * L.m) + kRows - 1) / kRows;
    if (L.m >= 1 && L.m <= kMaxRegM && row_blocks <= 65535) {
        switch (L.m) {
            case 1: launch_rows<1>(L, s); break;
            case 2: launch_rows<2>(L, s); break;
            case 3: launch_rows<3>(L, s); break;
            case 4: launch_rows<4>(L, s); break;
            case 5: launch_rows<5>(L, s); break;
            case 6: launch_rows<6>(L, s); break;
            case 7: launch_rows<7>(L, s); break;
            default: launch_rows<8>(L, s); break;
        }
        return cudaGetLastError();
    }
    fz_to_df_kernel<<<grid_blocks(total, kThreads), kThreads, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_ff_convert(const float4* src, const GridMap& sm, float4* dst, const GridMap& dm,
                              cudaStream_t s) {
    const int64_t n = (int64_t)dm.nx * dm.ny * dm.nz;
    if (n <= 0) return cudaSuccess;
    ff_convert_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(src, sm, dst, dm);
    return cudaGetLastError();
}

PP_CHECK_READER(check_flags_fz_to_df)

}  // namespace pp
