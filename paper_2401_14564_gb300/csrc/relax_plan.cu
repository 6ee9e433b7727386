// Pixel-to-warp plan for the relaxed scan (K2), built on the device from an
// earlier scan's FIRE iteration counts.
//
// A warp of K2 runs an 8x4 pixel tile until its slowest column is done, and
// every height change or cell reload of its other 31 lanes holds that column
// up (the lanes diverge).  On flake60 the heaviest column takes 1457 FIRE
// updates against 537 on average; run alone it takes 0.35 ms, inside its tile
// 0.56 ms, and the scan ends with it.  The plan moves the k heaviest columns
// out of their tiles into warps of `lanes` lanes each (their tiles run them as
// idle lanes), so those columns diverge only among themselves.  Which warp
// computes a pixel never changes a value: a planned scan writes the same bits.
//
// Layout of the plan buffer (int32 words, sizes from pp_relax_plan_size):
//   [0, 8)             header: [1] lowest bin taken, [2] columns above that bin,
//                      [3] / [4] selection counters
//   hist   [kBins]     columns per cost bin (cost >> shift)
//   cost   [npix]      sum over heights of the earlier scan's iters
//   list   [hb*lanes]  the selected pixels, -1 in unused slots (hb = ceil(k/lanes))
//   mask   [ceil(npix/32)]  bit p set when pixel p is in the list
#include <algorithm>

#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kBins = 2048;
constexpr int kHdr = 8;

__global__ void __launch_bounds__(256) plan_cost_kernel(const int* __restrict__ iters, int nz, int npix, int shift,
                                                        int* hist, int* cost) {
    __shared__ int sh[kBins];
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        long long c = 0;
        for (int k = 0; k < nz; ++k) c += max(__ldg(iters + (size_t)k * npix + p), 0);
        const int ci = (int)min(c, (long long)0x7fffffff);
        cost[p] = ci;
        atomicAdd(&sh[min(ci >> shift, kBins - 1)], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x)
        if (sh[b]) atomicAdd(hist + b, sh[b]);
}

// The bin T with (columns above T) < k <= (columns at or above T); T = 0 when fewer than k columns
// exist.  One thread: 2048 steps.
__global__ void plan_threshold_kernel(int* hdr, const int* hist, int k) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int above = 0, t = 0;
    for (int b = kBins - 1; b >= 0; --b) {
        if (above + hist[b] >= k) { t = b; break; }
        above += hist[b];
    }
    hdr[1] = t;
    hdr[2] = above;
    hdr[3] = 0;
    hdr[4] = 0;
}

__global__ void __launch_bounds__(256) plan_select_kernel(int* hdr, const int* __restrict__ cost, int npix, int shift,
                                                          int k, int* list, unsigned* mask) {
    const int t = hdr[1], above = hdr[2];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        const int bin = min(cost[p] >> shift, kBins - 1);
        int slot = k;
        if (bin > t) slot = atomicAdd(hdr + 3, 1);              // < above <= k - 1 by construction
        else if (bin == t) slot = above + atomicAdd(hdr + 4, 1);
        if (slot < k) {
            list[slot] = p;
            atomicOr(mask + (p >> 5), 1u << (p & 31));
        }
    }
}

}  // namespace

static_assert(kHdr + kBins == 8 + 2048, "relax_plan_list_offset assumes this header and histogram");

size_t relax_plan_words(int npix, int k, int lanes) {
    return relax_plan_mask_offset(npix, k, lanes) + ((size_t)npix + 31) / 32;
}

cudaError_t launch_relax_plan(const int* iters, int nz, int npix, int max_iter, int k, int lanes, int* plan,
                              cudaStream_t s) {
    // cost <= nz * max_iter: the shift that brings it under kBins
    long long top = (long long)nz * (long long)max(max_iter, 1);
    int shift = 0;
    while ((top >> shift) >= kBins) ++shift;
    const long long hb = ((long long)k + lanes - 1) / lanes;
    int* hdr = plan;
    int* hist = plan + kHdr;
    int* cost = hist + kBins;
    int* list = plan + relax_plan_list_offset(npix);
    unsigned* mask = reinterpret_cast<unsigned*>(plan + relax_plan_mask_offset(npix, k, lanes));
    cudaError_t e = cudaMemsetAsync(hdr, 0, (size_t)(kHdr + kBins) * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(list, 0xff, (size_t)(hb * lanes) * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mask, 0, (size_t)((npix + 31) / 32) * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (int)std::min<long long>(((long long)npix + 255) / 256, 2LL * sms);
    plan_cost_kernel<<<blocks, 256, 0, s>>>(iters, nz, npix, shift, hist, cost);
    plan_threshold_kernel<<<1, 32, 0, s>>>(hdr, hist, k);
    plan_select_kernel<<<blocks, 256, 0, s>>>(hdr, cost, npix, shift, k, list, mask);
    return cudaGetLastError();
}

}  // namespace pp
