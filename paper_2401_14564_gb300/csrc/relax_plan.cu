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

// Also clears the list (-1) and the mask for plan_select_kernel, which runs after it.
__global__ void __launch_bounds__(256) plan_cost_kernel(const int* __restrict__ iters, int nz, int npix, int shift,
                                                        int* hist, int* cost, int* list, int nlist, unsigned* mask,
                                                        int nmask) {
    __shared__ int sh[kBins];
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) sh[b] = 0;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    for (int q = gt; q < nlist; q += gs) list[q] = -1;
    for (int q = gt; q < nmask; q += gs) mask[q] = 0u;
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

// The bin T with (columns above T) < k <= (columns at or above T), and the count above it; T = 0
// when fewer than k columns exist.  One block of 1024 threads: thread t holds the bins 2047 - 2t and
// 2046 - 2t, and a scan over the threads (costliest bins first) finds the one bin where the running
// count reaches k.
__global__ void __launch_bounds__(1024) plan_threshold_kernel(int* hdr, const int* hist, int k) {
    static_assert(kBins == 2 * 1024, "two bins per thread");
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int h0 = hist[kBins - 1 - 2 * t], h1 = hist[kBins - 2 - 2 * t];
    int v = h0 + h1;
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int x = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += n;
        }
        wsum[lane] = x;
    }
    __syncthreads();
    const int before = (w ? wsum[w - 1] : 0) + v - (h0 + h1);  // columns in costlier bins
    const int incl0 = before + h0, incl1 = incl0 + h1;
    if (incl0 >= k && before < k) {
        hdr[1] = kBins - 1 - 2 * t;
        hdr[2] = before;
    } else if (incl1 >= k && incl0 < k) {
        hdr[1] = kBins - 2 - 2 * t;
        hdr[2] = incl0;
    } else if (t == 1023 && incl1 < k) {  // fewer than k columns: every one is taken
        hdr[1] = 0;
        hdr[2] = incl1 - h1;
    }
    if (t == 0) {
        hdr[3] = 0;
        hdr[4] = 0;
    }
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
    const cudaError_t e = cudaMemsetAsync(hdr, 0, (size_t)(kHdr + kBins) * sizeof(int), s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (int)std::min<long long>(((long long)npix + 255) / 256, 2LL * sms);
    plan_cost_kernel<<<blocks, 256, 0, s>>>(iters, nz, npix, shift, hist, cost, list, (int)(hb * lanes), mask,
                                            (npix + 31) / 32);
    plan_threshold_kernel<<<1, 1024, 0, s>>>(hdr, hist, k);
    plan_select_kernel<<<blocks, 256, 0, s>>>(hdr, cost, npix, shift, k, list, mask);
    return cudaGetLastError();
}

}  // namespace pp
