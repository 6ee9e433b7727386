// Read-bandwidth probe: a measurement aid of the benchmark, not part of the
// method.  The relaxed scan (K2) reads its corner values from a force-field
// slab that stays L2-resident; its roofline wants the bandwidth at which this
// GPU's L2 serves reads, which no stock kernel measures cleanly (a reduction
// is bound by its own arithmetic, a copy adds writes).  This kernel reads a
// buffer `passes` times with 16-byte loads that skip L1 (ld.global.cg), from
// enough resident threads to hide the latency, and sums what it reads so that
// no load is dead.
#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) read_probe_kernel(const float4* __restrict__ buf, long long n4,
                                                                   int passes, float* sink) {
    // passes x n4 loads in all, taken as one sequence that wraps around the buffer: each thread
    // issues kInFlight independent loads before it adds any of them, so a buffer smaller than
    // (threads x kInFlight x 16 B) still keeps enough bytes in flight to cover the L2 latency
    constexpr int kInFlight = 8;
    const long long stride = (long long)gridDim.x * kProbeThreads;
    const long long total = (long long)passes * n4;
    const long long step = stride % n4;
    long long j = (long long)blockIdx.x * kProbeThreads + threadIdx.x;
    long long i = j % n4;
    float4 acc[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    for (; j + (kInFlight - 1) * stride < total; j += kInFlight * stride) {
        float4 u[kInFlight];
#pragma unroll
        for (int q = 0; q < kInFlight; ++q) {
            u[q] = __ldcg(buf + i);
            i += step;
            if (i >= n4) i -= n4;
        }
#pragma unroll
        for (int q = 0; q < kInFlight; ++q) {
            float4& a = acc[q & 1];
            a.x += u[q].x; a.y += u[q].y; a.z += u[q].z; a.w += u[q].w;
        }
    }
    for (; j < total; j += stride) {
        const float4 u = __ldcg(buf + i);
        acc[0].x += u.x; acc[0].y += u.y; acc[0].z += u.z; acc[0].w += u.w;
        i += step;
        if (i >= n4) i -= n4;
    }
    const float s = (acc[0].x + acc[0].y) + (acc[0].z + acc[0].w) + (acc[1].x + acc[1].y) + (acc[1].z + acc[1].w);
    if (s == -1.2345678e-30f) *sink = s;  // keeps the sums (and so the loads) alive
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" {

pp_status pp_read_probe(const float* buf, size_t nfloats, int passes, float* sink, pp_stream stream) {
    set_error("");
    if (!buf || !sink) { set_error("pp_read_probe: NULL argument"); return PP_ERR_ARG; }
    if (reinterpret_cast<uintptr_t>(buf) % 16 != 0 || nfloats % 4 != 0 || nfloats == 0) {
        set_error("pp_read_probe: buf must be 16-byte aligned and hold a positive multiple of 4 floats");
        return PP_ERR_ARG;
    }
    if (passes < 1 || passes > 1000000) { set_error("pp_read_probe: passes must be in [1, 10^6]"); return PP_ERR_ARG; }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, read_probe_kernel, kProbeThreads, 0);
    if (e != cudaSuccess) return cuda_status(e, "pp_read_probe device query");
    read_probe_kernel<<<sms * (per_sm > 0 ? per_sm : 1), kProbeThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(buf), (long long)(nfloats / 4), passes, sink);
    return cuda_status(cudaGetLastError(), "pp_read_probe launch");
}

}  // extern "C"
