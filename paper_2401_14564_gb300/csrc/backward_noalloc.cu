// pp_backward_noalloc: pp_backward with its scratch taken from a fixed array
// inside the library instead of a caller-provided workspace.
//
// Some callers of this library cannot call cudaMalloc: code that runs inside a
// real-time acquisition or control loop, or a plugin inside a host program
// that forbids device allocations after start-up (cudaMalloc may block and
// synchronise the device), and C or Fortran callers that have no device
// allocator of their own.  For them the scratch of the adjoint lives in the
// file-scope array below: every GPU that loads this library holds those
// bytes until the process exits.
#include <string>

#include "pp_internal.cuh"

namespace pp {
namespace {

// Scratch of pp_backward: the 256-byte header plus one float4 per grid node,
// so grids of up to (32 MiB - 256 B) / 16 B = 2,097,136 stored nodes fit.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_backward_scratch[kStaticScratchBytes];

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// with the device current, on every call: a cached address would outlive a
// cudaDeviceReset or a new primary context, and the lookup costs nothing next
// to the adjoint.
pp_status scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_backward_scratch);
    if (e != cudaSuccess) return cuda_status(e, "pp_backward_noalloc cudaGetSymbolAddress");
    *out = p;
    return PP_OK;
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" {

size_t pp_backward_noalloc_capacity(void) { return kStaticScratchBytes; }

pp_status pp_backward_noalloc(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                              const float* ff, const pp_scan* scan, const pp_tip* tip,
                              const pp_df* df_params, const float* pos, const float* g_df,
                              const pp_grads* grads, pp_stream stream) {
    set_error("");
    // the same checks, in the same order and with the same status codes, as pp_backward
    BwdLaunch L;
    size_t adj_bytes = 0;
    pp_status st = backward_prepare("pp_backward_noalloc", atoms, probe, grid, ff, scan, tip, df_params, pos, g_df,
                                    grads, &L, &adj_bytes);
    if (st != PP_OK) return st;
    const size_t need = kBwdHeader + adj_bytes;
    if (need > kStaticScratchBytes) {
        set_error("pp_backward_noalloc: the grid needs " + std::to_string(need) +
                  " bytes of scratch but the library's static scratch holds " +
                  std::to_string(kStaticScratchBytes) + " bytes; use pp_backward with a caller workspace");
        return PP_ERR_CAPACITY;
    }
    void* ws = nullptr;
    st = scratch_address(&ws);
    if (st != PP_OK) return st;
    return backward_launch("pp_backward_noalloc", L, ws, adj_bytes, (cudaStream_t)stream);
}

}  // extern "C"
