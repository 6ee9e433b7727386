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
#include <mutex>
#include <string>

#include "pp_internal.cuh"

namespace pp {
namespace {

// Scratch of pp_backward: the 256-byte header plus one float4 per grid node,
// so grids of up to (32 MiB - 256 B) / 16 B = 2,097,136 stored nodes fit.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_backward_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
pp_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "pp_backward_noalloc cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("pp_backward_noalloc: device ordinal " + std::to_string(dev) + " beyond 63");
        return PP_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_backward_scratch);
        if (e != cudaSuccess) return cuda_status(e, "pp_backward_noalloc cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
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
    const size_t need = pp_backward_workspace(grid);
    if (need == 0) {
        set_error("pp_backward_noalloc: invalid grid");
        return PP_ERR_SHAPE;
    }
    if (need > kStaticScratchBytes) {
        set_error("pp_backward_noalloc: the grid needs " + std::to_string(need) +
                  " bytes of scratch but the library's static scratch holds " +
                  std::to_string(kStaticScratchBytes) + " bytes; use pp_backward with a caller workspace");
        return PP_ERR_CAPACITY;
    }
    void* ws = nullptr;
    const pp_status st = scratch_address(&ws);
    if (st != PP_OK) return st;
    return pp_backward(atoms, probe, grid, ff, scan, tip, df_params, pos, g_df, grads, ws, kStaticScratchBytes,
                       stream);
}

}  // extern "C"
