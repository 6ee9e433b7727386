// Internal definitions shared by the CUDA translation units of libpp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>

#include "pp.h"

namespace pp {

// Physical constants (own copies; SI-exact electron-volt).
constexpr double kCoulomb = 14.3996454784;          // k_e, eV*A/e^2
constexpr double kEvA2ToNm = 16.02176634;           // 1 eV/A^2 in N/m
constexpr double kNmToEvA2 = 1.0 / 16.02176634;     // 1 N/m in eV/A^2
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxDfHalfWidth = 31;                 // df stencil of at most 63 taps

// Separable node addressing: the float4 index of node (i,j,k) is
// X(i) + Y(j) + Z(k), each term ((v >> sh) * mul) + ((v & mask) << lsh).
// Linear layout: sh = mask = lsh = 0 and mul = 1, nx, nx*ny.  Bricked
// layout: sh = log2(brick side), mul = brick volume times the number of
// bricks before it along that axis, the remainder placed x-fastest inside.
struct AxisMap {
    int sh, mul, mask, lsh;
};

struct GridMap {
    AxisMap ax, ay, az;
    int nx, ny, nz;
    int64_t stored_nodes;  // node slots including brick padding
    int interp;            // 0: float4 (Fx, Fy, Fz, E) per node; 1: E per node (tricubic)
};

__host__ __device__ __forceinline__ int axis_off(const AxisMap& a, int v) {
    return ((v >> a.sh) * a.mul) + ((v & a.mask) << a.lsh);
}

__host__ __device__ __forceinline__ int node_index(const GridMap& g, int i, int j, int k) {
    return axis_off(g.ax, i) + axis_off(g.ay, j) + axis_off(g.az, k);
}

// Bounds-checked builds (-DPP_CHECKED: the library the bounds-check test loads, standing in for
// a memory checker): every global gather and scatter index of the kernels goes through
// checked(i, n, bit), which there records `bit` in this translation unit's flag word and
// substitutes index 0 when i is outside [0, n); in a normal build it returns i unchanged.
enum CheckBits : unsigned {
    kChkGridRead = 1u,    // force-field / energy grid reads
    kChkGridWrite = 2u,   // grid writes, grid-adjoint accumulation
    kChkScanRead = 4u,    // relaxed positions, Fz, loss weights read back
    kChkScanWrite = 8u,   // positions, Fz, iterations, df, eigenvalues written
    kChkFft = 16u,        // FFT scratch and input arrays
};
#ifdef PP_CHECKED
namespace {
__device__ unsigned int g_check_flags;  // one per translation unit
}
template <class I>
__device__ __forceinline__ I checked(I i, long long n, unsigned bit) {
    if ((unsigned long long)(long long)i < (unsigned long long)n) return i;
    atomicOr(&g_check_flags, bit);
    return I(0);
}
// Host function `fn` returning and clearing this translation unit's flag word.
#define PP_CHECK_READER(fn)                                           \
    unsigned int fn() {                                               \
        unsigned int v = 0, z = 0;                                    \
        cudaMemcpyFromSymbol(&v, g_check_flags, sizeof(v));           \
        cudaMemcpyToSymbol(g_check_flags, &z, sizeof(z));             \
        return v;                                                     \
    }
#else
template <class I>
__device__ __forceinline__ I checked(I i, long long, unsigned) { return i; }
#define PP_CHECK_READER(fn)
#endif

// Calls f(std::bool_constant<a>, std::bool_constant<b>, std::bool_constant<c>)
// for the runtime flags a, b, c: one place that turns the pair-term options
// (minimum image, Coulomb cutoff, tip quadrupole) into kernel template arguments.
template <class F>
inline auto with_flags(bool a, bool b, bool c, F&& f) {
    using T = std::true_type;
    using N = std::false_type;
    if (a) {
        if (b) return c ? f(T{}, T{}, T{}) : f(T{}, T{}, N{});
        return c ? f(T{}, N{}, T{}) : f(T{}, N{}, N{});
    }
    if (b) return c ? f(N{}, T{}, T{}) : f(N{}, T{}, N{});
    return c ? f(N{}, N{}, T{}) : f(N{}, N{}, N{});
}

// (z_top + d0z - z0) / dz and sdz / dz in FP64, each returned as a float and the float remainder
// (the relaxation's per-height cell coordinates, see relax_core.cuh).
__host__ __device__ inline void split_height_steps(float z_top, float d0z, float sdz, float z0, float dz, float* fz0,
                                                   float* fz0_lo, float* st, float* st_lo) {
    const double f = ((double)z_top + (double)d0z - (double)z0) / (double)dz;
    const double t = (double)sdz / (double)dz;
    *fz0 = (float)f;
    *fz0_lo = (float)(f - (double)*fz0);
    *st = (float)t;
    *st_lo = (float)(t - (double)*st);
}

// Host-side helpers (api.cu).
bool make_grid_map(const pp_grid* g, GridMap* out, std::string* why);
void set_error(const std::string& msg);
pp_status cuda_status(cudaError_t e, const char* what);
int df_half_width(double A_pp, double dz);
// coef[s + m] (s = -m..m) multiplies Fz at height index c + s for the output
// centred at c; includes the -(f0/2k) * 2/(pi a^2) prefactor and eV/A^2 -> N/m.
void df_stencil(double A_pp, double dz, double k, double f0, int m, float* coef);

// Launchers (one per kernel translation unit).
struct FFLaunch {
    const float *x, *y, *z, *R, *eps, *q;
    int n;
    float R_pp, eps_pp, kQ, core_frac, coul_rc;
    float kQzz;  // k_e Qzz / 2 (0: no tip quadrupole)
    int min_image;
    float Lx, Ly;
    float x0, y0, z0, dx, dy, dz;
    GridMap map;
    float4* ff;   // map.interp == 0
    float* ffE;   // map.interp == 1: energies only
    int zpt;  // z-nodes per thread: 4, 8 or 16
    int forces_only;  // 1: no energy sums, E slots written as 0 (map.interp == 0, not split)
    int split;     // 1: point charges per unit probe charge into ffel / ffelE, the rest into ff / ffE
    float4* ffel;  // split, map.interp == 0
    float* ffelE;  // split, map.interp == 1
    int kbeg, kend;  // node layers written: z index in [kbeg, kend) (0, nz for the whole grid)
};
cudaError_t launch_ff_assemble(const FFLaunch& L, cudaStream_t s);
// out = a + Q b over nfloats floats (16-byte aligned buffers; out may alias a)
cudaError_t launch_ff_combine(const float* a, const float* b, float Q, float* out, int64_t nfloats, cudaStream_t s);

struct RelaxLaunch {
    const float4* ff;   // map.interp == 0
    const float* ffE;   // map.interp == 1
    GridMap map;
    float gx0s, gy0s, gz0s, inv_dx, inv_dy, inv_dz;  // cell coordinate f = p * inv_d + g0s, g0s = -origin/d
    // z cell coordinate of the first height's rest position (z_top + d0z - z0) / dz and the step
    // sdz / dz per height, each a float and the float remainder of its FP64 value
    float fz0, fz0_lo, st, st_lo;
    int periodic_xy;
    int snx, sny, snz;
    float sx0, sy0, spx, spy, z_top, sdz;
    int layout;                           // 0 linear, 1 bricked
    float kx, ky, kR, R0, d0x, d0y, d0z;  // eV/A^2, A
    float R0sq, c0;                       // R0^2 and |d0|^2 - R0^2 (rounding residue of d0)
    int max_iter, n_min;
    float ftol2, dt0, dt_max, f_inc, f_dec, alpha0, f_alpha, inv_mass;
    int polish;  // Newton steps after FIRE stops below ftol (0: none)
    float* pos;
    float* fz;
    int* iters;
    int df_m;      // -1: no fused df
    float* df;
    int* zspan;    // nullable: [0] lowest, [1] highest node layer an interpolation read (atomic min / max)
    // nullable: a pixel-to-warp plan (relax_plan.cu): warps 0..plan_hblocks-1 run the listed pixels,
    // plan_lanes lanes each; the tiles after them skip the pixels whose mask bit is set
    const int* plan_list;
    const unsigned* plan_mask;
    int plan_hblocks, plan_lanes;
    float coef[2 * kMaxDfHalfWidth + 1];
};
cudaError_t launch_relax_scan(const RelaxLaunch& L, cudaStream_t s);

struct DfLaunch {
    const float* fz;
    float* df;
    int nz, npix, m;
    float coef[2 * kMaxDfHalfWidth + 1];
};
cudaError_t launch_fz_to_df(const DfLaunch& L, cudaStream_t s);
// Pixel-to-warp plan of the scan from an earlier scan's iteration counts (relax_plan.cu): buffer size in
// int32 words, and its build on the stream (k heaviest columns, `lanes` per warp).
size_t relax_plan_words(int npix, int k, int lanes);
cudaError_t launch_relax_plan(const int* iters, int nz, int npix, int max_iter, int k, int lanes, int* plan,
                              cudaStream_t s);
// Offsets of the plan's pixel list and mask inside the buffer (int32 words).
inline size_t relax_plan_list_offset(int npix) { return 8 + 2048 + (size_t)npix; }
inline size_t relax_plan_mask_offset(int npix, int k, int lanes) {
    return relax_plan_list_offset(npix) + (size_t)((k + lanes - 1) / lanes) * lanes;
}

struct BwdLaunch {
    // atoms and probe
    const float *ax, *ay, *az, *aR, *aeps, *aq;
    int n;
    float R_pp, eps_pp, kQ, ke, Q, core_frac, coul_rc;
    float Qzz, kQzz;  // tip quadrupole and k_e Qzz / 2
    int min_image;
    float Lx, Ly;
    // grid (node positions x0 + i*dx ..., cell coordinate p * inv_d + g0s)
    const float4* ff;
    const float* ffE;  // node energies of a tricubic grid (map.interp = 1), else null
    GridMap map;
    int layout;
    float x0, y0, z0, dx, dy, dz;
    float gx0s, gy0s, gz0s, inv_dx, inv_dy, inv_dz;
    int periodic_xy;
    // scan and tip springs (eV/A^2); nm converts a gradient per eV/A^2 into per N/m
    int snx, sny, snz;
    float sx0, sy0, spx, spy, z_top, sdz;
    float kx, ky, kR, R0, d0x, d0y, d0z, R0sq, c0, nm;
    // df stencil and the forward's saved state
    int m, nzo;
    float coef[2 * kMaxDfHalfWidth + 1];
    const float* pos;
    const float* g_df;
    // outputs (accumulated) and caller scratch
    float *gx, *gy, *gz, *gq, *gR, *geps, *gtip;
    float4* gbar;   // grid adjoint dL/dF_g (force grids)
    float* gbarE;   // grid adjoint dL/dE_g (energy grids)
    int* slab;
    float* qsum;    // {sum_i q_i C_i, sum_i q_i Cq_i} when Qzz != 0 (force grids)
    double* qsumd;  // the same sums on energy grids
};
cudaError_t launch_backward(const BwdLaunch& L, cudaStream_t s);
// Host side of the adjoint entry points (api.cu): argument checks into a prepared launch, then the
// launch on a workspace of kBwdHeader + adj_bytes bytes.  `who` prefixes the error messages.
pp_status backward_prepare(const std::string& who, const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                           const float* ff, const pp_scan* scan, const pp_tip* tip, const pp_df* dfp,
                           const float* pos, const float* g_df, const pp_grads* grads, BwdLaunch* L,
                           size_t* adj_bytes);
pp_status backward_launch(const std::string& who, BwdLaunch& L, void* ws, size_t adj_bytes, cudaStream_t s);

struct BatchArgs {
    const pp_mol_desc* descs;
    int nmol;
    pp_batch_params params;
    pp_atoms atoms;
    float* ff;
    float *pos, *fz, *df;
    int* iters;
    void* ws;
    int df_m;
    float coef[2 * kMaxDfHalfWidth + 1];
};
size_t batch_workspace_bytes(int nmol);
cudaError_t launch_batch(const BatchArgs& A, cudaStream_t s);

struct FftLaunch {
    const float *f, *g;  // sample field and tip density, [nz][ny][nx]
    float4* ff;          // (Fx, Fy, Fz, E) per node, linear layout
    void* ws;            // 3 complex values per node
    int nx, ny, nz;
    float dx, dy, dz;
    float scale, power;
    int accumulate;
};
size_t fft_workspace_bytes(int nx, int ny, int nz);
cudaError_t launch_fft_correlate(const FftLaunch& L, cudaStream_t s);

struct IetsLaunch {
    const float4* ff;   // map.interp == 0
    const float* ffE;   // map.interp == 1
    GridMap map;
    int layout;
    float gx0s, gy0s, gz0s, inv_dx, inv_dy, inv_dz;
    int periodic_xy;
    int snx, sny, snz;
    float sx0, sy0, spx, spy, z_top, sdz;
    float kx, ky, kR, R0, d0x, d0y, d0z, R0sq, c0;
    const float* pos;
    float* eig;
    float* hw;
    float hw_unit;  // hbar sqrt(1 eV/A^2 / m) in meV
};
cudaError_t launch_iets(const IetsLaunch& L, cudaStream_t s);

// Workspace of pp_backward: a 256-byte header (z-slab bounds) then the grid adjoint.
constexpr size_t kBwdHeader = 256;

cudaError_t launch_ff_convert(const float4* src, const GridMap& sm, float4* dst, const GridMap& dm,
                              cudaStream_t s);

}  // namespace pp
