// K6: many molecules in one persistent launch (force field -> relaxed scan ->
// df per molecule, exactly the single-molecule path of K1 + K2).
//
// Work items:  FF tile  = fw x (32/fw) grid columns x ZPT z-nodes of one molecule;
//              relax tile = rw x (32/rw) pixels x all heights of one molecule
// (fw, rw in {4, 8, 16} at launch time, ZPT in {4, 8} as a template argument;
// the shapes change the schedule, never a value).
// Every warp is an independent worker: lane 0 takes the next item index from
// a device counter.  The item list is a sequence of segments
//   FF(0), FF(1), R(0), FF(2), R(1), ..., FF(n-1), R(n-2), R(n-1)
// (prefix sums built by a planning kernel), so a relax tile of molecule m is
// handed out only after all force-field tiles of m were handed out -- and
// those never wait on anything, so every wait ends.  A relax tile still waits
// for its molecule's completion counter with a bounded spin (a timeout sets a
// status bit and the warp stops); force-field values written in this kernel
// are read back with plain cached loads after an acquire, never through the
// read-only path.  Many molecules' tiles are in flight at once, which fills
// the GPU even though one 128x128 scan is only 512 warps.
#include <cstring>

#include "ff_core.cuh"
#include "relax_core.cuh"

namespace pp {
namespace {

constexpr int kThreads = 128;  // 4 independent warps per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kMinCtas = 5;    // resident CTAs per SM the register budget is sized for

struct BatchLaunch {
    const pp_mol_desc* descs;
    int nmol;
    const float *ax, *ay, *az, *aR, *aeps, *aq;
    int n_atoms_total;
    float4* ff;
    long long ff_cap;
    float *pos, *fz, *df;
    int* iters;
    long long out_cap, df_cap;
    // probe (shared)
    float R_pp, eps_pp, kQ, core_frac, coul_rc, kQzz;
    int min_image, periodic_xy;
    // tip, FIRE and df stencil, under the names relax_pixel expects
    float kx, ky, kR, R0, d0x, d0y, d0z, R0sq, c0;
    int max_iter, n_min;
    float ftol2, dt0, dt_max, f_inc, f_dec, alpha0, f_alpha, inv_mass;
    float sdz;
    int df_m;
    const float* coef;  // in ws, written by the planning kernel
    // scratch
    unsigned long long* counter;
    int* status;
    long long* seg_start;  // [2 nmol + 1]
    int* done_ff;          // [nmol]
    float* coef_ws;
    long long spin_limit;
    int wait_extra;
    int forces_only;  // E slots written as 0, energy sums skipped
    int zpt;          // z-nodes per FF tile
    int fw_sh, rw_sh; // log2 of the FF and relax tile widths (4, 8 or 16 lanes along x)
    float coef_init[2 * kMaxDfHalfWidth + 1];
};

// Per-molecule geometry for relax_pixel (linear layout).
struct MolRelax {
    const float4* ff;
    GridMap map;
    float inv_dx, inv_dy, inv_dz, gx0s, gy0s, gz0s;
    float fz0, fz0_lo, st, st_lo;
    int periodic_xy;
    int snx, sny, snz;
    float sx0, sy0, spx, spy, z_top;
    float *pos, *fz, *df;
    int* iters;
};

__device__ __forceinline__ long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

__device__ __forceinline__ long long ff_tiles(const BatchLaunch& B, const pp_mol_desc& D) {
    return cdiv(D.nx, 1 << B.fw_sh) * cdiv(D.ny, 32 >> B.fw_sh) * cdiv(D.nz, B.zpt);
}
__device__ __forceinline__ long long relax_tiles(const BatchLaunch& B, const pp_mol_desc& D) {
    return cdiv(D.snx, 1 << B.rw_sh) * cdiv(D.sny, 32 >> B.rw_sh);
}

__device__ __forceinline__ bool finite_pos(float v) { return isfinite(v) && v > 0.f; }

// Every index a molecule's tiles will touch lies inside the caller's buffers.
__device__ bool mol_valid(const BatchLaunch& B, const pp_mol_desc& D) {
    if (D.nx < 2 || D.ny < 2 || D.nz < 2 || !finite_pos(D.dx) || !finite_pos(D.dy) || !finite_pos(D.dz)) return false;
    if (D.nx > (1 << 22) || D.ny > (1 << 22) || D.nz > (1 << 22)) return false;  // the cell lookup's fast floor
    if (!isfinite(D.x0) || !isfinite(D.y0) || !isfinite(D.z0)) return false;
    const long long nodes = (long long)D.nx * D.ny * D.nz;
    if (nodes >= (1LL << 31) || D.ff_offset < 0 || D.ff_offset + nodes > B.ff_cap) return false;
    if (D.n_atoms < 0 || D.atom_offset < 0 || (long long)D.atom_offset + D.n_atoms > B.n_atoms_total) return false;
    if (D.snx < 1 || D.sny < 1 || D.snz < 2 * B.df_m + 1) return false;
    if (!isfinite(D.sx0) || !isfinite(D.sy0) || !isfinite(D.spx) || !isfinite(D.spy) || !isfinite(D.z_top)) return false;
    const long long pts = (long long)D.snx * D.sny * D.snz;
    if (3 * pts >= (1LL << 31) || D.out_offset < 0 || D.out_offset + pts > B.out_cap) return false;
    const long long dfn = (long long)D.snx * D.sny * (D.snz - 2 * B.df_m);
    if (D.df_offset < 0 || D.df_offset + dfn > B.df_cap) return false;
    return true;
}

// Segment s of the item list -> (molecule, is force-field segment).
__device__ __forceinline__ void decode_segment(int s, int nmol, int& mol, bool& ff) {
    if (s == 0) { mol = 0; ff = true; }
    else if (s == 2 * nmol - 1) { mol = nmol - 1; ff = false; }
    else if (s & 1) { mol = (s + 1) >> 1; ff = true; }
    else { mol = (s >> 1) - 1; ff = false; }
}

__global__ void __launch_bounds__(1024) batch_plan_kernel(const BatchLaunch B) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        *B.counter = 0ULL;
        *B.status = 0;
        carry = 0;
    }
    for (int c = tid; c < 2 * B.df_m + 1; c += blockDim.x) B.coef_ws[c] = B.coef_init[c];
    for (int m = tid; m < B.nmol; m += blockDim.x) B.done_ff[m] = 0;
    __syncthreads();
    const int nseg = 2 * B.nmol;
    for (int base = 0; base < nseg; base += blockDim.x) {
        const int s = base + tid;
        long long len = 0;
        if (s < nseg) {
            int mol;
            bool ff;
            decode_segment(s, B.nmol, mol, ff);
            const pp_mol_desc D = B.descs[mol];
            if (mol_valid(B, D)) len = ff ? ff_tiles(B, D) : relax_tiles(B, D);
            else if (ff) atomicOr(B.status, PP_BATCH_BAD_DESC);
        }
        // inclusive block scan of len
        long long v = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            long long w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const long long before = carry + (warp > 0 ? wsum[warp - 1] : 0);
        if (s < nseg) B.seg_start[s] = before + v - len;
        __syncthreads();
        if (tid == 0) carry += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (tid == 0) B.seg_start[nseg] = carry;
}

__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void add_release(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// kZC: z-nodes computed (kZPT, or kZPT / 2 for a column's last tile when that many remain)
template <int kZPT, bool kMinImage, bool kCutoff, bool kQuad, bool kForcesOnly, int kZC = kZPT>
__device__ __forceinline__ void ff_tile(const BatchLaunch& B, const pp_mol_desc& D, long long tile, float4* s0,
                                        float4* s1, float4* s2, float4* s3, int lane) {
    constexpr int ZP = kZC / 2;
    const int fw = 1 << B.fw_sh;
    const long long tx_n = cdiv(D.nx, fw), ty_n = cdiv(D.ny, 32 >> B.fw_sh);
    const int tz = (int)(tile / (tx_n * ty_n));
    const long long r = tile - (long long)tz * tx_n * ty_n;
    const int ty = (int)(r / tx_n), tx = (int)(r - (long long)ty * tx_n);
    const int i = tx * fw + (lane & (fw - 1)), j = ty * (32 >> B.fw_sh) + (lane >> B.fw_sh), k0 = tz * kZPT;
    const float gx = D.x0 + i * D.dx, gy = D.y0 + j * D.dy;
    float2 gz[ZP];
#pragma unroll
    for (int t = 0; t < ZP; ++t) gz[t] = make_float2(D.z0 + (k0 + 2 * t) * D.dz, D.z0 + (k0 + 2 * t + 1) * D.dz);
    float2 fx[ZP], fy[ZP], fz[ZP], en[ZP];
#pragma unroll
    for (int t = 0; t < ZP; ++t) fx[t] = fy[t] = fz[t] = en[t] = make_float2(0.f, 0.f);
    const FFConst cst = ff_const(B.R_pp, B.eps_pp, B.kQ, B.core_frac, D.nx * D.dx, D.ny * D.dy,
                                 kCutoff ? B.coul_rc : 0.f, kQuad ? B.kQzz : 0.f);
    for (int base = 0; base < D.n_atoms; base += 32) {
        const int cnt = min(32, D.n_atoms - base);
        __syncwarp();
        if (lane < cnt) {
            const int g = D.atom_offset + base + lane;
            ff_stage_atom(cst, B.ax[g], B.ay[g], B.az[g], B.aR[g], B.aeps[g], B.aq[g], s0[lane], s1[lane], s2[lane],
                          s3[lane]);
        }
        __syncwarp();
        ff_accumulate<ZP, kMinImage, kCutoff, kQuad, true>(s0, s1, s2, s3, cnt, cst, gx, gy, gz, fx, fy, fz, en);
    }
    if (i < D.nx && j < D.ny) {
        const long long first = D.ff_offset + (long long)j * D.nx + i;
        const long long plane = (long long)D.nx * D.ny;
        auto at = [&](int k) { return checked(first + k * plane, (long long)B.ff_cap, kChkGridWrite); };
#pragma unroll
        for (int t = 0; t < ZP; ++t) {
            const int k = k0 + 2 * t;
            const float2 e = kForcesOnly ? make_float2(0.f, 0.f) : en[t];
            if (k < D.nz) B.ff[at(k)] = make_float4(fx[t].x, fy[t].x, fz[t].x, e.x);
            if (k + 1 < D.nz) B.ff[at(k + 1)] = make_float4(fx[t].y, fy[t].y, fz[t].y, e.y);
        }
    }
}

template <int kZPT, bool kMinImage, bool kCutoff, bool kQuad, bool kForcesOnly>
__global__ void __launch_bounds__(kThreads, kMinCtas) batch_kernel(const BatchLaunch B) {
    __shared__ float4 st[kWarps][4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long total = B.seg_start[2 * B.nmol];
    for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(B.counter, 1ULL);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        // segment holding item t: the last s with seg_start[s] <= t
        int lo = 0, hi = 2 * B.nmol - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.seg_start[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        int mol;
        bool ff;
        decode_segment(lo, B.nmol, mol, ff);
        const long long tile = t - B.seg_start[lo];
        const pp_mol_desc D = B.descs[mol];
        if (ff) {
            const long long per_z = cdiv(D.nx, 1 << B.fw_sh) * cdiv(D.ny, 32 >> B.fw_sh);
            const int k0 = (int)(tile / per_z) * kZPT;
            if (kZPT == 8 && D.nz - k0 <= 4)
                ff_tile<kZPT, kMinImage, kCutoff, kQuad, kForcesOnly, 4>(B, D, tile, st[warp][0], st[warp][1],
                                                                          st[warp][2], st[warp][3], lane);
            else
                ff_tile<kZPT, kMinImage, kCutoff, kQuad, kForcesOnly>(B, D, tile, st[warp][0], st[warp][1],
                                                                       st[warp][2], st[warp][3], lane);
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                add_release(B.done_ff + mol, 1);
            }
            continue;
        }
        // relax tile: wait (bounded) for every force-field tile of this molecule
        const int sff = mol == 0 ? 0 : 2 * mol - 1;
        const int need = (int)(B.seg_start[sff + 1] - B.seg_start[sff]) + B.wait_extra;
        int ok = 1;
        if (lane == 0) {
            long long polls = 0;
            while (load_acquire(B.done_ff + mol) < need) {
                if (++polls > B.spin_limit) {
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0) atomicOr(B.status, PP_BATCH_TIMEOUT);
            break;
        }
        __syncwarp();
        MolRelax G;
        G.ff = B.ff + D.ff_offset;
        G.map.nx = D.nx; G.map.ny = D.ny; G.map.nz = D.nz;
        G.map.ax = {0, 1, 0, 0};
        G.map.ay = {0, D.nx, 0, 0};
        G.map.az = {0, D.nx * D.ny, 0, 0};
        G.map.stored_nodes = (int64_t)D.nx * D.ny * D.nz;
        G.map.interp = 0;
        G.inv_dx = 1.f / D.dx; G.inv_dy = 1.f / D.dy; G.inv_dz = 1.f / D.dz;
        G.gx0s = (float)(-(double)D.x0 / (double)D.dx);
        G.gy0s = (float)(-(double)D.y0 / (double)D.dy);
        G.gz0s = (float)(-(double)D.z0 / (double)D.dz);
        split_height_steps(D.z_top, B.d0z, B.sdz, D.z0, D.dz, &G.fz0, &G.fz0_lo, &G.st, &G.st_lo);
        G.periodic_xy = B.periodic_xy;
        G.snx = D.snx; G.sny = D.sny; G.snz = D.snz;
        G.sx0 = D.sx0; G.sy0 = D.sy0; G.spx = D.spx; G.spy = D.spy; G.z_top = D.z_top;
        G.fz = B.fz + D.out_offset;
        G.pos = B.pos ? B.pos + 3 * D.out_offset : nullptr;
        G.iters = B.iters ? B.iters + D.out_offset : nullptr;
        G.df = B.df + D.df_offset;
        const int rw = 1 << B.rw_sh;
        const int tiles_x = (D.snx + rw - 1) / rw;
        const int ty = (int)(tile / tiles_x), tx = (int)(tile - (long long)ty * tiles_x);
        relax_pixel<0, true, false, true>(G, B, tx * rw + (lane & (rw - 1)), ty * (32 >> B.rw_sh) + (lane >> B.rw_sh));
    }
}

}  // namespace

size_t batch_workspace_bytes(int nmol) {
    if (nmol < 1) return 0;
    const size_t b = 320 + 8 * (2 * (size_t)nmol + 1) + 4 * (size_t)nmol;
    return (b + 15) & ~size_t(15);
}

cudaError_t launch_batch(const BatchArgs& A, cudaStream_t s) {
    BatchLaunch B;
    memset(&B, 0, sizeof(B));
    B.descs = A.descs; B.nmol = A.nmol;
    B.ax = A.atoms.x; B.ay = A.atoms.y; B.az = A.atoms.z; B.aR = A.atoms.R; B.aeps = A.atoms.eps; B.aq = A.atoms.q;
    B.n_atoms_total = A.atoms.n;
    B.ff = reinterpret_cast<float4*>(A.ff);
    B.ff_cap = A.params.ff_capacity;
    B.pos = A.pos; B.fz = A.fz; B.df = A.df; B.iters = A.iters;
    B.out_cap = A.params.out_capacity; B.df_cap = A.params.df_capacity;
    const pp_batch_params& P = A.params;
    B.R_pp = P.probe.R_pp; B.eps_pp = P.probe.eps_pp;
    B.kQ = (float)(kCoulomb * (double)P.probe.Q);
    B.kQzz = (float)(0.5 * kCoulomb * (double)P.probe.Qzz);
    B.core_frac = P.probe.core_frac; B.coul_rc = P.probe.coul_rc;
    B.min_image = P.probe.min_image; B.periodic_xy = P.periodic_xy;
    B.kx = (float)(P.tip.kx * kNmToEvA2); B.ky = (float)(P.tip.ky * kNmToEvA2); B.kR = (float)(P.tip.kR * kNmToEvA2);
    B.R0 = P.tip.R0; B.d0x = P.tip.d0x; B.d0y = P.tip.d0y;
    B.d0z = (float)(-sqrt((double)P.tip.R0 * P.tip.R0 - (double)P.tip.d0x * P.tip.d0x -
                          (double)P.tip.d0y * P.tip.d0y));
    B.R0sq = (float)((double)P.tip.R0 * P.tip.R0);
    B.c0 = (float)((double)B.d0x * B.d0x + (double)B.d0y * B.d0y + (double)B.d0z * B.d0z -
                   (double)P.tip.R0 * P.tip.R0);
    B.max_iter = P.fire.max_iter; B.n_min = P.fire.n_min;
    B.ftol2 = P.fire.ftol * P.fire.ftol;
    B.dt0 = P.fire.dt0; B.dt_max = P.fire.dt_max; B.f_inc = P.fire.f_inc; B.f_dec = P.fire.f_dec;
    B.alpha0 = P.fire.alpha0; B.f_alpha = P.fire.f_alpha; B.inv_mass = 1.f / P.fire.mass;
    B.sdz = P.scan_dz;
    B.df_m = A.df_m;
    for (int c = 0; c < 2 * A.df_m + 1; ++c) B.coef_init[c] = A.coef[c];
    char* w = reinterpret_cast<char*>(A.ws);
    B.counter = reinterpret_cast<unsigned long long*>(w);
    B.status = reinterpret_cast<int*>(w + 8);
    B.coef_ws = reinterpret_cast<float*>(w + 64);
    B.coef = B.coef_ws;
    B.seg_start = reinterpret_cast<long long*>(w + 320);
    B.done_ff = reinterpret_cast<int*>(w + 320 + 8 * (2 * (size_t)A.nmol + 1));
    B.spin_limit = P.spin_limit > 0 ? P.spin_limit : (1LL << 23);
    B.wait_extra = P.wait_extra;
    B.forces_only = P.ff_forces_only;
    B.zpt = P.ff_zpt > 0 ? P.ff_zpt : 8;
    const int fw = P.ff_tile_w > 0 ? P.ff_tile_w : 8, rw = P.relax_tile_w > 0 ? P.relax_tile_w : 8;
    B.fw_sh = fw == 4 ? 2 : (fw == 8 ? 3 : 4);
    B.rw_sh = rw == 4 ? 2 : (rw == 8 ? 3 : 4);

    batch_plan_kernel<<<1, 1024, 0, s>>>(B);
    const bool fo = B.forces_only != 0;
    const bool z4 = B.zpt == 4;
    const void* fn = with_flags(B.min_image != 0, B.coul_rc > 0.f, B.kQzz != 0.f, [fo, z4](auto mi, auto cut, auto quad) {
        constexpr bool MI = decltype(mi)::value, CUT = decltype(cut)::value, QUAD = decltype(quad)::value;
        if (z4) return fo ? (const void*)batch_kernel<4, MI, CUT, QUAD, true> : (const void*)batch_kernel<4, MI, CUT, QUAD, false>;
        return fo ? (const void*)batch_kernel<8, MI, CUT, QUAD, true> : (const void*)batch_kernel<8, MI, CUT, QUAD, false>;
    });
    int ctas = P.ctas;
    if (ctas <= 0) {
        int dev = 0, sms = 148, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
        ctas = sms * (per_sm > 0 ? per_sm : 1);
    }
    void* args[] = {&B};
    return cudaLaunchKernel(fn, dim3(ctas), dim3(kThreads), args, 0, s);
}

PP_CHECK_READER(check_flags_batch)

}  // namespace pp
