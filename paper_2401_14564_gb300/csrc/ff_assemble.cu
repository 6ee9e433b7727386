// K1: force-field grid assembly (Sec. 5.1.1 step 1).
//
// Every node g of the grid gets F_g = sum_i S_i(r) (r_g - r_i) and
// E_g = sum_i E_i(r), with, for atom i and the probe particle,
//   Lennard-Jones (Eq. LJ):  E = e_iPP [u6 - 2 u3],  S = 12 e_iPP (u6 - u3) / r^2,
//   u3 = (R_iPP^2 / r^2)^3, R_iPP = R_i + R_PP, e_iPP = sqrt(e_i e_PP);
//   Coulomb (Eq. point charges):  E = k_e Q q_i / r,  S = k_e Q q_i / r^3
//   (shifted-force variant when coul_rc > 0), F = -grad E (Sec. 2.2);
// r^2 is floored per pair at (core_frac R_iPP)^2; optionally the tip's axial
// quadrupole Qzz (Secs. 2.2.3, 2.2.5) in the sample's point-charge field,
//   E = (k_e q_i Qzz / 2) (3 dz^2 - r^2) / r^5, F = -grad E.
//
// This is compute-bound FP32 arithmetic with no dense contraction, so it runs
// on the FP32 pipes, not the tensor cores.  A CTA covers a 16x8 (x,y) tile of
// grid columns; each thread owns ZPT consecutive z-nodes of one column, so the
// lateral displacement of an atom is computed once per column and reused for
// all ZPT nodes.  The per-node arithmetic runs two z-nodes at a time on
// Blackwell's packed f32x2 FMA/MUL/ADD (one issue slot for two lanes' worth
// of FP32 work); only the core floor (no packed max) and the rsqrt stay
// scalar.  The Lennard-Jones terms are evaluated as polynomials in 1/r^6 with
// per-atom coefficients (12 e R^12, 12 e R^6, e R^12, 2 e R^6 with the mixed
// R = R_iPP, e = e_iPP), which takes 12 packed FP32 operations per pair of
// nodes for the forces and 3 more for the energy.  Atoms are staged into
// shared memory in chunks, with the mixing and these coefficients, k_e Q q_i
// and the floor radius^2 formed while staging, and each per-atom constant
// stored twice so that one 16-byte broadcast load yields a ready packed
// operand.
#include "ff_core.cuh"

namespace pp {
namespace {

constexpr int kTileX = 16;   // columns per CTA along x (two warps of 8)
constexpr int kTileY = 8;    // columns per CTA along y (two warps of 4)
constexpr int kThreads = kTileX * kTileY;
constexpr int kChunk = 256;  // atoms staged per pass

// kEnergy: write E alone, one float per node (tricubic grids); the force sums
// are then never formed (the compiler drops them with their stores).
// kSplit: the point-charge field per unit probe charge goes to a second grid
// (ffel / ffelE), the rest (LJ and the tip quadrupole) to the first.
// kForcesOnly: E slots written as 0; the energy sums are never formed (3 of
// the 15 packed FP32 operations per pair of nodes), the force sums are
// unchanged.
template <int ZPT, bool kMinImage, bool kCutoff, bool kQuad, bool kEnergy = false, bool kSplit = false,
          bool kForcesOnly = false>
__global__ void __launch_bounds__(kThreads) ff_assemble_kernel(const FFLaunch P) {
    static_assert(ZPT % 2 == 0, "z-nodes come in packed pairs");
    constexpr int ZP = ZPT / 2;
    __shared__ float4 s0[kChunk], s1[kChunk], s2[kChunk], s3[kChunk];

    // warp w covers an 8x4 sub-tile; lane -> (lane & 7, lane >> 3)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kTileX + (warp & 1) * 8 + (lane & 7);
    const int j = blockIdx.y * kTileY + (warp >> 1) * 4 + (lane >> 3);
    const int k0 = P.kbeg + blockIdx.z * ZPT;

    const float gx = P.x0 + i * P.dx;
    const float gy = P.y0 + j * P.dy;
    float2 gz[ZP];
#pragma unroll
    for (int t = 0; t < ZP; ++t) gz[t] = make_float2(P.z0 + (k0 + 2 * t) * P.dz, P.z0 + (k0 + 2 * t + 1) * P.dz);

    float2 fx[ZP], fy[ZP], fz[ZP], en[ZP];
    float2 fxe[ZP], fye[ZP], fze[ZP], ene[ZP];  // kSplit only
#pragma unroll
    for (int t = 0; t < ZP; ++t) fx[t] = fy[t] = fz[t] = en[t] = fxe[t] = fye[t] = fze[t] = ene[t] = make_float2(0.f, 0.f);

    const FFConst cst = ff_const(P.R_pp, P.eps_pp, P.kQ, P.core_frac, P.Lx, P.Ly, kCutoff ? P.coul_rc : 0.f,
                                 kQuad ? P.kQzz : 0.f);
    for (int base = 0; base < P.n; base += kChunk) {
        const int cnt = min(kChunk, P.n - base);
        __syncthreads();
        for (int a = threadIdx.x; a < cnt; a += kThreads) {
            const int g = base + a;
            ff_stage_atom(cst, P.x[g], P.y[g], P.z[g], P.R[g], P.eps[g], P.q[g], s0[a], s1[a], s2[a], s3[a]);
        }
        __syncthreads();
        // every thread of the block runs this (out-of-grid columns return only after it): the warp vote is safe
        ff_accumulate_impl<ZP, kMinImage, kCutoff, kQuad, kSplit, true>(s0, s1, s2, s3, cnt, cst, gx, gy, gz, fx, fy, fz, en,
                                                                  fxe, fye, fze, ene);
    }

    if (i >= P.map.nx || j >= P.map.ny) return;
    const int base_xy = axis_off(P.map.ax, i) + axis_off(P.map.ay, j);
    auto at = [&](int k) { return checked(base_xy + axis_off(P.map.az, k), P.map.stored_nodes, kChkGridWrite); };
    if constexpr (kEnergy) {
#pragma unroll
        for (int t = 0; t < ZP; ++t) {
            const int k = k0 + 2 * t;
            if (k < P.kend) P.ffE[at(k)] = en[t].x;
            if (k + 1 < P.kend) P.ffE[at(k + 1)] = en[t].y;
            if constexpr (kSplit) {
                if (k < P.kend) P.ffelE[at(k)] = ene[t].x;
                if (k + 1 < P.kend) P.ffelE[at(k + 1)] = ene[t].y;
            }
        }
    } else {
#pragma unroll
        for (int t = 0; t < ZP; ++t) {
            const int k = k0 + 2 * t;
            const float2 e = kForcesOnly ? make_float2(0.f, 0.f) : en[t];
            if (k < P.kend) P.ff[at(k)] = make_float4(fx[t].x, fy[t].x, fz[t].x, e.x);
            if (k + 1 < P.kend) P.ff[at(k + 1)] = make_float4(fx[t].y, fy[t].y, fz[t].y, e.y);
            if constexpr (kSplit) {
                if (k < P.kend)
                    P.ffel[at(k)] = make_float4(fxe[t].x, fye[t].x, fze[t].x, ene[t].x);
                if (k + 1 < P.kend)
                    P.ffel[at(k + 1)] = make_float4(fxe[t].y, fye[t].y, fze[t].y, ene[t].y);
            }
        }
    }
}

// out = a + Q b over n floats (a split force field recombined for probe charge Q): float4
// grid-stride body, the last n mod 4 floats by the first threads of CTA 0; out may alias a.
__global__ void ff_combine_kernel(const float* a, const float* __restrict__ b, float Q, float* out, int64_t n) {
    const int64_t n4 = n >> 2;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    float4* o4 = reinterpret_cast<float4*>(out);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 u = a4[i], v = __ldg(b4 + i);
        o4[i] = make_float4(fmaf(Q, v.x, u.x), fmaf(Q, v.y, u.y), fmaf(Q, v.z, u.z), fmaf(Q, v.w, u.w));
    }
    if (blockIdx.x == 0 && threadIdx.x < (int)(n & 3)) {
        const int64_t j = (n4 << 2) + threadIdx.x;
        out[j] = fmaf(Q, b[j], a[j]);
    }
}

template <int ZPT>
cudaError_t launch_zpt(const FFLaunch& L, cudaStream_t s) {
    dim3 grid((L.map.nx + kTileX - 1) / kTileX, (L.map.ny + kTileY - 1) / kTileY, (L.kend - L.kbeg + ZPT - 1) / ZPT);
    with_flags(L.min_image != 0, L.coul_rc > 0.f, L.kQzz != 0.f, [&](auto mi, auto cut, auto quad) {
        constexpr bool MI = decltype(mi)::value, CUT = decltype(cut)::value, QUAD = decltype(quad)::value;
        if (L.forces_only) ff_assemble_kernel<ZPT, MI, CUT, QUAD, false, false, true><<<grid, kThreads, 0, s>>>(L);
        else ff_assemble_kernel<ZPT, MI, CUT, QUAD><<<grid, kThreads, 0, s>>>(L);
        return 0;
    });
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ff_combine(const float* a, const float* b, float Q, float* out, int64_t nfloats, cudaStream_t s) {
    if (nfloats <= 0) return cudaSuccess;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = ((nfloats >> 2) + 255) / 256;
    // one wave of 8 resident 256-thread CTAs per SM, grid-stride inside
    const int blocks = (int)(want < 1 ? 1 : (want < 8LL * sms ? want : 8LL * sms));
    ff_combine_kernel<<<blocks, 256, 0, s>>>(a, b, Q, out, nfloats);
    return cudaGetLastError();
}

cudaError_t launch_ff_assemble(const FFLaunch& L, cudaStream_t s) {
    if (L.map.nx <= 0 || L.map.ny <= 0 || L.kend <= L.kbeg) return cudaSuccess;
    if (L.split) {  // one launch shape: 8 z-nodes per thread
        constexpr int ZPT = 8;
        dim3 grid((L.map.nx + kTileX - 1) / kTileX, (L.map.ny + kTileY - 1) / kTileY, (L.kend - L.kbeg + ZPT - 1) / ZPT);
        with_flags(L.min_image != 0, L.coul_rc > 0.f, L.kQzz != 0.f, [&](auto mi, auto cut, auto quad) {
            constexpr bool MI = decltype(mi)::value, CUT = decltype(cut)::value, QUAD = decltype(quad)::value;
            if (L.map.interp == 1) ff_assemble_kernel<ZPT, MI, CUT, QUAD, true, true><<<grid, kThreads, 0, s>>>(L);
            else ff_assemble_kernel<ZPT, MI, CUT, QUAD, false, true><<<grid, kThreads, 0, s>>>(L);
            return 0;
        });
        return cudaGetLastError();
    }
    if (L.map.interp == 1) {
        constexpr int ZPT = 8;
        dim3 grid((L.map.nx + kTileX - 1) / kTileX, (L.map.ny + kTileY - 1) / kTileY, (L.kend - L.kbeg + ZPT - 1) / ZPT);
        with_flags(L.min_image != 0, L.coul_rc > 0.f, L.kQzz != 0.f, [&](auto mi, auto cut, auto quad) {
            ff_assemble_kernel<ZPT, decltype(mi)::value, decltype(cut)::value, decltype(quad)::value, true>
                <<<grid, kThreads, 0, s>>>(L);
            return 0;
        });
        return cudaGetLastError();
    }
    // A column's last z-block would compute zpt - r nodes past the range when the layer count is not a
    // multiple of zpt (nz = 200 at 16: 13 x 16 = 208, 4 % of the arithmetic); those r layers go to a
    // second launch of a narrower shape instead (each node's sums are the same in every shape).
    const int zpt = (L.zpt == 4 || L.zpt == 16) ? L.zpt : 8;
    const int n = L.kend - L.kbeg, bulk = n - n % zpt, r = n - bulk;
    FFLaunch head = L, tail = L;
    head.kend = L.kbeg + bulk;
    tail.kbeg = L.kbeg + bulk;
    if (bulk > 0) {
        const cudaError_t e = zpt == 4 ? launch_zpt<4>(head, s) : zpt == 16 ? launch_zpt<16>(head, s) : launch_zpt<8>(head, s);
        if (e != cudaSuccess) return e;
    }
    if (r > 0) return r > 4 ? launch_zpt<8>(tail, s) : launch_zpt<4>(tail, s);
    return cudaSuccess;
}

PP_CHECK_READER(check_flags_ff_assemble)

}  // namespace pp
