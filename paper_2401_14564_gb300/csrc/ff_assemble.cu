// K1: force-field grid assembly (Sec. 5.1.1 step 1).
//
// Every node g of the grid gets F_g = sum_i S_i(r) (r_g - r_i) and
// E_g = sum_i E_i(r), with, for atom i and the probe particle,
//   Lennard-Jones (Eq. LJ):  E = e_iPP [u6 - 2 u3],  S = 12 e_iPP (u6 - u3) / r^2,
//   u3 = (R_iPP^2 / r^2)^3, R_iPP = R_i + R_PP, e_iPP = sqrt(e_i e_PP);
//   Coulomb (Eq. point charges):  E = k_e Q q_i / r,  S = k_e Q q_i / r^3
//   (shifted-force variant when coul_rc > 0), F = -grad E (Sec. 2.2);
// r^2 is floored per pair at (core_frac R_iPP)^2.
//
// The work is compute-bound FP32 arithmetic (no dense contraction, so no
// tensor cores): one rsqrt and ~18 FP32 instructions per node-atom pair.
// A CTA covers a 16x8 (x,y) tile of grid columns; each thread owns ZPT
// consecutive z-nodes of one column, so the lateral displacement of an atom
// is computed once per column and reused for all ZPT nodes.  Atoms are
// staged into shared memory in chunks of kChunk, with the per-atom mixing
// (R_iPP^2, 12 e_iPP, k_e Q q_i, floor radius^2, e_iPP) done while staging,
// and read back as warp-uniform broadcasts.
#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kTileX = 16;   // columns per CTA along x (two warps of 8)
constexpr int kTileY = 8;    // columns per CTA along y (two warps of 4)
constexpr int kThreads = kTileX * kTileY;
constexpr int kChunk = 256;  // atoms staged per pass

struct AtomA { float x, y, z, R2; };
struct AtomB { float E12, kq, rmin2, e; };

template <int ZPT, bool kMinImage, bool kCutoff>
__global__ void __launch_bounds__(kThreads) ff_assemble_kernel(const FFLaunch P) {
    __shared__ float4 sA[kChunk];
    __shared__ float4 sB[kChunk];

    // warp w covers an 8x4 sub-tile; lane -> (lane & 7, lane >> 3)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kTileX + (warp & 1) * 8 + (lane & 7);
    const int j = blockIdx.y * kTileY + (warp >> 1) * 4 + (lane >> 3);
    const int k0 = blockIdx.z * ZPT;

    const float gx = P.x0 + i * P.dx;
    const float gy = P.y0 + j * P.dy;
    float gz[ZPT];
#pragma unroll
    for (int t = 0; t < ZPT; ++t) gz[t] = P.z0 + (k0 + t) * P.dz;

    float fx[ZPT], fy[ZPT], fzz[ZPT], en[ZPT];
#pragma unroll
    for (int t = 0; t < ZPT; ++t) fx[t] = fy[t] = fzz[t] = en[t] = 0.f;

    const float invLx = kMinImage ? 1.f / P.Lx : 0.f;
    const float invLy = kMinImage ? 1.f / P.Ly : 0.f;
    const float irc2 = kCutoff ? 1.f / (P.coul_rc * P.coul_rc) : 0.f;
    const float rc2 = kCutoff ? P.coul_rc * P.coul_rc : 0.f;
    const float two_irc = kCutoff ? 2.f / P.coul_rc : 0.f;

    for (int base = 0; base < P.n; base += kChunk) {
        const int cnt = min(kChunk, P.n - base);
        __syncthreads();
        for (int a = threadIdx.x; a < cnt; a += kThreads) {
            const int g = base + a;
            const float Rij = P.R[g] + P.R_pp;
            const float eij = sqrtf(P.eps[g] * P.eps_pp);
            const float rmin = P.core_frac * Rij;
            sA[a] = make_float4(P.x[g], P.y[g], P.z[g], Rij * Rij);
            sB[a] = make_float4(12.f * eij, P.kQ * P.q[g], rmin * rmin, eij);
        }
        __syncthreads();
#pragma unroll 2
        for (int a = 0; a < cnt; ++a) {
            const float4 A = sA[a];
            const float4 B = sB[a];
            float rx = gx - A.x;
            float ry = gy - A.y;
            if (kMinImage) {
                rx = fmaf(-P.Lx, rintf(rx * invLx), rx);
                ry = fmaf(-P.Ly, rintf(ry * invLy), ry);
            }
            const float rxy2 = fmaf(rx, rx, ry * ry);
#pragma unroll
            for (int t = 0; t < ZPT; ++t) {
                const float rz = gz[t] - A.z;
                const float r2 = fmaxf(fmaf(rz, rz, rxy2), B.z);
                const float rs = rsqrtf(r2);
                const float ir2 = rs * rs;
                const float u = A.w * ir2;
                const float u3 = u * u * u;
                const float lj = fmaf(u3, u3, -u3);          // u6 - u3
                float f, e_el;
                if (kCutoff) {
                    const float t1 = (r2 < rc2) ? B.y * rs : 0.f;   // kq / r inside rc
                    f = fmaf(B.x, lj, t1) * ir2 - t1 * irc2;        // kq (1/r^3 - 1/(r rc^2))
                    e_el = fmaf(t1, r2 * irc2, t1) - ((r2 < rc2) ? B.y * two_irc : 0.f);
                } else {
                    e_el = B.y * rs;                                 // kq / r
                    f = fmaf(B.x, lj, e_el) * ir2;                   // 12 e (u6-u3)/r^2 + kq/r^3
                }
                fx[t] = fmaf(f, rx, fx[t]);
                fy[t] = fmaf(f, ry, fy[t]);
                fzz[t] = fmaf(f, rz, fzz[t]);
                en[t] = fmaf(B.w, u3 * (u3 - 2.f), en[t] + e_el);
            }
        }
    }

    if (i >= P.map.nx || j >= P.map.ny) return;
    const int base_xy = axis_off(P.map.ax, i) + axis_off(P.map.ay, j);
#pragma unroll
    for (int t = 0; t < ZPT; ++t) {
        const int k = k0 + t;
        if (k < P.map.nz) P.ff[base_xy + axis_off(P.map.az, k)] = make_float4(fx[t], fy[t], fzz[t], en[t]);
    }
}

template <int ZPT>
cudaError_t launch_zpt(const FFLaunch& L, cudaStream_t s) {
    dim3 grid((L.map.nx + kTileX - 1) / kTileX, (L.map.ny + kTileY - 1) / kTileY, (L.map.nz + ZPT - 1) / ZPT);
    const bool cut = L.coul_rc > 0.f;
    if (L.min_image && cut) ff_assemble_kernel<ZPT, true, true><<<grid, kThreads, 0, s>>>(L);
    else if (L.min_image) ff_assemble_kernel<ZPT, true, false><<<grid, kThreads, 0, s>>>(L);
    else if (cut) ff_assemble_kernel<ZPT, false, true><<<grid, kThreads, 0, s>>>(L);
    else ff_assemble_kernel<ZPT, false, false><<<grid, kThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ff_assemble(const FFLaunch& L, cudaStream_t s) {
    if (L.map.nx <= 0 || L.map.ny <= 0 || L.map.nz <= 0) return cudaSuccess;
    return launch_zpt<8>(L, s);
}

}  // namespace pp
