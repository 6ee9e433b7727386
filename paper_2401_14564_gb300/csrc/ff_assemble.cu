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
// This is compute-bound FP32 arithmetic with no dense contraction, so it runs
// on the FP32 pipes, not the tensor cores.  A CTA covers a 16x8 (x,y) tile of
// grid columns; each thread owns ZPT consecutive z-nodes of one column, so the
// lateral displacement of an atom is computed once per column and reused for
// all ZPT nodes.  The per-node arithmetic runs two z-nodes at a time on
// Blackwell's packed f32x2 FMA/MUL/ADD (one issue slot for two lanes' worth
// of FP32 work); only the core floor (no packed max) and the rsqrt stay
// scalar.  Atoms are staged into shared memory in chunks, with the per-atom
// mixing (R_iPP^2, 12 e_iPP, k_e Q q_i, floor radius^2, e_iPP) done while
// staging, and each per-atom constant stored twice so that one 16-byte
// broadcast load yields a ready packed operand.
#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kTileX = 16;   // columns per CTA along x (two warps of 8)
constexpr int kTileY = 8;    // columns per CTA along y (two warps of 4)
constexpr int kThreads = kTileX * kTileY;
constexpr int kChunk = 256;  // atoms staged per pass

// ---- packed FP32 pairs (PTX f32x2, sm_100 and later)
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2add(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Shared-memory record of one atom (64 B), constants duplicated for packed use.
//   s0 = (x, y, rmin^2, 0)   s1 = (-z, -z, R_iPP^2, R_iPP^2)
//   s2 = (12 e, 12 e, kq, kq) s3 = (e, e, 0, 0)
template <int ZPT, bool kMinImage, bool kCutoff>
__global__ void __launch_bounds__(kThreads) ff_assemble_kernel(const FFLaunch P) {
    static_assert(ZPT % 2 == 0, "z-nodes come in packed pairs");
    constexpr int ZP = ZPT / 2;
    __shared__ float4 s0[kChunk], s1[kChunk], s2[kChunk], s3[kChunk];

    // warp w covers an 8x4 sub-tile; lane -> (lane & 7, lane >> 3)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kTileX + (warp & 1) * 8 + (lane & 7);
    const int j = blockIdx.y * kTileY + (warp >> 1) * 4 + (lane >> 3);
    const int k0 = blockIdx.z * ZPT;

    const float gx = P.x0 + i * P.dx;
    const float gy = P.y0 + j * P.dy;
    float2 gz[ZP];
#pragma unroll
    for (int t = 0; t < ZP; ++t) gz[t] = make_float2(P.z0 + (k0 + 2 * t) * P.dz, P.z0 + (k0 + 2 * t + 1) * P.dz);

    float2 fx[ZP], fy[ZP], fz[ZP], en[ZP];
#pragma unroll
    for (int t = 0; t < ZP; ++t) fx[t] = fy[t] = fz[t] = en[t] = make_float2(0.f, 0.f);

    const float invLx = kMinImage ? 1.f / P.Lx : 0.f;
    const float invLy = kMinImage ? 1.f / P.Ly : 0.f;
    const float rc2 = kCutoff ? P.coul_rc * P.coul_rc : 0.f;
    const float irc2 = kCutoff ? 1.f / rc2 : 0.f;
    const float two_irc = kCutoff ? 2.f / P.coul_rc : 0.f;
    const float2 minus1 = make_float2(-1.f, -1.f);

    for (int base = 0; base < P.n; base += kChunk) {
        const int cnt = min(kChunk, P.n - base);
        __syncthreads();
        for (int a = threadIdx.x; a < cnt; a += kThreads) {
            const int g = base + a;
            const float Rij = P.R[g] + P.R_pp;
            const float eij = sqrtf(P.eps[g] * P.eps_pp);
            const float rmin = P.core_frac * Rij;
            const float kq = P.kQ * P.q[g];
            const float z = P.z[g];
            s0[a] = make_float4(P.x[g], P.y[g], rmin * rmin, 0.f);
            s1[a] = make_float4(-z, -z, Rij * Rij, Rij * Rij);
            s2[a] = make_float4(12.f * eij, 12.f * eij, kq, kq);
            s3[a] = make_float4(eij, eij, 0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 1
        for (int a = 0; a < cnt; ++a) {
            const float4 A0 = s0[a], A1 = s1[a], A2 = s2[a], A3 = s3[a];
            float rx = gx - A0.x;
            float ry = gy - A0.y;
            if (kMinImage) {
                rx = fmaf(-P.Lx, rintf(rx * invLx), rx);
                ry = fmaf(-P.Ly, rintf(ry * invLy), ry);
            }
            const float rxy2 = fmaf(rx, rx, ry * ry);
            const float2 RX = make_float2(rx, rx), RY = make_float2(ry, ry), RXY = make_float2(rxy2, rxy2);
            const float2 NZ = make_float2(A1.x, A1.y), R2 = make_float2(A1.z, A1.w);
            const float2 E12 = make_float2(A2.x, A2.y), KQ = make_float2(A2.z, A2.w);
            const float2 EE = make_float2(A3.x, A3.y);
#pragma unroll
            for (int t = 0; t < ZP; ++t) {
                const float2 rz = f2add(gz[t], NZ);
                float2 r2 = f2fma(rz, rz, RXY);
                r2.x = fmaxf(r2.x, A0.z);
                r2.y = fmaxf(r2.y, A0.z);
                const float2 rs = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                const float2 ir2 = f2mul(rs, rs);
                const float2 u = f2mul(R2, ir2);
                const float2 u3 = f2mul(f2mul(u, u), u);
                const float2 lj = f2mul(u3, f2add(u3, minus1));  // u6 - u3
                float2 eel = f2mul(KQ, rs);                         // kq / r
                float2 f;
                if (kCutoff) {
                    eel.x = (r2.x < rc2) ? eel.x : 0.f;
                    eel.y = (r2.y < rc2) ? eel.y : 0.f;
                    // kq (1/r^3 - 1/(r rc^2)) + 12 e (u6 - u3) / r^2
                    f = f2fma(eel, make_float2(-irc2, -irc2), f2mul(f2fma(E12, lj, eel), ir2));
                    // shifted-force energy kq (1/r + r/rc^2 - 2/rc)
                    float2 ee = f2fma(eel, f2mul(r2, make_float2(irc2, irc2)), eel);
                    ee.x -= (r2.x < rc2) ? KQ.x * two_irc : 0.f;
                    ee.y -= (r2.y < rc2) ? KQ.y * two_irc : 0.f;
                    eel = ee;
                } else {
                    f = f2mul(f2fma(E12, lj, eel), ir2);  // (12 e (u6 - u3) + kq / r) / r^2
                }
                fx[t] = f2fma(f, RX, fx[t]);
                fy[t] = f2fma(f, RY, fy[t]);
                fz[t] = f2fma(f, rz, fz[t]);
                en[t] = f2add(f2fma(EE, f2sub(lj, u3), en[t]), eel);  // e (u6 - 2 u3) + E_el
            }
        }
    }

    if (i >= P.map.nx || j >= P.map.ny) return;
    const int base_xy = axis_off(P.map.ax, i) + axis_off(P.map.ay, j);
#pragma unroll
    for (int t = 0; t < ZP; ++t) {
        const int k = k0 + 2 * t;
        if (k < P.map.nz) P.ff[base_xy + axis_off(P.map.az, k)] = make_float4(fx[t].x, fy[t].x, fz[t].x, en[t].x);
        if (k + 1 < P.map.nz)
            P.ff[base_xy + axis_off(P.map.az, k + 1)] = make_float4(fx[t].y, fy[t].y, fz[t].y, en[t].y);
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
