// Adjoint of the df image with respect to atoms and tip parameters.
//
// The paper has no gradients; this differentiates the same discrete model.
// For L = sum g_df * df:
//   K3^T  g_Fz = transpose of the df stencil applied to g_df (fused into K4);
//   K4    per relaxed point (pixel, height), at equilibrium G(p*) = 0 the
//         implicit function theorem gives dp*/dtheta = -J^{-1} dG/dtheta with
//         J = dG/dp (tip-spring Jacobian + exact Jacobian of the trilinear
//         interpolant), so with lambda = J^{-T} (dFz/dp)^T g_Fz:
//           dL/dtheta = g_Fz dFz/dtheta - lambda . dG/dtheta.
//         The grid values enter G through the trilinear weights, so the grid
//         adjoint is Gbar_g = -sum lambda w_g(p*) (float4 atomics); the tip
//         springs give dL/dkx = lambda_x e_x, dL/dky = lambda_y e_y, and
//         dL/dkR = g_Fz (|d|-R0) d_z/|d| + lambda.d (|d|-R0)/|d|;
//   K5    dL/dtheta_i = sum_g Gbar_g . dF_g/dtheta_i for every atom, by
//         recomputing the pair terms of the force-field grid (Eqs. LJ and
//         point charges, and the tip quadrupole when Qzz != 0) on the grid
//         nodes with a nonzero adjoint, restricted to the z-slab K4 touched;
//   fin   charges: dL/dq_i = k_e (Q C_i + (Qzz/2) Cq_i), dL/dQ = k_e sum_i q_i C_i,
//         dL/dQzz = (k_e/2) sum_i q_i Cq_i, with C_i = sum_g Gbar_g . delta c(r)
//         and Cq_i = sum_g Gbar_g . Phi (the quadrupole force per unit
//         k_e q_i Qzz / 2); eps via e_iPP = sqrt(e_i e_PP).
// No relaxation iterate is stored or replayed: only the saved p*.
#include "interp.cuh"

namespace pp {
namespace {

constexpr int kAdjThreads = 128;
constexpr int kFFBThreads = 64;
constexpr int kFFBNodes = 512;  // grid nodes staged per K5 CTA

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void init_kernel(const BwdLaunch P) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        P.slab[0] = 0x7fffffff;
        P.slab[1] = -1;
        P.gtip[0] = P.gtip[1] = P.gtip[2] = P.gtip[3] = P.gtip[4] = 0.f;
        P.qsum[0] = P.qsum[1] = 0.f;
        P.qsumd[0] = P.qsumd[1] = 0.0;
    }
    for (int a = t; a < P.n; a += gridDim.x * blockDim.x) {
        P.gx[a] = 0.f; P.gy[a] = 0.f; P.gz[a] = 0.f;
        P.gq[a] = 0.f; P.gR[a] = 0.f; P.geps[a] = 0.f;
    }
}

// g_Fz at height k = (df stencil)^T g_df: df[c] = sum_s coef[s+m] Fz[c+m+s].  With the half
// width M known at compile time the 2M+1 loads are independent and issue back to back; M < 0
// takes the run-time half width P.m.
template <int M>
__device__ __forceinline__ float df_transpose(const BwdLaunch& P, int k, int pix, int npix) {
    float gf = 0.f;
    if constexpr (M >= 0) {
        float t[2 * M + 1];
#pragma unroll
        for (int s = -M; s <= M; ++s) {
            const int c = k - M - s;
            t[s + M] = (c >= 0 && c < P.nzo)
                           ? __ldg(P.g_df + checked((int64_t)c * npix + pix, (long long)P.nzo * npix, kChkScanRead))
                           : 0.f;
        }
#pragma unroll
        for (int s = -M; s <= M; ++s) gf = fmaf(P.coef[s + M], t[s + M], gf);
    } else {
        for (int s = -P.m; s <= P.m; ++s) {
            const int c = k - P.m - s;
            if (c >= 0 && c < P.nzo)
                gf = fmaf(P.coef[s + P.m],
                          __ldg(P.g_df + checked((int64_t)c * npix + pix, (long long)P.nzo * npix, kChkScanRead)), gf);
        }
    }
    return gf;
}

// Grid-stride over the relaxed points: each thread sums its points' tip-parameter terms and
// z-slab bounds in registers, and a block adds them to the five shared scalars once (atomics
// from every warp to the same five addresses would serialise in L2).
// On a tricubic energy grid (kTri) J takes minus the Hessian of the interpolant and the grid
// adjoint is one scalar per node, Ebar_g = sum lambda . grad w_g(p*) over the 64 stencil nodes
// (F_S = -sum_g E_g grad w_g).
template <int LAYOUT, int M, bool kTri>
__global__ void __launch_bounds__(kAdjThreads) relax_adjoint_kernel(const BwdLaunch P) {
    __shared__ float sred[3][kAdjThreads / 32];
    __shared__ int sk[2][kAdjThreads / 32];
    const int npix = P.snx * P.sny;
    const int64_t total = (int64_t)npix * P.snz;
    float gkx = 0.f, gky = 0.f, gkR = 0.f;
    int kmin = 0x7fffffff, kmax = -1;
    for (int64_t o = (int64_t)blockIdx.x * kAdjThreads + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * kAdjThreads) {
        const int k = (int)(o / npix), pix = (int)(o - (int64_t)k * npix);
        // the relaxed position is loaded together with the g_df taps (one memory round trip)
        const int64_t o3 = checked(3 * o, 3 * total, kChkScanRead);
        const float px = __ldg(P.pos + o3), py = __ldg(P.pos + o3 + 1), pz = __ldg(P.pos + o3 + 2);
        const float gf = df_transpose<M>(P, k, pix, npix);
        if (gf != 0.f) {
            const int i = pix % P.snx, j = pix / P.snx;
            const float ax = fmaf((float)i, P.spx, P.sx0), ay = fmaf((float)j, P.spy, P.sy0);
            // d = p - anchor with the anchor height z_top - k sdz carried exactly as az + az_lo (the
            // product's rounding by an FMA, the difference's by a two-sum): a rounding common to
            // every point of a height would sum coherently in the tip-parameter sums
            float az, az_lo;
            {
                const float p_hi = __fmul_rn((float)k, P.sdz), p_lo = fmaf((float)k, P.sdz, -p_hi);
                two_sum(P.z_top, -p_hi, az, az_lo);
                az_lo -= p_lo;
            }
            const float dx = px - ax, dy = py - ay, dz = (pz - az) - az_lo;
            const float ex = dx - P.d0x, ey = dy - P.d0y, ez = dz - P.d0z;
            // q = |d|^2 - R0^2 without cancellation, as in the forward kernel
            const float q = fmaf(2.f * P.d0x + ex, ex, fmaf(2.f * P.d0y + ey, ey, fmaf(2.f * P.d0z + ez, ez, P.c0)));
            const float d2 = P.R0sq + q;
            const float rs = rsqrtf(d2);
            const float dn = d2 * rs;
            const float ext = __fdividef(q, fmaf(P.R0, dn, d2));  // (|d| - R0) / |d|
            const float ar = -P.kR * ext;                          // -kR (1 - R0/|d|)
            const float br = -P.kR * P.R0 * rs * rs * rs;          // -kR R0 / |d|^3
            // J = dF_T/dd + dF_S/dp
            const Cells cl = locate(P, px, py, pz);
            float J[3][3];
            if constexpr (kTri) {
                float ec[64];
                tricubic_load(P.ffE, P.map, cl, P.periodic_xy, ec);
                tricubic_jacobian(ec, cl, P.inv_dx, P.inv_dy, P.inv_dz, J);
            } else {
                float4 v[8];
                load_corners<LAYOUT>(P.ff, P.map, cl, v);
                trilinear_jacobian(v, cl, P.inv_dx, P.inv_dy, P.inv_dz, J);
            }
            const float dd[3] = {dx, dy, dz};
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) J[a][b] += (a == b ? ar : 0.f) + br * dd[a] * dd[b];
            J[0][0] -= P.kx;
            J[1][1] -= P.ky;
            // dFz/dp = kR [(1 - R0/|d|) z_hat + R0 d_z d / |d|^3]
            const float r0 = -br * dz * dx * gf, r1 = -br * dz * dy * gf, r2 = (-ar - br * dz * dz) * gf;
            // solve J^T lambda = r by the adjugate
            const float a00 = J[0][0], a01 = J[1][0], a02 = J[2][0];
            const float a10 = J[0][1], a11 = J[1][1], a12 = J[2][1];
            const float a20 = J[0][2], a21 = J[1][2], a22 = J[2][2];
            const float c00 = a11 * a22 - a12 * a21, c01 = a02 * a21 - a01 * a22, c02 = a01 * a12 - a02 * a11;
            const float c10 = a12 * a20 - a10 * a22, c11 = a00 * a22 - a02 * a20, c12 = a02 * a10 - a00 * a12;
            const float c20 = a10 * a21 - a11 * a20, c21 = a01 * a20 - a00 * a21, c22 = a00 * a11 - a01 * a10;
            const float det = a00 * c00 + a01 * c10 + a02 * c20;
            if (det != 0.f && isfinite(det)) {
                const float id = 1.f / det;
                const float lx = (c00 * r0 + c01 * r1 + c02 * r2) * id;
                const float ly = (c10 * r0 + c11 * r1 + c12 * r2) * id;
                const float lz = (c20 * r0 + c21 * r1 + c22 * r2) * id;
                gkx = fmaf(lx, ex, gkx);
                gky = fmaf(ly, ey, gky);
                gkR += gf * ext * dz + (lx * dx + ly * dy + lz * dz) * ext;
                if constexpr (kTri) {
                    // Ebar_g += lambda . grad w_g, w_g = wx_a wy_b wz_c:
                    //   = wz_c (lx' dwx_a wy_b + ly' wx_a dwy_b) + lz' dwz_c wx_a wy_b, l' = lambda dt/dp
                    float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
                    cr_weights(cl.x.t, wx, dwx);
                    cr_weights(cl.y.t, wy, dwy);
                    cr_weights(cl.z.t, wz, dwz);
                    const float lxs = lx * cl.x.dtdf * P.inv_dx, lys = ly * cl.y.dtdf * P.inv_dy;
                    const float lzs = lz * cl.z.dtdf * P.inv_dz;
                    int xo[4], yo[4], zo[4];
                    stencil4(cl.x, P.map.nx, P.periodic_xy != 0, 1, xo);
                    stencil4(cl.y, P.map.ny, P.periodic_xy != 0, P.map.ay.mul, yo);
                    stencil4(cl.z, P.map.nz, false, P.map.az.mul, zo);
#pragma unroll
                    for (int b = 0; b < 4; ++b)
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const float pab = fmaf(lxs * dwx[a], wy[b], lys * wx[a] * dwy[b]);
                            const float qab = wx[a] * wy[b];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float v = fmaf(wz[c], pab, lzs * dwz[c] * qab);
                                if (v != 0.f)
                                    atomicAdd(P.gbarE + checked(zo[c] + yo[b] + xo[a], P.map.stored_nodes, kChkGridWrite),
                                              v);
                            }
                        }
                    kmin = min(kmin, max(cl.z.i0 - 1, 0));
                    kmax = max(kmax, min(cl.z.i1 + 1, P.map.nz - 1));
                } else {
                    // grid adjoint: Gbar += -lambda w_g at the 8 corners
                    int idx[8];
                    corner_index<LAYOUT>(P.map, cl, idx);
                    float w[8];
                    corner_weights(cl, w);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (w[c] != 0.f)
                            atomicAdd(P.gbar + checked(idx[c], P.map.stored_nodes, kChkGridWrite),
                                      make_float4(-lx * w[c], -ly * w[c], -lz * w[c], 0.f));
                    kmin = min(kmin, cl.z.i0);
                    kmax = max(kmax, cl.z.i1);
                }
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    gkx = warp_sum(gkx);
    gky = warp_sum(gky);
    gkR = warp_sum(gkR);
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if (lane == 0) {
        sred[0][warp] = gkx;
        sred[1][warp] = gky;
        sred[2][warp] = gkR;
        sk[0][warp] = kmin;
        sk[1][warp] = kmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kAdjThreads / 32; ++w) {
            gkx += sred[0][w];
            gky += sred[1][w];
            gkR += sred[2][w];
            kmin = min(kmin, sk[0][w]);
            kmax = max(kmax, sk[1][w]);
        }
        if (gkx != 0.f) atomicAdd(P.gtip + 0, gkx * P.nm);
        if (gky != 0.f) atomicAdd(P.gtip + 1, gky * P.nm);
        if (gkR != 0.f) atomicAdd(P.gtip + 2, gkR * P.nm);
        if (kmax >= 0) {
            atomicMin(P.slab + 0, kmin);
            atomicMax(P.slab + 1, kmax);
        }
    }
}

// K5: per-atom contraction of the grid adjoint with the pair derivatives.
// A CTA stages kFFBNodes consecutive nodes (logical x-fastest order), keeps
// those with a nonzero adjoint, and each thread then sweeps them for one atom,
// accumulating (dx, dy, dz, dR, de_iPP, C, Cq) in registers.  The kept nodes
// are stored in pairs, (x0, x1, y0, y1), (z0, z1, gx0, gx1), (gy0, gy1, gz0,
// gz1), so that two nodes go through each packed f32x2 instruction (the floor
// test, the rsqrt and the minimum image stay per node).
__device__ __forceinline__ float2 sel2(bool c0, bool c1, float2 a, float2 b) {
    return make_float2(c0 ? a.x : b.x, c1 ? a.y : b.y);
}

template <bool kMinImage, bool kCutoff, bool kQuad>
__global__ void __launch_bounds__(kFFBThreads) ff_backward_kernel(const BwdLaunch P) {
    __shared__ float4 sxy[kFFBNodes / 2];  // (x0, x1, y0, y1)
    __shared__ float4 szg[kFFBNodes / 2];  // (z0, z1, gx0, gx1)
    __shared__ float4 sgg[kFFBNodes / 2];  // (gy0, gy1, gz0, gz1)
    __shared__ int scount;
    const int nx = P.map.nx, ny = P.map.ny;
    const int64_t nxy = (int64_t)nx * ny;
    const int64_t first = (int64_t)blockIdx.x * kFFBNodes;
    const int klo = P.slab[0], khi = P.slab[1];
    if (khi < 0) return;
    const int kfirst = (int)(first / nxy), klast = (int)((first + kFFBNodes - 1) / nxy);
    if (klast < klo || kfirst > khi) return;
    if (threadIdx.x == 0) scount = 0;
    __syncthreads();
    float* fxy = reinterpret_cast<float*>(sxy);
    float* fzg = reinterpret_cast<float*>(szg);
    float* fgg = reinterpret_cast<float*>(sgg);
    const int64_t total = nxy * P.map.nz;
    for (int t = threadIdx.x; t < kFFBNodes; t += kFFBThreads) {
        const int64_t g = first + t;
        bool keep = false;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        int i = 0, j = 0, k = 0;
        if (g < total) {
            k = (int)(g / nxy);
            const int64_t r = g - (int64_t)k * nxy;
            j = (int)(r / nx);
            i = (int)(r - (int64_t)j * nx);
            a = P.gbar[checked(node_index(P.map, i, j, k), P.map.stored_nodes, kChkGridRead)];
            keep = (a.x != 0.f) || (a.y != 0.f) || (a.z != 0.f);
        }
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if ((threadIdx.x & 31) == 0 && mask) base = atomicAdd(&scount, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const int slot = base + __popc(mask & ((1u << (threadIdx.x & 31)) - 1u));
            const int q = (slot >> 1) * 4, l = slot & 1;
            fxy[q + l] = P.x0 + i * P.dx;
            fxy[q + 2 + l] = P.y0 + j * P.dy;
            fzg[q + l] = P.z0 + k * P.dz;
            fzg[q + 2 + l] = a.x;
            fgg[q + l] = a.y;
            fgg[q + 2 + l] = a.z;
        }
    }
    __syncthreads();
    const int cnt = scount;
    if (cnt == 0) return;
    if ((cnt & 1) && threadIdx.x == 0) {
        // pad the last pair with a copy of its node and a zero adjoint (it adds nothing)
        const int q = (cnt >> 1) * 4;
        fxy[q + 1] = fxy[q];
        fxy[q + 3] = fxy[q + 2];
        fzg[q + 1] = fzg[q];
        fzg[q + 3] = 0.f;
        fgg[q + 1] = 0.f;
        fgg[q + 3] = 0.f;
    }
    __syncthreads();
    const int npairs = (cnt + 1) >> 1;
    const float rc2 = kCutoff ? P.coul_rc * P.coul_rc : 0.f;
    const float irc2 = kCutoff ? 1.f / rc2 : 0.f;
    const float invLx = kMinImage ? 1.f / P.Lx : 0.f, invLy = kMinImage ? 1.f / P.Ly : 0.f;
    const float2 TWELVE = make_float2(12.f, 12.f), EIGHT = make_float2(8.f, 8.f), M14 = make_float2(-14.f, -14.f);
    const float2 M6 = make_float2(-6.f, -6.f), M3 = make_float2(-3.f, -3.f), CF = make_float2(P.core_frac, P.core_frac);
    float qC = 0.f, qCq = 0.f;  // this thread's q_i C_i and q_i Cq_i (tip quadrupole only)
    for (int a0 = 0; a0 < P.n; a0 += kFFBThreads) {
        const int ia = a0 + threadIdx.x;
        const unsigned live = __ballot_sync(0xffffffffu, ia < P.n);  // this warp's lanes with an atom
        if (ia >= P.n) break;
        const float ax = P.ax[ia], ay = P.ay[ia], azz = P.az[ia];
        const float Rij = P.aR[ia] + P.R_pp;
        const float eij = sqrtf(P.aeps[ia] * P.eps_pp);
        const float qq = P.kQ * P.aq[ia];
        const float rmin2 = (P.core_frac * Rij) * (P.core_frac * Rij);
        const float kqq = kQuad ? P.kQzz * P.aq[ia] : 0.f;
        const float2 AX = make_float2(ax, ax), AY = make_float2(ay, ay), AZ = make_float2(azz, azz);
        const float2 RR2 = make_float2(Rij * Rij, Rij * Rij), EIJ = make_float2(eij, eij), QQ = make_float2(qq, qq);
        const float2 E12 = make_float2(12.f * eij, 12.f * eij), E12R = make_float2(12.f * eij / Rij, 12.f * eij / Rij);
        float2 GPX = make_float2(0.f, 0.f), GPY = GPX, GPZ = GPX, GR = GPX, GE = GPX, CC = GPX, CQ = GPX;
        for (int pr = 0; pr < npairs; ++pr) {
            const float4 A = sxy[pr], B = szg[pr], G = sgg[pr];
            float2 DX = f2sub(make_float2(A.x, A.y), AX), DY = f2sub(make_float2(A.z, A.w), AY);
            const float2 DZ = f2sub(make_float2(B.x, B.y), AZ);
            const float2 GX = make_float2(B.z, B.w), GY = make_float2(G.x, G.y), GZ = make_float2(G.z, G.w);
            if (kMinImage) {
                DX.x = fmaf(-P.Lx, rintf(DX.x * invLx), DX.x);
                DX.y = fmaf(-P.Lx, rintf(DX.y * invLx), DX.y);
                DY.x = fmaf(-P.Ly, rintf(DY.x * invLy), DY.x);
                DY.y = fmaf(-P.Ly, rintf(DY.y * invLy), DY.y);
            }
            const float2 R2raw = f2fma(DX, DX, f2fma(DY, DY, f2mul(DZ, DZ)));
            const bool c0 = R2raw.x < rmin2, c1 = R2raw.y < rmin2;  // core floor per node
            const float2 R2v = make_float2(c0 ? rmin2 : R2raw.x, c1 ? rmin2 : R2raw.y);
            // kFar: both nodes lie at or beyond coul_rc from every live lane's atom (a warp vote), so
            // each in-range test below is false and is taken as such: the cut point-charge and
            // quadrupole terms become the zeros they select, and their arithmetic drops out
            auto pair = [&](auto far_t) {
                constexpr bool kFar = decltype(far_t)::value;
                auto in_rc = [&](float r2v) { return !kFar && r2v < rc2; };
                const float2 RS = make_float2(rsqrtf(R2v.x), rsqrtf(R2v.y));
                const float2 IR2 = f2mul(RS, RS);
                const float2 U = f2mul(RR2, IR2);
                const float2 S6 = f2mul(f2mul(U, U), U);
                const float2 S12 = f2mul(S6, S6);
                const float2 SLJ = f2mul(f2mul(TWELVE, f2sub(S12, S6)), IR2);                 // LJ S per unit e_iPP
                const float2 DSLJDR = f2mul(f2mul(E12, f2fma(EIGHT, S6, f2mul(M14, S12))), f2mul(IR2, RS));
                const float2 DSLJDRR = f2mul(f2mul(E12R, f2fma(TWELVE, S12, f2mul(M6, S6))), IR2);
                float2 Cv, DC;
                if (kCutoff) {
                    const bool i0 = in_rc(R2v.x), i1 = in_rc(R2v.y);
                    const float2 z = make_float2(0.f, 0.f);
                    Cv = sel2(i0, i1, f2mul(RS, f2sub(IR2, make_float2(irc2, irc2))), z);     // 1/r^3 - 1/(r rc^2)
                    DC = sel2(i0, i1, f2mul(IR2, f2fma(M3, IR2, make_float2(irc2, irc2))), z);  // -3/r^4 + 1/(r^2 rc^2)
                } else {
                    Cv = f2mul(RS, IR2);
                    DC = f2mul(M3, f2mul(IR2, IR2));
                }
                const float2 S = f2fma(EIJ, SLJ, f2mul(QQ, Cv));
                const float2 DSDR = f2fma(QQ, DC, DSLJDR);
                const float2 AD = f2fma(GX, DX, f2fma(GY, DY, f2mul(GZ, DZ)));
                const float2 RAD = sel2(c0, c1, make_float2(0.f, 0.f), f2mul(f2mul(DSDR, AD), RS));  // dS/dr (a.delta)/r
                GPX = f2sub(GPX, f2fma(S, GX, f2mul(RAD, DX)));
                GPY = f2sub(GPY, f2fma(S, GY, f2mul(RAD, DY)));
                GPZ = f2sub(GPZ, f2fma(S, GZ, f2mul(RAD, DZ)));
                GR = f2fma(AD, sel2(c0, c1, f2fma(DSDR, CF, DSLJDRR), DSLJDRR), GR);
                GE = f2fma(AD, SLJ, GE);
                CC = f2fma(AD, Cv, CC);
                if (kQuad) {
                    // Phi = A delta - 6 dz r^-5 z_hat, A = 15 dz^2 r^-7 - 3 r^-5 (cut off at rc)
                    const bool q0 = !kCutoff || in_rc(R2v.x), q1 = !kCutoff || in_rc(R2v.y);
                    const float2 z = make_float2(0.f, 0.f);
                    const float2 IR5 = f2mul(f2mul(IR2, IR2), RS), IR7 = f2mul(IR5, IR2), DZ2 = f2mul(DZ, DZ);
                    const float2 Aq = sel2(q0, q1, f2fma(f2mul(make_float2(15.f, 15.f), DZ2), IR7, f2mul(M3, IR5)), z);
                    const float2 A6 = sel2(q0, q1, f2mul(make_float2(6.f, 6.f), f2mul(DZ, IR5)), z);
                    CQ = f2fma(Aq, AD, f2fma(f2mul(make_float2(-1.f, -1.f), A6), GZ, CQ));  // a . Phi
                    // a . dPhi/dr at fixed delta, and the z row of a^T dPhi/d delta at fixed r
                    const float2 W = sel2(q0, q1,
                                          f2mul(RS, f2fma(f2fma(f2mul(make_float2(-105.f, -105.f), DZ2), IR7,
                                                                f2mul(make_float2(15.f, 15.f), IR5)),
                                                          AD, f2mul(f2mul(make_float2(30.f, 30.f), DZ), f2mul(IR5, GZ)))),
                                          z);
                    const float2 ZROW = sel2(q0, q1,
                                             f2fma(f2mul(make_float2(30.f, 30.f), f2mul(DZ, IR7)), AD,
                                                   f2mul(f2mul(M6, IR5), GZ)),
                                             z);
                    const float2 WR = sel2(c0, c1, z, f2mul(W, RS));  // r follows delta unless floored
                    const float2 MK = make_float2(-kqq, -kqq);
                    GPX = f2fma(MK, f2fma(Aq, GX, f2mul(WR, DX)), GPX);
                    GPY = f2fma(MK, f2fma(Aq, GY, f2mul(WR, DY)), GPY);
                    GPZ = f2fma(MK, f2fma(Aq, GZ, f2fma(WR, DZ, ZROW)), GPZ);
                    GR = sel2(c0, c1, f2fma(make_float2(kqq * P.core_frac, kqq * P.core_frac), W, GR), GR);
                }
            };
            if (kCutoff && __all_sync(live, R2v.x >= rc2 && R2v.y >= rc2)) pair(std::true_type{});
            else pair(std::false_type{});
        }
        const float gpx = GPX.x + GPX.y, gpy = GPY.x + GPY.y, gpz = GPZ.x + GPZ.y;
        const float gRr = GR.x + GR.y, ge = GE.x + GE.y, C = CC.x + CC.y, Cq = CQ.x + CQ.y;
        atomicAdd(P.gx + ia, gpx);
        atomicAdd(P.gy + ia, gpy);
        atomicAdd(P.gz + ia, gpz);
        atomicAdd(P.gR + ia, gRr);
        atomicAdd(P.geps + ia, ge);
        if (kQuad) {
            atomicAdd(P.gq + ia, fmaf(P.Q, C, 0.5f * P.Qzz * Cq));  // per unit k_e
            qC = fmaf(P.aq[ia], C, qC);
            qCq = fmaf(P.aq[ia], Cq, qCq);
        } else {
            atomicAdd(P.gq + ia, C);
        }
    }
    if (kQuad) {
        qC = warp_sum(qC);
        qCq = warp_sum(qCq);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(P.qsum + 0, qC);
            atomicAdd(P.qsum + 1, qCq);
        }
    }
}

// s + t with the rounding error carried in c (Kahan): the f32x2 instructions are not reassociated.
__device__ __forceinline__ void kahan_add(float2& s, float2& c, float2 t) {
    const float2 y = f2sub(t, c);
    const float2 u = f2add(s, y);
    c = f2sub(f2sub(u, s), y);
    s = u;
}

// K5 on an energy grid: dL/dtheta_i = sum_g Ebar_g dE_g/dtheta_i.  Same staging as the force
// variant, with the nodes' scalar adjoints in pairs, (x0, x1, y0, y1), (z0, z1, e0, e1).  Per
// node, with delta = r_g - r_i and r = |delta| (floored at core_frac R_iPP):
//   position  -dE/d delta = F: S delta (+ cq Phi), and inside the floor only the quadrupole's
//             explicit dz term remains (r is then constant in delta);
//   R_iPP     12 e (s12 - s6) / R, or core_frac (qq de_el/dr + cq deq/dr) inside the floor;
//   e_iPP     s12 - 2 s6 per unit e_iPP;  charges  C = sum Ebar e_el, Cq = sum Ebar eq,
// with e_el = 1/r (shifted-force: 1/r + r/rc^2 - 2/rc) and eq = 3 dz^2/r^5 - 1/r^3.
// The node adjoint sums to zero over every stencil (the weight gradients do), so the charge
// sums are differences of terms about r/dx larger than themselves (thousands of times larger
// for the long-ranged e_el): C and Cq are accumulated with compensation, and the cross-CTA
// sums of q_i C_i and q_i Cq_i (dL/dQ, dL/dQzz, which cancel again across a neutral molecule)
// in FP64.
template <bool kMinImage, bool kCutoff, bool kQuad>
__global__ void __launch_bounds__(kFFBThreads) ff_backward_energy_kernel(const BwdLaunch P) {
    __shared__ float4 sxy[kFFBNodes / 2];  // (x0, x1, y0, y1)
    __shared__ float4 sze[kFFBNodes / 2];  // (z0, z1, e0, e1)
    __shared__ int scount;
    const int nx = P.map.nx, ny = P.map.ny;
    const int64_t nxy = (int64_t)nx * ny;
    const int64_t first = (int64_t)blockIdx.x * kFFBNodes;
    const int klo = P.slab[0], khi = P.slab[1];
    if (khi < 0) return;
    const int kfirst = (int)(first / nxy), klast = (int)((first + kFFBNodes - 1) / nxy);
    if (klast < klo || kfirst > khi) return;
    if (threadIdx.x == 0) scount = 0;
    __syncthreads();
    float* fxy = reinterpret_cast<float*>(sxy);
    float* fze = reinterpret_cast<float*>(sze);
    const int64_t total = nxy * P.map.nz;
    for (int t = threadIdx.x; t < kFFBNodes; t += kFFBThreads) {
        const int64_t g = first + t;
        bool keep = false;
        float e = 0.f;
        int i = 0, j = 0, k = 0;
        if (g < total) {
            k = (int)(g / nxy);
            const int64_t r = g - (int64_t)k * nxy;
            j = (int)(r / nx);
            i = (int)(r - (int64_t)j * nx);
            e = P.gbarE[checked(node_index(P.map, i, j, k), P.map.stored_nodes, kChkGridRead)];
            keep = e != 0.f;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if ((threadIdx.x & 31) == 0 && mask) base = atomicAdd(&scount, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const int slot = base + __popc(mask & ((1u << (threadIdx.x & 31)) - 1u));
            const int q = (slot >> 1) * 4, l = slot & 1;
            fxy[q + l] = P.x0 + i * P.dx;
            fxy[q + 2 + l] = P.y0 + j * P.dy;
            fze[q + l] = P.z0 + k * P.dz;
            fze[q + 2 + l] = e;
        }
    }
    __syncthreads();
    const int cnt = scount;
    if (cnt == 0) return;
    if ((cnt & 1) && threadIdx.x == 0) {
        const int q = (cnt >> 1) * 4;  // pad the last pair with its node and a zero adjoint
        fxy[q + 1] = fxy[q];
        fxy[q + 3] = fxy[q + 2];
        fze[q + 1] = fze[q];
        fze[q + 3] = 0.f;
    }
    __syncthreads();
    const int npairs = (cnt + 1) >> 1;
    const float rc2 = kCutoff ? P.coul_rc * P.coul_rc : 0.f;
    const float irc = kCutoff ? 1.f / P.coul_rc : 0.f, irc2 = irc * irc;
    const float invLx = kMinImage ? 1.f / P.Lx : 0.f, invLy = kMinImage ? 1.f / P.Ly : 0.f;
    const float2 TWELVE = make_float2(12.f, 12.f), M2 = make_float2(-2.f, -2.f);
    const float2 Z2 = make_float2(0.f, 0.f);
    double qC = 0.0, qCq = 0.0;  // this thread's q_i C_i and q_i Cq_i, summed in FP64
    for (int a0 = 0; a0 < P.n; a0 += kFFBThreads) {
        const int ia = a0 + threadIdx.x;
        if (ia >= P.n) break;
        const float ax = P.ax[ia], ay = P.ay[ia], azz = P.az[ia];
        const float Rij = P.aR[ia] + P.R_pp;
        const float eij = sqrtf(P.aeps[ia] * P.eps_pp);
        const float qq = P.kQ * P.aq[ia];
        const float rmin2 = (P.core_frac * Rij) * (P.core_frac * Rij);
        const float kqq = kQuad ? P.kQzz * P.aq[ia] : 0.f;
        const float2 AX = make_float2(ax, ax), AY = make_float2(ay, ay), AZ = make_float2(azz, azz);
        const float2 RR2 = make_float2(Rij * Rij, Rij * Rij), EIJ = make_float2(eij, eij), QQ = make_float2(qq, qq);
        const float2 E12R = make_float2(12.f * eij / Rij, 12.f * eij / Rij);
        const float2 QCF = make_float2(qq * P.core_frac, qq * P.core_frac);
        const float2 KCF = make_float2(kqq * P.core_frac, kqq * P.core_frac), KQ = make_float2(kqq, kqq);
        float2 GPX = Z2, GPY = Z2, GPZ = Z2, GR = Z2, GE = Z2, CC = Z2, CQ = Z2;
        float2 KC = Z2, KQ2 = Z2;  // compensations of CC and CQ
        for (int pr = 0; pr < npairs; ++pr) {
            const float4 A = sxy[pr], B = sze[pr];
            float2 DX = f2sub(make_float2(A.x, A.y), AX), DY = f2sub(make_float2(A.z, A.w), AY);
            const float2 DZ = f2sub(make_float2(B.x, B.y), AZ);
            const float2 EB = make_float2(B.z, B.w);
            if (kMinImage) {
                DX.x = fmaf(-P.Lx, rintf(DX.x * invLx), DX.x);
                DX.y = fmaf(-P.Lx, rintf(DX.y * invLx), DX.y);
                DY.x = fmaf(-P.Ly, rintf(DY.x * invLy), DY.x);
                DY.y = fmaf(-P.Ly, rintf(DY.y * invLy), DY.y);
            }
            const float2 R2raw = f2fma(DX, DX, f2fma(DY, DY, f2mul(DZ, DZ)));
            const bool c0 = R2raw.x < rmin2, c1 = R2raw.y < rmin2;
            const float2 R2v = make_float2(c0 ? rmin2 : R2raw.x, c1 ? rmin2 : R2raw.y);
            const float2 RS = make_float2(rsqrtf(R2v.x), rsqrtf(R2v.y));
            const float2 IR2 = f2mul(RS, RS);
            const float2 U = f2mul(RR2, IR2);
            const float2 S6 = f2mul(f2mul(U, U), U);
            const float2 S12 = f2mul(S6, S6);
            float2 Cv, EEL, DE;
            if (kCutoff) {
                const bool i0 = R2v.x < rc2, i1 = R2v.y < rc2;
                const float2 R = f2mul(R2v, RS);
                Cv = sel2(i0, i1, f2mul(RS, f2sub(IR2, make_float2(irc2, irc2))), Z2);
                EEL = sel2(i0, i1, f2fma(R, make_float2(irc2, irc2), f2sub(RS, make_float2(2.f * irc, 2.f * irc))), Z2);
                DE = sel2(i0, i1, f2sub(make_float2(irc2, irc2), IR2), Z2);
            } else {
                Cv = f2mul(RS, IR2);
                EEL = RS;
                DE = f2mul(make_float2(-1.f, -1.f), IR2);
            }
            // S = e 12 (s12 - s6) / r^2 + qq c
            const float2 S = f2fma(f2mul(EIJ, f2mul(TWELVE, f2sub(S12, S6))), IR2, f2mul(QQ, Cv));
            float2 FS = S;       // coefficient of delta in F (zero inside the floor)
            float2 FZ = Z2;      // extra z component of F
            float2 GRc = f2mul(QCF, DE);  // dE/dR inside the floor
            if (kQuad) {
                const bool q0 = !kCutoff || R2v.x < rc2, q1 = !kCutoff || R2v.y < rc2;
                const float2 IR5 = f2mul(f2mul(IR2, IR2), RS), DZ2 = f2mul(DZ, DZ);
                const float2 T = f2mul(DZ2, IR2);  // dz^2 / r^2
                // Phi = (15 dz^2/r^7 - 3/r^5) delta - (6 dz/r^5) z_hat
                const float2 Aq = sel2(q0, q1, f2mul(IR5, f2fma(make_float2(15.f, 15.f), T, make_float2(-3.f, -3.f))), Z2);
                const float2 A6 = sel2(q0, q1, f2mul(make_float2(6.f, 6.f), f2mul(DZ, IR5)), Z2);
                const float2 EQ = sel2(q0, q1, f2mul(f2mul(RS, IR2), f2fma(make_float2(3.f, 3.f), T, make_float2(-1.f, -1.f))), Z2);
                const float2 DEQ = sel2(q0, q1, f2mul(f2mul(IR2, IR2), f2fma(make_float2(-15.f, -15.f), T, make_float2(3.f, 3.f))), Z2);
                FS = f2fma(KQ, Aq, FS);
                FZ = f2mul(KQ, A6);  // F_z gets -cq 6 dz / r^5 (subtracted below)
                GRc = f2fma(KCF, DEQ, GRc);
                kahan_add(CQ, KQ2, f2mul(EB, EQ));
            }
            const float2 EF = sel2(c0, c1, Z2, f2mul(EB, FS));
            GPX = f2fma(EF, DX, GPX);
            GPY = f2fma(EF, DY, GPY);
            GPZ = f2sub(f2fma(EF, DZ, GPZ), f2mul(EB, FZ));
            GR = f2fma(EB, sel2(c0, c1, GRc, f2mul(E12R, f2sub(S12, S6))), GR);
            GE = f2fma(EB, f2fma(M2, S6, S12), GE);
            kahan_add(CC, KC, f2mul(EB, EEL));
        }
        const float gpx = GPX.x + GPX.y, gpy = GPY.x + GPY.y, gpz = GPZ.x + GPZ.y;
        const double Cd = ((double)CC.x - KC.x) + ((double)CC.y - KC.y);
        const double Cqd = ((double)CQ.x - KQ2.x) + ((double)CQ.y - KQ2.y);
        const float gRr = GR.x + GR.y, ge = GE.x + GE.y, C = (float)Cd, Cq = (float)Cqd;
        atomicAdd(P.gx + ia, gpx);
        atomicAdd(P.gy + ia, gpy);
        atomicAdd(P.gz + ia, gpz);
        atomicAdd(P.gR + ia, gRr);
        atomicAdd(P.geps + ia, ge);
        atomicAdd(P.gq + ia, fmaf(P.Q, C, 0.5f * P.Qzz * Cq));  // per unit k_e
        qC += (double)P.aq[ia] * Cd;
        if (kQuad) qCq += (double)P.aq[ia] * Cqd;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        qC += __shfl_xor_sync(0xffffffffu, qC, o);
        qCq += __shfl_xor_sync(0xffffffffu, qCq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (qC != 0.0) atomicAdd(P.qsumd + 0, qC);
        if (kQuad && qCq != 0.0) atomicAdd(P.qsumd + 1, qCq);
    }
}

// Charges and well depths from the accumulated sums; dL/dQ by a block reduction
// (with a tip quadrupole, or on an energy grid, K5 has already combined the charge
// terms and summed q_i C_i and q_i Cq_i).
__global__ void finalize_kernel(const BwdLaunch P) {
    __shared__ float red[32];
    if (P.Qzz != 0.f || P.map.interp) {
        for (int a = threadIdx.x; a < P.n; a += blockDim.x) {
            P.gq[a] *= P.ke;
            const float eij = sqrtf(P.aeps[a] * P.eps_pp);
            P.geps[a] = eij > 0.f ? P.geps[a] * P.eps_pp / (2.f * eij) : 0.f;
        }
        if (threadIdx.x == 0) {
            P.gtip[3] = P.map.interp ? (float)((double)P.ke * P.qsumd[0]) : P.ke * P.qsum[0];
            P.gtip[4] = P.map.interp ? (float)(0.5 * (double)P.ke * P.qsumd[1]) : 0.5f * P.ke * P.qsum[1];
        }
        return;
    }
    float acc = 0.f;
    for (int a = threadIdx.x; a < P.n; a += blockDim.x) {
        const float C = P.gq[a] * P.ke;  // sum (a.delta) k_e c
        acc = fmaf(P.aq[a], C, acc);
        P.gq[a] = P.Q * C;
        const float eij = sqrtf(P.aeps[a] * P.eps_pp);
        P.geps[a] = eij > 0.f ? P.geps[a] * P.eps_pp / (2.f * eij) : 0.f;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        v = warp_sum(v);
        if (threadIdx.x == 0) P.gtip[3] = v;
    }
}

template <int LAYOUT, int M>
void launch_adjoint_m(const BwdLaunch& L, int blocks, cudaStream_t s) {
    if constexpr (LAYOUT == 0) {
        if (L.map.interp) {  // energy grids are stored in the linear layout
            relax_adjoint_kernel<0, M, true><<<blocks, kAdjThreads, 0, s>>>(L);
            return;
        }
    }
    relax_adjoint_kernel<LAYOUT, M, false><<<blocks, kAdjThreads, 0, s>>>(L);
}

// Compile-time stencil half widths 1..8 (A_pp / dz up to 16), the run-time loop beyond.
template <int LAYOUT>
void launch_adjoint_layout(const BwdLaunch& L, int blocks, cudaStream_t s) {
    switch (L.m) {
        case 1: launch_adjoint_m<LAYOUT, 1>(L, blocks, s); break;
        case 2: launch_adjoint_m<LAYOUT, 2>(L, blocks, s); break;
        case 3: launch_adjoint_m<LAYOUT, 3>(L, blocks, s); break;
        case 4: launch_adjoint_m<LAYOUT, 4>(L, blocks, s); break;
        case 5: launch_adjoint_m<LAYOUT, 5>(L, blocks, s); break;
        case 6: launch_adjoint_m<LAYOUT, 6>(L, blocks, s); break;
        case 7: launch_adjoint_m<LAYOUT, 7>(L, blocks, s); break;
        case 8: launch_adjoint_m<LAYOUT, 8>(L, blocks, s); break;
        default: launch_adjoint_m<LAYOUT, -1>(L, blocks, s); break;
    }
}

void launch_adjoint(const BwdLaunch& L, int blocks, cudaStream_t s) {
    if (L.layout == 0) launch_adjoint_layout<0>(L, blocks, s);
    else launch_adjoint_layout<1>(L, blocks, s);
}

}  // namespace

cudaError_t launch_backward(const BwdLaunch& L, cudaStream_t s) {
    init_kernel<<<(L.n + 255) / 256 + 1, 256, 0, s>>>(L);
    const int64_t total = (int64_t)L.snx * L.sny * L.snz;
    // one wave of resident blocks (8 per SM at this register count), grid-stride inside
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (total + kAdjThreads - 1) / kAdjThreads;
    const int blocks = (int)(need < 8LL * sms ? (need > 0 ? need : 1) : 8LL * sms);
    launch_adjoint(L, blocks, s);
    if (L.n > 0) {
        const int64_t nodes = (int64_t)L.map.nx * L.map.ny * L.map.nz;
        const int fb = (int)((nodes + kFFBNodes - 1) / kFFBNodes);
        with_flags(L.min_image != 0, L.coul_rc > 0.f, L.Qzz != 0.f, [&](auto mi, auto cut, auto quad) {
            constexpr bool MI = decltype(mi)::value, CUT = decltype(cut)::value, QUAD = decltype(quad)::value;
            if (L.map.interp) ff_backward_energy_kernel<MI, CUT, QUAD><<<fb, kFFBThreads, 0, s>>>(L);
            else ff_backward_kernel<MI, CUT, QUAD><<<fb, kFFBThreads, 0, s>>>(L);
            return 0;
        });
    }
    finalize_kernel<<<1, 256, 0, s>>>(L);
    return cudaGetLastError();
}

PP_CHECK_READER(check_flags_backward)

}  // namespace pp
