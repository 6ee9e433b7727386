// K9: IETS map (Sec. 3.3) -- vibration modes of the probe particle at its
// relaxed position.  The lateral CO mode is softened or stiffened by the
// curvature of the tip-sample potential; per relaxed point this kernel forms
// the stiffness K = -(J + J^T)/2, J = dG/dp = tip-spring Jacobian + exact
// Jacobian of the trilinear force interpolant (the same J the adjoint uses),
// or, on a tricubic energy grid, minus the Hessian of the energy interpolant,
// and writes its three eigenvalues ascending (cyclic Jacobi rotations, FP32,
// stopped once the off-diagonal part is below FP32 resolution) and the mode
// energies hbar sqrt(lambda/m).
#include "interp.cuh"

namespace pp {
namespace {

constexpr int kThreads = 128;

// One Jacobi rotation zeroing a[p][q] of a symmetric 3x3 (Rutishauser's tangent form).
__device__ __forceinline__ void jacobi_rotate(float a[3][3], int p, int q) {
    const float apq = a[p][q];
    if (fabsf(apq) < 1e-30f) return;
    const float th = (a[q][q] - a[p][p]) / (2.f * apq);
    const float t = copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
    const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
    }
}

template <int LAYOUT, bool kTricubic>
__global__ void __launch_bounds__(kThreads) iets_kernel(const IetsLaunch P) {
    const int npix = P.snx * P.sny;
    const int64_t total = (int64_t)npix * P.snz;
    const int64_t o = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (o >= total) return;
    const int k = (int)(o / npix), pix = (int)(o - (int64_t)k * npix);
    const int i = pix % P.snx, j = pix / P.snx;
    const int64_t o3 = checked(3 * o, 3 * total, kChkScanRead);
    const float px = __ldg(P.pos + o3), py = __ldg(P.pos + o3 + 1), pz = __ldg(P.pos + o3 + 2);
    const float dx = px - fmaf((float)i, P.spx, P.sx0), dy = py - fmaf((float)j, P.spy, P.sy0);
    float az, az_lo;  // anchor height z_top - k sdz as az + az_lo, as in K4
    {
        const float p_hi = __fmul_rn((float)k, P.sdz), p_lo = fmaf((float)k, P.sdz, -p_hi);
        two_sum(P.z_top, -p_hi, az, az_lo);
        az_lo -= p_lo;
    }
    const float dz = (pz - az) - az_lo;
    const float ex = dx - P.d0x, ey = dy - P.d0y, ez = dz - P.d0z;
    const float q = fmaf(2.f * P.d0x + ex, ex, fmaf(2.f * P.d0y + ey, ey, fmaf(2.f * P.d0z + ez, ez, P.c0)));
    const float d2 = P.R0sq + q;
    const float rs = rsqrtf(d2);
    const float dn = d2 * rs;
    const float ar = -P.kR * __fdividef(q, fmaf(P.R0, dn, d2));  // -kR (1 - R0/|d|)
    const float br = -P.kR * P.R0 * rs * rs * rs;                // -kR R0 / |d|^3
    const Cells cl = locate(P, px, py, pz);
    float J[3][3];
    if constexpr (kTricubic) {
        float ec[64];
        tricubic_load(P.ffE, P.map, cl, P.periodic_xy, ec);
        tricubic_jacobian(ec, cl, P.inv_dx, P.inv_dy, P.inv_dz, J);
    } else {
        float4 v[8];
        load_corners<LAYOUT>(P.ff, P.map, cl, v);
        trilinear_jacobian(v, cl, P.inv_dx, P.inv_dy, P.inv_dz, J);
    }
    const float dd[3] = {dx, dy, dz};
    float a[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int n = 0; n < 3; ++n)
            a[m][n] = -0.5f * (J[m][n] + J[n][m]) - ((m == n ? ar : 0.f) + br * dd[m] * dd[n]);
    a[0][0] += P.kx;
    a[1][1] += P.ky;
    // cyclic sweeps until every off-diagonal element is below the FP32 resolution of the diagonal
    // (the eigenvalue error is then a few ulps of |a|, also for a degenerate pair, where closed
    // forms through acos lose half the digits); at most 5, the warp leaving together
    const unsigned lanes = __activemask();
    for (int sweep = 0; sweep < 5; ++sweep) {
        const float off = fmaf(a[0][1], a[0][1], fmaf(a[0][2], a[0][2], a[1][2] * a[1][2]));
        const float diag = fmaf(a[0][0], a[0][0], fmaf(a[1][1], a[1][1], a[2][2] * a[2][2]));
        if (__all_sync(lanes, off <= 3.5527137e-15f * diag)) break;  // (2^-24)^2
        jacobi_rotate(a, 0, 1);
        jacobi_rotate(a, 0, 2);
        jacobi_rotate(a, 1, 2);
    }
    float e0 = a[0][0], e1 = a[1][1], e2 = a[2][2], t;
    if (e0 > e1) { t = e0; e0 = e1; e1 = t; }
    if (e1 > e2) { t = e1; e1 = e2; e2 = t; }
    if (e0 > e1) { t = e0; e0 = e1; e1 = t; }
    const int64_t w3 = checked(3 * o, 3 * total, kChkScanWrite);
    P.eig[w3] = e0;
    P.eig[w3 + 1] = e1;
    P.eig[w3 + 2] = e2;
    if (P.hw) {
        P.hw[w3] = e0 > 0.f ? P.hw_unit * sqrtf(e0) : 0.f;
        P.hw[w3 + 1] = e1 > 0.f ? P.hw_unit * sqrtf(e1) : 0.f;
        P.hw[w3 + 2] = e2 > 0.f ? P.hw_unit * sqrtf(e2) : 0.f;
    }
}

}  // namespace

cudaError_t launch_iets(const IetsLaunch& L, cudaStream_t s) {
    const int64_t total = (int64_t)L.snx * L.sny * L.snz;
    const int blocks = (int)((total + kThreads - 1) / kThreads);
    if (L.map.interp == 1) iets_kernel<0, true><<<blocks, kThreads, 0, s>>>(L);
    else if (L.layout == 0) iets_kernel<0, false><<<blocks, kThreads, 0, s>>>(L);
    else iets_kernel<1, false><<<blocks, kThreads, 0, s>>>(L);
    return cudaGetLastError();
}

PP_CHECK_READER(check_flags_iets)

}  // namespace pp
