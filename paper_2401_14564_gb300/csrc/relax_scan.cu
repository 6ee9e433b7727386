// K2: relaxed tip scan (Sec. 5.1.1 step 2) with an optional fused df epilogue.
//
// One thread owns one pixel column and walks its heights from the top down:
// the PP starts at anchor + d0 for the first height and at p*(k-1) - dz z_hat
// (the tip moved down by dz, the deflection kept) for the others, and is
// relaxed by FIRE on G(p) = F_T(p) + F_S(p) (Eq. F_PP), with the tip springs
// of Eq. F_tip and F_S trilinearly interpolated from the force grid.  The tip
// force is read out as Fz = -F^T_{R,z} = kR (|d| - R0) d_z / |d| (Sec. 2.1).
//
// The FIRE state is e = d - d0, the deflection from the spring's rest
// displacement.  Then |d|^2 - R0^2 = (2 d0 + e).e + (|d0|^2 - R0^2) is formed
// without cancellation, so the radial extension and Fz keep full FP32
// relative precision however stiff the spring (with d itself the extension
// would be quantised at ulp(R0) ~ 5e-7 A, i.e. 3e-4 eV/A at 1e4 N/m).
//
// Lanes of a warp cover an 8x4 pixel tile, so the 32 PPs sit in neighbouring
// grid cells and their corner loads share L1 lines.  Each lane advances to its
// next height as soon as it has converged; the warp only waits for its
// slowest lane once, at the end of the columns, not at every height.
// Interpolation is done by hand in FP32 from eight float4 corner loads on the
// read-only path (hardware texture filtering carries only 8 fractional bits
// in its weights, which would cost the 1e-3 A position parity).
#include "interp.cuh"

namespace pp {
namespace {

constexpr int kThreads = 32;  // one warp per CTA: an 8x4 pixel tile (evens out warps per SM)
constexpr int kTileX = 8;
constexpr int kTileY = 4;

// Radial factor s = -kR (|d| - R0) / |d| with d = d0 + e, from
// q = |d|^2 - R0^2 = (2 d0 + e).e + c0 and (|d| - R0)/|d| = q / (|d|^2 + R0 |d|).
__device__ __forceinline__ float radial_factor(const RelaxLaunch& P, float3 e) {
    const float q = fmaf(2.f * P.d0x + e.x, e.x, fmaf(2.f * P.d0y + e.y, e.y, fmaf(2.f * P.d0z + e.z, e.z, P.c0)));
    const float d2 = P.R0sq + q;
    const float dn = d2 * rsqrtf(d2);
    return -P.kR * __fdividef(q, fmaf(P.R0, dn, d2));
}

__device__ __forceinline__ float3 total_force_tip(const RelaxLaunch& P, float3 e, float s, float3 Fs) {
    float3 G;
    G.x = fmaf(s, P.d0x + e.x, fmaf(-P.kx, e.x, Fs.x));
    G.y = fmaf(s, P.d0y + e.y, fmaf(-P.ky, e.y, Fs.y));
    G.z = fmaf(s, P.d0z + e.z, Fs.z);
    return G;
}

template <int LAYOUT>
__global__ void __launch_bounds__(kThreads) relax_scan_kernel(const RelaxLaunch P) {
    const int lane = threadIdx.x;
    const int i = blockIdx.x * kTileX + (lane & 7);
    const int j = blockIdx.y * kTileY + (lane >> 3);
    const bool valid = (i < P.snx) && (j < P.sny);
    const int npix = P.snx * P.sny;
    const int pix = j * P.snx + i;

    // rest position of the PP under this pixel's anchor, without the height
    const float bx = fmaf((float)i, P.spx, P.sx0) + P.d0x;
    const float by = fmaf((float)j, P.spy, P.sy0) + P.d0y;

    float3 e = make_float3(0.f, 0.f, 0.f), v = make_float3(0.f, 0.f, 0.f);
    float dt = P.dt0, alpha = P.alpha0;
    int npos = 0, it = 0, k = 0;
    bool active = valid;
    // Corner values of the cell holding the PP, reloaded only when the PP
    // changes cell (a converging PP rarely does after its first steps).
    float4 cv[8];
    int cell_x = -1, cell_y = -1, cell_z = -1;
    while (__any_sync(0xffffffffu, active)) {
        if (!active) continue;
        const float az = P.z_top - k * P.sdz;
        const float s = radial_factor(P, e);
        const Cells cl = locate(P, bx + e.x, by + e.y, (az + P.d0z) + e.z);
        if (cl.x.i0 != cell_x || cl.y.i0 != cell_y || cl.z.i0 != cell_z) {
            load_corners<LAYOUT>(P.ff, P.map, cl, cv);
            cell_x = cl.x.i0;
            cell_y = cl.y.i0;
            cell_z = cl.z.i0;
        }
        const float3 Fs = trilinear(cv, cl);
        const float3 G = total_force_tip(P, e, s, Fs);
        const float g2 = fmaf(G.x, G.x, fmaf(G.y, G.y, G.z * G.z));
        if (g2 < P.ftol2 || it >= P.max_iter) {
            // converged (or out of iterations) at height k: write, then go one height down
            // keeping the deflection e (the warm start p*(k-1) - dz z_hat)
            const int o = k * npix + pix;
            P.fz[o] = -s * (P.d0z + e.z);  // kR (|d| - R0) d_z / |d|
            if (P.pos) {
                P.pos[3 * o] = bx + e.x;
                P.pos[3 * o + 1] = by + e.y;
                P.pos[3 * o + 2] = (az + P.d0z) + e.z;
            }
            if (P.iters) P.iters[o] = it;
            ++k;
            active = k < P.snz;
            v = make_float3(0.f, 0.f, 0.f);
            dt = P.dt0;
            alpha = P.alpha0;
            npos = 0;
            it = 0;
            continue;
        }
        if (it > 0) {
            const float pw = fmaf(G.x, v.x, fmaf(G.y, v.y, G.z * v.z));
            if (pw > 0.f) {
                const float v2 = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
                const float c = alpha * (v2 * rsqrtf(v2)) * rsqrtf(g2);  // alpha |v| / |G|
                const float om = 1.f - alpha;
                v.x = fmaf(om, v.x, c * G.x);
                v.y = fmaf(om, v.y, c * G.y);
                v.z = fmaf(om, v.z, c * G.z);
                if (npos > P.n_min) {
                    dt = fminf(dt * P.f_inc, P.dt_max);
                    alpha *= P.f_alpha;
                }
                ++npos;
            } else {
                v = make_float3(0.f, 0.f, 0.f);
                dt *= P.f_dec;
                alpha = P.alpha0;
                npos = 0;
            }
        }
        const float h = dt * P.inv_mass;
        v.x = fmaf(h, G.x, v.x);
        v.y = fmaf(h, G.y, v.y);
        v.z = fmaf(h, G.z, v.z);
        e.x = fmaf(dt, v.x, e.x);
        e.y = fmaf(dt, v.y, e.y);
        e.z = fmaf(dt, v.z, e.z);
        ++it;
    }

    if (P.df_m >= 0 && valid) {
        // Fused df: this thread wrote its own Fz column above (program order makes it visible).
        const int m = P.df_m;
        for (int c = m; c < P.snz - m; ++c) {
            float acc = 0.f;
            for (int t = -m; t <= m; ++t) acc = fmaf(P.coef[t + m], P.fz[(c + t) * npix + pix], acc);
            P.df[(c - m) * npix + pix] = acc;
        }
    }
}

}  // namespace

cudaError_t launch_relax_scan(const RelaxLaunch& L, cudaStream_t s) {
    dim3 grid((L.snx + kTileX - 1) / kTileX, (L.sny + kTileY - 1) / kTileY, 1);
    if (L.layout == 0) relax_scan_kernel<0><<<grid, kThreads, 0, s>>>(L);
    else relax_scan_kernel<1><<<grid, kThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace pp
