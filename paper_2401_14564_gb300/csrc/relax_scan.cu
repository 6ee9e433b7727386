// K2: relaxed tip scan (Sec. 5.1.1 step 2) with an optional fused df epilogue.
//
// One thread owns one pixel column and walks its heights from the top down:
// the PP starts at anchor + d0 for the first height and at p*(k-1) - dz z_hat
// (the tip moved down by dz, the deflection kept) for the others, and is
// relaxed by FIRE on G(p) = F_T(p) + F_S(p) (Eq. F_PP), with the tip springs
// of Eq. F_tip and F_S trilinearly interpolated from the force grid.  The tip
// force is read out as Fz = -F^T_{R,z} = kR (|d| - R0) d_z / |d| (Sec. 2.1).
//
// Interpolation is done by hand in FP32 from eight float4 corner loads on the
// read-only path (hardware texture filtering carries only 8 fractional bits
// in its weights, which would cost the 1e-3 A position parity).  Lanes of a
// warp cover an 8x4 pixel tile, so the 32 PPs sit in neighbouring grid cells
// and their corner loads share cache lines.  Each lane runs its own FIRE
// state; lanes that have converged idle until the whole warp is done, and the
// warp then moves to the next height together.
#include "pp_internal.cuh"

namespace pp {
namespace {

constexpr int kTileX = 16;
constexpr int kTileY = 8;
constexpr int kThreads = kTileX * kTileY;

struct Cell {
    int i0, i1;
    float t;
};

__device__ __forceinline__ Cell axis_cell(float p, float o, float inv_h, int n, int periodic) {
    float f = (p - o) * inv_h;
    f = fminf(fmaxf(f, -1.0e7f), 1.0e7f);  // keeps the integer conversion defined for any input
    const float fl = floorf(f);
    int i = (int)fl;
    Cell c;
    if (periodic) {
        int m = i % n;
        if (m < 0) m += n;
        c.i0 = m;
        c.i1 = (m + 1 == n) ? 0 : m + 1;
        c.t = f - fl;
    } else {
        i = min(max(i, 0), n - 2);
        c.i0 = i;
        c.i1 = i + 1;
        c.t = fminf(fmaxf(f - (float)i, 0.f), 1.f);
    }
    return c;
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Trilinear interpolation of (Fx, Fy, Fz) at p.
__device__ __forceinline__ float3 sample_force(const RelaxLaunch& P, float px, float py, float pz) {
    const Cell cx = axis_cell(px, P.gx0, P.inv_dx, P.map.nx, P.periodic_xy);
    const Cell cy = axis_cell(py, P.gy0, P.inv_dy, P.map.ny, P.periodic_xy);
    const Cell cz = axis_cell(pz, P.gz0, P.inv_dz, P.map.nz, 0);
    const int x0 = axis_off(P.map.ax, cx.i0), x1 = axis_off(P.map.ax, cx.i1);
    const int y0 = axis_off(P.map.ay, cy.i0), y1 = axis_off(P.map.ay, cy.i1);
    const int z0 = axis_off(P.map.az, cz.i0), z1 = axis_off(P.map.az, cz.i1);
    const float4 c000 = __ldg(P.ff + (x0 + y0 + z0));
    const float4 c100 = __ldg(P.ff + (x1 + y0 + z0));
    const float4 c010 = __ldg(P.ff + (x0 + y1 + z0));
    const float4 c110 = __ldg(P.ff + (x1 + y1 + z0));
    const float4 c001 = __ldg(P.ff + (x0 + y0 + z1));
    const float4 c101 = __ldg(P.ff + (x1 + y0 + z1));
    const float4 c011 = __ldg(P.ff + (x0 + y1 + z1));
    const float4 c111 = __ldg(P.ff + (x1 + y1 + z1));
    float3 F;
    F.x = lerpf(lerpf(lerpf(c000.x, c100.x, cx.t), lerpf(c010.x, c110.x, cx.t), cy.t),
                lerpf(lerpf(c001.x, c101.x, cx.t), lerpf(c011.x, c111.x, cx.t), cy.t), cz.t);
    F.y = lerpf(lerpf(lerpf(c000.y, c100.y, cx.t), lerpf(c010.y, c110.y, cx.t), cy.t),
                lerpf(lerpf(c001.y, c101.y, cx.t), lerpf(c011.y, c111.y, cx.t), cy.t), cz.t);
    F.z = lerpf(lerpf(lerpf(c000.z, c100.z, cx.t), lerpf(c010.z, c110.z, cx.t), cy.t),
                lerpf(lerpf(c001.z, c101.z, cx.t), lerpf(c011.z, c111.z, cx.t), cy.t), cz.t);
    return F;
}

// G = F_T + F_S for the displacement d = p - a (Eq. F_PP with Eq. F_tip).
// The radial term uses the correctly rounded |d|, so |d| = R0 gives exactly 0.
__device__ __forceinline__ float3 total_force(const RelaxLaunch& P, float3 a, float3 d) {
    const float d2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
    const float s = -P.kR * (sqrtf(d2) - P.R0) * rsqrtf(d2);  // -kR (|d| - R0) / |d|
    const float3 Fs = sample_force(P, a.x + d.x, a.y + d.y, a.z + d.z);
    float3 G;
    G.x = fmaf(s, d.x, fmaf(-P.kx, d.x - P.d0x, Fs.x));
    G.y = fmaf(s, d.y, fmaf(-P.ky, d.y - P.d0y, Fs.y));
    G.z = fmaf(s, d.z, Fs.z);
    return G;
}

__global__ void __launch_bounds__(kThreads) relax_scan_kernel(const RelaxLaunch P) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kTileX + (warp & 1) * 8 + (lane & 7);
    const int j = blockIdx.y * kTileY + (warp >> 1) * 4 + (lane >> 3);
    const bool valid = (i < P.snx) && (j < P.sny);
    const int npix = P.snx * P.sny;
    const int pix = j * P.snx + i;

    float3 a;
    a.x = P.sx0 + i * P.spx;
    a.y = P.sy0 + j * P.spy;
    // The FIRE state is the displacement d = p - anchor: lowering the tip by dz
    // with d unchanged is exactly the warm start p*(k-1) - dz z_hat.
    float3 d = make_float3(P.d0x, P.d0y, P.d0z);

    for (int k = 0; k < P.snz; ++k) {
        a.z = P.z_top - k * P.sdz;

        float3 v = make_float3(0.f, 0.f, 0.f);
        float dt = P.dt0, alpha = P.alpha0;
        int npos = 0, it = 0;
        bool active = valid;
        // Lanes run their own FIRE; the warp leaves the loop once no lane is active.
        while (__any_sync(0xffffffffu, active)) {
            if (active) {
                const float3 G = total_force(P, a, d);
                const float g2 = fmaf(G.x, G.x, fmaf(G.y, G.y, G.z * G.z));
                if (g2 < P.ftol2 || it >= P.max_iter) {
                    active = false;
                } else {
                    if (it > 0) {
                        const float pw = fmaf(G.x, v.x, fmaf(G.y, v.y, G.z * v.z));
                        if (pw > 0.f) {
                            const float vn = sqrtf(fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z)));
                            const float c = alpha * vn * rsqrtf(g2);
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
                    d.x = fmaf(dt, v.x, d.x);
                    d.y = fmaf(dt, v.y, d.y);
                    d.z = fmaf(dt, v.z, d.z);
                    ++it;
                }
            }
        }
        if (valid) {
            const float d2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
            const int o = k * npix + pix;
            P.fz[o] = P.kR * (sqrtf(d2) - P.R0) * rsqrtf(d2) * d.z;  // kR (|d| - R0) d_z / |d|
            if (P.pos) {
                P.pos[3 * o] = a.x + d.x;
                P.pos[3 * o + 1] = a.y + d.y;
                P.pos[3 * o + 2] = a.z + d.z;
            }
            if (P.iters) P.iters[o] = it;
        }
    }

    if (P.df_m >= 0 && valid) {
        // Fused df: this thread wrote its own Fz column above (program order makes it visible).
        const int m = P.df_m;
        for (int c = m; c < P.snz - m; ++c) {
            float s = 0.f;
            for (int t = -m; t <= m; ++t) s = fmaf(P.coef[t + m], P.fz[(c + t) * npix + pix], s);
            P.df[(c - m) * npix + pix] = s;
        }
    }
}

}  // namespace

cudaError_t launch_relax_scan(const RelaxLaunch& L, cudaStream_t s) {
    dim3 grid((L.snx + kTileX - 1) / kTileX, (L.sny + kTileY - 1) / kTileY, 1);
    relax_scan_kernel<<<grid, kThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace pp
