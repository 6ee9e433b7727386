// FIRE relaxation of one pixel column (Sec. 5.1.1 step 2; Eqs. F_PP, F_tip;
// Sec. 2.1 readout; Eq. df epilogue), shared by the single-grid scan (K2) and
// the batched persistent kernel (K6).  G_t supplies the grid, scan and output
// fields and Q_t the tip, FIRE and df-stencil fields, under the names of
// RelaxLaunch (K2 passes its launch struct as both).
//
// The FIRE state is e = d - d0, the deflection from the spring's rest
// displacement: |d|^2 - R0^2 = (2 d0 + e).e + (|d0|^2 - R0^2) is then formed
// without cancellation, so the radial extension and Fz keep full FP32
// relative precision however stiff the spring.  Each lane advances to its
// next height as soon as it has converged (the warm start p*(k-1) - dz z_hat
// keeps e); the warp waits for its slowest lane only at the end.  The 8
// corner values of the PP's cell are cached in registers and reloaded only
// when the PP changes cell.
#pragma once

#include "interp.cuh"

namespace pp {

// Radial factor s = -kR (|d| - R0) / |d| with d = d0 + e, from
// q = |d|^2 - R0^2 = (2 d0 + e).e + c0 and (|d| - R0)/|d| = q / (|d|^2 + R0 |d|).
template <class Q_t>
__device__ __forceinline__ float radial_factor(const Q_t& P, float3 e) {
    const float q = fmaf(2.f * P.d0x + e.x, e.x, fmaf(2.f * P.d0y + e.y, e.y, fmaf(2.f * P.d0z + e.z, e.z, P.c0)));
    const float d2 = P.R0sq + q;
    const float dn = d2 * rsqrtf(d2);
    return -P.kR * __fdividef(q, fmaf(P.R0, dn, d2));
}

// Height k of a scan, shared by every pixel of that height: the anchor z and the z cell coordinate
// of the PP's rest position (anchor + d0z - z0) / dz, each as a float plus the float remainder of
// its exact value.  A rounding left in a value every pixel of a height shares would move that
// whole height coherently (by up to half an ulp of the coordinate, ~5e-7 A at 8 A): invisible in
// one pixel, but it adds up over the image in the tip-parameter gradients, whose sums cancel to
// a small fraction of their terms.  With the remainders carried, the roundings left are those of
// per-pixel sums, which vary from pixel to pixel.  The first height's cell coordinate and the
// step sdz / dz come as float pairs formed in FP64 once per launch (the single scan, on the host)
// or once per work item (the batch) (fz0, fz0_lo, st, st_lo); each later height is an exact
// float-float step (FP64 is a slow pipe on this part).
struct Height {
    float az, az_lo;  // anchor z
    float fz, fz_lo;  // z cell coordinate of anchor + d0z
};

template <class G_t>
__device__ __forceinline__ Height height_first(const G_t& P) {
    Height h;
    h.az = P.z_top;
    h.az_lo = 0.f;
    h.fz = P.fz0;
    h.fz_lo = P.fz0_lo;
    return h;
}

// One height down: anchor - sdz and cell coordinate - sdz / dz, in float-float.
template <class G_t, class Q_t>
__device__ __forceinline__ void height_next(Height& h, const G_t& P, const Q_t& Q) {
    float s, e;
    two_sum(h.az, -Q.sdz, s, e);
    e = __fadd_rn(e, h.az_lo);
    h.az = __fadd_rn(s, e);
    h.az_lo = __fsub_rn(e, __fsub_rn(h.az, s));
    two_sum(h.fz, -P.st, s, e);
    e = __fadd_rn(e, __fsub_rn(h.fz_lo, P.st_lo));
    h.fz = __fadd_rn(s, e);
    h.fz_lo = __fsub_rn(e, __fsub_rn(h.fz, s));
}

// Cells of the PP at lateral position (px, py) and deflection ez below height h's rest position.
// The three axes take the in-range path together and share one range test: a branch per axis
// on every FIRE iteration's dependency chain cost more than the arithmetic (the slowest pixel
// column alone went from 650 to 494 cycles per iteration; identical cells).
template <class L>
__device__ __forceinline__ Cells locate_h(const L& P, float px, float py, const Height& h, float ez) {
    const float fx = fmaf(px, P.inv_dx, P.gx0s), fy = fmaf(py, P.inv_dy, P.gy0s);
    const float fz = h.fz + fmaf(ez, P.inv_dz, h.fz_lo);
    Cells c;
    c.x = axis_fast(fx);
    c.y = axis_fast(fy);
    c.z = axis_fast(fz);
    if (((unsigned)c.x.i0 > (unsigned)(P.map.nx - 2)) | ((unsigned)c.y.i0 > (unsigned)(P.map.ny - 2)) |
        ((unsigned)c.z.i0 > (unsigned)(P.map.nz - 2))) {
        c.x = axis_cell(fx, P.map.nx, P.periodic_xy);
        c.y = axis_cell(fy, P.map.ny, P.periodic_xy);
        c.z = axis_cell(fz, P.map.nz, 0);
    }
    return c;
}

template <class Q_t>
__device__ __forceinline__ float3 total_force_tip(const Q_t& P, float3 e, float s, float3 Fs) {
    float3 G;
    G.x = fmaf(s, P.d0x + e.x, fmaf(-P.kx, e.x, Fs.x));
    G.y = fmaf(s, P.d0y + e.y, fmaf(-P.ky, e.y, Fs.y));
    G.z = fmaf(s, P.d0z + e.z, Fs.z);
    return G;
}

// Adds the tip springs' Jacobian dF_T/dp = s I - kR R0 d d^T / |d|^3 - diag(kx, ky, 0) (Eq. F_tip,
// s = -kR (|d| - R0)/|d|, d = d0 + e) to J.
template <class Q_t>
__device__ __forceinline__ void add_spring_jacobian(const Q_t& P, float3 e, float s, float J[3][3]) {
    const float q = fmaf(2.f * P.d0x + e.x, e.x, fmaf(2.f * P.d0y + e.y, e.y, fmaf(2.f * P.d0z + e.z, e.z, P.c0)));
    const float rs = rsqrtf(P.R0sq + q);
    const float br = -P.kR * P.R0 * rs * rs * rs;
    const float d[3] = {P.d0x + e.x, P.d0y + e.y, P.d0z + e.z};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) J[a][b] += (a == b ? s : 0.f) + br * d[a] * d[b];
    J[0][0] -= P.kx;
    J[1][1] -= P.ky;
}

// x = J^{-1} b by the adjugate; false when J is singular.
__device__ __forceinline__ bool solve3(const float J[3][3], float3 b, float3& x) {
    const float c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1], c01 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    const float c02 = J[0][1] * J[1][2] - J[0][2] * J[1][1], c10 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const float c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0], c12 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    const float c20 = J[1][0] * J[2][1] - J[1][1] * J[2][0], c21 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    const float c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const float det = J[0][0] * c00 + J[0][1] * c10 + J[0][2] * c20;
    if (!(det != 0.f) || !isfinite(det)) return false;
    const float id = 1.f / det;
    x = make_float3((c00 * b.x + c01 * b.y + c02 * b.z) * id, (c10 * b.x + c11 * b.y + c12 * b.z) * id,
                    (c20 * b.x + c21 * b.y + c22 * b.z) * id);
    return true;
}

// Widens [lo, hi] to the node layers a lookup in cell c reads: the cell's two layers (trilinear), or
// the four of its stencil, clamped into the grid (tricubic).
template <bool kTricubic>
__device__ __forceinline__ void note_layers(const Cells& c, int nz, int& lo, int& hi) {
    lo = min(lo, kTricubic ? max(c.z.i0 - 1, 0) : c.z.i0);
    hi = max(hi, kTricubic ? min(c.z.i1 + 1, nz - 1) : c.z.i1);
}

// One lane's pixel column (i, j) of an 8x4 pixel tile: all heights, FIRE per
// height, outputs, and the fused df epilogue.  Each lane loops until its own
// column is done; the lanes of a warp still issue together while they are in
// the same part of the loop.  kWarpVote instead keeps the whole warp in the
// loop until its last lane is done (a vote per iteration; all 32 lanes must
// call): the single-grid scan runs 4.5 % faster without it, the persistent
// batch kernel, whose warps go on to other work items, 35 % slower.  kCoherent
// selects plain cached loads of the force field instead of the read-only
// path, for grids written earlier in the same kernel.  kTricubic takes F_S
// from the tricubic energy grid P.ffE (linear layout) instead of the
// trilinear force grid.  kPolish adds, where FIRE stopped below ftol, up to
// Q.polish Newton steps p <- p - J^{-1} G with the exact Jacobian (springs +
// interpolant), each kept only if it lowers |G| (the equilibrium the implicit
// adjoint differentiates, to the FP32 resolution of G).  kSpan: returns the lowest and highest node
// layer this lane's lookups read ((INT_MAX, INT_MIN) for a lane outside the scan, and always without
// kSpan).
template <int LAYOUT, bool kCoherent, bool kTricubic = false, bool kWarpVote = false, bool kPolish = false,
          bool kSpan = false, class G_t, class Q_t>
__device__ __forceinline__ int2 relax_pixel(const G_t& P, const Q_t& Q, int i, int j) {
    const bool valid = (i < P.snx) && (j < P.sny);
    const int npix = P.snx * P.sny;
    const int pix = j * P.snx + i;

    // rest position of the PP under this pixel's anchor, without the height
    const float bx = fmaf((float)i, P.spx, P.sx0) + Q.d0x;
    const float by = fmaf((float)j, P.spy, P.sy0) + Q.d0y;

    float3 e = make_float3(0.f, 0.f, 0.f), v = make_float3(0.f, 0.f, 0.f);
    float dt = Q.dt0, alpha = Q.alpha0;
    int npos = 0, it = 0, k = 0;
    bool active = valid;
    // Corner values of the cell holding the PP, reloaded only when the PP
    // changes cell (a converging PP rarely does after its first steps).
    float4 cv[8];
    float ec[kTricubic ? 64 : 1];  // tricubic: the cached stencil energies
    int cell_x = -1, cell_y = -1, cell_z = -1;
    int zlo = 0x7fffffff, zhi = -0x7fffffff - 1;
    Height hk = height_first(P);
    while (kWarpVote ? __any_sync(0xffffffffu, active) : active) {
        if (kWarpVote && !active) continue;
        const float s = radial_factor(Q, e);
        const Cells cl = locate_h(P, bx + e.x, by + e.y, hk, e.z);
        float3 Fs;
        if constexpr (kTricubic) {
            // the 64 stencil energies stay in registers until the PP changes cell
            if (cl.x.i0 != cell_x || cl.y.i0 != cell_y || cl.z.i0 != cell_z) {
                tricubic_load(P.ffE, P.map, cl, P.periodic_xy, ec);
                if constexpr (kSpan) note_layers<true>(cl, P.map.nz, zlo, zhi);
                cell_x = cl.x.i0;
                cell_y = cl.y.i0;
                cell_z = cl.z.i0;
            }
            Fs = tricubic_eval(ec, cl, P.inv_dx, P.inv_dy, P.inv_dz);
        } else {
            if (cl.x.i0 != cell_x || cl.y.i0 != cell_y || cl.z.i0 != cell_z) {
                load_corners<LAYOUT, kCoherent>(P.ff, P.map, cl, cv);
                if constexpr (kSpan) note_layers<false>(cl, P.map.nz, zlo, zhi);
                cell_x = cl.x.i0;
                cell_y = cl.y.i0;
                cell_z = cl.z.i0;
            }
            Fs = trilinear(cv, cl);
        }
        const float3 G = total_force_tip(Q, e, s, Fs);
        const float g2 = fmaf(G.x, G.x, fmaf(G.y, G.y, G.z * G.z));
        if (g2 < Q.ftol2 || it >= Q.max_iter) {
            // converged (or out of iterations) at height k: write, then go one height down
            // keeping the deflection e (the warm start p*(k-1) - dz z_hat)
            float sw = s;
            if constexpr (kPolish) {
                if (it < Q.max_iter) {
                    Cells cc = cl;
                    float gc2 = g2;
                    float3 Gc = G;
                    for (int n = 0; n < Q.polish; ++n) {
                        float J[3][3];
                        if constexpr (kTricubic) tricubic_jacobian(ec, cc, P.inv_dx, P.inv_dy, P.inv_dz, J);
                        else trilinear_jacobian(cv, cc, P.inv_dx, P.inv_dy, P.inv_dz, J);
                        add_spring_jacobian(Q, e, sw, J);
                        float3 dp;
                        if (!solve3(J, make_float3(-Gc.x, -Gc.y, -Gc.z), dp)) break;
                        const float3 et = make_float3(e.x + dp.x, e.y + dp.y, e.z + dp.z);
                        const float st = radial_factor(Q, et);
                        const Cells ct = locate_h(P, bx + et.x, by + et.y, hk, et.z);
                        float3 Ft;
                        if constexpr (kTricubic) {
                            if (ct.x.i0 != cell_x || ct.y.i0 != cell_y || ct.z.i0 != cell_z) {
                                tricubic_load(P.ffE, P.map, ct, P.periodic_xy, ec);
                                if constexpr (kSpan) note_layers<true>(ct, P.map.nz, zlo, zhi);
                                cell_x = ct.x.i0;
                                cell_y = ct.y.i0;
                                cell_z = ct.z.i0;
                            }
                            Ft = tricubic_eval(ec, ct, P.inv_dx, P.inv_dy, P.inv_dz);
                        } else {
                            if (ct.x.i0 != cell_x || ct.y.i0 != cell_y || ct.z.i0 != cell_z) {
                                load_corners<LAYOUT, kCoherent>(P.ff, P.map, ct, cv);
                                if constexpr (kSpan) note_layers<false>(ct, P.map.nz, zlo, zhi);
                                cell_x = ct.x.i0;
                                cell_y = ct.y.i0;
                                cell_z = ct.z.i0;
                            }
                            Ft = trilinear(cv, ct);
                        }
                        const float3 Gt = total_force_tip(Q, et, st, Ft);
                        const float gt2 = fmaf(Gt.x, Gt.x, fmaf(Gt.y, Gt.y, Gt.z * Gt.z));
                        if (!(gt2 < gc2)) break;  // no progress: FP32 resolution of G reached
                        e = et;
                        sw = st;
                        cc = ct;
                        Gc = Gt;
                        gc2 = gt2;
                    }
                }
            }
            const int o = checked(k * npix + pix, (long long)npix * P.snz, kChkScanWrite);
            P.fz[o] = -sw * (Q.d0z + e.z);  // kR (|d| - R0) d_z / |d|
            if (P.pos) {
                // anchor + (d0 + e): the rounding of the stored coordinate is then independent of
                // the pixel's neighbours, so p - anchor recomputed from it (the adjoint, the IETS
                // map) carries no error common to a whole height; (anchor + d0) + e would round
                // anchor + d0 the same way for every pixel of a height, a bias that sums coherently
                // in the tip-parameter gradients
                P.pos[3 * o] = fmaf((float)i, P.spx, P.sx0) + (Q.d0x + e.x);
                P.pos[3 * o + 1] = fmaf((float)j, P.spy, P.sy0) + (Q.d0y + e.y);
                P.pos[3 * o + 2] = hk.az + ((Q.d0z + e.z) + hk.az_lo);
            }
            if (P.iters) P.iters[o] = it;
            ++k;
            active = k < P.snz;
            height_next(hk, P, Q);
            v = make_float3(0.f, 0.f, 0.f);
            dt = Q.dt0;
            alpha = Q.alpha0;
            npos = 0;
            it = 0;
            continue;
        }
        {
            // FIRE velocity mixing, or the reset after an uphill step, as selects rather than
            // branches (lanes disagree on pw > 0 at different iterations; a branch serialised both
            // paths and added a reconvergence to every iteration's chain): the values taken are
            // those of the branching form.  v = 0 on a height's first iteration, where v2 = 0 and
            // the unused mixed velocity is NaN.
            const float pw = fmaf(G.x, v.x, fmaf(G.y, v.y, G.z * v.z));
            const bool up = (it > 0) && (pw > 0.f);
            const bool down = (it > 0) && !(pw > 0.f);
            const float v2 = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
            // alpha |v| / |G| with one reciprocal root (the floor only keeps a product that
            // underflows, after many step halvings, from giving 0 * inf)
            const float c = alpha * v2 * rsqrtf(fmaxf(v2 * g2, 1e-37f));
            const float om = 1.f - alpha;
            const float mx = fmaf(om, v.x, c * G.x), my = fmaf(om, v.y, c * G.y), mz = fmaf(om, v.z, c * G.z);
            const bool grow = up && (npos > Q.n_min);
            v.x = up ? mx : (down ? 0.f : v.x);
            v.y = up ? my : (down ? 0.f : v.y);
            v.z = up ? mz : (down ? 0.f : v.z);
            dt = grow ? fminf(dt * Q.f_inc, Q.dt_max) : (down ? dt * Q.f_dec : dt);
            alpha = grow ? alpha * Q.f_alpha : (down ? Q.alpha0 : alpha);
            npos = up ? npos + 1 : (down ? 0 : npos);
        }
        const float h = dt * Q.inv_mass;
        v.x = fmaf(h, G.x, v.x);
        v.y = fmaf(h, G.y, v.y);
        v.z = fmaf(h, G.z, v.z);
        e.x = fmaf(dt, v.x, e.x);
        e.y = fmaf(dt, v.y, e.y);
        e.z = fmaf(dt, v.z, e.z);
        ++it;
    }

    if (Q.df_m >= 0 && valid) {
        // Fused df: this thread wrote its own Fz column above (program order makes it visible).
        const int m = Q.df_m;
        for (int c = m; c < P.snz - m; ++c) {
            float acc = 0.f;
            for (int t = -m; t <= m; ++t)
                acc = fmaf(Q.coef[t + m], P.fz[checked((c + t) * npix + pix, (long long)npix * P.snz, kChkScanRead)],
                           acc);
            P.df[checked((c - m) * npix + pix, (long long)npix * (P.snz - 2 * m), kChkScanWrite)] = acc;
        }
    }
    return make_int2(zlo, zhi);
}


}  // namespace pp
