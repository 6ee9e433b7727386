// Device helpers shared by the relaxation (K2) and its adjoint (K4): packed
// FP32 pairs, grid-cell location, corner loads and the trilinear force
// interpolant (Sec. 5.1.1 step 2) with its exact Jacobian.
#pragma once

#include "pp_internal.cuh"

namespace pp {

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
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float t) {
    return f2fma(make_float2(t, t), f2sub(b, a), a);
}
__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// s + e = a + b exactly (Knuth's two-sum; the _rn intrinsics keep each step a single rounding that
// no multiply-add contraction may merge).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct Cell {
    int i0, i1;
    float t;     // fraction in [0, 1]
    float dtdf;  // d t / d f: 1 inside, 0 where the fraction is clamped
};

// The in-range part of axis_cell alone (the caller checks the range).
__device__ __forceinline__ Cell axis_fast(float f) {
    Cell c;
    const float mg = __fadd_rd(f, 12582912.f);
    c.i0 = __float_as_int(mg) - 0x4B400000;
    c.i1 = c.i0 + 1;
    c.t = __fsub_rn(f, __fsub_rn(mg, 12582912.f));
    c.dtdf = 1.f;
    return c;
}

// Cell along one axis from the scaled coordinate f = (p - o) / h.  In-range
// cells (0 <= i <= n-2, the usual case) take a few instructions; the rest
// wrap (periodic) or clamp (index in [0, n-2], fraction in [0, 1]).  The fast
// path floors by adding 1.5 * 2^23 rounded down: for |f| < 2^22 the sum is
// 1.5 * 2^23 + floor(f) exactly, so its bits less those of 1.5 * 2^23 are
// floor(f) and the sum less 1.5 * 2^23 is floor(f) as a float (two adds and an
// integer subtract on the ALU pipes instead of two conversions on the
// long-latency ones, on every FIRE iteration's dependency chain).  Anything
// outside [0, n-2] (negative, huge, NaN) takes the slow path, which floors
// again with the saturating conversion, so any input ends up in range.
__device__ __forceinline__ Cell axis_cell(float f, int n, int periodic) {
    Cell c = axis_fast(f);
    if ((unsigned)c.i0 > (unsigned)(n - 2)) {
        c.i0 = __float2int_rd(f);  // floor, saturating (NaN -> 0)
        if (periodic) {
            const float nf = (float)n;
            float g = fminf(fmaxf(f, -1.0e7f), 1.0e7f);
            g = fmaf(-nf, floorf(g / nf), g);  // [0, n] up to rounding
            c.i0 = min(max(__float2int_rd(g), 0), n - 1);
            c.i1 = (c.i0 + 1 == n) ? 0 : c.i0 + 1;
            c.t = fminf(fmaxf(g - (float)c.i0, 0.f), 1.f);
        } else {
            const int i = min(max(c.i0, 0), n - 2);
            const float t = f - (float)i;
            c.dtdf = (t > 0.f && t < 1.f) ? 1.f : 0.f;
            c.t = fminf(fmaxf(t, 0.f), 1.f);
            c.i0 = i;
            c.i1 = i + 1;
        }
    }
    return c;
}

struct Cells {
    Cell x, y, z;
};


// Cells of the point (px, py, pz): the three in-range paths, then one range test for all axes
// (a branch per axis costs more than the arithmetic on a dependency chain).
template <class L>
__device__ __forceinline__ Cells locate(const L& P, float px, float py, float pz) {
    const float fx = fmaf(px, P.inv_dx, P.gx0s), fy = fmaf(py, P.inv_dy, P.gy0s), fz = fmaf(pz, P.inv_dz, P.gz0s);
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

template <int LAYOUT>
__device__ __forceinline__ int off_x(const GridMap& m, int i) { return LAYOUT == 0 ? i : axis_off(m.ax, i); }
template <int LAYOUT>
__device__ __forceinline__ int off_y(const GridMap& m, int j) { return LAYOUT == 0 ? j * m.ay.mul : axis_off(m.ay, j); }
template <int LAYOUT>
__device__ __forceinline__ int off_z(const GridMap& m, int k) { return LAYOUT == 0 ? k * m.az.mul : axis_off(m.az, k); }

// Storage indices of the 8 corners, ordered c[(dz*2 + dy)*2 + dx].
template <int LAYOUT>
__device__ __forceinline__ void corner_index(const GridMap& m, const Cells& c, int idx[8]) {
    const int x0 = off_x<LAYOUT>(m, c.x.i0), x1 = off_x<LAYOUT>(m, c.x.i1);
    const int y0 = off_y<LAYOUT>(m, c.y.i0), y1 = off_y<LAYOUT>(m, c.y.i1);
    const int z0 = off_z<LAYOUT>(m, c.z.i0), z1 = off_z<LAYOUT>(m, c.z.i1);
    const int r00 = y0 + z0, r10 = y1 + z0, r01 = y0 + z1, r11 = y1 + z1;
    idx[0] = r00 + x0; idx[1] = r00 + x1; idx[2] = r10 + x0; idx[3] = r10 + x1;
    idx[4] = r01 + x0; idx[5] = r01 + x1; idx[6] = r11 + x0; idx[7] = r11 + x1;
}

// kCoherent = false: read-only path (grids not written during the kernel);
// true: plain L1-cached loads, for grids another warp wrote in this kernel.
template <int LAYOUT, bool kCoherent = false>
__device__ __forceinline__ void load_corners(const float4* __restrict__ ff, const GridMap& m, const Cells& c,
                                             float4 v[8]) {
    int idx[8];
    corner_index<LAYOUT>(m, c, idx);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int i = checked(idx[q], m.stored_nodes, kChkGridRead);
        v[q] = kCoherent ? __ldca(ff + i) : __ldg(ff + i);
    }
}

// Trilinear interpolant of (Fx, Fy, Fz); (Fx, Fy) as packed pairs.
__device__ __forceinline__ float3 trilinear(const float4 v[8], const Cells& c) {
    const float tx = c.x.t, ty = c.y.t, tz = c.z.t;
    const float2 a00 = lerp2(make_float2(v[0].x, v[0].y), make_float2(v[1].x, v[1].y), tx);
    const float2 a10 = lerp2(make_float2(v[2].x, v[2].y), make_float2(v[3].x, v[3].y), tx);
    const float2 a01 = lerp2(make_float2(v[4].x, v[4].y), make_float2(v[5].x, v[5].y), tx);
    const float2 a11 = lerp2(make_float2(v[6].x, v[6].y), make_float2(v[7].x, v[7].y), tx);
    const float2 fxy = lerp2(lerp2(a00, a10, ty), lerp2(a01, a11, ty), tz);
    const float fz = lerpf(lerpf(lerpf(v[0].z, v[1].z, tx), lerpf(v[2].z, v[3].z, tx), ty),
                           lerpf(lerpf(v[4].z, v[5].z, tx), lerpf(v[6].z, v[7].z, tx), ty), tz);
    return make_float3(fxy.x, fxy.y, fz);
}

template <int LAYOUT, class L>
__device__ __forceinline__ float3 sample_force(const L& P, float px, float py, float pz) {
    const Cells c = locate(P, px, py, pz);
    float4 v[8];
    load_corners<LAYOUT>(P.ff, P.map, c, v);
    return trilinear(v, c);
}

// ---- tricubic interpolation of the node energies (grids with interp = 1)

// Cubic convolution (Catmull-Rom) weights of nodes i-1..i+2 at fraction t and
// their derivatives in t:
//   w = ((-t^3+2t^2-t), (3t^3-5t^2+2), (-3t^3+4t^2+t), (t^3-t^2)) / 2.
__device__ __forceinline__ void cr_weights(float t, float w[4], float dw[4]) {
    const float t2 = t * t, tm = t - 1.f;
    w[0] = -0.5f * t * tm * tm;
    w[1] = fmaf(t2, fmaf(1.5f, t, -2.5f), 1.f);
    w[2] = t * fmaf(t, fmaf(-1.5f, t, 2.f), 0.5f);
    w[3] = 0.5f * t2 * tm;
    dw[0] = fmaf(t, fmaf(-1.5f, t, 2.f), -0.5f);
    dw[1] = t * fmaf(4.5f, t, -5.f);
    dw[2] = fmaf(t, fmaf(-4.5f, t, 4.f), 0.5f);
    dw[3] = t * fmaf(1.5f, t, -1.f);
}

// Offsets of the 4 stencil nodes i0-1, i0, i1, i1+1 along one axis: they
// wrap like the cell on a periodic axis and clamp into [0, n-1] otherwise.
__device__ __forceinline__ void stencil4(const Cell& c, int n, bool periodic, int mul, int off[4]) {
    int im = c.i0 - 1, ip = c.i1 + 1;
    if (periodic) {
        im = c.i0 == 0 ? n - 1 : im;
        ip = c.i1 == n - 1 ? 0 : ip;
    } else {
        im = max(im, 0);
        ip = min(ip, n - 1);
    }
    off[0] = im * mul;
    off[1] = c.i0 * mul;
    off[2] = c.i1 * mul;
    off[3] = ip * mul;
}

// The 64 stencil energies of the located cell, ec[(cz*4 + b)*4 + a] for
// nodes (i0-1+a, j0-1+b, k0-1+cz) with the wrap/clamp of stencil4.
__device__ __forceinline__ void tricubic_load(const float* __restrict__ E, const GridMap& m, const Cells& c,
                                              int periodic, float ec[64]) {
    int xo[4], yo[4], zo[4];
    stencil4(c.x, m.nx, periodic != 0, 1, xo);
    stencil4(c.y, m.ny, periodic != 0, m.ay.mul, yo);
    stencil4(c.z, m.nz, false, m.az.mul, zo);
#pragma unroll
    for (int cz = 0; cz < 4; ++cz)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a)
                ec[(cz * 4 + b) * 4 + a] = __ldg(E + checked(zo[cz] + yo[b] + xo[a], m.stored_nodes, kChkGridRead));
}

// Second derivatives in t of the cubic convolution weights.
__device__ __forceinline__ void cr_weights2(float t, float d2w[4]) {
    d2w[0] = fmaf(-3.f, t, 2.f);   // (-6t + 4)/2
    d2w[1] = fmaf(9.f, t, -5.f);   // (18t - 10)/2
    d2w[2] = fmaf(-9.f, t, 4.f);   // (-18t + 8)/2
    d2w[3] = fmaf(3.f, t, -1.f);   // (6t - 2)/2
}

// Exact Jacobian J[a][b] = dF_a/dp_b = -d2E/dp_a dp_b of the tricubic interpolant from the
// stencil energies (symmetric; zero rows/columns along axes whose fraction is clamped).
__device__ __forceinline__ void tricubic_jacobian(const float ec[64], const Cells& c, float inv_dx, float inv_dy,
                                                  float inv_dz, float J[3][3]) {
    float wx[4], dwx[4], ddx[4], wy[4], dwy[4], ddy[4], wz[4], dwz[4], ddz[4];
    cr_weights(c.x.t, wx, dwx);
    cr_weights(c.y.t, wy, dwy);
    cr_weights(c.z.t, wz, dwz);
    cr_weights2(c.x.t, ddx);
    cr_weights2(c.y.t, ddy);
    cr_weights2(c.z.t, ddz);
    // H_ab from row sums R0 = sum wx e, R1 = sum dwx e, R2 = sum ddx e, then along y and z
    float hxx = 0.f, hyy = 0.f, hzz = 0.f, hxy = 0.f, hxz = 0.f, hyz = 0.f;
#pragma unroll
    for (int cz = 0; cz < 4; ++cz) {
        float s00 = 0.f, s01 = 0.f, s02 = 0.f, s10 = 0.f, s11 = 0.f, s20 = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float* e = ec + (cz * 4 + b) * 4;
            float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                r0 = fmaf(wx[a], e[a], r0);
                r1 = fmaf(dwx[a], e[a], r1);
                r2 = fmaf(ddx[a], e[a], r2);
            }
            s00 = fmaf(wy[b], r0, s00);
            s01 = fmaf(dwy[b], r0, s01);
            s02 = fmaf(ddy[b], r0, s02);
            s10 = fmaf(wy[b], r1, s10);
            s11 = fmaf(dwy[b], r1, s11);
            s20 = fmaf(wy[b], r2, s20);
        }
        hxx = fmaf(wz[cz], s20, hxx);
        hyy = fmaf(wz[cz], s02, hyy);
        hzz = fmaf(ddz[cz], s00, hzz);
        hxy = fmaf(wz[cz], s11, hxy);
        hxz = fmaf(dwz[cz], s10, hxz);
        hyz = fmaf(dwz[cz], s01, hyz);
    }
    const float sx = c.x.dtdf * inv_dx, sy = c.y.dtdf * inv_dy, sz = c.z.dtdf * inv_dz;
    J[0][0] = -hxx * sx * sx; J[1][1] = -hyy * sy * sy; J[2][2] = -hzz * sz * sz;
    J[0][1] = J[1][0] = -hxy * sx * sy;
    J[0][2] = J[2][0] = -hxz * sx * sz;
    J[1][2] = J[2][1] = -hyz * sy * sz;
}

// F = -grad E of the tricubic interpolant from the cached stencil energies: the 64 values are
// contracted along x into (value, x-derivative) pairs, then along y and z, two sums per packed
// instruction.  Where a fraction is clamped (outside the grid in z, or x,y without periodicity)
// that derivative is zero, as for trilinear.
__device__ __forceinline__ float3 tricubic_eval(const float ec[64], const Cells& c, float inv_dx, float inv_dy,
                                                float inv_dz) {
    float wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
    cr_weights(c.x.t, wx, dwx);
    cr_weights(c.y.t, wy, dwy);
    cr_weights(c.z.t, wz, dwz);
    float2 WX[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) WX[a] = make_float2(wx[a], dwx[a]);
    float2 gzx = make_float2(0.f, 0.f);
    float gy = 0.f;
#pragma unroll
    for (int cz = 0; cz < 4; ++cz) {
        float2 s02 = make_float2(0.f, 0.f);
        float s1 = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float* e = ec + (cz * 4 + b) * 4;
            float2 r = f2mul(WX[0], make_float2(e[0], e[0]));
            r = f2fma(WX[1], make_float2(e[1], e[1]), r);
            r = f2fma(WX[2], make_float2(e[2], e[2]), r);
            r = f2fma(WX[3], make_float2(e[3], e[3]), r);
            s02 = f2fma(make_float2(wy[b], wy[b]), r, s02);
            s1 = fmaf(dwy[b], r.x, s1);
        }
        gzx = f2fma(make_float2(dwz[cz], wz[cz]), s02, gzx);
        gy = fmaf(wz[cz], s1, gy);
    }
    return make_float3(-gzx.y * (c.x.dtdf * inv_dx), -gy * (c.y.dtdf * inv_dy), -gzx.x * (c.z.dtdf * inv_dz));
}

// Trilinear weights of the 8 corners (same order as corner_index).
__device__ __forceinline__ void corner_weights(const Cells& c, float w[8]) {
    const float wx[2] = {1.f - c.x.t, c.x.t}, wy[2] = {1.f - c.y.t, c.y.t}, wz[2] = {1.f - c.z.t, c.z.t};
#pragma unroll
    for (int q = 0; q < 8; ++q) w[q] = wz[q >> 2] * wy[(q >> 1) & 1] * wx[q & 1];
}

// Exact Jacobian J[a][b] = dF_a / dp_b of the trilinear interpolant: the
// x-derivative is the (y,z)-bilinear blend of the x-differences times dt/dx,
// and likewise for y and z.
__device__ __forceinline__ void trilinear_jacobian(const float4 v[8], const Cells& c, float inv_dx, float inv_dy,
                                                   float inv_dz, float J[3][3]) {
    const float wx[2] = {1.f - c.x.t, c.x.t}, wy[2] = {1.f - c.y.t, c.y.t}, wz[2] = {1.f - c.z.t, c.z.t};
    const float sx = c.x.dtdf * inv_dx, sy = c.y.dtdf * inv_dy, sz = c.z.dtdf * inv_dz;
    float3 gx = make_float3(0.f, 0.f, 0.f), gy = gx, gz = gx;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int cz = 0; cz < 2; ++cz) {
            const float4 hi = v[(cz * 2 + b) * 2 + 1], lo = v[(cz * 2 + b) * 2];
            const float w = wy[b] * wz[cz];
            gx.x = fmaf(w, hi.x - lo.x, gx.x);
            gx.y = fmaf(w, hi.y - lo.y, gx.y);
            gx.z = fmaf(w, hi.z - lo.z, gx.z);
        }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int cz = 0; cz < 2; ++cz) {
            const float4 hi = v[(cz * 2 + 1) * 2 + a], lo = v[(cz * 2) * 2 + a];
            const float w = wx[a] * wz[cz];
            gy.x = fmaf(w, hi.x - lo.x, gy.x);
            gy.y = fmaf(w, hi.y - lo.y, gy.y);
            gy.z = fmaf(w, hi.z - lo.z, gy.z);
        }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const float4 hi = v[(2 + b) * 2 + a], lo = v[b * 2 + a];
            const float w = wx[a] * wy[b];
            gz.x = fmaf(w, hi.x - lo.x, gz.x);
            gz.y = fmaf(w, hi.y - lo.y, gz.y);
            gz.z = fmaf(w, hi.z - lo.z, gz.z);
        }
    J[0][0] = gx.x * sx; J[0][1] = gy.x * sy; J[0][2] = gz.x * sz;
    J[1][0] = gx.y * sx; J[1][1] = gy.y * sy; J[1][2] = gz.y * sz;
    J[2][0] = gx.z * sx; J[2][1] = gy.z * sy; J[2][2] = gz.z * sz;
}

}  // namespace pp
