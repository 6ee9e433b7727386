// Pair-sum core of the force-field grid assembly (Sec. 5.1.1 step 1;
// Eqs. LJ and point charges; F = -grad E, Sec. 2.2), shared by K1 and the
// batched kernel K6.
//
// Atoms are staged as 64-byte records in shared memory, each per-atom
// constant stored twice so that one 16-byte broadcast load yields a ready
// packed f32x2 operand:
//   s0 = (x, y, rmin^2, kqq)   s1 = (-z, -z, a, a)
//   s2 = (-b, -b, kq, kq)      s3 = (c, c, -d, -d)
// with R = R_iPP = R_i + R_PP, e = e_iPP = sqrt(e_i e_PP), a = 12 e R^12,
// b = 12 e R^6, c = e R^12, d = 2 e R^6, kq = k_e Q q_i, kqq = k_e Qzz q_i / 2
// and rmin = core_frac R.  With u3 = (R^2 / r^2)^3 the Lennard-Jones terms
// are then polynomials in 1/r^6:
//   12 e (u3^2 - u3) = (a / r^6 - b) / r^6,   e (u3^2 - 2 u3) = (c / r^6 - d) / r^6.
// A thread accumulates ZP packed pairs of z-nodes of one grid column: per
// node and atom, with delta = r_node - r_atom,
//   F += [(a / r^6 - b) / r^8 + kq / r^3] delta,
//   E += (c / r^6 - d) / r^6 + kq / r,
// with r^2 floored at rmin^2 (shifted-force Coulomb when kCutoff), and with
// the tip quadrupole (kQuad; cut off at coul_rc when kCutoff)
//   F += kqq [(15 dz^2/r^2 - 3) delta - 6 dz z_hat] / r^5,
//   E += kqq (3 dz^2 - r^2) / r^5.
#pragma once

#include "interp.cuh"

namespace pp {

struct FFConst {
    float R_pp, eps_pp, kQ, core_frac, kQzz;
    float Lx, Ly, invLx, invLy;  // minimum-image period
    float rc2, irc2, two_irc;    // shifted-force cutoff
};

__device__ __forceinline__ FFConst ff_const(float R_pp, float eps_pp, float kQ, float core_frac, float Lx, float Ly,
                                            float coul_rc, float kQzz) {
    FFConst c;
    c.R_pp = R_pp; c.eps_pp = eps_pp; c.kQ = kQ; c.core_frac = core_frac; c.kQzz = kQzz;
    c.Lx = Lx; c.Ly = Ly;
    c.invLx = 1.f / Lx; c.invLy = 1.f / Ly;
    c.rc2 = coul_rc * coul_rc;
    c.irc2 = coul_rc > 0.f ? 1.f / c.rc2 : 0.f;
    c.two_irc = coul_rc > 0.f ? 2.f / coul_rc : 0.f;
    return c;
}

// Mixing rules and the staged record of one atom.
__device__ __forceinline__ void ff_stage_atom(const FFConst& c, float x, float y, float z, float R, float eps, float q,
                                              float4& s0, float4& s1, float4& s2, float4& s3) {
    const float Rij = R + c.R_pp;
    const float eij = sqrtf(eps * c.eps_pp);
    const float rmin = c.core_frac * Rij;
    const float R2 = Rij * Rij;
    const float R6 = R2 * R2 * R2;
    const float R12 = R6 * R6;
    const float kq = c.kQ * q;
    const float kqq = c.kQzz * q;
    s0 = make_float4(x, y, rmin * rmin, kqq);
    s1 = make_float4(-z, -z, 12.f * eij * R12, 12.f * eij * R12);
    s2 = make_float4(-12.f * eij * R6, -12.f * eij * R6, kq, kq);
    s3 = make_float4(eij * R12, eij * R12, -2.f * eij * R6, -2.f * eij * R6);
}

// kSplit: the point-charge terms go to (fxe, fye, fze, ene) instead (staged with kq = k_e q_i, i.e.
// per unit probe charge), the LJ and quadrupole terms stay in (fx, fy, fz, en).
// kFloorVote (all 32 lanes of the warp call): r^2 = rxy^2 + rz^2 >= rxy^2, so where every lane's
// column passes the atom laterally at or beyond the core radius the floor max(r^2, floor^2) is r^2
// for all its nodes; the warp votes once per atom and then skips the two scalar max per node pair
// (the same bits; the floor binds only for columns within the core radius of an atom, a few % of
// the warp-atom pairs).  Likewise with kCutoff: where every lane's column passes the atom at or
// beyond coul_rc, every node's r^2 >= rc^2 and the cut terms are the zeros the in-range tests would
// select (the same expressions with those tests known false: the same bits), so the point-charge
// (and quadrupole) arithmetic drops out; on a laterally periodic slab most atoms are that far.
template <int ZP, bool kMinImage, bool kCutoff, bool kQuad, bool kSplit, bool kFloorVote = false>
__device__ __forceinline__ void ff_accumulate_impl(const float4* s0, const float4* s1, const float4* s2,
                                                   const float4* s3, int cnt, const FFConst& c, float gx, float gy,
                                                   const float2 (&gz)[ZP], float2 (&fx)[ZP], float2 (&fy)[ZP],
                                                   float2 (&fz)[ZP], float2 (&en)[ZP], float2 (&fxe)[ZP],
                                                   float2 (&fye)[ZP], float2 (&fze)[ZP], float2 (&ene)[ZP]) {
    const float2 minus3 = make_float2(-3.f, -3.f), minus6 = make_float2(-6.f, -6.f);
    const float2 three = make_float2(3.f, 3.f), fifteen = make_float2(15.f, 15.f);
#pragma unroll 1
    for (int a = 0; a < cnt; ++a) {
        const float4 A0 = s0[a], A1 = s1[a], A2 = s2[a], A3 = s3[a];
        float rx = gx - A0.x;
        float ry = gy - A0.y;
        if (kMinImage) {
            rx = fmaf(-c.Lx, rintf(rx * c.invLx), rx);
            ry = fmaf(-c.Ly, rintf(ry * c.invLy), ry);
        }
        const float rxy2 = fmaf(rx, rx, ry * ry);
        const float2 RX = make_float2(rx, rx), RY = make_float2(ry, ry), RXY = make_float2(rxy2, rxy2);
        const float2 NZ = make_float2(A1.x, A1.y), LA = make_float2(A1.z, A1.w);
        const float2 LB = make_float2(A2.x, A2.y), KQ = make_float2(A2.z, A2.w);
        const float2 EC = make_float2(A3.x, A3.y), ED = make_float2(A3.z, A3.w);
        const float2 KQQ = make_float2(A0.w, A0.w);
        auto body = [&](auto floor_t, auto far_t) {
            constexpr bool kFloor = decltype(floor_t)::value;
            constexpr bool kFar = decltype(far_t)::value;  // every node of every lane beyond coul_rc
            auto in_rc = [&](float r2v) { return !kFar && r2v < c.rc2; };
#pragma unroll
            for (int t = 0; t < ZP; ++t) {
                const float2 rz = f2add(gz[t], NZ);
                float2 r2 = f2fma(rz, rz, RXY);
                if (kFloor) {
                    r2.x = fmaxf(r2.x, A0.z);
                    r2.y = fmaxf(r2.y, A0.z);
                }
                const float2 rs = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                const float2 ir2 = f2mul(rs, rs);
                const float2 ir4 = f2mul(ir2, ir2);
                const float2 ir6 = f2mul(ir4, ir2);
                const float2 lj = f2mul(f2fma(LA, ir6, LB), ir6);  // 12 e (u6 - u3)
                float2 eel;  // kq / r (cut and shifted when kCutoff); formed when needed
                float2 f;    // radial factor of every term (of the LJ and quadrupole terms when kSplit)
                float2 fe;   // kSplit: radial factor of the point-charge term
                if (kCutoff) {
                    eel = f2mul(KQ, rs);
                    eel.x = in_rc(r2.x) ? eel.x : 0.f;
                    eel.y = in_rc(r2.y) ? eel.y : 0.f;
                    if (kSplit) {
                        fe = f2fma(eel, make_float2(-c.irc2, -c.irc2), f2mul(eel, ir2));  // kq (1/r^3 - 1/(r rc^2))
                        f = f2mul(lj, ir2);
                    } else {
                        // kq (1/r^3 - 1/(r rc^2)) + 12 e (u6 - u3) / r^2
                        f = f2fma(eel, make_float2(-c.irc2, -c.irc2), f2mul(f2add(lj, eel), ir2));
                    }
                    // shifted-force energy kq (1/r + r/rc^2 - 2/rc)
                    float2 ee = f2fma(eel, f2mul(r2, make_float2(c.irc2, c.irc2)), eel);
                    ee.x -= in_rc(r2.x) ? KQ.x * c.two_irc : 0.f;
                    ee.y -= in_rc(r2.y) ? KQ.y * c.two_irc : 0.f;
                    eel = ee;
                } else if (kSplit) {
                    eel = f2mul(KQ, rs);
                    fe = f2mul(eel, ir2);
                    f = f2mul(lj, ir2);
                } else {
                    eel = f2mul(KQ, rs);                // formed only for the quadrupole's energy sum
                    f = f2mul(f2fma(KQ, rs, lj), ir2);  // (12 e (u6 - u3) + kq / r) / r^2
                }
                float2 fzf = f;
                float2 eq = make_float2(0.f, 0.f);  // quadrupole energy
                if (kQuad) {
                    float2 c5 = f2mul(KQQ, f2mul(ir4, rs));  // kqq / r^5
                    if (kCutoff) {
                        c5.x = in_rc(r2.x) ? c5.x : 0.f;
                        c5.y = in_rc(r2.y) ? c5.y : 0.f;
                    }
                    const float2 rz2 = f2mul(rz, rz);
                    f = f2fma(c5, f2fma(f2mul(rz2, ir2), fifteen, minus3), f);  // + kqq (15 dz^2/r^2 - 3) / r^5
                    fzf = f2fma(c5, minus6, f);                                 // axial -6 kqq dz / r^5
                    // + kqq (3 dz^2 - r^2) / r^5
                    if (kSplit) eq = f2mul(c5, f2sub(f2mul(rz2, three), r2));
                    else eel = f2fma(c5, f2sub(f2mul(rz2, three), r2), eel);
                }
                fx[t] = f2fma(f, RX, fx[t]);
                fy[t] = f2fma(f, RY, fy[t]);
                fz[t] = f2fma(fzf, rz, fz[t]);
                if (kSplit) {
                    en[t] = f2add(f2fma(f2fma(EC, ir6, ED), ir6, en[t]), eq);  // e (u6 - 2 u3) + E_quad
                    fxe[t] = f2fma(fe, RX, fxe[t]);
                    fye[t] = f2fma(fe, RY, fye[t]);
                    fze[t] = f2fma(fe, rz, fze[t]);
                    ene[t] = f2add(ene[t], eel);
                } else if (kCutoff || kQuad) {
                    en[t] = f2add(f2fma(f2fma(EC, ir6, ED), ir6, en[t]), eel);  // e (u6 - 2 u3) + E_el (+ E_quad)
                } else {
                    en[t] = f2fma(KQ, rs, f2fma(f2fma(EC, ir6, ED), ir6, en[t]));  // e (u6 - 2 u3) + kq / r
                }
            }
        };
        const bool clear = kFloorVote && __all_sync(0xffffffffu, rxy2 >= A0.z);
        const bool far = kFloorVote && kCutoff && __all_sync(0xffffffffu, rxy2 >= c.rc2);
        if (clear) {
            if (far) body(std::false_type{}, std::true_type{});
            else body(std::false_type{}, std::false_type{});
        } else {
            if (far) body(std::true_type{}, std::true_type{});
            else body(std::true_type{}, std::false_type{});
        }
    }
}

template <int ZP, bool kMinImage, bool kCutoff, bool kQuad, bool kFloorVote = false>
__device__ __forceinline__ void ff_accumulate(const float4* s0, const float4* s1, const float4* s2, const float4* s3,
                                              int cnt, const FFConst& c, float gx, float gy, const float2 (&gz)[ZP],
                                              float2 (&fx)[ZP], float2 (&fy)[ZP], float2 (&fz)[ZP], float2 (&en)[ZP]) {
    ff_accumulate_impl<ZP, kMinImage, kCutoff, kQuad, false, kFloorVote>(s0, s1, s2, s3, cnt, c, gx, gy, gz, fx, fy,
                                                                         fz, en, fx, fy, fz, en);
}

}  // namespace pp
