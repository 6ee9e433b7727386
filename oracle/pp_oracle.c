/*
 * FP64 CPU oracle of the Probe-Particle Model hot path (LJ + point charges).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and the two share
 * no code, header, table or constant.
 *
 * Everything here is the plain definition of the discrete model, written as
 * loops in double precision:
 *   - force-field grid by direct pair sum over all sample atoms (Sec. 5.1.1,
 *     step 1), pair terms from Eq. (LJ) with the mixing rules R_iPP = R_i+R_PP,
 *     e_iPP = sqrt(e_i e_PP) and Eq. (point-charge electrostatics), F = -grad E
 *     (Sec. 2.2);
 *   - trilinear interpolation of the force grid (Sec. 5.1.1, step 2);
 *   - tip springs of Eq. (F_tip), total PP force of Eq. (F_PP), FIRE
 *     relaxation (Sec. 5.1.1, step 2; Bitzek et al. 2006), warm-started from
 *     the previous height, followed by a Newton polish with the exact 3x3
 *     Jacobian to |G| < 1e-11 eV/A;
 *   - tip force Fz = -F^T_{R,z} at the relaxed PP (Sec. 2.1);
 *   - frequency shift of Eq. (df) by product integration of a piecewise
 *     linear Fz against the kernel u / sqrt(a^2 - u^2), a = A/2;
 *   - the implicit-function adjoint of all of the above (the paper has no
 *     gradients; this is the derivative of the same discrete model);
 *   - optionally tricubic interpolation of the grid potential instead of
 *     trilinear interpolation of the grid forces (Sec. 5.1.1 step 2: the
 *     paper's suggestion for larger spacings with no stored forces);
 *   - the cross-correlation force fields of the Hartree-potential and
 *     full-density models (Eqs. El_conv and Pauli_FDBM) on periodic grids,
 *     by direct summation, with the spectral derivative for F;
 *   - optionally an axial point quadrupole on the probe (Secs. 2.2.3, 2.2.5: the CO
 *     tip's quadrupolar charge distribution) in the field of the sample's
 *     point charges.
 *
 * Readings of the paper that the code fixes (all units: A, eV, e):
 *   d0 = (d0x, d0y, -sqrt(R0^2 - d0x^2 - d0y^2)): the PP hangs below the tip;
 *   per-pair r^2 floor (core_frac * R_iPP)^2, displacement left unscaled;
 *   grid nodes x_i = x0 + i*dx, periodic in x,y when periodic_xy, clamped in z
 *   (cell index in [0, nz-2], fraction in [0,1]);
 *   spring constants are given in N/m and converted with 1 eV/A^2 = 16.02176634
 *   N/m; Coulomb constant 14.3996454784 eV*A/e^2;
 *   tricubic = tensor product of 1D cubic convolution (Catmull-Rom) through
 *   the node energies: weights of nodes i-1..i+2 at fraction t are
 *   ((-t^3+2t^2-t), (3t^3-5t^2+2), (-3t^3+4t^2+t), (t^3-t^2)) / 2, i.e. the
 *   cubic Hermite curve with central-difference slopes; F = -grad E_interp is
 *   continuous across cell faces.  Periodic in x,y; in z the cell index and
 *   fraction clamp as for trilinear and stencil nodes clamp into [0, nz-1];
 *   the tip quadrupole Qzz (e*A^2) is the second moment sum_k q_k z_k^2 of an
 *   axial charge distribution with no net charge or dipole, rigidly attached
 *   to the PP (no rotation, Sec. 2.2.3); its energy in the sample potential
 *   V(r) = k_e sum_i q_i / |r - r_i| is (Qzz/2) d^2V/dz^2, per atom
 *   E = (k_e q_i Qzz / 2) (3 dz^2 - r^2) / r^5; with coul_rc > 0 the term is
 *   cut off (not shifted) at r >= coul_rc; inside the core floor r is
 *   replaced by the floor radius, as for the other pair terms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_KE 14.3996454784          /* Coulomb constant, eV*A/e^2 */
#define OR_EVA2_TO_NM 16.02176634    /* 1 eV/A^2 in N/m (SI: 1 eV = 1.602176634e-19 J) */
#define OR_NM_TO_EVA2 (1.0 / OR_EVA2_TO_NM) /* 1 N/m in eV/A^2 */
#define OR_PI 3.14159265358979323846

typedef struct { int n; const double *x, *y, *z, *R, *eps, *q; } or_atoms;
typedef struct { double R_pp, eps_pp, Q, coul_rc; int min_image; double core_frac; double Qzz; } or_probe;
/* Lx, Ly: minimum-image period; 0 means the grid's own extent nx*dx, ny*dy
 * (a window of a larger periodic grid passes the full grid's extent).
 * interp: 0 trilinear interpolation of the node forces, 1 tricubic
 * interpolation of the node energies with F = -grad of the interpolant. */
typedef struct {
    int nx, ny, nz; double x0, y0, z0, dx, dy, dz; int periodic_xy; double Lx, Ly; int interp;
} or_grid;
typedef struct { double kx, ky, kR, R0, d0x, d0y; } or_tip; /* springs in N/m */
typedef struct { int nx, ny, nz; double x0, y0, px, py, z_top, dz; } or_scan;
typedef struct {
    int max_iter; double ftol, dt0, dt_max, f_inc, f_dec, alpha0, f_alpha, mass; int n_min;
} or_fire;
typedef struct { double A_pp, k, f0; } or_df; /* A (peak-to-peak), N/m, Hz */

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ pairs */

/* One sample atom seen from point r.  The pair force is S * delta. */
typedef struct {
    double d[3];        /* delta = r - r_i (minimum image when enabled) */
    double r;           /* distance after the core floor */
    int clamped;        /* the floor replaced |delta| */
    double S, E;        /* force factor and energy */
    double dSdr;        /* dS/dr at fixed R_iPP */
    double dSdR;        /* total dS/dR_iPP, including the floor's R-dependence */
    double S_lj_e;      /* LJ part of S per unit e_iPP */
    double S_el_qq;     /* Coulomb part of S per unit k_e Q q_i */
    double e_ij;        /* e_iPP */
    /* tip quadrupole, per unit k_e q_i Qzz / 2 (zero when Qzz = 0 or beyond coul_rc) */
    double Phi[3];      /* force */
    double eq;          /* energy */
    double dPhi[9];     /* dPhi_a / d delta_b, the floored r held fixed when clamped */
    double dPhi_dr[3];  /* dPhi_a / dr at fixed delta */
    /* energy derivatives (adjoint of an energy grid): LJ + Coulomb part, then the quadrupole's
     * per unit k_e q_i Qzz / 2; inside the floor r is the floor radius, constant in delta */
    double E_lj_e;      /* LJ energy per unit e_iPP */
    double E_el_qq;     /* Coulomb energy per unit k_e Q q_i */
    double dE_dd[3];    /* dE / d delta */
    double dE_dR;       /* dE / dR_iPP */
    double deq_dd[3];   /* d eq / d delta */
    double deq_dr;      /* d eq / dr at fixed delta */
} or_pair;

/* Quadrupole pair term as a function of delta and r (r = |delta| unless floored):
 *   e = 3 dz^2 / r^5 - 1 / r^3,
 *   Phi = -grad e = (15 dz^2 / r^7 - 3 / r^5) delta - (6 dz / r^5) z_hat. */
static void quad_eval(const double d[3], double r, int clamped, or_pair* o) {
    const double dz = d[2];
    const double r2 = r * r, r5 = r2 * r2 * r, r7 = r5 * r2;
    const double A = 15.0 * dz * dz / r7 - 3.0 / r5;
    o->eq = 3.0 * dz * dz / r5 - 1.0 / (r2 * r);
    for (int a = 0; a < 3; ++a) o->Phi[a] = A * d[a];
    o->Phi[2] -= 6.0 * dz / r5;
    /* partials at fixed r */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) o->dPhi[a * 3 + b] = (a == b ? A : 0.0);
    for (int a = 0; a < 3; ++a) o->dPhi[a * 3 + 2] += 30.0 * dz * d[a] / r7;
    o->dPhi[2 * 3 + 2] -= 6.0 / r5;
    /* energy: eq = 3 dz^2 / r^5 - 1 / r^3 */
    o->deq_dr = -15.0 * dz * dz / (r5 * r) + 3.0 / (r2 * r2);
    if (clamped) {
        o->deq_dd[0] = o->deq_dd[1] = 0.0;
        o->deq_dd[2] = 6.0 * dz / r5;
    } else {
        for (int a = 0; a < 3; ++a) o->deq_dd[a] = -o->Phi[a];
    }
    /* dPhi/dr at fixed delta */
    const double dA = -105.0 * dz * dz / (r7 * r) + 15.0 / (r5 * r);
    for (int a = 0; a < 3; ++a) o->dPhi_dr[a] = dA * d[a];
    o->dPhi_dr[2] += 30.0 * dz / (r5 * r);
    if (!clamped && r > 0.0)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) o->dPhi[a * 3 + b] += o->dPhi_dr[a] * d[b] / r;
}

static void pair_eval(const or_atoms* A, int i, const or_probe* P, double Lx, double Ly,
                      const double pt[3], or_pair* o) {
    double dx = pt[0] - A->x[i], dy = pt[1] - A->y[i], dz = pt[2] - A->z[i];
    if (P->min_image) {
        dx -= Lx * nearbyint(dx / Lx);
        dy -= Ly * nearbyint(dy / Ly);
    }
    o->d[0] = dx; o->d[1] = dy; o->d[2] = dz;
    const double Rij = A->R[i] + P->R_pp;              /* mixing rule, Eq. (LJ) */
    const double eij = sqrt(A->eps[i] * P->eps_pp);    /* mixing rule, Eq. (LJ) */
    const double qq = OR_KE * P->Q * A->q[i];          /* Eq. (point charges) */
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double rmin = P->core_frac * Rij;
    double r;
    if (r2 < rmin * rmin) { r = rmin; o->clamped = 1; }
    else { r = sqrt(r2); o->clamped = 0; }
    o->r = r;
    o->e_ij = eij;
    /* E_LJ = e [(R/r)^12 - 2 (R/r)^6];  F = -dE/dr rhat = 12 e [(R/r)^12 - (R/r)^6] / r^2 * delta */
    const double s6 = pow(Rij / r, 6.0);
    const double s12 = s6 * s6;
    o->S_lj_e = 12.0 * (s12 - s6) / (r * r);
    const double E_lj = eij * (s12 - 2.0 * s6);
    const double dSlj_dr = 12.0 * eij * (-14.0 * s12 + 8.0 * s6) / (r * r * r);
    const double dSlj_dR = 12.0 * eij * (12.0 * s12 - 6.0 * s6) / (Rij * r * r);
    /* E_el = qq / r (optionally shifted-force truncated at rc) */
    double c, e_el, dc_dr, de_dr;
    if (P->coul_rc > 0.0) {
        const double rc = P->coul_rc;
        if (r < rc) {
            c = 1.0 / (r * r * r) - 1.0 / (rc * rc * r);
            e_el = 1.0 / r - 1.0 / rc + (r - rc) / (rc * rc);
            dc_dr = -3.0 / (r * r * r * r) + 1.0 / (rc * rc * r * r);
            de_dr = -1.0 / (r * r) + 1.0 / (rc * rc);
        } else {
            c = 0.0; e_el = 0.0; dc_dr = 0.0; de_dr = 0.0;
        }
    } else {
        c = 1.0 / (r * r * r);
        e_el = 1.0 / r;
        dc_dr = -3.0 / (r * r * r * r);
        de_dr = -1.0 / (r * r);
    }
    o->S_el_qq = c;
    o->S = eij * o->S_lj_e + qq * c;
    o->E = E_lj + qq * e_el;
    o->E_lj_e = s12 - 2.0 * s6;
    o->E_el_qq = e_el;
    if (o->clamped) {
        /* r = core_frac R_iPP: the LJ energy is the constant e (cf^-12 - 2 cf^-6) */
        o->dE_dd[0] = o->dE_dd[1] = o->dE_dd[2] = 0.0;
        o->dE_dR = qq * de_dr * P->core_frac;
    } else {
        for (int a = 0; a < 3; ++a) o->dE_dd[a] = -o->S * o->d[a];  /* F = -grad E */
        o->dE_dR = 12.0 * eij * (s12 - s6) / Rij;
    }
    if (P->Qzz != 0.0 && !(P->coul_rc > 0.0 && r >= P->coul_rc)) {
        quad_eval(o->d, r, o->clamped, o);
    } else {
        memset(o->Phi, 0, sizeof o->Phi);
        memset(o->dPhi, 0, sizeof o->dPhi);
        memset(o->dPhi_dr, 0, sizeof o->dPhi_dr);
        memset(o->deq_dd, 0, sizeof o->deq_dd);
        o->eq = 0.0;
        o->deq_dr = 0.0;
    }
    o->dSdr = dSlj_dr + qq * dc_dr;
    o->dSdR = dSlj_dR + (o->clamped ? o->dSdr * P->core_frac : 0.0);
}

/* Sample force and energy at r by direct sum (the definition of a grid node value). */
static int sample_point(const or_atoms* A, const or_probe* P, double Lx, double Ly,
                        const double r[3], double out[4], double Js[9]) {
    double F[3] = {0, 0, 0}, E = 0.0;
    int core = 0;
    if (Js) memset(Js, 0, 9 * sizeof(double));
    for (int i = 0; i < A->n; ++i) {
        or_pair p;
        pair_eval(A, i, P, Lx, Ly, r, &p);
        const double cq = 0.5 * OR_KE * P->Qzz * A->q[i];  /* tip quadrupole, per atom */
        for (int a = 0; a < 3; ++a) F[a] += p.S * p.d[a] + cq * p.Phi[a];
        E += p.E + cq * p.eq;
        core |= p.clamped;
        if (Js) {
            for (int a = 0; a < 3; ++a) {
                Js[a * 3 + a] += p.S;
                if (!p.clamped && p.r > 0.0)
                    for (int b = 0; b < 3; ++b) Js[a * 3 + b] += p.dSdr * p.d[a] * p.d[b] / p.r;
                for (int b = 0; b < 3; ++b) Js[a * 3 + b] += cq * p.dPhi[a * 3 + b];
            }
        }
    }
    out[0] = F[0]; out[1] = F[1]; out[2] = F[2]; out[3] = E;
    return core;
}

static void grid_period(const or_grid* G, double* Lx, double* Ly) {
    *Lx = G->Lx > 0.0 ? G->Lx : G->nx * G->dx;
    *Ly = G->Ly > 0.0 ? G->Ly : G->ny * G->dy;
}

/* Force-field grid, layout [nz][ny][nx][4] = (Fx, Fy, Fz, E); core[node] = 1 where a pair hit the floor. */
int or_make_ff(const or_atoms* A, const or_probe* P, const or_grid* G, double* ff,
               unsigned char* core, int nthreads) {
    if (!A || !P || !G || !ff || G->nx < 2 || G->ny < 2 || G->nz < 2) return 1;
    set_threads(nthreads);
    double Lx, Ly;
    grid_period(G, &Lx, &Ly);
    const long nxy = (long)G->nx * G->ny;
    const long total = nxy * G->nz;
#pragma omp parallel for schedule(static)
    for (long g = 0; g < total; ++g) {
        const long k = g / nxy, rem = g % nxy, j = rem / G->nx, i = rem % G->nx;
        double r[3] = {G->x0 + i * G->dx, G->y0 + j * G->dy, G->z0 + k * G->dz};
        int c = sample_point(A, P, Lx, Ly, r, ff + 4 * g, NULL);
        if (core) core[g] = (unsigned char)c;
    }
    return 0;
}

/* Sample force/energy at arbitrary points pts[npts][3] (grid-free). */
int or_ff_points(const or_atoms* A, const or_probe* P, const or_grid* G, int npts,
                 const double* pts, double* out, unsigned char* core, int nthreads) {
    if (!A || !P || !G || npts < 0) return 1;
    set_threads(nthreads);
    double Lx, Ly;
    grid_period(G, &Lx, &Ly);
#pragma omp parallel for schedule(static)
    for (int t = 0; t < npts; ++t) {
        int c = sample_point(A, P, Lx, Ly, pts + 3 * t, out + 4 * t, NULL);
        if (core) core[t] = (unsigned char)c;
    }
    return 0;
}

/* ------------------------------------------------------------ interpolation */

static void axis_locate(double p, double o, double h, int n, int periodic,
                        long* i0, long* i1, double* t, double* dtdp) {
    const double f = (p - o) / h;
    const double fl = floor(f);
    long i = (long)fl;
    double tt = f - fl, d = 1.0 / h;
    if (periodic) {
        long m = i % n;
        if (m < 0) m += n;
        *i0 = m;
        *i1 = (m + 1) % n;
    } else {
        if (i < 0) i = 0;
        if (i > n - 2) i = n - 2;
        tt = f - (double)i;
        if (tt < 0.0) { tt = 0.0; d = 0.0; }
        else if (tt > 1.0) { tt = 1.0; d = 0.0; }
        *i0 = i;
        *i1 = i + 1;
    }
    *t = tt;
    *dtdp = d;
}

/* Trilinear interpolant of (Fx,Fy,Fz) at p and, optionally, its exact Jacobian
 * J[a*3+b] = dF_a/dp_b and the 8 corner node indices and weights. */
static void interp_tricubic(const double* ff, const or_grid* G, const double p[3], double* E, double F[3],
                            double* J);

static void interp(const double* ff, const or_grid* G, const double p[3], double F[3], double* J,
                   long node[8], double w8[8]) {
    if (G->interp == 1) {  /* energy grid: no corner list */
        interp_tricubic(ff, G, p, NULL, F, J);
        return;
    }
    long ix[2], iy[2], iz[2];
    double tx, ty, tz, gx, gy, gz;
    axis_locate(p[0], G->x0, G->dx, G->nx, G->periodic_xy, &ix[0], &ix[1], &tx, &gx);
    axis_locate(p[1], G->y0, G->dy, G->ny, G->periodic_xy, &iy[0], &iy[1], &ty, &gy);
    axis_locate(p[2], G->z0, G->dz, G->nz, 0, &iz[0], &iz[1], &tz, &gz);
    const double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty}, wz[2] = {1.0 - tz, tz};
    const double sx[2] = {-gx, gx}, sy[2] = {-gy, gy}, sz[2] = {-gz, gz};
    F[0] = F[1] = F[2] = 0.0;
    if (J) memset(J, 0, 9 * sizeof(double));
    int c = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e, ++c) {
                const long g = (iz[a] * G->ny + iy[b]) * G->nx + ix[e];
                const double* v = ff + 4 * g;
                const double w = wz[a] * wy[b] * wx[e];
                for (int m = 0; m < 3; ++m) F[m] += w * v[m];
                if (J) {
                    const double dw[3] = {wz[a] * wy[b] * sx[e], wz[a] * sy[b] * wx[e], sz[a] * wy[b] * wx[e]};
                    for (int m = 0; m < 3; ++m)
                        for (int n = 0; n < 3; ++n) J[m * 3 + n] += dw[n] * v[m];
                }
                if (node) { node[c] = g; w8[c] = w; }
            }
}

/* Stencil of 4 nodes (i-1 .. i+2) around p along one axis for the tricubic
 * interpolant, with the fraction t in the cell [i, i+1] and dt/dp (0 where
 * clamped); same cell and fraction as axis_locate. */
static void axis_stencil(double p, double o, double h, int n, int periodic, long idx[4], double* t,
                         double* dtdp) {
    long i0, i1;
    axis_locate(p, o, h, n, periodic, &i0, &i1, t, dtdp);
    for (int q = 0; q < 4; ++q) {
        long k = i0 - 1 + q;
        if (periodic) {
            k %= n;
            if (k < 0) k += n;
        } else {
            if (k < 0) k = 0;
            if (k > n - 1) k = n - 1;
        }
        idx[q] = k;
    }
}

/* Catmull-Rom (cubic convolution, a = -1/2) weights of nodes -1, 0, 1, 2 at t,
 * and their first and second derivatives in t. */
static void cr_weights(double t, double w[4], double dw[4], double d2w[4]) {
    const double t2 = t * t, t3 = t2 * t;
    w[0] = 0.5 * (-t3 + 2.0 * t2 - t);
    w[1] = 0.5 * (3.0 * t3 - 5.0 * t2 + 2.0);
    w[2] = 0.5 * (-3.0 * t3 + 4.0 * t2 + t);
    w[3] = 0.5 * (t3 - t2);
    dw[0] = 0.5 * (-3.0 * t2 + 4.0 * t - 1.0);
    dw[1] = 0.5 * (9.0 * t2 - 10.0 * t);
    dw[2] = 0.5 * (-9.0 * t2 + 8.0 * t + 1.0);
    dw[3] = 0.5 * (3.0 * t2 - 2.0 * t);
    d2w[0] = 0.5 * (-6.0 * t + 4.0);
    d2w[1] = 0.5 * (18.0 * t - 10.0);
    d2w[2] = 0.5 * (-18.0 * t + 8.0);
    d2w[3] = 0.5 * (6.0 * t - 2.0);
}

/* Tricubic interpolant of the node energies ff[g][3] at p: E, F = -grad E and,
 * optionally, J[a*3+b] = dF_a/dp_b = -d2E/dp_a dp_b. */
static void interp_tricubic(const double* ff, const or_grid* G, const double p[3], double* E, double F[3],
                            double* J) {
    long ix[4], iy[4], iz[4];
    double tx, ty, tz, sx, sy, sz;
    axis_stencil(p[0], G->x0, G->dx, G->nx, G->periodic_xy, ix, &tx, &sx);
    axis_stencil(p[1], G->y0, G->dy, G->ny, G->periodic_xy, iy, &ty, &sy);
    axis_stencil(p[2], G->z0, G->dz, G->nz, 0, iz, &tz, &sz);
    double wx[4], dwx[4], d2wx[4], wy[4], dwy[4], d2wy[4], wz[4], dwz[4], d2wz[4];
    cr_weights(tx, wx, dwx, d2wx);
    cr_weights(ty, wy, dwy, d2wy);
    cr_weights(tz, wz, dwz, d2wz);
    double e = 0.0, g[3] = {0, 0, 0}, H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a) {
                const double v = ff[4 * ((iz[c] * G->ny + iy[b]) * G->nx + ix[a]) + 3];
                e += wx[a] * wy[b] * wz[c] * v;
                g[0] += dwx[a] * wy[b] * wz[c] * v;
                g[1] += wx[a] * dwy[b] * wz[c] * v;
                g[2] += wx[a] * wy[b] * dwz[c] * v;
                if (J) {
                    H[0] += d2wx[a] * wy[b] * wz[c] * v;
                    H[4] += wx[a] * d2wy[b] * wz[c] * v;
                    H[8] += wx[a] * wy[b] * d2wz[c] * v;
                    H[1] += dwx[a] * dwy[b] * wz[c] * v;
                    H[2] += dwx[a] * wy[b] * dwz[c] * v;
                    H[5] += wx[a] * dwy[b] * dwz[c] * v;
                }
            }
    const double s[3] = {sx, sy, sz};
    if (E) *E = e;
    for (int m = 0; m < 3; ++m) F[m] = -g[m] * s[m];
    if (J) {
        H[3] = H[1];
        H[6] = H[2];
        H[7] = H[5];
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) J[m * 3 + n] = -H[m * 3 + n] * s[m] * s[n];
    }
}

int or_interp_points(const double* ff, const or_grid* G, int npts, const double* pts,
                     double* F, double* J) {
    for (int t = 0; t < npts; ++t) interp(ff, G, pts + 3 * t, F + 3 * t, J ? J + 9 * t : NULL, NULL, NULL);
    return 0;
}

/* Interpolated energy at pts: tricubic grids only (trilinear grids interpolate forces). */
int or_interp_energy_points(const double* ff, const or_grid* G, int npts, const double* pts, double* E) {
    if (G->interp != 1) return 1;
    double F[3];
    for (int t = 0; t < npts; ++t) interp_tricubic(ff, G, pts + 3 * t, E + t, F, NULL);
    return 0;
}

/* --------------------------------------------------------------- tip model */

typedef struct { double kx, ky, kR, R0, d0x, d0y, d0z; } tip_si; /* eV/A^2 */

static tip_si tip_units(const or_tip* T) {
    tip_si t;
    t.kx = T->kx * OR_NM_TO_EVA2;
    t.ky = T->ky * OR_NM_TO_EVA2;
    t.kR = T->kR * OR_NM_TO_EVA2;
    t.R0 = T->R0;
    t.d0x = T->d0x;
    t.d0y = T->d0y;
    t.d0z = -sqrt(fmax(T->R0 * T->R0 - T->d0x * T->d0x - T->d0y * T->d0y, 0.0));
    return t;
}

/* Eq. (F_tip): F^T = -k_R (|d| - R0) d/|d| - k_xy (.) (d - d0), k_xy = (kx, ky, 0). */
static void tip_force(const tip_si* t, const double d[3], double F[3], double* J) {
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double s = -t->kR * (dn - t->R0) / dn;
    F[0] = s * d[0] - t->kx * (d[0] - t->d0x);
    F[1] = s * d[1] - t->ky * (d[1] - t->d0y);
    F[2] = s * d[2];
    if (J) {
        /* dF/dd = -kR [(1 - R0/|d|) I + R0 d d^T / |d|^3] - diag(kx, ky, 0) */
        const double a = -t->kR * (1.0 - t->R0 / dn);
        const double b = -t->kR * t->R0 / (dn * dn * dn);
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) J[m * 3 + n] = (m == n ? a : 0.0) + b * d[m] * d[n];
        J[0] -= t->kx;
        J[4] -= t->ky;
    }
}

/* Tip force on the cantilever, Fz = -F^T_{R,z} = kR (|d| - R0) d_z / |d| (Sec. 2.1). */
static double tip_fz(const tip_si* t, const double d[3]) {
    const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    return t->kR * (dn - t->R0) * d[2] / dn;
}

/* ---------------------------------------------------------- PP relaxation */

typedef struct {
    const double* ff;   /* grid mode when non-NULL */
    const or_grid* G;
    const or_atoms* A;  /* direct (grid-free) mode when ff == NULL */
    const or_probe* P;
    double Lx, Ly;
    tip_si tip;
} or_model;

/* Total PP force G(p) = F^T + F^S of Eq. (F_PP) and optionally its Jacobian. */
static void total_force(const or_model* M, const double anchor[3], const double p[3],
                        double Gv[3], double* J) {
    double d[3] = {p[0] - anchor[0], p[1] - anchor[1], p[2] - anchor[2]};
    double Ft[3], Fs[3], Jt[9], Js[9];
    tip_force(&M->tip, d, Ft, J ? Jt : NULL);
    if (M->ff) {
        interp(M->ff, M->G, p, Fs, J ? Js : NULL, NULL, NULL);
    } else {
        double o[4];
        sample_point(M->A, M->P, M->Lx, M->Ly, p, o, J ? Js : NULL);
        Fs[0] = o[0]; Fs[1] = o[1]; Fs[2] = o[2];
    }
    for (int m = 0; m < 3; ++m) Gv[m] = Ft[m] + Fs[m];
    if (J)
        for (int m = 0; m < 9; ++m) J[m] = Jt[m] + Js[m];
}

static double norm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

/* FIRE (Bitzek et al. 2006) with semi-implicit Euler steps.  Each iteration:
 * evaluate G; stop if |G| < ftol; from the second iteration on, if G.v > 0 mix
 * v <- (1-alpha) v + alpha |v| G/|G| and, after more than n_min such steps in a
 * row, grow dt (capped at dt_max) and shrink alpha; if G.v <= 0 zero v, halve
 * dt and reset alpha; then v += dt G / m, p += dt v.  Returns the number of
 * position updates; *res gets the last evaluated |G|. */
static int fire_relax(const or_model* M, const or_fire* Fp, const double anchor[3], double p[3],
                      double* res) {
    double v[3] = {0, 0, 0}, Gv[3];
    double dt = Fp->dt0, alpha = Fp->alpha0;
    int npos = 0, it = 0;
    double g = 0.0;
    for (it = 0; it < Fp->max_iter; ++it) {
        total_force(M, anchor, p, Gv, NULL);
        g = norm3(Gv);
        if (g < Fp->ftol) break;
        if (it > 0) {
            const double P = Gv[0] * v[0] + Gv[1] * v[1] + Gv[2] * v[2];
            if (P > 0.0) {
                const double vn = norm3(v);
                for (int m = 0; m < 3; ++m) v[m] = (1.0 - alpha) * v[m] + alpha * vn * Gv[m] / g;
                if (npos > Fp->n_min) {
                    dt = fmin(dt * Fp->f_inc, Fp->dt_max);
                    alpha *= Fp->f_alpha;
                }
                ++npos;
            } else {
                v[0] = v[1] = v[2] = 0.0;
                dt *= Fp->f_dec;
                alpha = Fp->alpha0;
                npos = 0;
            }
        }
        for (int m = 0; m < 3; ++m) {
            v[m] += dt * Gv[m] / Fp->mass;
            p[m] += dt * v[m];
        }
    }
    if (it == Fp->max_iter) {
        total_force(M, anchor, p, Gv, NULL);
        g = norm3(Gv);
    }
    *res = g;
    return it;
}

/* Solve the 3x3 system A x = b by Gaussian elimination with partial pivoting. */
static int solve3(const double* Ain, const double* b, double* x) {
    double A[3][4];
    for (int m = 0; m < 3; ++m) {
        for (int n = 0; n < 3; ++n) A[m][n] = Ain[m * 3 + n];
        A[m][3] = b[m];
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return 1;
        if (piv != c)
            for (int n = 0; n < 4; ++n) { double t = A[c][n]; A[c][n] = A[piv][n]; A[piv][n] = t; }
        for (int r = c + 1; r < 3; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int n = c; n < 4; ++n) A[r][n] -= f * A[c][n];
        }
    }
    for (int m = 2; m >= 0; --m) {
        double s = A[m][3];
        for (int n = m + 1; n < 3; ++n) s -= A[m][n] * x[n];
        x[m] = s / A[m][m];
    }
    return 0;
}

/* Newton iterations p <- p - J^{-1} G with backtracking on |G|, to |G| < tol. */
static int newton_polish(const or_model* M, const double anchor[3], double p[3], double tol,
                         double* res) {
    double Gv[3], J[9], dp[3], q[3], Gq[3];
    for (int it = 0; it < 200; ++it) {
        total_force(M, anchor, p, Gv, J);
        const double g = norm3(Gv);
        *res = g;
        if (g < tol) return 1;
        const double rhs[3] = {-Gv[0], -Gv[1], -Gv[2]};
        if (solve3(J, rhs, dp)) return 0;
        double step = 1.0;
        int moved = 0;
        while (step > 1e-10) {
            for (int m = 0; m < 3; ++m) q[m] = p[m] + step * dp[m];
            total_force(M, anchor, q, Gq, NULL);
            if (norm3(Gq) < g) { moved = 1; break; }
            step *= 0.5;
        }
        if (!moved) return 0;
        p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
    }
    total_force(M, anchor, p, Gv, NULL);
    *res = norm3(Gv);
    return *res < tol;
}

/* Eigenvalues of a symmetric 3x3 matrix by cyclic Jacobi rotations, ascending in ev[3]. */
static void sym3_eigs(const double* S, double ev[3]) {
    double a[3][3];
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) a[m][n] = S[m * 3 + n];
    for (int sweep = 0; sweep < 50; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        if (off < 1e-30) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int P = pq == 2 ? 1 : 0, Q = pq == 0 ? 1 : 2;
            if (fabs(a[P][Q]) < 1e-300) continue;
            const double th = 0.5 * atan2(2.0 * a[P][Q], a[Q][Q] - a[P][P]);
            const double c = cos(th), s = sin(th);
            for (int k = 0; k < 3; ++k) {
                const double akp = a[k][P], akq = a[k][Q];
                a[k][P] = c * akp - s * akq;
                a[k][Q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {
                const double apk = a[P][k], aqk = a[Q][k];
                a[P][k] = c * apk - s * aqk;
                a[Q][k] = s * apk + c * aqk;
            }
        }
    }
    ev[0] = a[0][0]; ev[1] = a[1][1]; ev[2] = a[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2 - i; ++j)
            if (ev[j] > ev[j + 1]) { const double t = ev[j]; ev[j] = ev[j + 1]; ev[j + 1] = t; }
}

static double sym3_min_eig(const double* S) {
    double ev[3];
    sym3_eigs(S, ev);
    return ev[0];
}

/* Relax the listed pixel columns over all scan heights.
 *   ff == NULL selects the grid-free model (F^S by direct pair sum at p).
 *   cols[c] = j*scan.nx + i.  Outputs per column c and height k (index c*nz+k):
 *   pos[3], fz, iters (FIRE updates), res (|G| after FIRE), lam (smallest
 *   eigenvalue of the symmetrised stiffness -J at the final p), ok (Newton
 *   reached |G| < polish_tol; 1 when polishing is off).
 *   Warm start: p(0) = anchor + d0, p(k) = p(k-1) - dz z_hat.  With
 *   polish_tol > 0 the polished p(k-1) seeds height k. */
int or_relax_columns(const double* ff, const or_grid* G, const or_atoms* A, const or_probe* P,
                     const or_scan* S, const or_tip* T, const or_fire* Fp, int ncols,
                     const int* cols, double polish_tol, double* pos, double* fz, int* iters,
                     double* res, double* lam, int* ok, int nthreads) {
    if (!G || !S || !T || !Fp || !cols || ncols < 0) return 1;
    if (!ff && (!A || !P)) return 1;
    set_threads(nthreads);
    or_model M;
    M.ff = ff; M.G = G; M.A = A; M.P = P;
    grid_period(G, &M.Lx, &M.Ly);
    M.tip = tip_units(T);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < ncols; ++c) {
        const int i = cols[c] % S->nx, j = cols[c] / S->nx;
        double p[3];
        for (int k = 0; k < S->nz; ++k) {
            const double anchor[3] = {S->x0 + i * S->px, S->y0 + j * S->py, S->z_top - k * S->dz};
            if (k == 0) {
                p[0] = anchor[0] + M.tip.d0x;
                p[1] = anchor[1] + M.tip.d0y;
                p[2] = anchor[2] + M.tip.d0z;
            } else {
                p[2] -= S->dz;
            }
            double r = 0.0;
            const int it = fire_relax(&M, Fp, anchor, p, &r);
            int good = 1;
            if (polish_tol > 0.0) {
                double r2;
                good = newton_polish(&M, anchor, p, polish_tol, &r2);
            }
            double Gv[3], J[9], Ks[9];
            total_force(&M, anchor, p, Gv, J);
            for (int m = 0; m < 3; ++m)
                for (int n = 0; n < 3; ++n) Ks[m * 3 + n] = -0.5 * (J[m * 3 + n] + J[n * 3 + m]);
            const double d[3] = {p[0] - anchor[0], p[1] - anchor[1], p[2] - anchor[2]};
            const long o = (long)c * S->nz + k;
            if (pos) { pos[3 * o] = p[0]; pos[3 * o + 1] = p[1]; pos[3 * o + 2] = p[2]; }
            if (fz) fz[o] = tip_fz(&M.tip, d);
            if (iters) iters[o] = it;
            if (res) res[o] = r;
            if (lam) lam[o] = sym3_min_eig(Ks);
            if (ok) ok[o] = good;
        }
    }
    return 0;
}

/* IETS map (Sec. 3.3): the probe particle's vibration modes at the relaxed
 * position p*: stiffness K = -(J + J^T)/2 with J = dG/dp (tip springs + exact
 * trilinear Jacobian, or the direct-sum Jacobian when ff == NULL), its three
 * eigenvalues ascending (eV/A^2) in eig[3*o..], and the mode energies
 * hbar*sqrt(lambda/m) in meV in hw[3*o..] (0 where lambda <= 0) for a mass in
 * atomic mass units.  pos and outputs in scan layout [nz][ny][nx]. */
int or_iets(const double* ff, const or_grid* G, const or_atoms* A, const or_probe* P, const or_scan* S,
            const or_tip* T, const double* pos, double mass_amu, double* eig, double* hw, int nthreads) {
    if (!G || !S || !T || !pos || !eig || !(mass_amu > 0.0)) return 1;
    if (!ff && (!A || !P)) return 1;
    set_threads(nthreads);
    or_model M;
    M.ff = ff; M.G = G; M.A = A; M.P = P;
    grid_period(G, &M.Lx, &M.Ly);
    M.tip = tip_units(T);
    /* hbar sqrt(eV A^-2 / amu) in meV: SI constants */
    const double hbar = 1.054571817e-34, ev = 1.602176634e-19, amu = 1.66053906660e-27;
    const double unit = hbar * sqrt(ev / 1e-20 / amu) / ev * 1e3;
    const long npix = (long)S->nx * S->ny, total = npix * S->nz;
#pragma omp parallel for schedule(static)
    for (long o = 0; o < total; ++o) {
        const int k = (int)(o / npix);
        const long px = o % npix;
        const int i = (int)(px % S->nx), j = (int)(px / S->nx);
        const double anchor[3] = {S->x0 + i * S->px, S->y0 + j * S->py, S->z_top - k * S->dz};
        double Gv[3], J[9], K[9], ev3[3];
        total_force(&M, anchor, pos + 3 * o, Gv, J);
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) K[m * 3 + n] = -0.5 * (J[m * 3 + n] + J[n * 3 + m]);
        sym3_eigs(K, ev3);
        for (int m = 0; m < 3; ++m) {
            eig[3 * o + m] = ev3[m];
            if (hw) hw[3 * o + m] = ev3[m] > 0.0 ? unit * sqrt(ev3[m] / mass_amu) : 0.0;
        }
    }
    return 0;
}

/* ---------------------------------------------------------- frequency shift */

static double prim1(double u, double a) { return -sqrt(fmax(a * a - u * u, 0.0)); }
static double prim2(double u, double a) {
    double s = u / a;
    if (s > 1.0) s = 1.0;
    if (s < -1.0) s = -1.0;
    return 0.5 * a * a * asin(s) - 0.5 * u * sqrt(fmax(a * a - u * u, 0.0));
}

/* Weights W_j (j = -m..m, stored at W[j+m]) with
 *   integral_{-a}^{a} u f(u) / sqrt(a^2 - u^2) du = sum_j W_j f(j h)
 * exactly for every f that is linear between the nodes u_j = j h; m = ceil(a/h).
 * Uses the primitives of u/sqrt(a^2-u^2) and u^2/sqrt(a^2-u^2). Returns m. */
int or_df_weights(double a, double h, double* W) {
    const int m = (int)ceil(a / h - 1e-9);
    if (!W) return m;
    for (int j = 0; j <= 2 * m; ++j) W[j] = 0.0;
    for (int j = -m; j < m; ++j) {
        const double uj = j * h, uj1 = (j + 1) * h;
        const double lo = fmax(uj, -a), hi = fmin(uj1, a);
        if (!(lo < hi)) continue;
        const double I1 = prim1(hi, a) - prim1(lo, a);
        const double I2 = prim2(hi, a) - prim2(lo, a);
        W[j + m] += (uj1 * I1 - I2) / h;
        W[j + 1 + m] += (I2 - uj * I1) / h;
    }
    return m;
}

/* Eq. (df): df(z_c) = -(f0/2k) (8/(pi A^2)) integral_{-A/2}^{A/2} u Fz(z_c+u)/sqrt(A^2/4-u^2) du.
 * fz[nz][npix] at tip heights z_k = z_top - k dz (k grows downward), df[nz-2m][npix]
 * labelled by the centre index c = m..nz-1-m.  Fz in eV/A, k in N/m, f0 in Hz. */
int or_fz_to_df(const double* fz, int nz, int npix, double dz, const or_df* D, double* df) {
    const double a = 0.5 * D->A_pp;
    const int m = or_df_weights(a, dz, NULL);
    if (nz < 2 * m + 1 || npix < 0) return 1;
    double* W = (double*)malloc((2 * m + 1) * sizeof(double));
    or_df_weights(a, dz, W);
    const double pref = -(D->f0 / (2.0 * D->k)) * (2.0 / (OR_PI * a * a)) * OR_EVA2_TO_NM;
    for (int c = m; c <= nz - 1 - m; ++c)
        for (int px = 0; px < npix; ++px) {
            double s = 0.0;
            for (int j = -m; j <= m; ++j) s += W[j + m] * fz[(long)(c - j) * npix + px];
            df[(long)(c - m) * npix + px] = pref * s;
        }
    free(W);
    return 0;
}

/* ------------------------------------------------------------------ adjoint */

/* Accumulate a . dF/d(theta_i) for one pair into the per-atom gradients
 * g[0..2] (position), g[3] (R_i), g[4] (eps_i), g[5] (q_i), *gQ and *gQzz. */
static void pair_grad(const or_pair* p, const or_atoms* A, int i, const or_probe* P,
                      const double a[3], double* g, double* gQ, double* gQzz) {
    const double ad = a[0] * p->d[0] + a[1] * p->d[1] + a[2] * p->d[2];
    for (int m = 0; m < 3; ++m) {
        double v = p->S * a[m];
        if (!p->clamped && p->r > 0.0) v += p->dSdr * ad * p->d[m] / p->r;
        g[m] -= v;  /* delta = r - r_i, d delta / d r_i = -I */
    }
    g[3] += ad * p->dSdR;
    if (p->e_ij > 0.0) g[4] += ad * p->S_lj_e * P->eps_pp / (2.0 * p->e_ij);
    g[5] += ad * OR_KE * P->Q * p->S_el_qq;
    *gQ += ad * OR_KE * A->q[i] * p->S_el_qq;
    if (P->Qzz != 0.0) {
        const double cq = 0.5 * OR_KE * P->Qzz * A->q[i];
        const double aPhi = a[0] * p->Phi[0] + a[1] * p->Phi[1] + a[2] * p->Phi[2];
        for (int m = 0; m < 3; ++m)
            g[m] -= cq * (a[0] * p->dPhi[m] + a[1] * p->dPhi[3 + m] + a[2] * p->dPhi[6 + m]);
        if (p->clamped)
            g[3] += cq * P->core_frac * (a[0] * p->dPhi_dr[0] + a[1] * p->dPhi_dr[1] + a[2] * p->dPhi_dr[2]);
        g[5] += 0.5 * OR_KE * P->Qzz * aPhi;
        *gQzz += 0.5 * OR_KE * A->q[i] * aPhi;
    }
}

/* Accumulate eb * dE/d(theta_i) for one pair into the per-atom gradients (energy grids). */
static void pair_grad_energy(const or_pair* p, const or_atoms* A, int i, const or_probe* P, double eb, double* g,
                             double* gQ, double* gQzz) {
    const double cq = 0.5 * OR_KE * P->Qzz * A->q[i];
    for (int m = 0; m < 3; ++m) g[m] -= eb * (p->dE_dd[m] + cq * p->deq_dd[m]);  /* d delta / d r_i = -I */
    g[3] += eb * (p->dE_dR + (p->clamped ? cq * p->deq_dr * P->core_frac : 0.0));
    if (p->e_ij > 0.0) g[4] += eb * p->E_lj_e * P->eps_pp / (2.0 * p->e_ij);
    g[5] += eb * (OR_KE * P->Q * p->E_el_qq + 0.5 * OR_KE * P->Qzz * p->eq);
    *gQ += eb * OR_KE * A->q[i] * p->E_el_qq;
    *gQzz += eb * 0.5 * OR_KE * A->q[i] * p->eq;
}

/* The 64 stencil nodes of the tricubic interpolant at p and the gradients in p of their
 * weights, grad w_g(p) (zero along an axis whose fraction is clamped). */
static void tricubic_grad_weights(const or_grid* G, const double p[3], long node[64], double gw[64][3]) {
    long ix[4], iy[4], iz[4];
    double tx, ty, tz, sx, sy, sz;
    axis_stencil(p[0], G->x0, G->dx, G->nx, G->periodic_xy, ix, &tx, &sx);
    axis_stencil(p[1], G->y0, G->dy, G->ny, G->periodic_xy, iy, &ty, &sy);
    axis_stencil(p[2], G->z0, G->dz, G->nz, 0, iz, &tz, &sz);
    double wx[4], dwx[4], d2wx[4], wy[4], dwy[4], d2wy[4], wz[4], dwz[4], d2wz[4];
    cr_weights(tx, wx, dwx, d2wx);
    cr_weights(ty, wy, dwy, d2wy);
    cr_weights(tz, wz, dwz, d2wz);
    int q = 0;
    for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a, ++q) {
                node[q] = (iz[c] * G->ny + iy[b]) * G->nx + ix[a];
                gw[q][0] = dwx[a] * wy[b] * wz[c] * sx;
                gw[q][1] = wx[a] * dwy[b] * wz[c] * sy;
                gw[q][2] = wx[a] * wy[b] * dwz[c] * sz;
            }
}

/* Gradient of L = sum_c sum_pix g_df[c][pix] * df[c][pix] with respect to the
 * atoms (x, y, z, q, R, eps) and the tip (kx, ky, kR in per N/m, Q), by the
 * implicit function theorem at the relaxed positions pos[nz][ny][nx][3]:
 *   g_Fz = K^T g_df;  J^T lambda = g_Fz grad_p Fz;
 *   dL/dtheta = g_Fz dFz/dtheta - lambda . dG/dtheta.
 * Grid mode (ff != NULL): the grid adjoint Gbar_g = -sum lambda w_g(p*) is
 * contracted with the pair derivatives of every node value; on a tricubic
 * energy grid the node values are energies, F_S = -sum_g E_g grad w_g, and
 * the grid adjoint is the scalar Ebar_g = sum lambda . grad w_g(p*),
 * contracted with the pair energies' derivatives.  Direct mode:
 * the pair derivatives are taken at p* itself.
 * gtip = {dL/dkx, dL/dky, dL/dkR, dL/dQ, dL/dQzz}.  grid_adj (optional) gets Gbar [nz][ny][nx][3]
 * (on an energy grid Ebar in component 0, the others zero). */
int or_backward(const double* ff, const or_grid* G, const or_atoms* A, const or_probe* P,
                const or_scan* S, const or_tip* T, const or_df* D, const double* pos,
                const double* g_df, double* grads /*[n][6]*/, double* gtip, double* grid_adj,
                int nthreads) {
    if (!G || !A || !P || !S || !T || !D || !pos || !g_df || !grads || !gtip) return 1;
    set_threads(nthreads);
    or_model M;
    M.ff = ff; M.G = G; M.A = A; M.P = P;
    grid_period(G, &M.Lx, &M.Ly);
    M.tip = tip_units(T);
    const tip_si* t = &M.tip;
    const int nz = S->nz;
    const long npix = (long)S->nx * S->ny;
    const double a = 0.5 * D->A_pp;
    const int m = or_df_weights(a, S->dz, NULL);
    if (nz < 2 * m + 1) return 1;
    double* W = (double*)malloc((2 * m + 1) * sizeof(double));
    or_df_weights(a, S->dz, W);
    const double pref = -(D->f0 / (2.0 * D->k)) * (2.0 / (OR_PI * a * a)) * OR_EVA2_TO_NM;
    /* g_Fz = K^T g_df */
    double* gfz = (double*)calloc((size_t)nz * npix, sizeof(double));
    for (int c = m; c <= nz - 1 - m; ++c)
        for (long px = 0; px < npix; ++px) {
            const double gd = g_df[(long)(c - m) * npix + px];
            for (int j = -m; j <= m; ++j) gfz[(long)(c - j) * npix + px] += pref * W[j + m] * gd;
        }
    free(W);
    const long nnode = (long)G->nx * G->ny * G->nz;
    double* gbar = ff ? (double*)calloc((size_t)nnode * 3, sizeof(double)) : NULL;
    double* lam = (double*)calloc((size_t)nz * npix * 3, sizeof(double));
    double gkx = 0, gky = 0, gkR = 0;
    for (int k = 0; k < nz; ++k)
        for (long px = 0; px < npix; ++px) {
            const long o = (long)k * npix + px;
            const double gf = gfz[o];
            if (gf == 0.0) continue;
            const int i = (int)(px % S->nx), j = (int)(px / S->nx);
            const double anchor[3] = {S->x0 + i * S->px, S->y0 + j * S->py, S->z_top - k * S->dz};
            const double* p = pos + 3 * o;
            const double d[3] = {p[0] - anchor[0], p[1] - anchor[1], p[2] - anchor[2]};
            const double dn = norm3(d);
            double Gv[3], J[9], JT[9];
            total_force(&M, anchor, p, Gv, J);
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) JT[r * 3 + s] = J[s * 3 + r];
            /* grad_p Fz = kR [(1 - R0/|d|) z_hat + R0 d_z d / |d|^3] */
            double gphi[3];
            for (int r = 0; r < 3; ++r) gphi[r] = t->kR * t->R0 * d[2] * d[r] / (dn * dn * dn);
            gphi[2] += t->kR * (1.0 - t->R0 / dn);
            double rhs[3] = {gf * gphi[0], gf * gphi[1], gf * gphi[2]}, l[3];
            if (solve3(JT, rhs, l)) continue;
            lam[3 * o] = l[0]; lam[3 * o + 1] = l[1]; lam[3 * o + 2] = l[2];
            /* tip parameters: dG/dkx = -(d_x - d0x) x_hat, ... (internal units) */
            gkx += l[0] * (d[0] - t->d0x);
            gky += l[1] * (d[1] - t->d0y);
            gkR += gf * (dn - t->R0) * d[2] / dn + (l[0] * d[0] + l[1] * d[1] + l[2] * d[2]) * (dn - t->R0) / dn;
            if (gbar && G->interp == 1) {
                /* F_S = -sum_g E_g grad w_g: dL/dE_g = -lambda . (-grad w_g) */
                long node[64];
                double gw[64][3];
                tricubic_grad_weights(G, p, node, gw);
                for (int q = 0; q < 64; ++q) gbar[3 * node[q]] += l[0] * gw[q][0] + l[1] * gw[q][1] + l[2] * gw[q][2];
            } else if (gbar) {
                long node[8];
                double w8[8], F[3];
                interp(ff, G, p, F, NULL, node, w8);
                for (int c8 = 0; c8 < 8; ++c8)
                    for (int r = 0; r < 3; ++r) gbar[3 * node[c8] + r] -= l[r] * w8[c8];
            }
        }
    gtip[0] = gkx * OR_NM_TO_EVA2;
    gtip[1] = gky * OR_NM_TO_EVA2;
    gtip[2] = gkR * OR_NM_TO_EVA2;
    double gQ_total = 0.0, gQzz_total = 0.0;
    const int n = A->n;
    double* gQ_atom = (double*)calloc((size_t)n, sizeof(double));
    double* gQzz_atom = (double*)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int ia = 0; ia < n; ++ia) {
        double g[6] = {0, 0, 0, 0, 0, 0}, gQ = 0.0, gQzz = 0.0;
        if (gbar) {
            const long nxy = (long)G->nx * G->ny;
            for (long gi = 0; gi < nnode; ++gi) {
                const double* av = gbar + 3 * gi;
                if (av[0] == 0.0 && av[1] == 0.0 && av[2] == 0.0) continue;
                const long kk = gi / nxy, rem = gi % nxy, jj = rem / G->nx, ii = rem % G->nx;
                const double r[3] = {G->x0 + ii * G->dx, G->y0 + jj * G->dy, G->z0 + kk * G->dz};
                or_pair pr;
                pair_eval(A, ia, P, M.Lx, M.Ly, r, &pr);
                if (G->interp == 1)
                    pair_grad_energy(&pr, A, ia, P, av[0], g, &gQ, &gQzz);
                else
                    pair_grad(&pr, A, ia, P, av, g, &gQ, &gQzz);
            }
        } else {
            for (long o = 0; o < (long)nz * npix; ++o) {
                const double* l = lam + 3 * o;
                if (l[0] == 0.0 && l[1] == 0.0 && l[2] == 0.0) continue;
                const double av[3] = {-l[0], -l[1], -l[2]};
                or_pair pr;
                pair_eval(A, ia, P, M.Lx, M.Ly, pos + 3 * o, &pr);
                pair_grad(&pr, A, ia, P, av, g, &gQ, &gQzz);
            }
        }
        for (int r = 0; r < 6; ++r) grads[6 * ia + r] = g[r];
        gQ_atom[ia] = gQ;
        gQzz_atom[ia] = gQzz;
    }
    for (int ia = 0; ia < n; ++ia) {
        gQ_total += gQ_atom[ia];
        gQzz_total += gQzz_atom[ia];
    }
    gtip[3] = gQ_total;
    gtip[4] = gQzz_total;
    if (grid_adj && gbar) memcpy(grid_adj, gbar, (size_t)nnode * 3 * sizeof(double));
    free(gQ_atom);
    free(gQzz_atom);
    free(gbar);
    free(lam);
    free(gfz);
    return 0;
}

/* ------------------------------------------------- FFT-type force fields */

/* Spectral derivative weights of periodic samples along one axis (n even):
 * the derivative of the trigonometric interpolant with its Nyquist term
 * dropped, written in real space, f'_i = sum_j D_{i-j} f_j with
 * D_0 = 0 and D_m = (pi / (n h)) (-1)^m cot(pi m / n). */
static double spectral_d(long m, long n, double h) {
    m %= n;
    if (m < 0) m += n;
    if (m == 0) return 0.0;
    const double sgn = (m % 2) ? -1.0 : 1.0;
    return OR_PI / ((double)n * h) * sgn / tan(OR_PI * (double)m / (double)n);
}

static double powered(double v, double p) {
    if (p == 1.0) return v;
    return v > 0.0 ? pow(v, p) : 0.0;
}

/* Cross-correlation force field of Eqs. (El_conv) and (Pauli_FDBM) on a grid
 * periodic in x, y and z: the sample field f (Hartree potential, or density)
 * seen by the tip's density g placed at every node n,
 *   E[n] = scale * dV * sum_h g[h]^p f[n + h]^p      (indices modulo the grid),
 * with dV = dx dy dz, g[h] the tip density at offset h from the PP, p = 1 for
 * electrostatics (scale = 1) and p = beta, scale = A for the Pauli term (the
 * product [g f]^beta factors into g^beta f^beta); F = -grad E by the spectral
 * derivative of each axis.  ff[n] = (Fx, Fy, Fz, E), layout [nz][ny][nx][4].
 * p != 1 takes densities: negative samples count as 0.  Sizes must be even. */
int or_correlate(const double* f, const double* g, const or_grid* G, double scale, double p, double* ff,
                 int nthreads) {
    if (!f || !g || !G || !ff) return 1;
    const long nx = G->nx, ny = G->ny, nz = G->nz;
    if (nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2) return 1;
    set_threads(nthreads);
    const long nxy = nx * ny, N = nxy * nz;
    const double dV = G->dx * G->dy * G->dz;
    double* fp = (double*)malloc((size_t)N * sizeof(double));
    double* gp = (double*)malloc((size_t)N * sizeof(double));
    double* E = (double*)malloc((size_t)N * sizeof(double));
    for (long q = 0; q < N; ++q) {
        fp[q] = powered(f[q], p);
        gp[q] = powered(g[q], p);
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        const long k = n / nxy, j = (n % nxy) / nx, i = n % nx;
        double s = 0.0;
        for (long c = 0; c < nz; ++c)
            for (long b = 0; b < ny; ++b)
                for (long a = 0; a < nx; ++a) {
                    const double gv = gp[(c * ny + b) * nx + a];
                    if (gv == 0.0) continue;
                    s += gv * fp[(((k + c) % nz) * ny + (j + b) % ny) * nx + (i + a) % nx];
                }
        E[n] = scale * dV * s;
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        const long k = n / nxy, j = (n % nxy) / nx, i = n % nx;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (long a = 0; a < nx; ++a) gx += spectral_d(i - a, nx, G->dx) * E[(k * ny + j) * nx + a];
        for (long b = 0; b < ny; ++b) gy += spectral_d(j - b, ny, G->dy) * E[(k * ny + b) * nx + i];
        for (long c = 0; c < nz; ++c) gz += spectral_d(k - c, nz, G->dz) * E[(c * ny + j) * nx + i];
        ff[4 * n] = -gx;
        ff[4 * n + 1] = -gy;
        ff[4 * n + 2] = -gz;
        ff[4 * n + 3] = E[n];
    }
    free(fp);
    free(gp);
    free(E);
    return 0;
}

/* E[n] alone at the listed nodes (for spot checks of large grids). */
int or_correlate_nodes(const double* f, const double* g, const or_grid* G, double scale, double p, int nnodes,
                       const long* nodes, double* E, int nthreads) {
    if (!f || !g || !G || !nodes || !E) return 1;
    const long nx = G->nx, ny = G->ny, nz = G->nz, nxy = nx * ny;
    set_threads(nthreads);
    const double dV = G->dx * G->dy * G->dz;
#pragma omp parallel for schedule(static)
    for (int t = 0; t < nnodes; ++t) {
        const long n = nodes[t];
        const long k = n / nxy, j = (n % nxy) / nx, i = n % nx;
        double s = 0.0;
        for (long c = 0; c < nz; ++c)
            for (long b = 0; b < ny; ++b)
                for (long a = 0; a < nx; ++a) {
                    const double gv = powered(g[(c * ny + b) * nx + a], p);
                    if (gv == 0.0) continue;
                    s += gv * powered(f[(((k + c) % nz) * ny + (j + b) % ny) * nx + (i + a) % nx], p);
                }
        E[t] = scale * dV * s;
    }
    return 0;
}
