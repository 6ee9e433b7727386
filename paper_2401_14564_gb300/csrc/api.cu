// C ABI of libpp: argument checks, unit conversion, launch.
#include <math.h>
#include <nvtx3/nvToolsExt.h>

#include <cstring>
#include <string>
#include <vector>

#include "pp_internal.cuh"

namespace pp {

static thread_local std::string g_error;

// NVTX range around an entry point's host side (validation and enqueue), named after the
// entry point, so that a timeline tool shows which call issued which kernels.  Without an
// attached tool a push or pop costs a branch.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

void set_error(const std::string& msg) { g_error = msg; }

pp_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PP_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return PP_ERR_CUDA;
}

static bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }
static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
static bool finite_pos(float v) { return isfinite(v) && v > 0.f; }

bool make_grid_map(const pp_grid* g, GridMap* out, std::string* why) {
    if (!g) { *why = "grid is NULL"; return false; }
    if (g->nx < 2 || g->ny < 2 || g->nz < 2) { *why = "grid needs nx, ny, nz >= 2"; return false; }
    // (the cell lookup's fast floor is exact below 2^22 nodes per axis)
    if (g->nx > (1 << 22) || g->ny > (1 << 22) || g->nz > (1 << 22)) { *why = "grid axes hold at most 2^22 nodes"; return false; }
    if (!finite_pos(g->dx) || !finite_pos(g->dy) || !finite_pos(g->dz)) { *why = "grid spacing must be > 0"; return false; }
    if (!isfinite(g->x0) || !isfinite(g->y0) || !isfinite(g->z0)) { *why = "grid origin must be finite"; return false; }
    if (g->periodic_xy != 0 && g->periodic_xy != 1) { *why = "periodic_xy must be 0 or 1"; return false; }
    if (g->interp != 0 && g->interp != 1) { *why = "interp must be 0 (trilinear) or 1 (tricubic)"; return false; }
    if (g->interp == 1 && g->layout != 0) { *why = "tricubic (energy) grids use the linear layout"; return false; }
    GridMap m;
    m.nx = g->nx; m.ny = g->ny; m.nz = g->nz;
    m.interp = g->interp;
    if (g->layout == 0) {
        const int64_t n = (int64_t)g->nx * g->ny * g->nz;
        if (n >= (int64_t(1) << 31)) { *why = "grid has 2^31 or more nodes"; return false; }
        m.ax = {0, 1, 0, 0};
        m.ay = {0, g->nx, 0, 0};
        m.az = {0, g->nx * g->ny, 0, 0};
        m.stored_nodes = n;
    } else if (g->layout == 1) {
        if (!pow2_in(g->bx, 1, 16) || !pow2_in(g->by, 1, 16) || !pow2_in(g->bz, 1, 16)) {
            *why = "brick sides must be powers of two in [1, 16]";
            return false;
        }
        const int lx = ilog2(g->bx), ly = ilog2(g->by), lz = ilog2(g->bz), lb = lx + ly + lz;
        const int64_t nbx = (g->nx + g->bx - 1) / g->bx, nby = (g->ny + g->by - 1) / g->by;
        const int64_t nbz = (g->nz + g->bz - 1) / g->bz;
        const int64_t n = (nbx * nby * nbz) << lb;
        if (n >= (int64_t(1) << 31)) { *why = "bricked grid has 2^31 or more slots"; return false; }
        m.ax = {lx, 1 << lb, g->bx - 1, 0};
        m.ay = {ly, (int)(nbx << lb), g->by - 1, lx};
        m.az = {lz, (int)((nbx * nby) << lb), g->bz - 1, lx + ly};
        m.stored_nodes = n;
    } else {
        *why = "layout must be 0 (linear) or 1 (bricked)";
        return false;
    }
    *out = m;
    return true;
}

int df_half_width(double A_pp, double dz) {
    if (!(A_pp > 0.0) || !(dz > 0.0) || !isfinite(A_pp) || !isfinite(dz)) return -1;
    const double m = ceil(0.5 * A_pp / dz - 1e-9);
    return m > 1e6 ? -1 : (int)m;
}

// W(u_j), u_j = j*dz (j = -m..m): exact quadrature weights of
// integral_{-a}^{a} u f(u) / sqrt(a^2 - u^2) du for f linear between nodes.
// On [u_j, u_j+1] the hat functions are (u_{j+1} - u)/h and (u - u_j)/h, so
// each interval needs the two moments of the kernel, integral u/sqrt and
// integral u^2/sqrt, taken from their antiderivatives -sqrt(a^2-u^2) and
// (a^2/2) asin(u/a) - (u/2) sqrt(a^2-u^2).
static void giessibl_weights(double a, double h, int m, std::vector<double>& W) {
    W.assign(2 * m + 1, 0.0);
    auto root = [a](double u) { return sqrt(fmax(a * a - u * u, 0.0)); };
    auto m1 = [&](double u) { return -root(u); };
    auto m2 = [&](double u) {
        const double s = fmin(fmax(u / a, -1.0), 1.0);
        return 0.5 * a * a * asin(s) - 0.5 * u * root(u);
    };
    for (int j = -m; j < m; ++j) {
        const double ul = j * h, ur = (j + 1) * h;
        const double lo = fmax(ul, -a), hi = fmin(ur, a);
        if (hi <= lo) continue;
        const double k1 = m1(hi) - m1(lo), k2 = m2(hi) - m2(lo);
        W[j + m] += (ur * k1 - k2) / h;      // left node's hat
        W[j + 1 + m] += (k2 - ul * k1) / h;  // right node's hat
    }
}

void df_stencil(double A_pp, double dz, double k, double f0, int m, float* coef) {
    const double a = 0.5 * A_pp;
    std::vector<double> W;
    giessibl_weights(a, dz, m, W);
    const double pref = -(f0 / (2.0 * k)) * (2.0 / (kPi * a * a)) * kEvA2ToNm;
    // Fz at height index c+s sits at u = -s*dz from the centre: heights fall as the index grows
    for (int s = -m; s <= m; ++s) coef[s + m] = (float)(pref * W[-s + m]);
}

#ifdef PP_CHECKED
// flag readers of the kernel translation units (bounds-checked builds)
unsigned int check_flags_ff_assemble();
unsigned int check_flags_relax_scan();
unsigned int check_flags_fz_to_df();
unsigned int check_flags_backward();
unsigned int check_flags_batch();
unsigned int check_flags_iets();
unsigned int check_flags_fft();
#endif

}  // namespace pp

using namespace pp;

extern "C" {

const char* pp_last_error(void) { return g_error.c_str(); }

pp_status pp_check_flags(unsigned int* flags) {
    g_error.clear();
    if (!flags) { set_error("pp_check_flags: NULL argument"); return PP_ERR_ARG; }
    *flags = 0;
#ifdef PP_CHECKED
    pp_status st = cuda_status(cudaDeviceSynchronize(), "pp_check_flags sync");
    if (st != PP_OK) return st;
    *flags = check_flags_ff_assemble() | check_flags_relax_scan() | check_flags_fz_to_df() | check_flags_backward() |
             check_flags_batch() | check_flags_iets() | check_flags_fft();
    return PP_OK;
#else
    set_error("pp_check_flags: not a bounds-checked build (compile with -DPP_CHECKED)");
    return PP_ERR_UNSUPPORTED;
#endif
}

size_t pp_ff_floats(const pp_grid* grid) {
    GridMap m;
    std::string why;
    if (!make_grid_map(grid, &m, &why)) return 0;
    return (size_t)m.stored_nodes * (m.interp ? 1 : 4);
}

int pp_df_margin(float A_pp, float dz) { return df_half_width(A_pp, dz); }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Validation and launch shared by pp_make_ff, pp_make_ff_tuned and pp_make_ff_split.
// layers: NULL for the whole grid (padding zeroed), else the node layers [layers[0], layers[1]) to write.
static pp_status make_ff_impl(const char* name, const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                              float* ff, float* ff_el, int zpt, int forces_only, pp_stream stream,
                              const int* layers = nullptr) {
    const std::string who(name);
    if (!atoms || !probe || !grid || !ff) { set_error(who + ": NULL argument"); return PP_ERR_ARG; }
    if (atoms->n < 0) { set_error(who + ": atoms->n < 0"); return PP_ERR_ARG; }
    if (atoms->n > 0 && (!atoms->x || !atoms->y || !atoms->z || !atoms->R || !atoms->eps || !atoms->q)) {
        set_error(who + ": NULL atom array");
        return PP_ERR_ARG;
    }
    if (!(probe->core_frac > 0.f && probe->core_frac < 1.f)) { set_error(who + ": core_frac must be in (0,1)"); return PP_ERR_ARG; }
    if (!(probe->eps_pp >= 0.f) || !isfinite(probe->R_pp) || !isfinite(probe->Q) || !(probe->coul_rc >= 0.f) ||
        !isfinite(probe->Qzz)) {
        set_error(who + ": invalid probe parameters");
        return PP_ERR_ARG;
    }
    if (probe->min_image != 0 && probe->min_image != 1) { set_error(who + ": min_image must be 0 or 1"); return PP_ERR_ARG; }
    if (!aligned16(ff) || (ff_el && !aligned16(ff_el))) { set_error(who + ": grids must be 16-byte aligned"); return PP_ERR_ARG; }
    if (ff_el == ff) { set_error(who + ": ff and ff_el must be different buffers"); return PP_ERR_ARG; }
    GridMap map;
    std::string why;
    if (!make_grid_map(grid, &map, &why)) { set_error(who + ": " + why); return PP_ERR_SHAPE; }
    if (forces_only && map.interp) { set_error(who + ": ff_forces_only on an energy-only (interp = 1) grid"); return PP_ERR_ARG; }
    const int kbeg = layers ? layers[0] : 0, kend = layers ? layers[1] : grid->nz;
    if (kbeg < 0 || kend <= kbeg || kend > grid->nz) {
        set_error(who + ": node layers must satisfy 0 <= k_begin < k_end <= nz");
        return PP_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!layers && map.stored_nodes > (int64_t)grid->nx * grid->ny * grid->nz) {
        for (float* g : {ff, ff_el}) {
            if (!g) continue;
            pp_status st = cuda_status(cudaMemsetAsync(g, 0, (size_t)map.stored_nodes * 16, s), (who + " memset").c_str());
            if (st != PP_OK) return st;
        }
    }
    FFLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.x = atoms->x; L.y = atoms->y; L.z = atoms->z; L.R = atoms->R; L.eps = atoms->eps; L.q = atoms->q;
    L.n = atoms->n;
    L.R_pp = probe->R_pp;
    L.eps_pp = probe->eps_pp;
    // split: the point-charge grid is per unit probe charge
    L.kQ = (float)(kCoulomb * (ff_el ? 1.0 : (double)probe->Q));
    L.kQzz = (float)(0.5 * kCoulomb * (double)probe->Qzz);
    L.core_frac = probe->core_frac;
    L.coul_rc = probe->coul_rc;
    L.min_image = probe->min_image;
    L.Lx = grid->nx * grid->dx;
    L.Ly = grid->ny * grid->dy;
    L.x0 = grid->x0; L.y0 = grid->y0; L.z0 = grid->z0;
    L.dx = grid->dx; L.dy = grid->dy; L.dz = grid->dz;
    L.map = map;
    L.ff = map.interp ? nullptr : reinterpret_cast<float4*>(ff);
    L.ffE = map.interp ? ff : nullptr;
    L.zpt = zpt;
    L.forces_only = forces_only;
    L.split = ff_el != nullptr;
    L.ffel = (ff_el && !map.interp) ? reinterpret_cast<float4*>(ff_el) : nullptr;
    L.ffelE = (ff_el && map.interp) ? ff_el : nullptr;
    L.kbeg = kbeg;
    L.kend = kend;
    return cuda_status(launch_ff_assemble(L, s), (who + " launch").c_str());
}

pp_status pp_make_ff(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid, float* ff,
                     pp_stream stream) {
    Range range("pp_make_ff");
    g_error.clear();
    return make_ff_impl("pp_make_ff", atoms, probe, grid, ff, nullptr, 8, 0, stream);
}

pp_status pp_make_ff_tuned(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid, float* ff,
                           const pp_tuning* tuning, pp_stream stream) {
    Range range("pp_make_ff_tuned");
    g_error.clear();
    const int zpt = (tuning && tuning->ff_zpt) ? tuning->ff_zpt : 8;
    if (zpt != 4 && zpt != 8 && zpt != 16) { set_error("pp_make_ff_tuned: ff_zpt must be 4, 8 or 16"); return PP_ERR_ARG; }
    const int forces_only = tuning ? tuning->ff_forces_only : 0;
    if (forces_only != 0 && forces_only != 1) { set_error("pp_make_ff_tuned: ff_forces_only must be 0 or 1"); return PP_ERR_ARG; }
    return make_ff_impl("pp_make_ff_tuned", atoms, probe, grid, ff, nullptr, zpt, forces_only, stream);
}

pp_status pp_make_ff_layers(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid, float* ff,
                            const pp_tuning* tuning, int k_begin, int k_end, pp_stream stream) {
    Range range("pp_make_ff_layers");
    g_error.clear();
    const int zpt = (tuning && tuning->ff_zpt) ? tuning->ff_zpt : 8;
    if (zpt != 4 && zpt != 8 && zpt != 16) { set_error("pp_make_ff_layers: ff_zpt must be 4, 8 or 16"); return PP_ERR_ARG; }
    const int forces_only = tuning ? tuning->ff_forces_only : 0;
    if (forces_only != 0 && forces_only != 1) { set_error("pp_make_ff_layers: ff_forces_only must be 0 or 1"); return PP_ERR_ARG; }
    const int layers[2] = {k_begin, k_end};
    return make_ff_impl("pp_make_ff_layers", atoms, probe, grid, ff, nullptr, zpt, forces_only, stream, layers);
}

pp_status pp_make_ff_split(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid, float* ff,
                           float* ff_el, pp_stream stream) {
    Range range("pp_make_ff_split");
    g_error.clear();
    if (!ff_el) { set_error("pp_make_ff_split: NULL ff_el"); return PP_ERR_ARG; }
    return make_ff_impl("pp_make_ff_split", atoms, probe, grid, ff, ff_el, 8, 0, stream);
}

pp_status pp_ff_combine(const float* ff, const float* ff_el, float Q, const pp_grid* grid, float* out,
                        pp_stream stream) {
    Range range("pp_ff_combine");
    g_error.clear();
    if (!ff || !ff_el || !grid || !out) { set_error("pp_ff_combine: NULL argument"); return PP_ERR_ARG; }
    if (!isfinite(Q)) { set_error("pp_ff_combine: Q must be finite"); return PP_ERR_ARG; }
    if (!aligned16(ff) || !aligned16(ff_el) || !aligned16(out)) {
        set_error("pp_ff_combine: grids must be 16-byte aligned");
        return PP_ERR_ARG;
    }
    GridMap map;
    std::string why;
    if (!make_grid_map(grid, &map, &why)) { set_error("pp_ff_combine: " + why); return PP_ERR_SHAPE; }
    const int64_t nfloats = map.stored_nodes * (map.interp ? 1 : 4);
    return cuda_status(launch_ff_combine(ff, ff_el, Q, out, nfloats, (cudaStream_t)stream), "pp_ff_combine launch");
}

static bool check_tip_fire(const pp_tip* tip, const pp_fire* fire, std::string* why) {
    if (!(tip->kR > 0.f) || !(tip->R0 > 0.f) || !(tip->kx >= 0.f) || !(tip->ky >= 0.f) ||
        !isfinite(tip->kR) || !isfinite(tip->kx) || !isfinite(tip->ky) || !isfinite(tip->d0x) || !isfinite(tip->d0y)) {
        *why = "invalid tip springs";
        return false;
    }
    if (!(tip->d0x * tip->d0x + tip->d0y * tip->d0y < tip->R0 * tip->R0)) { *why = "|(d0x, d0y)| must be < R0"; return false; }
    if (fire->max_iter < 0 || !(fire->ftol > 0.f) || !(fire->dt0 > 0.f) || !(fire->dt_max > 0.f) ||
        !(fire->f_inc >= 1.f) || !(fire->f_dec > 0.f && fire->f_dec <= 1.f) || !(fire->alpha0 >= 0.f && fire->alpha0 <= 1.f) ||
        !(fire->f_alpha > 0.f && fire->f_alpha <= 1.f) || !(fire->mass > 0.f) || fire->n_min < 0 ||
        fire->polish < 0 || fire->polish > 16) {
        *why = "invalid FIRE parameters";
        return false;
    }
    return true;
}

// pp_relax_scan, and pp_relax_scan_ex with its options (checked by the caller).
static pp_status relax_scan_impl(const char* name, const float* ff, const pp_grid* grid, const pp_scan* scan,
                                 const pp_tip* tip, const pp_fire* fire, float* pos, float* fz, int* iters,
                                 const pp_df* fused_df, float* df, int* zspan, const pp_scan_opts* opts,
                                 pp_stream stream) {
    const std::string who(name);
    if (!ff || !grid || !scan || !tip || !fire || !fz) { set_error(who + ": NULL argument"); return PP_ERR_ARG; }
    if (!aligned16(ff)) { set_error(who + ": ff must be 16-byte aligned"); return PP_ERR_ARG; }
    GridMap map;
    std::string why;
    if (!make_grid_map(grid, &map, &why)) { set_error(who + ": " + why); return PP_ERR_SHAPE; }
    if (scan->nx < 1 || scan->ny < 1 || scan->nz < 1) { set_error(who + ": scan sizes must be >= 1"); return PP_ERR_SHAPE; }
    if ((int64_t)scan->nx * scan->ny * scan->nz * 3 >= (int64_t(1) << 31)) {
        set_error(who + ": scan too large for one call");
        return PP_ERR_SHAPE;
    }
    if (!isfinite(scan->x0) || !isfinite(scan->y0) || !isfinite(scan->px) || !isfinite(scan->py) ||
        !isfinite(scan->z_top) || !finite_pos(scan->dz)) {
        set_error(who + ": invalid scan geometry");
        return PP_ERR_ARG;
    }
    if (!check_tip_fire(tip, fire, &why)) { set_error(who + ": " + why); return PP_ERR_ARG; }
    RelaxLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.ff = map.interp ? nullptr : reinterpret_cast<const float4*>(ff);
    L.ffE = map.interp ? ff : nullptr;
    L.map = map;
    L.inv_dx = 1.f / grid->dx; L.inv_dy = 1.f / grid->dy; L.inv_dz = 1.f / grid->dz;
    L.gx0s = (float)(-(double)grid->x0 / grid->dx);
    L.gy0s = (float)(-(double)grid->y0 / grid->dy);
    L.gz0s = (float)(-(double)grid->z0 / grid->dz);
    L.periodic_xy = grid->periodic_xy;
    L.snx = scan->nx; L.sny = scan->ny; L.snz = scan->nz;
    L.sx0 = scan->x0; L.sy0 = scan->y0; L.spx = scan->px; L.spy = scan->py;
    L.z_top = scan->z_top; L.sdz = scan->dz;
    L.kx = (float)(tip->kx * kNmToEvA2);
    L.ky = (float)(tip->ky * kNmToEvA2);
    L.kR = (float)(tip->kR * kNmToEvA2);
    L.R0 = tip->R0;
    L.d0x = tip->d0x;
    L.d0y = tip->d0y;
    L.d0z = (float)(-sqrt((double)tip->R0 * tip->R0 - (double)tip->d0x * tip->d0x - (double)tip->d0y * tip->d0y));
    L.R0sq = (float)((double)tip->R0 * tip->R0);
    L.c0 = (float)((double)L.d0x * L.d0x + (double)L.d0y * L.d0y + (double)L.d0z * L.d0z - (double)tip->R0 * tip->R0);
    split_height_steps(scan->z_top, L.d0z, scan->dz, grid->z0, grid->dz, &L.fz0, &L.fz0_lo, &L.st, &L.st_lo);
    L.layout = grid->layout;
    L.max_iter = fire->max_iter;
    L.n_min = fire->n_min;
    L.ftol2 = fire->ftol * fire->ftol;
    L.dt0 = fire->dt0; L.dt_max = fire->dt_max; L.f_inc = fire->f_inc; L.f_dec = fire->f_dec;
    L.alpha0 = fire->alpha0; L.f_alpha = fire->f_alpha; L.inv_mass = 1.f / fire->mass;
    L.polish = fire->polish;
    L.pos = pos; L.fz = fz; L.iters = iters;
    L.df_m = -1;
    L.df = nullptr;
    if (fused_df && df) {
        if (!finite_pos(fused_df->k) || !isfinite(fused_df->f0)) { set_error(who + ": invalid df parameters"); return PP_ERR_ARG; }
        const int m = df_half_width(fused_df->A_pp, scan->dz);
        if (m < 0) { set_error(who + ": invalid df amplitude"); return PP_ERR_ARG; }
        if (m > kMaxDfHalfWidth) { set_error(who + ": df stencil wider than 63 taps"); return PP_ERR_UNSUPPORTED; }
        if (scan->nz < 2 * m + 1) { set_error(who + ": fewer heights than the df stencil"); return PP_ERR_SHAPE; }
        L.df_m = m;
        L.df = df;
        df_stencil(fused_df->A_pp, scan->dz, fused_df->k, fused_df->f0, m, L.coef);
    }
    L.zspan = zspan;
    if (opts && opts->plan) {
        const int npix = scan->nx * scan->ny;
        const int* plan = static_cast<const int*>(opts->plan);
        L.plan_list = plan + relax_plan_list_offset(npix);
        L.plan_mask = reinterpret_cast<const unsigned*>(plan + relax_plan_mask_offset(npix, opts->plan_k, opts->plan_lanes));
        L.plan_lanes = opts->plan_lanes;
        L.plan_hblocks = (opts->plan_k + opts->plan_lanes - 1) / opts->plan_lanes;
    }
    if (zspan) {
        // (INT_MAX, INT_MIN) before the scan folds its lanes' layers in by atomic min / max
        for (int h = 0; h < 2; ++h) {
            const pp_status st = cuda_status(cudaMemsetAsync(zspan + h, h ? 0x80 : 0x7f, sizeof(int),
                                                             (cudaStream_t)stream), (who + " memset").c_str());
            if (st != PP_OK) return st;
        }
    }
    return cuda_status(launch_relax_scan(L, (cudaStream_t)stream), (who + " launch").c_str());
}

pp_status pp_relax_scan(const float* ff, const pp_grid* grid, const pp_scan* scan, const pp_tip* tip,
                        const pp_fire* fire, float* pos, float* fz, int* iters, const pp_df* fused_df, float* df,
                        pp_stream stream) {
    Range range("pp_relax_scan");
    g_error.clear();
    return relax_scan_impl("pp_relax_scan", ff, grid, scan, tip, fire, pos, fz, iters, fused_df, df, nullptr, nullptr,
                           stream);
}

pp_status pp_relax_scan_ex(const float* ff, const pp_grid* grid, const pp_scan* scan, const pp_tip* tip,
                           const pp_fire* fire, float* pos, float* fz, int* iters, const pp_df* fused_df, float* df,
                           const pp_scan_opts* opts, pp_stream stream) {
    Range range("pp_relax_scan_ex");
    g_error.clear();
    const char* who = "pp_relax_scan_ex";
    if (!opts) { set_error("pp_relax_scan_ex: NULL opts"); return PP_ERR_ARG; }
    if (opts->zspan && ((uintptr_t)opts->zspan & 3u) != 0) {
        set_error("pp_relax_scan_ex: zspan must be 4-byte aligned");
        return PP_ERR_ARG;
    }
    if (opts->plan) {
        if (((uintptr_t)opts->plan & 3u) != 0) { set_error("pp_relax_scan_ex: plan must be 4-byte aligned"); return PP_ERR_ARG; }
        if (opts->plan_k < 1 || opts->plan_lanes < 1 || opts->plan_lanes > 32 || !scan ||
            (int64_t)opts->plan_k > (int64_t)scan->nx * scan->ny) {
            set_error("pp_relax_scan_ex: plan_k must be in [1, nx*ny] and plan_lanes in [1, 32]");
            return PP_ERR_ARG;
        }
    }
    return relax_scan_impl(who, ff, grid, scan, tip, fire, pos, fz, iters, fused_df, df, opts->zspan, opts, stream);
}

size_t pp_relax_plan_size(const pp_scan* scan, int k, int lanes) {
    if (!scan || scan->nx < 1 || scan->ny < 1 || lanes < 1 || lanes > 32 || k < 1 ||
        (int64_t)scan->nx * scan->ny >= (int64_t(1) << 30) || (int64_t)k > (int64_t)scan->nx * scan->ny)
        return 0;
    return relax_plan_words(scan->nx * scan->ny, k, lanes) * sizeof(int);
}

pp_status pp_relax_plan(const int* iters, const pp_scan* scan, int max_iter, int k, int lanes, void* plan,
                        pp_stream stream) {
    Range range("pp_relax_plan");
    g_error.clear();
    if (!iters || !scan || !plan) { set_error("pp_relax_plan: NULL argument"); return PP_ERR_ARG; }
    if (((uintptr_t)plan & 3u) != 0 || ((uintptr_t)iters & 3u) != 0) {
        set_error("pp_relax_plan: iters and plan must be 4-byte aligned");
        return PP_ERR_ARG;
    }
    if (scan->nx < 1 || scan->ny < 1 || scan->nz < 1 ||
        (int64_t)scan->nx * scan->ny * scan->nz * 3 >= (int64_t(1) << 31)) {
        set_error("pp_relax_plan: invalid scan size");
        return PP_ERR_SHAPE;
    }
    if (max_iter < 0) { set_error("pp_relax_plan: max_iter < 0"); return PP_ERR_ARG; }
    if (pp_relax_plan_size(scan, k, lanes) == 0) {
        set_error("pp_relax_plan: k must be in [1, nx*ny] and lanes in [1, 32]");
        return PP_ERR_ARG;
    }
    return cuda_status(launch_relax_plan(iters, scan->nz, scan->nx * scan->ny, max_iter, k, lanes,
                                         static_cast<int*>(plan), (cudaStream_t)stream),
                       "pp_relax_plan launch");
}

pp_status pp_fz_to_df(const float* fz, int nz, int npix, float dz, const pp_df* dfp, float* df, pp_stream stream) {
    Range range("pp_fz_to_df");
    g_error.clear();
    if (!dfp) { set_error("pp_fz_to_df: NULL argument"); return PP_ERR_ARG; }
    if (nz < 1 || npix < 0) { set_error("pp_fz_to_df: nz >= 1 and npix >= 0 required"); return PP_ERR_SHAPE; }
    if (npix > 0 && (!fz || !df)) { set_error("pp_fz_to_df: NULL argument"); return PP_ERR_ARG; }
    if (!finite_pos(dz) || !finite_pos(dfp->k) || !isfinite(dfp->f0)) { set_error("pp_fz_to_df: invalid parameters"); return PP_ERR_ARG; }
    const int m = df_half_width(dfp->A_pp, dz);
    if (m < 0) { set_error("pp_fz_to_df: invalid amplitude"); return PP_ERR_ARG; }
    if (m > kMaxDfHalfWidth) { set_error("pp_fz_to_df: df stencil wider than 63 taps"); return PP_ERR_UNSUPPORTED; }
    if (nz < 2 * m + 1) { set_error("pp_fz_to_df: fewer heights than the df stencil"); return PP_ERR_SHAPE; }
    DfLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.fz = fz; L.df = df; L.nz = nz; L.npix = npix; L.m = m;
    if (npix == 0) return PP_OK;
    df_stencil(dfp->A_pp, dz, dfp->k, dfp->f0, m, L.coef);
    return cuda_status(launch_fz_to_df(L, (cudaStream_t)stream), "pp_fz_to_df launch");
}

size_t pp_backward_workspace(const pp_grid* grid) {
    GridMap m;
    std::string why;
    if (!make_grid_map(grid, &m, &why)) return 0;
    return kBwdHeader + (size_t)m.stored_nodes * (m.interp ? 4 : 16);
}

}  // extern "C"

namespace pp {

// Every check of the adjoint's arguments except those of the workspace, in the order pp_backward
// has always made them (so that pp_backward and pp_backward_noalloc return the same status for
// the same arguments); on success fills *Lp (all but the workspace fields) and the grid adjoint's
// byte count *adj_bytes.
pp_status backward_prepare(const std::string& who, const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                           const float* ff, const pp_scan* scan, const pp_tip* tip, const pp_df* dfp,
                           const float* pos, const float* g_df, const pp_grads* grads, BwdLaunch* Lp,
                           size_t* adj_bytes_out) {
    if (!atoms || !probe || !grid || !ff || !scan || !tip || !dfp || !pos || !g_df || !grads) {
        set_error(who + ": NULL argument");
        return PP_ERR_ARG;
    }
    if (atoms->n < 0) { set_error(who + ": atoms->n < 0"); return PP_ERR_ARG; }
    if (atoms->n > 0 && (!atoms->x || !atoms->y || !atoms->z || !atoms->R || !atoms->eps || !atoms->q ||
                         !grads->x || !grads->y || !grads->z || !grads->q || !grads->R || !grads->eps)) {
        set_error(who + ": NULL atom or gradient array");
        return PP_ERR_ARG;
    }
    if (!grads->tip) { set_error(who + ": NULL tip gradient"); return PP_ERR_ARG; }
    if (!aligned16(ff)) { set_error(who + ": ff must be 16-byte aligned"); return PP_ERR_ARG; }
    if (!(probe->core_frac > 0.f && probe->core_frac < 1.f) || !(probe->eps_pp >= 0.f) || !(probe->coul_rc >= 0.f) ||
        (probe->min_image != 0 && probe->min_image != 1) || !isfinite(probe->Q) || !isfinite(probe->Qzz)) {
        set_error(who + ": invalid probe parameters");
        return PP_ERR_ARG;
    }
    GridMap map;
    std::string why;
    if (!make_grid_map(grid, &map, &why)) { set_error(who + ": " + why); return PP_ERR_SHAPE; }
    if (scan->nx < 1 || scan->ny < 1 || scan->nz < 1 ||
        (int64_t)scan->nx * scan->ny * scan->nz * 3 >= (int64_t(1) << 31)) {
        set_error(who + ": invalid scan size");
        return PP_ERR_SHAPE;
    }
    if (!finite_pos(scan->dz)) { set_error(who + ": invalid scan geometry"); return PP_ERR_ARG; }
    pp_fire dummy = {1, 1.f, 1.f, 1.f, 1.f, 1.f, 0.f, 1.f, 1.f, 0, 0};
    if (!check_tip_fire(tip, &dummy, &why)) { set_error(who + ": " + why); return PP_ERR_ARG; }
    if (!finite_pos(dfp->k) || !isfinite(dfp->f0)) { set_error(who + ": invalid df parameters"); return PP_ERR_ARG; }
    const int m = df_half_width(dfp->A_pp, scan->dz);
    if (m < 0) { set_error(who + ": invalid df amplitude"); return PP_ERR_ARG; }
    if (m > kMaxDfHalfWidth) { set_error(who + ": df stencil wider than 63 taps"); return PP_ERR_UNSUPPORTED; }
    if (scan->nz < 2 * m + 1) { set_error(who + ": fewer heights than the df stencil"); return PP_ERR_SHAPE; }
    const size_t adj_bytes = (size_t)map.stored_nodes * (map.interp ? 4 : 16);
    *adj_bytes_out = adj_bytes;
    BwdLaunch& L = *Lp;
    std::memset(&L, 0, sizeof(L));
    L.ax = atoms->x; L.ay = atoms->y; L.az = atoms->z; L.aR = atoms->R; L.aeps = atoms->eps; L.aq = atoms->q;
    L.n = atoms->n;
    L.R_pp = probe->R_pp; L.eps_pp = probe->eps_pp;
    L.kQ = (float)(kCoulomb * (double)probe->Q);
    L.ke = (float)kCoulomb;
    L.Q = probe->Q;
    L.Qzz = probe->Qzz;
    L.kQzz = (float)(0.5 * kCoulomb * (double)probe->Qzz);
    L.core_frac = probe->core_frac; L.coul_rc = probe->coul_rc; L.min_image = probe->min_image;
    L.Lx = grid->nx * grid->dx; L.Ly = grid->ny * grid->dy;
    L.ff = map.interp ? nullptr : reinterpret_cast<const float4*>(ff);
    L.ffE = map.interp ? ff : nullptr;
    L.map = map;
    L.layout = grid->layout;
    L.x0 = grid->x0; L.y0 = grid->y0; L.z0 = grid->z0; L.dx = grid->dx; L.dy = grid->dy; L.dz = grid->dz;
    L.inv_dx = 1.f / grid->dx; L.inv_dy = 1.f / grid->dy; L.inv_dz = 1.f / grid->dz;
    L.gx0s = (float)(-(double)grid->x0 / grid->dx);
    L.gy0s = (float)(-(double)grid->y0 / grid->dy);
    L.gz0s = (float)(-(double)grid->z0 / grid->dz);
    L.periodic_xy = grid->periodic_xy;
    L.snx = scan->nx; L.sny = scan->ny; L.snz = scan->nz;
    L.sx0 = scan->x0; L.sy0 = scan->y0; L.spx = scan->px; L.spy = scan->py; L.z_top = scan->z_top; L.sdz = scan->dz;
    L.kx = (float)(tip->kx * kNmToEvA2); L.ky = (float)(tip->ky * kNmToEvA2); L.kR = (float)(tip->kR * kNmToEvA2);
    L.R0 = tip->R0; L.d0x = tip->d0x; L.d0y = tip->d0y;
    L.d0z = (float)(-sqrt((double)tip->R0 * tip->R0 - (double)tip->d0x * tip->d0x - (double)tip->d0y * tip->d0y));
    L.R0sq = (float)((double)tip->R0 * tip->R0);
    L.c0 = (float)((double)L.d0x * L.d0x + (double)L.d0y * L.d0y + (double)L.d0z * L.d0z - (double)tip->R0 * tip->R0);
    L.nm = (float)kNmToEvA2;
    L.m = m;
    L.nzo = scan->nz - 2 * m;
    df_stencil(dfp->A_pp, scan->dz, dfp->k, dfp->f0, m, L.coef);
    L.pos = pos;
    L.g_df = g_df;
    L.gx = grads->x; L.gy = grads->y; L.gz = grads->z; L.gq = grads->q; L.gR = grads->R; L.geps = grads->eps;
    L.gtip = grads->tip;
    return PP_OK;
}

// Points the prepared launch at the workspace ws (kBwdHeader + adj_bytes bytes, 16-byte aligned),
// clears the grid adjoint and enqueues the adjoint kernels.
pp_status backward_launch(const std::string& who, BwdLaunch& L, void* ws, size_t adj_bytes, cudaStream_t s) {
    L.slab = reinterpret_cast<int*>(ws);
    L.qsum = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + 16);
    L.gbar = L.map.interp ? nullptr : reinterpret_cast<float4*>(reinterpret_cast<char*>(ws) + kBwdHeader);
    L.gbarE = L.map.interp ? reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + kBwdHeader) : nullptr;
    L.qsumd = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + 32);
    pp_status st = cuda_status(cudaMemsetAsync(reinterpret_cast<char*>(ws) + kBwdHeader, 0, adj_bytes, s),
                               (who + " memset").c_str());
    if (st != PP_OK) return st;
    return cuda_status(launch_backward(L, s), (who + " launch").c_str());
}

}  // namespace pp

extern "C" {

pp_status pp_backward(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid, const float* ff,
                      const pp_scan* scan, const pp_tip* tip, const pp_df* dfp, const float* pos, const float* g_df,
                      const pp_grads* grads, void* ws, size_t ws_bytes, pp_stream stream) {
    Range range("pp_backward");
    g_error.clear();
    if (!ws) { set_error("pp_backward: NULL argument"); return PP_ERR_ARG; }
    if (!aligned16(ws)) { set_error("pp_backward: ws must be 16-byte aligned"); return PP_ERR_ARG; }
    BwdLaunch L;
    size_t adj_bytes = 0;
    const pp_status st = backward_prepare("pp_backward", atoms, probe, grid, ff, scan, tip, dfp, pos, g_df, grads, &L,
                                          &adj_bytes);
    if (st != PP_OK) return st;
    const size_t need = kBwdHeader + adj_bytes;
    if (ws_bytes < need) {
        set_error("pp_backward: workspace too small (need " + std::to_string(need) + " bytes)");
        return PP_ERR_CAPACITY;
    }
    return backward_launch("pp_backward", L, ws, adj_bytes, (cudaStream_t)stream);
}

size_t pp_batch_workspace(int nmol) { return batch_workspace_bytes(nmol); }

pp_status pp_batch_run(const pp_mol_desc* descs, int nmol, const pp_batch_params* bp, const pp_atoms* atoms,
                       float* ff, float* pos, float* fz, int* iters, float* df, void* ws, size_t ws_bytes,
                       pp_stream stream) {
    Range range("pp_batch_run");
    g_error.clear();
    if (!descs || !bp || !atoms || !ff || !fz || !df || !ws) { set_error("pp_batch_run: NULL argument"); return PP_ERR_ARG; }
    if (nmol < 1 || nmol > (1 << 24)) { set_error("pp_batch_run: nmol must be in [1, 2^24]"); return PP_ERR_SHAPE; }
    if (atoms->n < 0 || (atoms->n > 0 && (!atoms->x || !atoms->y || !atoms->z || !atoms->R || !atoms->eps || !atoms->q))) {
        set_error("pp_batch_run: invalid packed atoms");
        return PP_ERR_ARG;
    }
    if (!aligned16(ff) || !aligned16(ws)) { set_error("pp_batch_run: ff and ws must be 16-byte aligned"); return PP_ERR_ARG; }
    const pp_probe* probe = &bp->probe;
    if (!(probe->core_frac > 0.f && probe->core_frac < 1.f) || !(probe->eps_pp >= 0.f) || !(probe->coul_rc >= 0.f) ||
        !isfinite(probe->R_pp) || !isfinite(probe->Q) || !isfinite(probe->Qzz) ||
        (probe->min_image != 0 && probe->min_image != 1)) {
        set_error("pp_batch_run: invalid probe parameters");
        return PP_ERR_ARG;
    }
    std::string why;
    if (!check_tip_fire(&bp->tip, &bp->fire, &why)) { set_error("pp_batch_run: " + why); return PP_ERR_ARG; }
    if (bp->fire.polish != 0) { set_error("pp_batch_run: the Newton polish is not available in batches"); return PP_ERR_UNSUPPORTED; }
    {
        auto width_ok = [](int w) { return w == 0 || w == 4 || w == 8 || w == 16; };
        if (!width_ok(bp->ff_tile_w) || !width_ok(bp->relax_tile_w) ||
            !(bp->ff_zpt == 0 || bp->ff_zpt == 4 || bp->ff_zpt == 8)) {
            set_error("pp_batch_run: tile widths must be 0, 4, 8 or 16 and ff_zpt 0, 4 or 8");
            return PP_ERR_ARG;
        }
    }
    if (!finite_pos(bp->scan_dz) || (bp->periodic_xy != 0 && bp->periodic_xy != 1)) {
        set_error("pp_batch_run: invalid scan_dz or periodic_xy");
        return PP_ERR_ARG;
    }
    if (bp->ff_capacity < 0 || bp->out_capacity < 0 || bp->df_capacity < 0 || bp->n_atoms_total < 0 ||
        bp->n_atoms_total > atoms->n || bp->ctas < 0 || bp->spin_limit < 0 || bp->wait_extra < 0 ||
        (bp->ff_forces_only != 0 && bp->ff_forces_only != 1)) {
        set_error("pp_batch_run: invalid capacities or launch settings");
        return PP_ERR_ARG;
    }
    if (!finite_pos(bp->df.k) || !isfinite(bp->df.f0)) { set_error("pp_batch_run: invalid df parameters"); return PP_ERR_ARG; }
    const int m = df_half_width(bp->df.A_pp, bp->scan_dz);
    if (m < 0) { set_error("pp_batch_run: invalid df amplitude"); return PP_ERR_ARG; }
    if (m > kMaxDfHalfWidth) { set_error("pp_batch_run: df stencil wider than 63 taps"); return PP_ERR_UNSUPPORTED; }
    const size_t need = batch_workspace_bytes(nmol);
    if (ws_bytes < need) {
        set_error("pp_batch_run: workspace too small (need " + std::to_string(need) + " bytes)");
        return PP_ERR_CAPACITY;
    }
    BatchArgs A;
    std::memset(&A, 0, sizeof(A));
    A.descs = descs; A.nmol = nmol; A.params = *bp; A.atoms = *atoms;
    A.ff = ff; A.pos = pos; A.fz = fz; A.df = df; A.iters = iters; A.ws = ws;
    A.df_m = m;
    df_stencil(bp->df.A_pp, bp->scan_dz, bp->df.k, bp->df.f0, m, A.coef);
    return cuda_status(launch_batch(A, (cudaStream_t)stream), "pp_batch_run launch");
}

pp_status pp_batch_status(const void* ws, int* flags, pp_stream stream) {
    g_error.clear();
    if (!ws || !flags) { set_error("pp_batch_status: NULL argument"); return PP_ERR_ARG; }
    int st = 0;
    cudaStream_t s = (cudaStream_t)stream;
    pp_status r = cuda_status(cudaMemcpyAsync(&st, reinterpret_cast<const char*>(ws) + 8, sizeof(int),
                                              cudaMemcpyDeviceToHost, s), "pp_batch_status copy");
    if (r != PP_OK) return r;
    r = cuda_status(cudaStreamSynchronize(s), "pp_batch_status sync");
    if (r != PP_OK) return r;
    *flags = st;
    if (st & PP_BATCH_TIMEOUT) { set_error("pp_batch_run: a bounded wait ran out"); return PP_ERR_TIMEOUT; }
    if (st & PP_BATCH_BAD_DESC) { set_error("pp_batch_run: invalid descriptor(s) skipped"); return PP_ERR_CAPACITY; }
    return PP_OK;
}

pp_status pp_iets(const float* ff, const pp_grid* grid, const pp_scan* scan, const pp_tip* tip, const float* pos,
                  float mass_amu, float* eig, float* hw, pp_stream stream) {
    Range range("pp_iets");
    g_error.clear();
    if (!ff || !grid || !scan || !tip || !pos || !eig) { set_error("pp_iets: NULL argument"); return PP_ERR_ARG; }
    if (!aligned16(ff)) { set_error("pp_iets: ff must be 16-byte aligned"); return PP_ERR_ARG; }
    if (!finite_pos(mass_amu)) { set_error("pp_iets: mass must be > 0"); return PP_ERR_ARG; }
    GridMap map;
    std::string why;
    if (!make_grid_map(grid, &map, &why)) { set_error("pp_iets: " + why); return PP_ERR_SHAPE; }

    if (scan->nx < 1 || scan->ny < 1 || scan->nz < 1 ||
        (int64_t)scan->nx * scan->ny * scan->nz * 3 >= (int64_t(1) << 31)) {
        set_error("pp_iets: invalid scan size");
        return PP_ERR_SHAPE;
    }
    if (!finite_pos(scan->dz)) { set_error("pp_iets: invalid scan geometry"); return PP_ERR_ARG; }
    pp_fire dummy = {1, 1.f, 1.f, 1.f, 1.f, 1.f, 0.f, 1.f, 1.f, 0, 0};
    if (!check_tip_fire(tip, &dummy, &why)) { set_error("pp_iets: " + why); return PP_ERR_ARG; }
    IetsLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.ff = map.interp ? nullptr : reinterpret_cast<const float4*>(ff);
    L.ffE = map.interp ? ff : nullptr;
    L.map = map;
    L.layout = grid->layout;
    L.inv_dx = 1.f / grid->dx; L.inv_dy = 1.f / grid->dy; L.inv_dz = 1.f / grid->dz;
    L.gx0s = (float)(-(double)grid->x0 / grid->dx);
    L.gy0s = (float)(-(double)grid->y0 / grid->dy);
    L.gz0s = (float)(-(double)grid->z0 / grid->dz);
    L.periodic_xy = grid->periodic_xy;
    L.snx = scan->nx; L.sny = scan->ny; L.snz = scan->nz;
    L.sx0 = scan->x0; L.sy0 = scan->y0; L.spx = scan->px; L.spy = scan->py; L.z_top = scan->z_top; L.sdz = scan->dz;
    L.kx = (float)(tip->kx * kNmToEvA2); L.ky = (float)(tip->ky * kNmToEvA2); L.kR = (float)(tip->kR * kNmToEvA2);
    L.R0 = tip->R0; L.d0x = tip->d0x; L.d0y = tip->d0y;
    L.d0z = (float)(-sqrt((double)tip->R0 * tip->R0 - (double)tip->d0x * tip->d0x - (double)tip->d0y * tip->d0y));
    L.R0sq = (float)((double)tip->R0 * tip->R0);
    L.c0 = (float)((double)L.d0x * L.d0x + (double)L.d0y * L.d0y + (double)L.d0z * L.d0z - (double)tip->R0 * tip->R0);
    L.pos = pos; L.eig = eig; L.hw = hw;
    // hbar sqrt(1 eV/A^2 / (m amu)) in meV, from SI constants
    const double hbar = 1.054571817e-34, ev = 1.602176634e-19, amu = 1.66053906660e-27;
    L.hw_unit = (float)(hbar * sqrt(ev / 1e-20 / (amu * mass_amu)) / ev * 1e3);
    return cuda_status(launch_iets(L, (cudaStream_t)stream), "pp_iets launch");
}

pp_status pp_ff_convert(const float* src, const pp_grid* src_grid, float* dst, const pp_grid* dst_grid,
                        pp_stream stream) {
    Range range("pp_ff_convert");
    g_error.clear();
    if (!src || !dst || !src_grid || !dst_grid) { set_error("pp_ff_convert: NULL argument"); return PP_ERR_ARG; }
    if (!aligned16(src) || !aligned16(dst)) { set_error("pp_ff_convert: buffers must be 16-byte aligned"); return PP_ERR_ARG; }
    GridMap sm, dm;
    std::string why;
    if (!make_grid_map(src_grid, &sm, &why) || !make_grid_map(dst_grid, &dm, &why)) {
        set_error("pp_ff_convert: " + why);
        return PP_ERR_SHAPE;
    }
    if (sm.interp || dm.interp) { set_error("pp_ff_convert: tricubic (energy) grids are not supported"); return PP_ERR_UNSUPPORTED; }
    if (sm.nx != dm.nx || sm.ny != dm.ny || sm.nz != dm.nz) { set_error("pp_ff_convert: node counts differ"); return PP_ERR_SHAPE; }
    cudaStream_t s = (cudaStream_t)stream;
    if (dm.stored_nodes > (int64_t)dm.nx * dm.ny * dm.nz) {
        pp_status st = cuda_status(cudaMemsetAsync(dst, 0, (size_t)dm.stored_nodes * 16, s), "pp_ff_convert memset");
        if (st != PP_OK) return st;
    }
    return cuda_status(launch_ff_convert(reinterpret_cast<const float4*>(src), sm, reinterpret_cast<float4*>(dst), dm, s),
                       "pp_ff_convert launch");
}

}  // extern "C"

static bool pow2_fft(int n) { return n >= 2 && n <= 1024 && (n & (n - 1)) == 0; }

static bool fft_grid(const pp_grid* grid, GridMap* map, std::string* why, pp_status* st) {
    if (!make_grid_map(grid, map, why)) { *st = PP_ERR_SHAPE; return false; }
    if (grid->layout != 0 || map->interp != 0) {
        *why = "needs a linear force grid (layout 0, interp 0)";
        *st = PP_ERR_UNSUPPORTED;
        return false;
    }
    if (!pow2_fft(grid->nx) || !pow2_fft(grid->ny) || !pow2_fft(grid->nz)) {
        *why = "grid sizes must be powers of two in [2, 1024]";
        *st = PP_ERR_UNSUPPORTED;
        return false;
    }
    return true;
}

size_t pp_fft_workspace(const pp_grid* grid) {
    GridMap m;
    std::string why;
    pp_status st;
    if (!grid || !fft_grid(grid, &m, &why, &st)) return 0;
    return fft_workspace_bytes(grid->nx, grid->ny, grid->nz);
}

pp_status pp_fft_correlate(const float* f, const float* g, const pp_grid* grid, float scale, float power,
                           int accumulate, float* ff, void* ws, size_t ws_bytes, pp_stream stream) {
    Range range("pp_fft_correlate");
    g_error.clear();
    if (!f || !g || !grid || !ff || !ws) { set_error("pp_fft_correlate: NULL argument"); return PP_ERR_ARG; }
    if (!isfinite(scale) || !(power > 0.f) || !isfinite(power) || (accumulate != 0 && accumulate != 1)) {
        set_error("pp_fft_correlate: scale must be finite, power > 0, accumulate 0 or 1");
        return PP_ERR_ARG;
    }
    if (!aligned16(f) || !aligned16(g) || !aligned16(ff) || !aligned16(ws)) {
        set_error("pp_fft_correlate: f, g, ff and ws must be 16-byte aligned");
        return PP_ERR_ARG;
    }
    GridMap map;
    std::string why;
    pp_status st = PP_OK;
    if (!fft_grid(grid, &map, &why, &st)) { set_error("pp_fft_correlate: " + why); return st; }
    const size_t need = fft_workspace_bytes(grid->nx, grid->ny, grid->nz);
    if (ws_bytes < need) {
        set_error("pp_fft_correlate: workspace too small (need " + std::to_string(need) + " bytes)");
        return PP_ERR_CAPACITY;
    }
    FftLaunch L;
    L.f = f; L.g = g;
    L.ff = reinterpret_cast<float4*>(ff);
    L.ws = ws;
    L.nx = grid->nx; L.ny = grid->ny; L.nz = grid->nz;
    L.dx = grid->dx; L.dy = grid->dy; L.dz = grid->dz;
    L.scale = scale; L.power = power; L.accumulate = accumulate;
    return cuda_status(launch_fft_correlate(L, (cudaStream_t)stream), "pp_fft_correlate launch");
}
