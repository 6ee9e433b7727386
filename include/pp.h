/*
 * pp.h -- C ABI of the GB300 (sm_103a) Probe-Particle Model hot path.
 *
 * Three stages of the paper's two-step scheme (Sec. 5.1.1) plus its tip
 * readout and frequency shift (Sec. 2.1), each a CUDA kernel:
 *
 *   pp_make_ff     force-field grid from Lennard-Jones (Eq. LJ, mixing rules
 *                  R_iPP = R_i + R_PP, e_iPP = sqrt(e_i e_PP)) and point-charge
 *                  Coulomb (Eq. point charges) pair sums, F = -grad E (Sec. 2.2);
 *   pp_relax_scan  relaxed tip scan: per pixel, heights from the top down, FIRE
 *                  on F_PP = F_T + F_S (Eq. F_PP, Eq. F_tip) with F_S trilinearly
 *                  interpolated from the grid (Sec. 5.1.1 step 2), warm-started
 *                  from the previous height; output Fz = -F^T_{R,z} (Sec. 2.1);
 *   pp_fz_to_df    Fz(z) -> frequency shift df by Eq. df (Giessibl kernel).
 *
 * Conventions shared by every entry point
 *   Units      Angstrom, eV, elementary charge; spring constants and the
 *              cantilever stiffness in N/m; f0 in Hz; df in Hz.
 *   Memory     Every array argument is DEVICE memory owned by the caller,
 *              unless its comment says host.  The library allocates nothing
 *              and keeps no pointer after the call returns (its kernels may
 *              still be running on `stream`).
 *   Execution  All work is enqueued on `stream` (a cudaStream_t; NULL = the
 *              legacy default stream).  No call synchronises the host except
 *              pp_batch_status, which reads a status word back.
 *   Errors     Every call returns a pp_status; nothing throws across the ABI.
 *              Shapes, sizes and NULL pointers are checked on the host before
 *              any launch; a failed check launches nothing.  PP_ERR_CUDA means
 *              a launch failed (the CUDA error string is in pp_last_error()).
 *              Device data is not scanned.
 *   Threads    Calls are thread-safe; pp_last_error() is per host thread.
 *   Device     The current CUDA device of the calling thread is used.
 */
#ifndef PP_H_
#define PP_H_

#include <stddef.h>

#if defined(__GNUC__)
#define PP_API __attribute__((visibility("default")))
#else
#define PP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PP_OK = 0,
    PP_ERR_ARG = 1,         /* NULL pointer or a parameter out of range      */
    PP_ERR_SHAPE = 2,       /* inconsistent or unsupported sizes             */
    PP_ERR_CUDA = 3,        /* a CUDA launch or call failed                  */
    PP_ERR_CAPACITY = 4,    /* a caller buffer (workspace) is too small      */
    PP_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up            */
    PP_ERR_UNSUPPORTED = 6  /* a valid request this build does not implement */
} pp_status;

typedef void* pp_stream; /* cudaStream_t */

/* Sample atoms, structure of arrays, n >= 0.  Device pointers to n floats. */
typedef struct {
    int n;
    const float *x, *y, *z; /* positions, A                                  */
    const float *R;         /* LJ radius R_i, A (mixing: R_iPP = R_i + R_PP)  */
    const float *eps;       /* LJ well depth e_i >= 0, eV (e_iPP = sqrt(e_i e_PP)) */
    const float *q;         /* point charge q_i, e                           */
} pp_atoms;

/* Probe particle.  The pair force is floored per pair at
 * r^2 >= (core_frac * R_iPP)^2 (displacement unscaled) so that no value is
 * infinite; coul_rc > 0 selects a shifted-force Coulomb truncated at coul_rc
 * (F = k_e Q q (1/r^2 - 1/rc^2) r_hat for r < rc, 0 beyond); min_image = 1
 * sums each atom's nearest lateral periodic image, period = grid extent
 * (nx*dx, ny*dy).
 * Qzz != 0 adds the CO tip's quadrupolar charge distribution (Secs. 2.2.3,
 * 2.2.5; the paper's point-charge simulations use -0.05 e*A^2): an axial
 * point quadrupole of second moment Qzz = sum q_k z_k^2 (no net charge or
 * dipole) riding on the PP without rotation, with energy (Qzz/2) d^2V/dz^2 in
 * the sample's point-charge potential, i.e. per atom, with delta = r - r_i,
 *   E = (k_e q_i Qzz / 2) (3 dz^2 - r^2) / r^5,
 *   F = (k_e q_i Qzz / 2) [(15 dz^2/r^7 - 3/r^5) delta - (6 dz/r^5) z_hat];
 * r is the floored distance; with coul_rc > 0 the term is cut off (not
 * shifted) at r >= coul_rc. */
typedef struct {
    float R_pp, eps_pp; /* A, eV                       */
    float Q;            /* probe charge, e             */
    float coul_rc;      /* A; 0 = plain Coulomb        */
    int min_image;      /* 0 or 1                      */
    float core_frac;    /* floor radius / R_iPP, in (0, 1) */
    float Qzz;          /* tip quadrupole, e*A^2; 0 = none */
} pp_probe;

/* Regular force-field grid: node (i,j,k) sits at (x0+i*dx, y0+j*dy, z0+k*dz).
 * Interpolation wraps i,j periodically when periodic_xy = 1, else clamps; it
 * always clamps in z (cell index in [0, nz-2], fraction in [0,1]).
 * layout 0: node (i,j,k) at index (k*ny + j)*nx + i.
 * layout 1: bricks of bx*by*bz nodes (each a power of two, 1..16), bricks in
 *           x-fastest order, nodes x-fastest inside a brick; dimensions are
 *           padded up to whole bricks.  pp_ff_floats() gives the size.
 * interp 0: every node holds 4 floats (Fx, Fy, Fz, E) in eV/A and eV (E = 0
 *           when assembled with ff_forces_only) and the scan interpolates the
 *           forces trilinearly (Sec. 5.1.1 step 2).
 * interp 1: every node holds the energy E only (eV), layout 0; the scan
 *           interpolates E tricubically (the paper's suggestion for larger
 *           spacings without stored forces) and takes F = -grad of the
 *           interpolant: along each axis the cubic convolution (Catmull-Rom)
 *           weights of nodes i-1..i+2 at fraction t,
 *           ((-t^3+2t^2-t), (3t^3-5t^2+2), (-3t^3+4t^2+t), (t^3-t^2)) / 2,
 *           stencil nodes wrapping like the cell (periodic) or clamped into
 *           the grid (z, and x,y when not periodic).
 * Each axis holds 2..2^22 nodes.  The buffer must be 16-byte aligned. */
typedef struct {
    int nx, ny, nz;
    float x0, y0, z0;
    float dx, dy, dz;
    int periodic_xy;
    int layout;
    int bx, by, bz;
    int interp;  /* 0 trilinear forces, 1 tricubic energy */
} pp_grid;

/* Tip springs of Eq. F_tip, with d = r_PP - r_TIP and
 * d0 = (d0x, d0y, -sqrt(R0^2 - d0x^2 - d0y^2)) (the PP hangs below the tip):
 *   F_T = -kR (|d| - R0) d/|d| - (kx (d_x - d0x), ky (d_y - d0y), 0). */
typedef struct {
    float kx, ky, kR; /* N/m */
    float R0;         /* A   */
    float d0x, d0y;   /* A   */
} pp_tip;

/* Tip anchors: pixel (i,j) at height index k is at
 * (x0 + i*px, y0 + j*py, z_top - k*dz), k = 0..nz-1 (approaching the sample). */
typedef struct {
    int nx, ny, nz;
    float x0, y0, px, py;
    float z_top, dz;
} pp_scan;

/* FIRE (Bitzek et al. 2006), semi-implicit Euler.  Per height: v = 0,
 * dt = dt0, alpha = alpha0.  Each iteration evaluates G = F_PP and stops when
 * |G| < ftol (eV/A) or after max_iter position updates; from the second
 * iteration on, G.v > 0 mixes v <- (1-alpha) v + alpha |v| G/|G| and, after
 * more than n_min such steps in a row, sets dt <- min(dt*f_inc, dt_max),
 * alpha <- alpha*f_alpha; G.v <= 0 sets v = 0, dt <- dt*f_dec,
 * alpha <- alpha0.  Then v += dt G/mass, p += dt v.
 * polish (0..16, 0 = off) adds, at every height where FIRE stopped below
 * ftol, up to that many Newton steps p <- p - J^{-1} G with the exact
 * Jacobian J = dG/dp (tip springs + the interpolant's), each kept only if it
 * lowers |G|: the relaxed point then sits at the equilibrium G = 0 to the
 * FP32 resolution of G, as the implicit adjoint (pp_backward) assumes.  The
 * iteration counts are FIRE's alone.  pp_batch_run requires polish = 0. */
typedef struct {
    int max_iter;
    float ftol, dt0, dt_max, f_inc, f_dec, alpha0, f_alpha, mass;
    int n_min;
    int polish;
} pp_fire;

/* Cantilever of Eq. df: A_pp is the PEAK-TO-PEAK amplitude (A), k the
 * stiffness (N/m), f0 the base frequency (Hz). */
typedef struct {
    float A_pp, k, f0;
} pp_df;

/* Number of floats of a force-field buffer for `grid` (4 per stored node,
 * brick padding included; 1 per node for interp = 1); 0 if the grid is invalid. */
PP_API size_t pp_ff_floats(const pp_grid* grid);

/* Half-width in samples of the df stencil: m = ceil(A_pp/2 / dz).  A scan of
 * nz heights yields nz - 2m df values per pixel (centre labelling); -1 if the
 * arguments are invalid. */
PP_API int pp_df_margin(float A_pp, float dz);

/* FF grid assembly (Sec. 5.1.1 step 1; Eqs. LJ and point charges; Sec. 2.2).
 * Writes all nodes of `ff` (pp_ff_floats(grid) floats, padding nodes
 * included) with (Fx, Fy, Fz, E) = sum over atoms of the pair force and
 * energy at the node, or E alone when grid->interp = 1 (then the launch
 * shape is fixed and tuning is ignored).  atoms->n may be 0 (all zeros).  Errors: PP_ERR_ARG
 * (NULL, core_frac outside (0,1), negative eps), PP_ERR_SHAPE (nx, ny, nz < 2,
 * spacing <= 0, brick not a power of two), PP_ERR_CUDA. */
PP_API pp_status pp_make_ff(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                     float* ff, pp_stream stream);

/* pp_make_ff with the point-charge electrostatics kept apart, for scanning the
 * probe charge Q without reassembling the grid: `ff` gets the Lennard-Jones
 * terms (and the tip quadrupole when probe->Qzz != 0), `ff_el` the Coulomb
 * field of the sample's point charges per unit probe charge (Eq. point
 * charges with Q = 1; shifted-force when coul_rc > 0); probe->Q is not used.
 * F = ff + Q ff_el is the grid pp_make_ff writes for charge Q (up to FP32
 * rounding of the two sums); pp_ff_combine forms it.  Both buffers hold
 * pp_ff_floats(grid) floats in the grid's layout (energies only when
 * grid->interp = 1), 16-byte aligned and distinct.  Launch shape fixed (8
 * z-nodes per thread).  Errors as pp_make_ff. */
PP_API pp_status pp_make_ff_split(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                                  float* ff, float* ff_el, pp_stream stream);

/* out = ff + Q ff_el over the pp_ff_floats(grid) floats of a split grid (any
 * layout or interp; padding included), i.e. the grid for probe charge Q.
 * `out` may be `ff` itself.  HBM-bound elementwise pass (12 bytes moved per
 * float).  Errors: PP_ERR_ARG (NULL, unaligned, Q not finite), PP_ERR_SHAPE,
 * PP_ERR_CUDA. */
PP_API pp_status pp_ff_combine(const float* ff, const float* ff_el, float Q, const pp_grid* grid, float* out,
                               pp_stream stream);

/* Options of pp_make_ff_tuned.  ff_zpt (the launch shape, picked by the
 * autotuner) is the number of consecutive z-nodes each thread accumulates, 4,
 * 8 or 16; 0 = 8.  ff_forces_only = 1 skips the energy sums of an interp = 0
 * grid and writes 0 in every E slot: the scan reads only the forces (Sec.
 * 5.1.1 step 2), and the forces are bit for bit those of ff_forces_only = 0
 * (the default, E written). */
typedef struct {
    int ff_zpt;
    int ff_forces_only;
} pp_tuning;

/* pp_make_ff with an explicit launch shape; the forces written are the same
 * sums (identical arithmetic per node), and so are the energies unless
 * ff_forces_only.  Errors as pp_make_ff, plus PP_ERR_ARG for an unsupported
 * ff_zpt, an ff_forces_only other than 0 or 1, or ff_forces_only on an
 * interp = 1 grid (which holds nothing but E).  tuning may be NULL. */
PP_API pp_status pp_make_ff_tuned(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                                  float* ff, const pp_tuning* tuning, pp_stream stream);

/* pp_make_ff_tuned restricted to the node layers k_begin <= k < k_end (every
 * x and y): those nodes get exactly the values pp_make_ff_tuned writes there
 * (each node's sums do not depend on which nodes share its launch); every
 * other node of ff, and the padding nodes of a bricked layout (which
 * pp_make_ff zeroes), are left as they are.  The paper has no counterpart: it
 * lets a caller assemble the layers a scan reads first and the rest on
 * another stream while the scan runs (the grid is still complete when both
 * have finished).  tuning may be NULL.  Errors as pp_make_ff_tuned, plus
 * PP_ERR_ARG unless 0 <= k_begin < k_end <= nz. */
PP_API pp_status pp_make_ff_layers(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                                   float* ff, const pp_tuning* tuning, int k_begin, int k_end,
                                   pp_stream stream);

/* Relaxed tip scan (Sec. 5.1.1 step 2; Eqs. F_PP, F_tip; Sec. 2.1 readout).
 * F_S comes from the grid by trilinear force interpolation, or by the
 * gradient of the tricubic energy interpolant when grid->interp = 1.
 * One thread per pixel walks the heights k = 0..nz-1: start p = anchor + d0
 * at k = 0 and p = p*(k-1) - dz z_hat after that, relax by FIRE, write
 *   pos[((k*ny + j)*nx + i)*3 + c]  relaxed PP position (nullable),
 *   fz[(k*ny + j)*nx + i]           Fz = kR (|d| - R0) d_z/|d|, eV/A,
 *   iters[(k*ny + j)*nx + i]        FIRE position updates; == max_iter when
 *                                   |G| < ftol was not reached (nullable).
 * Non-convergence is reported through iters only.  When fused_df and df are
 * both non-NULL the same launch also writes df[(c*ny + j)*nx + i],
 * c = 0..nz-2m-1, exactly as pp_fz_to_df would.  Errors: PP_ERR_ARG,
 * PP_ERR_SHAPE (grid invalid, scan sizes < 1, nz < 2m+1 with fused df),
 * PP_ERR_UNSUPPORTED (m > 31), PP_ERR_CUDA. */
PP_API pp_status pp_relax_scan(const float* ff, const pp_grid* grid, const pp_scan* scan,
                        const pp_tip* tip, const pp_fire* fire,
                        float* pos, float* fz, int* iters,
                        const pp_df* fused_df, float* df, pp_stream stream);

/* Options of pp_relax_scan_ex (neither changes an output bit; the paper has
 * no counterpart to either).
 *   zspan  DEVICE int[2] (4-byte aligned, caller-owned) or NULL: receives the
 *          lowest and highest node layer k the scan's interpolations read,
 *          over every FIRE iteration and Newton step of every pixel
 *          (trilinear: the two layers of each cell used; tricubic: the four
 *          stencil layers, clamped to the grid); the call initialises it on
 *          the stream.  A scan whose layers lie inside those already assembled
 *          read nothing else: the check a caller makes after overlapping the
 *          scan with pp_make_ff_layers of the other layers (and, if it fails,
 *          runs the scan again on the complete grid).
 *   plan   DEVICE pixel-to-warp plan from pp_relax_plan for a scan of the same
 *          nx and ny, built with plan_k and plan_lanes, or NULL: the plan's
 *          pixels run in warps of plan_lanes lanes ahead of the 8x4 pixel
 *          tiles, which skip them.  A stale plan (another image's) costs time,
 *          never correctness. */
typedef struct {
    int* zspan;
    const int* plan;
    int plan_k;
    int plan_lanes;
} pp_scan_opts;

/* pp_relax_scan with the options above: the same outputs, bit for bit.
 * Errors as pp_relax_scan, plus PP_ERR_ARG for a NULL opts, an unaligned
 * zspan or plan, plan_k outside [1, nx*ny] or plan_lanes outside [1, 32]. */
PP_API pp_status pp_relax_scan_ex(const float* ff, const pp_grid* grid, const pp_scan* scan,
                                  const pp_tip* tip, const pp_fire* fire,
                                  float* pos, float* fz, int* iters,
                                  const pp_df* fused_df, float* df, const pp_scan_opts* opts,
                                  pp_stream stream);

/* Bytes of a pixel-to-warp plan for a scan of nx x ny pixels (any nz): 0 when
 * k is outside [1, nx*ny], lanes outside [1, 32] or the scan invalid. */
PP_API size_t pp_relax_plan_size(const pp_scan* scan, int k, int lanes);

/* Builds a plan in `plan` (DEVICE, 4-byte aligned, pp_relax_plan_size bytes)
 * from an earlier scan's iteration counts iters[k][j][i] (DEVICE, the layout
 * pp_relax_scan writes, nz heights; max_iter the FIRE limit it ran with): the
 * cost of pixel column (i, j) is its FIRE updates summed over the heights,
 * and the plan lists the k costliest columns (among equal costs at the
 * boundary, any), to run `lanes` to a warp.  A K2 warp runs 32 columns until
 * its slowest is done, and the other lanes' height changes and cell reloads
 * hold that column up; columns of similar cost in narrow warps finish
 * sooner.  Nothing of the paper's method changes: which warp computes a pixel
 * never changes its value.  Errors: PP_ERR_ARG (NULL, unaligned, k, lanes or
 * max_iter invalid), PP_ERR_SHAPE (scan sizes), PP_ERR_CUDA. */
PP_API pp_status pp_relax_plan(const int* iters, const pp_scan* scan, int max_iter, int k, int lanes,
                               void* plan, pp_stream stream);

/* Frequency shift of Eq. df.  fz[k*npix + p] holds Fz (eV/A) at tip heights
 * z_k = z_top - k*dz; df[c*npix + p] (Hz), c = 0..nz-2m-1, is centred at
 * z_{c+m}.  Fz is taken piecewise linear between the heights and integrated
 * exactly against u/sqrt(a^2 - u^2), a = A_pp/2.  npix = 0 is a no-op (fz and df
 * may then be NULL).  Errors: PP_ERR_ARG,
 * PP_ERR_SHAPE (nz < 2m+1), PP_ERR_UNSUPPORTED (m > 31), PP_ERR_CUDA. */
PP_API pp_status pp_fz_to_df(const float* fz, int nz, int npix, float dz, const pp_df* df_params,
                      float* df, pp_stream stream);

/* Layout conversion of a force-field buffer: src laid out as `src_grid`,
 * dst as `dst_grid`; the two must describe the same nodes (nx, ny, nz) and
 * may differ in layout and brick shape.  Padding nodes of dst are zeroed.
 * Errors: PP_ERR_ARG, PP_ERR_SHAPE, PP_ERR_UNSUPPORTED (interp = 1 grids),
 * PP_ERR_CUDA. */
PP_API pp_status pp_ff_convert(const float* src, const pp_grid* src_grid, float* dst,
                        const pp_grid* dst_grid, pp_stream stream);

/* ---------------------------------------------------------------- batches
 * Many molecules of uneven size in one persistent launch (a7; the paper's
 * batch generator for ML datasets, Sec. 4.4, motivates it; the method per
 * molecule is exactly pp_make_ff + pp_relax_scan with fused df).  Grids are
 * linear layout; all molecules share the probe, tip, FIRE, df parameters,
 * the scan height step and the periodic_xy flag. */
typedef struct {
    long long ff_offset;  /* float4 index of this molecule's grid in the packed ff buffer  */
    long long out_offset; /* index of its [snz][sny][snx] block in fz and iters (x3 in pos) */
    long long df_offset;  /* index of its [snz-2m][sny][snx] block in df                    */
    int atom_offset;      /* first atom in the packed atom arrays                           */
    int n_atoms;          /* >= 0                                                           */
    int nx, ny, nz;       /* grid nodes (>= 2 each)                                         */
    float x0, y0, z0, dx, dy, dz;
    int snx, sny, snz;    /* scan pixels and heights                                        */
    float sx0, sy0, spx, spy, z_top;
} pp_mol_desc;

typedef struct {
    pp_probe probe;
    pp_tip tip;
    pp_fire fire;
    pp_df df;
    float scan_dz;          /* height step of every scan, A                                  */
    int periodic_xy;        /* interpolation wrap of every grid (0 or 1)                      */
    long long ff_capacity;  /* float4 slots in ff                                             */
    long long out_capacity; /* entries in fz and iters (pos holds 3x)                         */
    long long df_capacity;  /* entries in df                                                  */
    int n_atoms_total;      /* length of the packed atom arrays                               */
    int ctas;               /* persistent CTAs of 128 threads; 0 = fill the GPU               */
    long long spin_limit;   /* polls (~128 ns apart) before a relax item stops waiting for its
                               molecule's force field; 0 = 1<<23 (about one second)           */
    int wait_extra;         /* test hook, 0 in normal use: relax items wait for this many more
                               force-field tiles than exist, so every wait runs out            */
    int ff_forces_only;     /* 1: every grid's E slots written as 0 and the energy sums skipped
                               (the forces, and so all scan outputs, are unchanged); 0 or 1    */
    /* Work-item shapes (picked by the autotuner; every choice computes the same values bit for
     * bit, only the scheduling differs).  0 selects the default in brackets. */
    int ff_tile_w;          /* force-field tile width in grid columns along x: 4, 8 or 16 [8]; the
                               tile is ff_tile_w x (32 / ff_tile_w) columns                    */
    int ff_zpt;             /* z-nodes per force-field tile: 4 or 8 [8]                         */
    int relax_tile_w;       /* relax tile width in pixels along x: 4, 8 or 16 [8]; the tile is
                               relax_tile_w x (32 / relax_tile_w) pixels, all heights          */
} pp_batch_params;

/* Status bits reported by pp_batch_status. */
#define PP_BATCH_BAD_DESC 1 /* a descriptor was invalid or overran a buffer: that molecule was skipped */
#define PP_BATCH_TIMEOUT 2  /* a bounded wait ran out: some relax tiles were not computed            */

/* Scratch bytes of pp_batch_run for nmol molecules (0 if nmol < 1). */
PP_API size_t pp_batch_workspace(int nmol);

/* One launch over all molecules: a planning kernel validates every device
 * descriptor (bad ones are skipped and flagged) and lays out a work list of
 * force-field tiles (ff_tile_w x 32/ff_tile_w columns x ff_zpt z-nodes) and
 * relax tiles (relax_tile_w x 32/relax_tile_w pixels, all heights) ordered
 * FF(0), FF(1), R(0), FF(2), R(1), ...; then a
 * persistent kernel whose warps pull items from a device counter.  A relax
 * tile waits (bounded, see spin_limit) until every force-field tile of its
 * molecule is done; items are handed out in list order, so the force field
 * it waits for is always being computed by running warps.  Writes, per
 * molecule, the force field, fz, df and (nullable) pos and iters exactly as
 * pp_make_ff + pp_relax_scan (fused df) on that molecule alone (the grid's E
 * slots 0 when params->ff_forces_only).  descs is a
 * DEVICE array of nmol descriptors; atoms are packed device arrays; ws is
 * 16-byte aligned scratch of pp_batch_workspace(nmol) bytes.  Nothing is
 * synchronised: the launch can be captured in a CUDA graph and replayed.
 * Errors detected on the host: PP_ERR_ARG, PP_ERR_SHAPE, PP_ERR_CAPACITY,
 * PP_ERR_UNSUPPORTED, PP_ERR_CUDA; errors found on the device are reported
 * by pp_batch_status. */
PP_API pp_status pp_batch_run(const pp_mol_desc* descs, int nmol, const pp_batch_params* params,
                              const pp_atoms* atoms, float* ff, float* pos, float* fz, int* iters,
                              float* df, void* ws, size_t ws_bytes, pp_stream stream);

/* Device-side status of the last pp_batch_run on `ws`: waits for `stream`,
 * then stores the PP_BATCH_* bits in *flags (host int).  Returns
 * PP_ERR_TIMEOUT if a wait ran out, PP_ERR_CAPACITY if a descriptor was bad,
 * else PP_OK.  This call synchronises the host with the stream. */
PP_API pp_status pp_batch_status(const void* ws, int* flags, pp_stream stream);

/* Gradients of pp_backward, device arrays owned by the caller: x, y, z, q, R,
 * eps hold n floats each (dL/dx_i in 1/A, dL/dq_i per e, dL/dR_i per A,
 * dL/deps_i per eV); tip holds 5 floats {dL/dkx, dL/dky, dL/dkR (per N/m),
 * dL/dQ (per e), dL/dQzz (per e*A^2)}.  pp_backward overwrites all of them. */
typedef struct {
    float *x, *y, *z, *q, *R, *eps;
    float* tip;
} pp_grads;

/* Bytes of scratch pp_backward needs for `grid`: a 256-byte header plus the
 * grid adjoint, one float4 per stored node (one float on an interp = 1
 * grid); 0 if the grid is invalid. */
PP_API size_t pp_backward_workspace(const pp_grid* grid);

/* Gradient of L = sum_{c,pix} g_df[c][pix] * df[c][pix] with respect to the
 * atoms (x, y, z, q, R, eps) and the tip (kx, ky, kR, Q, Qzz).  The paper has no
 * gradients: this is the implicit-function adjoint of the same discrete
 * model at the relaxed positions of a forward pass -- for every relaxed point
 * J^T lambda = (dFz/dp)^T g_Fz with J the exact 3x3 Jacobian of F_T + F_S
 * (trilinear interpolant included), g_Fz the transpose of the df stencil
 * (Eq. df) applied to g_df, then a grid adjoint -lambda (x) trilinear weights
 * contracted with the pair derivatives of Eqs. LJ and point charges on the
 * nodes it touches.  On a tricubic energy grid (interp = 1) J holds minus the
 * Hessian of the energy interpolant, the grid adjoint is the scalar
 * lambda . grad w_g over the 64 stencil nodes of each point, and it is
 * contracted with the derivatives of the pair energies.  Inputs: the forward's atoms, probe, grid, force field
 * `ff`, scan, tip and df parameters, and its relaxed positions
 * pos[nz][ny][nx][3]; g_df[nz-2m][ny][nx].  Points where FIRE stopped at
 * max_iter are differentiated as if converged.  Scratch `ws` (16-byte
 * aligned, >= pp_backward_workspace(grid) bytes) is overwritten; FP32
 * atomics make the sums order-dependent at rounding level.  Errors:
 * PP_ERR_ARG, PP_ERR_SHAPE, PP_ERR_CAPACITY (ws too small), PP_ERR_UNSUPPORTED
 * (df stencil wider than 63 taps), PP_ERR_CUDA. */
PP_API pp_status pp_backward(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                             const float* ff, const pp_scan* scan, const pp_tip* tip,
                             const pp_df* df_params, const float* pos, const float* g_df,
                             const pp_grads* grads, void* ws, size_t ws_bytes, pp_stream stream);

/* pp_backward without a caller workspace.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code in
 * a real-time acquisition or control loop, or a plugin whose host forbids
 * device allocations after start-up (cudaMalloc may block and synchronise
 * the device), and C or Fortran callers without a device allocator.  It
 * computes exactly what pp_backward computes, taking its scratch from a
 * 32 MiB array that every GPU loading this library holds until the process
 * exits; it allocates nothing itself.  Grids whose pp_backward_workspace()
 * exceeds pp_backward_noalloc_capacity() bytes (about 2.1 million stored
 * nodes) are rejected with PP_ERR_CAPACITY.  Every call looks up the
 * array's device address on the current device (cudaGetSymbolAddress), so a
 * device reset or a new context leaves later calls valid; the first call on a
 * device may load the library's code there, so make it before any stream
 * capture.  All calls share the one array and it keeps the last call's
 * contents (each call clears what must start at zero): calls that overlap on
 * the GPU -- on different streams, or from different threads -- race and
 * must be serialised by the caller.  Inputs, outputs and errors as
 * pp_backward. */
PP_API pp_status pp_backward_noalloc(const pp_atoms* atoms, const pp_probe* probe, const pp_grid* grid,
                                     const float* ff, const pp_scan* scan, const pp_tip* tip,
                                     const pp_df* df_params, const float* pos, const float* g_df,
                                     const pp_grads* grads, pp_stream stream);

/* Bytes of the static scratch behind pp_backward_noalloc. */
PP_API size_t pp_backward_noalloc_capacity(void);

/* IETS map (Sec. 3.3): the probe particle's vibration modes at its relaxed
 * positions pos[nz][ny][nx][3] (from pp_relax_scan with the same ff, grid,
 * scan and tip).  Per point, the stiffness K = -(J + J^T)/2 with J the exact
 * Jacobian of F_T + F_S (tip springs + trilinear interpolant); writes its
 * eigenvalues ascending to eig[((k*ny + j)*nx + i)*3 + c] (eV/A^2) and, when
 * hw is not NULL, the mode energies hbar sqrt(lambda/m) in meV (0 where
 * lambda <= 0) for a probe mass of mass_amu atomic mass units.  The two
 * lower eigenvalues are the lateral modes the IETS signal follows.  On a
 * tricubic energy grid (interp = 1) F_S's Jacobian is minus the Hessian of the
 * energy interpolant.  Errors: PP_ERR_ARG, PP_ERR_SHAPE, PP_ERR_CUDA. */
PP_API pp_status pp_iets(const float* ff, const pp_grid* grid, const pp_scan* scan, const pp_tip* tip,
                         const float* pos, float mass_amu, float* eig, float* hw, pp_stream stream);

/* Bytes of scratch pp_fft_correlate needs for `grid`: three complex FP32
 * arrays in a padded layout, 3 * nz * ((nx + 16) * ny + 16) * 8 bytes; 0 if
 * the grid is invalid or not supported by it. */
PP_API size_t pp_fft_workspace(const pp_grid* grid);

/* Cross-correlation force field of the Hartree-potential and full-density
 * models (Eqs. El_conv and Pauli_FDBM, evaluated by the convolution theorem
 * as in Sec. 5.1.2): for a sample field f (the Hartree potential V_S in V,
 * or the density rho_S in e/A^3) and the tip's density g (e/A^3, g[h] at
 * offset h from the PP, wrapped), on a grid periodic along x, y and z,
 *   E[n] = scale * dx dy dz * sum_h g[h]^p f[n + h]^p   (indices modulo the grid),
 * F = -grad E by the spectral derivative (Nyquist terms dropped).  With
 * scale = 1, p = 1 this is the electrostatic energy of Eq. El_conv; with
 * scale = A, p = beta the Pauli energy of Eq. Pauli_FDBM ([g f]^beta =
 * g^beta f^beta; negative density samples count as 0 when p != 1).  f and g
 * are device arrays [nz][ny][nx] of floats, 16-byte aligned; ff is a force-field buffer of the
 * grid (layout 0, interp 0): (Fx, Fy, Fz, E) per node is written
 * (accumulate = 0) or added to what ff holds (accumulate = 1), e.g. to the
 * Lennard-Jones grid of pp_make_ff.  ws: pp_fft_workspace(grid) bytes,
 * 16-byte aligned, overwritten.  nx, ny, nz must be powers of two in
 * [2, 1024].  Errors: PP_ERR_ARG, PP_ERR_SHAPE, PP_ERR_UNSUPPORTED (sizes,
 * bricked or energy-only grid), PP_ERR_CAPACITY (ws too small), PP_ERR_CUDA. */
PP_API pp_status pp_fft_correlate(const float* f, const float* g, const pp_grid* grid, float scale, float power,
                                  int accumulate, float* ff, void* ws, size_t ws_bytes, pp_stream stream);

/* Bounds-checked builds (libpp_checked.so, compiled with PP_CHECKED defined):
 * every global gather and scatter index of the kernels is tested against
 * the size of its array; an index outside it sets a bit and is replaced by
 * 0 (the result is then wrong, never an out-of-bounds access).  Bits: 1 grid
 * read, 2 grid write or grid-adjoint accumulation, 4 scan array read
 * (positions, Fz, loss weights), 8 scan array write, 16 FFT arrays.
 * pp_check_flags synchronises the device, stores the bits set since the last
 * call in *flags and clears them.  In a normal build *flags = 0 and it
 * returns PP_ERR_UNSUPPORTED. */
PP_API pp_status pp_check_flags(unsigned int* flags);

/* Read-bandwidth probe (a measurement aid of the benchmark; the paper has no
 * counterpart): reads the nfloats floats of buf `passes` times with 16-byte
 * loads that bypass L1, from every resident thread of a full-GPU grid, and
 * writes nothing but (never, in practice) one float to *sink.  Timing it on a
 * buffer well inside the L2 gives the L2 read bandwidth the relaxed scan's
 * roofline is stated against.  buf: device, 16-byte aligned, nfloats a
 * positive multiple of 4; sink: one device float.  Errors: PP_ERR_ARG,
 * PP_ERR_CUDA. */
PP_API pp_status pp_read_probe(const float* buf, size_t nfloats, int passes, float* sink, pp_stream stream);

/* Message of the last failed call on this host thread ("" if none). */
PP_API const char* pp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PP_H_ */
