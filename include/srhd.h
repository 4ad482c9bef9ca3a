/*
 * srhd.h - C ABI of libsrhd.so, the GB300 (sm_103a) per-patch fluid update of
 * special-relativistic hydrodynamics with the Taub-Mathews equation of state,
 * following Tseng, Schive & Chiueh, "GAMER-SR" (arXiv 2012.11130).
 *
 * Conventions (all entry points)
 *   Units c = m = k_B = 1 (Section 1); T means k_B T / m c^2.
 *   Primitive variables W = (rho, U^x, U^y, U^z, p): proper density, spatial
 *   four-velocity (Eq. new expression of Lorentz factor), pressure.
 *   Conserved variables U = (D, M^x, M^y, M^z, Etilde): D = rho gamma
 *   (Eq. density), M = D h U (Eq. momentum), Etilde = E - D (Eq. ETilde).
 *   Arrays are structure-of-arrays: variable v of element i is at
 *   base[v * var_stride + i]. Patch arrays are [npatch][5][cells] with
 *   x fastest: a ghosted patch holds 12^3 cells (an 8^3 interior plus two
 *   ghost cells on every side, Section 3.1), an interior patch 8^3 cells.
 *   Precision: SRHD_FP64 = double storage and double arithmetic;
 *   SRHD_MIXED = float storage, float arithmetic, except the cancelling sum
 *   A D^2 = Etilde (Etilde + 2D) - |M|^2 behind the left-hand side A of
 *   Eq. (transcendental equation) / Eq. (Unphysical result), which is formed
 *   in double in every conserved-to-primitive conversion;
 *   SRHD_MIXED_CF = as SRHD_MIXED but with A formed by compensated float
 *   arithmetic (see srhd_prec).
 *
 * Ownership and execution
 *   Every data pointer is a caller-owned DEVICE pointer on the context's
 *   device unless stated otherwise. The library allocates device memory only
 *   in srhd_create (the context's scratch) and in srhd_advance_uniform_host
 *   (its stage), and frees it in srhd_destroy.
 *   Calls are asynchronous on the given stream (a cudaStream_t passed as
 *   void*, NULL = legacy default stream) and never synchronise the device;
 *   srhd_advance_uniform_host alone waits, for its own work only.
 *   A context must not be used by two streams at once: its scratch is
 *   shared by the calls that use it (srhd_advance_patches with dt_next,
 *   srhd_cfl_dt).
 *
 * Errors
 *   Every call returns an srhd_status. Argument errors are detected on the
 *   host before any launch (SRHD_ERR_ARG) and launch failures are reported
 *   as SRHD_ERR_CUDA; srhd_last_error() returns a description of the last
 *   failure on the calling thread. Device-side outcomes (unphysical cells,
 *   retries, Newton non-convergence) are written to the caller's status
 *   arrays; no kernel traps, asserts or spins, and every loop is bounded.
 */
#ifndef SRHD_H
#define SRHD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum srhd_status {
  SRHD_OK = 0,
  SRHD_ERR_ARG = 1,   /* invalid argument (null pointer, size, enum, ...) */
  SRHD_ERR_CUDA = 2,  /* a CUDA runtime call or launch failed */
} srhd_status;

typedef enum srhd_prec {
  SRHD_FP64 = 0,     /* double storage, double arithmetic */
  SRHD_MIXED = 1,    /* float storage and arithmetic; the cancelling sum A D^2
                        of Eq. (transcendental equation) in double */
  SRHD_MIXED_CF = 2, /* float storage and arithmetic; A of Eq. (transcendental
                        equation) from error-free float products and a
                        compensated float sum (about 2^-44 of the cancelling
                        terms instead of 2^-53), so no double arithmetic at
                        all; element type float */
} srhd_prec;

typedef enum srhd_riemann { SRHD_HLLC = 0, SRHD_HLLE = 1 } srhd_riemann;
typedef enum srhd_cfl_mode { SRHD_CFL_SIGNAL = 0, SRHD_CFL_LIGHT = 1 } srhd_cfl_mode;
typedef enum srhd_bc { SRHD_BC_PERIODIC = 0, SRHD_BC_OUTFLOW = 1 } srhd_bc;

/* Energy formulation (Sections 2.1, 2.3 and 4). SRHD_SCHEME_REDUCED is the
 * paper's scheme: the fifth conserved variable is Etilde = E - D with flux
 * (Etilde + p) U^j / gamma (Eq. ETilde evolution) and conversions by
 * Eq. E_D and the Etilde form of Eq. transcendental equation.
 * SRHD_SCHEME_TOTAL is the "original scheme" the paper compares against: the
 * fifth variable is the total energy E = D h gamma - p with flux M^j
 * (Eq. E evoltion), inverted from (E/D)^2 - (|M|/D)^2 - 1, whose error grows
 * as 4 eps / (3T) for cold gas (Eq. OriRelativeError). */
typedef enum srhd_scheme { SRHD_SCHEME_REDUCED = 0, SRHD_SCHEME_TOTAL = 1 } srhd_scheme;

/* Per-cell status codes written by srhd_con2pri (cell_status). */
enum {
  SRHD_CELL_OK = 0,
  SRHD_CELL_UNPHYSICAL = 1, /* Eq. (Unphysical result) fails: A <= eps_machine
                               (2e-16, Section 3.3); outputs are NaN */
  SRHD_CELL_NOCONV = 2,     /* Newton-Raphson hit its iteration cap; outputs
                               hold the last iterate */
};

/* Per-patch status of srhd_advance_patches / srhd_flux_patches:
 * (code << 8) | retries, where retries (0..255) counts the limiter
 * reductions of Section 3.3 (1) and code is a bit set of: */
enum {
  SRHD_PATCH_UNPHYSICAL = 1, /* still unphysical with piecewise-constant data */
  SRHD_PATCH_BAD_INPUT = 2,  /* a cell of the ghosted input is unphysical */
  SRHD_PATCH_NOCONV = 4,     /* some Newton solve hit its iteration cap */
  SRHD_PATCH_STAGE_TIMEOUT = 8, /* ghosted batches and uniform grids: the
                               asynchronous copy of the next tile into shared
                               memory did not complete within
                               about a second (a device fault); the CTA that
                               waited stopped, so this patch and the later
                               patches of that CTA were not updated, and
                               dt_next is NaN */
};

/* Run-time parameters (Sections 3.1-3.3). */
/* Equation of state (Section 2.2): the Taub-Mathews EoS of the paper, or the
 * polytropic EoS h = 1 + Gamma/(Gamma-1) T that the paper keeps for pure
 * non-relativistic (Gamma = 5/3) or ultra-relativistic (Gamma = 4/3) gas. */
typedef enum srhd_eos { SRHD_EOS_TM = 0, SRHD_EOS_POLYTROPIC = 1 } srhd_eos;

typedef struct srhd_params {
  double cfl;             /* C_CFL of Eq. (time_step_sound_speed); default 0.5 */
  double theta;           /* minmod coefficient of the PLM limiter; default 1.5 */
  double retry_factor;    /* limiter reduction per retry (Section 3.3); 0.75 */
  double theta_floor;     /* below theta_floor * theta the retry uses theta = 0
                             (piecewise constant); default 1e-2 */
  int32_t riemann;        /* srhd_riemann; default SRHD_HLLC */
  int32_t cfl_mode;       /* srhd_cfl_mode; default SRHD_CFL_SIGNAL */
  int32_t ndim;           /* active dimensions in the CFL bound
                             (Eq. time_step_U_max uses 3); default 3 */
  int32_t newton_max_iter;/* Newton iteration cap; 0 = 50 (FP64) / 30 (FP32) */
  int32_t patch_variant;  /* launch variant of the fused patch kernel, 0..3
                             (threads per CTA, CTAs per SM, one or two Newton
                             solves per thread); 0 = default. Results do not
                             depend on it beyond rounding-free reordering of
                             independent work; chosen by an autotuner. */
  int32_t scheme;         /* srhd_scheme; default SRHD_SCHEME_REDUCED. Applies to
                             every call of the context: the fifth conserved
                             variable of all arrays is then E instead of Etilde */
  int32_t eos;            /* srhd_eos; default SRHD_EOS_TM. Applies to every call
                             of the context. SRHD_EOS_POLYTROPIC runs one fixed
                             launch configuration of the patch kernel
                             (patch_variant is then ignored). */
  double gamma;           /* Gamma of SRHD_EOS_POLYTROPIC, 1 < gamma <= 5/3;
                             default 5/3 (ignored for SRHD_EOS_TM) */
} srhd_params;

typedef struct srhd_ctx srhd_ctx;

/* Fills *p with the defaults listed above. Returns SRHD_ERR_ARG if p is NULL. */
srhd_status srhd_default_params(srhd_params* p);

/* Creates a context on the current CUDA device: validates *p (NULL means
 * defaults), queries the SM count and allocates the scratch used by the CFL
 * reduction. *ctx receives the handle (NULL on failure). */
srhd_status srhd_create(srhd_ctx** ctx, const srhd_params* p);

/* Frees the context and its scratch. The caller must make sure no work that
 * uses the context is still running. NULL is accepted. */
srhd_status srhd_destroy(srhd_ctx* ctx);

/* Description of the last error on the calling thread ("" if none). */
const char* srhd_last_error(void);

/* Primitive -> conserved, n independent cells (Section 2.3: Eq. density,
 * Eq. momentum, Eq. T_to_HTilde, Eq. E_D, with f from Eq. transcendental
 * equation).
 *   prim  [5 * var_stride] input, cons [5 * var_stride] output, element type
 *         double (SRHD_FP64) or float (SRHD_MIXED); var_stride >= n.
 *   Cells with rho <= 0 or p <= 0 produce NaN. n == 0 is a no-op. */
srhd_status srhd_prim2con(srhd_ctx* ctx, srhd_prec prec, const void* prim, void* cons,
                          int64_t n, int64_t var_stride, void* stream);

/* Conserved -> primitive, n independent cells (Section 2.3: the root of
 * Eq. transcendental equation, f(htilde) = A, then Eq. four-velocity, Eq. new
 * expression of Lorentz factor, Eq. density, Eq. T of h, Eq. p=rhoT). The
 * kernels solve the same equation for the same root by Newton-Raphson in the
 * conic parameter tau = h - T - 1 of the TM hyperbola (h - 4T)(h - T) = 1,
 * in which f is a ratio of polynomials, starting from
 * tau0 = A / (1 + sqrt(1 + A)) (the root for |M| = 0) instead of the
 * htilde guesses of Appendix A; htilde and T follow from tau in closed form.
 * A is formed in double (SRHD_FP64, SRHD_MIXED) or by compensated float
 * arithmetic (SRHD_MIXED_CF) and checked against Eq. (Unphysical result).
 *   cons, prim as in srhd_prim2con.
 *   cell_status [n] int32 (nullable): SRHD_CELL_* per cell. */
srhd_status srhd_con2pri(srhd_ctx* ctx, srhd_prec prec, const void* cons, void* prim,
                         int64_t n, int64_t var_stride, int32_t* cell_status, void* stream);

/* Riemann fluxes of a batch of ghosted patches: the first part of
 * srhd_advance_patches (con2pri of the tile, PLM, MUSCL-Hancock half step,
 * con2pri of the predicted face states, HLLC/HLLE; Section 3.1), stopping
 * before the update.
 *   cons_ghosted [npatch][5][12^3]; face_flux [npatch][3][5][576] output,
 *   direction d faces ordered with extent 9 along d and 8 across, x fastest
 *   (face index i along d sits between interior cells i-1 and i);
 *   dt_dh [npatch][2] device doubles (dt, dh) per patch;
 *   patch_status [npatch] int32 (nullable): code bits only (no retry is made
 *   without an update). */
srhd_status srhd_flux_patches(srhd_ctx* ctx, srhd_prec prec, const void* cons_ghosted,
                              void* face_flux, int32_t npatch, const double* dt_dh,
                              int32_t* patch_status, void* stream);

/* One MUSCL-Hancock step of a batch of independent ghosted patches
 * (Sections 3.1-3.3): con2pri, PLM with the hybrid van Leer / generalised
 * minmod limiter, Hancock half step, con2pri of predicted face states,
 * HLLC (HLLE option and fallback), conservative update (Eq. conservative
 * form with Eq. ETilde evolution), the unphysical check Eq. (Unphysical
 * result) with the whole-patch limiter retry, and optionally the CFL time
 * step of the updated state (Eqs. time_step_U_max, SMax,
 * time_step_sound_speed).
 *   cons_ghosted [npatch][5][12^3] input (not modified).
 *   cons_out     [npatch][5][8^3] output; must not overlap the input.
 *   patch_face_flux (nullable) [npatch][6][5][64]: fluxes through the six
 *                patch faces (-x,+x,-y,+y,-z,+z), 8x8 each, for coarse-fine
 *                flux correction.
 *   npatch >= 0; dt_dh [npatch][2] device doubles (dt, dh) per patch.
 *   worklist (nullable) [npatch] int32: the launch processes patches
 *                worklist[0..npatch) (indices into every per-patch array);
 *                NULL means 0..npatch-1. Indices are not range checked on
 *                the device; the caller guarantees they are valid.
 *   dt_next (nullable): one device double receiving min over the processed
 *                patches of C_CFL dh / S_max of the updated cells, or NaN if
 *                some updated cell is unphysical.
 *   patch_status (nullable) [npatch] int32, see SRHD_PATCH_*. */
srhd_status srhd_advance_patches(srhd_ctx* ctx, srhd_prec prec, const void* cons_ghosted,
                                 void* cons_out, void* patch_face_flux, int32_t npatch,
                                 const double* dt_dh, const int32_t* worklist, double* dt_next,
                                 int32_t* patch_status, void* stream);

/* srhd_advance_patches on patches p0 .. p0+n-1 of a uniform grid resident on
 * the device, tiled as in srhd_fill_ghosts_uniform, without a ghosted copy:
 * the kernel reads each patch's 12^3 tile (two ghost cells, periodic or
 * outflow per axis) from the patch and its neighbours in `interior` while
 * it loads the tile (the same values srhd_fill_ghosts_uniform writes, so
 * the results are identical to fill + srhd_advance_patches).
 *   interior [npx*npy*npz][5][8^3]; bc[3] host srhd_bc of x, y, z;
 *   0 <= p0, n >= 0, p0 + n <= npx*npy*npz;
 *   cons_out [n][5][8^3] (row i: patch p0+i) must not overlap interior;
 *   patch_face_flux (nullable) [n][6][5][64], dt_dh [n][2], patch_status
 *   (nullable) [n] and dt_next (nullable) as srhd_advance_patches. */
srhd_status srhd_advance_uniform(srhd_ctx* ctx, srhd_prec prec, const void* interior,
                                 int32_t npx, int32_t npy, int32_t npz, const int32_t* bc,
                                 int32_t p0, int32_t n, void* cons_out, void* patch_face_flux,
                                 const double* dt_dh, double* dt_next, int32_t* patch_status,
                                 void* stream);

/* Conserved-to-primitive conversion (Section 2.3, Eqs. transcendental
 * equation and p = rho T; unphysical states per Eq. Unphysical result) of
 * npatch interior patches into the primitive-cache layout of
 * srhd_advance_uniform_prim:
 *   cons [npatch][5][8^3] (D, M^x, M^y, M^z, Etilde);
 *   prim_out [npatch][6][8^3] = (rho, U^x, U^y, U^z, p, tau), where tau is
 *   the converged root-finding variable of the conversion (the conic
 *   parameter h - T - 1 of the TM EoS, htilde for the polytropic EoS);
 *   all six are NaN for an unphysical cell. Storage type as prec. */
srhd_status srhd_con2pri_patches(srhd_ctx* ctx, srhd_prec prec, const void* cons, int64_t npatch,
                                 void* prim_out, void* stream);

/* srhd_advance_uniform with a primitive cache: each step's update phase
 * already converts the new state (for the CFL bound of Section 3.2, and as
 * the check of Eq. Unphysical result), so it also writes those primitives,
 * and the next step gathers the primitives of its tiles from them instead
 * of converting every tile cell again (about 2.7 conversions per updated
 * cell, because neighbouring tiles overlap). The method and its results are
 * those of srhd_advance_uniform, up to the rounding of the Newton root
 * (the cached conversion starts from the cell's previous root).
 *   interior [npx*npy*npz][5][8^3] and prim_in [npx*npy*npz][6][8^3]: the
 *   state and its primitives (from srhd_con2pri_patches, or prim_out of the
 *   previous step over the whole grid); a cell whose cached primitives are
 *   NaN or non-positive (rho, p) makes every patch that reads it
 *   SRHD_PATCH_BAD_INPUT;
 *   cons_out [n][5][8^3] and prim_out [n][6][8^3] (row i: patch p0+i), the
 *   new state and its primitives (NaN where unphysical); neither may
 *   overlap interior or prim_in;
 *   bc, p0, n, patch_face_flux, dt_dh, dt_next, patch_status as in
 *   srhd_advance_uniform. */
srhd_status srhd_advance_uniform_prim(srhd_ctx* ctx, srhd_prec prec, const void* interior,
                                      const void* prim_in, int32_t npx, int32_t npy, int32_t npz,
                                      const int32_t* bc, int32_t p0, int32_t n, void* cons_out,
                                      void* prim_out, void* patch_face_flux, const double* dt_dh,
                                      double* dt_next, int32_t* patch_status, void* stream);

/* One VL step (the predictor-corrector integrator GAMER-SR offers beside
 * MUSCL-Hancock, Section 3.1) of a batch of independent patches with THREE
 * ghost cells per side: a first-order unsplit predictor to the half step
 * (Riemann fluxes between the piecewise-constant cell states), con2pri of
 * the predicted state, then PLM reconstruction of it (no Hancock step),
 * conserved face states, Riemann flux and the conservative update, with the
 * Eq. (Unphysical result) check and the limiter retry of the corrector
 * (Section 3.3) and the optional CFL bound, as srhd_advance_patches. An
 * unphysical predicted state marks the patch SRHD_PATCH_UNPHYSICAL and its
 * output NaN (the predictor does not depend on the limiter).
 *   cons_ghosted [npatch][5][14^3] input (8^3 interior, 3 ghost cells per
 *   side, x fastest); every other argument as srhd_advance_patches (the
 *   patch_variant parameter does not apply; eos and scheme do). */
srhd_status srhd_advance_patches_vl(srhd_ctx* ctx, srhd_prec prec, const void* cons_ghosted,
                                    void* cons_out, void* patch_face_flux, int32_t npatch,
                                    const double* dt_dh, const int32_t* worklist,
                                    double* dt_next, int32_t* patch_status, void* stream);

/* CFL time step (Section 3.2) of a batch of interior patches:
 * dt_out = min over all cells of C_CFL dh / S_max (signal mode) or
 * C_CFL dh (light mode); NaN if some cell is unphysical.
 *   cons [npatch][5][8^3]; dt_out: one device double. */
srhd_status srhd_cfl_dt(srhd_ctx* ctx, srhd_prec prec, const void* cons, int32_t npatch,
                        double dh, double* dt_out, void* stream);

/* Ghost-zone fill of a uniform grid tiled by npx*npy*npz patches (patch
 * (ix,iy,iz) at index (iz*npy + iy)*npx + ix), with periodic or outflow
 * (zero-gradient copy) boundaries per axis. Not part of the paper's solver:
 * a harness for uniform-grid runs, where all patches are on one level.
 *   interior [np][5][8^3] input, ghosted [np][5][12^3] output;
 *   bc[3] host array of srhd_bc for x, y, z. */
srhd_status srhd_fill_ghosts_uniform(srhd_ctx* ctx, srhd_prec prec, const void* interior,
                                     void* ghosted, int32_t npx, int32_t npy, int32_t npz,
                                     const int32_t* bc, void* stream);

/* ---- AMR: the steps around the per-patch update in a patch hierarchy ----
 * Section 3.1: data live in 8^3 patches on levels l = 0, 1, ... (level l has
 * a cell 2^l times finer than level 0) and level l takes two substeps per
 * step of level l-1. The calls below work on one array of all patches of
 * all levels, [ntotal][5][8^3] (a patch is an index into it); the caller
 * builds the maps from its hierarchy (paper_2012_11130_gb300/amr.py does).
 * They move data only and are HBM-bound. Map entries are range checked on
 * the device: an invalid entry gives NaN (fill) or is skipped. */

/* Ghost-zone fill of the patches p0 .. p0+n-1 (all cells of their 12^3
 * tiles, interior included), from a source map. The paper fills the ghost
 * zones of a fine patch from its own level where that level covers them and
 * otherwise from the coarser level (Section 3.3 (3)); here the coarse value is the
 * coarse cell containing the ghost cell (piecewise-constant prolongation,
 * conservative and physical whenever the coarse state is), interpolated
 * linearly in time between the coarse level's states before and after its
 * step. Boundary conditions are encoded in the map (a copy of an edge cell
 * for outflow, a wrapped cell for periodic, a fixed state for inflow).
 *   cur, prev [ntotal][5][8^3]: the latest interior states of all patches,
 *       and those before each level's latest step;
 *   ghosted [ntotal][5][12^3] output (rows p0 .. p0+n-1 written);
 *   map [ntotal][12^3] int32 (row p for patch p), per tile cell:
 *       q >= 0, bit 30 clear: copy of cur cell q (q = patch * 512 + cell,
 *             cell = (k*8 + j)*8 + i);
 *       q >= 0, bit 30 set (SRHD_AMR_COARSE): (1-w) prev[q'] + w cur[q'],
 *             q' = q without bit 30;
 *       q < 0: special state -1-q of `special` [nspecial][5] (device, may
 *             be NULL when nspecial == 0);
 *   ntotal >= 1, 0 <= p0, n >= 0, p0 + n <= ntotal, 0 <= w <= 1. */
#define SRHD_AMR_COARSE (1 << 30)
srhd_status srhd_amr_fill_ghosts(srhd_ctx* ctx, srhd_prec prec, const void* cur,
                                 const void* prev, void* ghosted, const int32_t* map,
                                 int32_t ntotal, int32_t p0, int32_t n, double w,
                                 const void* special, int32_t nspecial, void* stream);

/* srhd_amr_fill_ghosts and srhd_advance_patches in one launch, without the
 * ghosted copy: the patch kernel reads each listed patch's 12^3 tile through
 * its map row while it loads the tile. Tile cell c of patch p takes
 *   map[p][c] >= 0 without SRHD_AMR_COARSE: level_state[q];
 *   with SRHD_AMR_COARSE: (1-w) coarse_old[q'] + w coarse_new[q'];
 *   < 0: special state -1-map[p][c] (NaN if out of range or invalid),
 * i.e. the tile srhd_amr_fill_ghosts writes with cur = level_state for the
 * first kind and (prev, cur) = (coarse_old, coarse_new) for the second, and
 * the step and its outputs are those of srhd_advance_patches on that tile
 * (bit-identical results). A driver copies the level's state to prev first
 * and passes level_state = coarse_old = prev, coarse_new = cur,
 * cons_out = cur.
 *   level_state, coarse_old, coarse_new [ntotal][5][8^3]; map [ntotal][12^3];
 *   cons_out [ntotal][5][8^3]: rows of the processed patches written; they
 *       must not be rows that the map rows of the processed patches read;
 *   npatch, worklist (nullable: 0..npatch-1, indices < ntotal, not checked
 *   on the device), dt_dh [ntotal][2], patch_face_flux (nullable)
 *   [ntotal][6][5][64], dt_next, patch_status (nullable) [ntotal] as
 *   srhd_advance_patches; w, special, nspecial as srhd_amr_fill_ghosts. */
srhd_status srhd_advance_amr(srhd_ctx* ctx, srhd_prec prec, const void* level_state,
                             const void* coarse_old, const void* coarse_new, const int32_t* map,
                             int32_t ntotal, double w, const void* special, int32_t nspecial,
                             void* cons_out, void* patch_face_flux, int32_t npatch,
                             const double* dt_dh, const int32_t* worklist, double* dt_next,
                             int32_t* patch_status, void* stream);

/* Restriction: each listed parent patch takes, in every cell, the mean of
 * the 2x2x2 cells of its child covering that cell (volume average, so the
 * mass, momentum and energy of the coarse level equal those of the fine one
 * where it is refined).
 *   cur [ntotal][5][8^3] in/out;
 *   children [nparent][9] int32: parent index, then the children of octants
 *       cx + 2 cy + 4 cz (cx = 1 for the child of larger x). */
srhd_status srhd_amr_restrict(srhd_ctx* ctx, srhd_prec prec, void* cur,
                              const int32_t* children, int32_t nparent, int32_t ntotal,
                              void* stream);

/* Coarse-fine flux correction (Section 3.3 (4), the correction that keeps the
 * composite grid conservative): the coarse cells on a patch face bordering
 * the finer level are corrected by U += s (dt/dh) (F_coarse - <F_fine>),
 * s = +1 on a high face and -1 on a low one, with F_coarse the patch-face
 * flux of the coarse step and <F_fine> the mean of the fine patch-face fluxes
 * over the 2x2 fine faces covering the coarse face and over the two fine
 * substeps; a cell on several such faces takes their corrections in the
 * face order below. A cell whose corrected state fails Eq. (Unphysical
 * result) (D > 0 and A > 2e-16, A in double from the stored values, in the
 * context's scheme) keeps its uncorrected state, as the paper prescribes;
 * this breaks exact conservation on that cell only.
 *   cur [ntotal][5][8^3] in/out;
 *   flux_coarse, flux_fine0, flux_fine1 [ntotal][6][5][64]: patch-face
 *       fluxes (srhd_advance_patches' patch_face_flux) of the coarse step and
 *       of the two fine substeps;
 *   faces [nrows][25] int32: coarse patch, then for faces -x,+x,-y,+y,-z,+z
 *       the four fine patches across it, ordered qa + 2 qb by quadrant (qa
 *       along the lower transverse axis), or -1 for a face that does not
 *       border the finer level; a coarse patch appears in one row only;
 *   dt_dh [ntotal][2] device doubles (the coarse patch's dt, dh);
 *   skipped (nullable): one device int32 to which the number of cells whose
 *       correction was skipped is added (atomically; the caller zeroes it). */
srhd_status srhd_amr_flux_correct(srhd_ctx* ctx, srhd_prec prec, void* cur,
                                  const void* flux_coarse, const void* flux_fine0,
                                  const void* flux_fine1, const int32_t* faces, int32_t nrows,
                                  const double* dt_dh, int32_t ntotal, int32_t* skipped,
                                  void* stream);

/* Limited linear prolongation of the ghost cells that a fine level takes
 * from the coarser level (Section 3.3 (3), ghost-zone interpolation): the
 * conserved variables are interpolated, and where that gives a state failing
 * Eq. (Unphysical result) the primitive variables (rho, U^x, U^y, U^z, p) are
 * interpolated instead and converted back (always physical). Per axis the
 * slope is the minmod of the two one-sided differences of the coarse cell
 * with its neighbours; the fine cell centre lies a quarter of a coarse cell
 * below or above the coarse centre along each axis. Coarse states are taken
 * at the fine substep's time, (1 - w) prev + w cur, as in
 * srhd_amr_fill_ghosts. The results go to rows of a special-state array that
 * the maps of srhd_amr_fill_ghosts and srhd_advance_amr then reference
 * (paper_2012_11130_gb300/amr.py builds such maps and tables).
 *   cur, prev [ntotal][5][8^3]: coarse states after and before the coarse
 *       level's step;
 *   table [nrows][8] int32 per fine ghost cell: the coarse cell containing
 *       it, its neighbours along -x, +x, -y, +y, -z, +z (flat indices
 *       patch * 512 + cell; -1 where the coarse level does not cover the
 *       neighbour, which gives a zero one-sided difference), then parity
 *       bits (bit d set: the fine cell is in the upper half along axis d);
 *   out [nrows][5] output (rows of the special-state array); a row whose
 *       coarse cell index is out of range gives NaN;
 *   fallbacks (nullable): one device int32 to which the number of rows
 *       interpolated in primitive variables is added (the caller zeroes it);
 *   0 <= w <= 1. */
srhd_status srhd_amr_prolong(srhd_ctx* ctx, srhd_prec prec, const void* cur, const void* prev,
                             const int32_t* table, int32_t nrows, int32_t ntotal, double w,
                             void* out, int32_t* fallbacks, void* stream);

/* srhd_fill_ghosts_uniform restricted to the patches p0 .. p0+n-1, so that a
 * caller can fill and advance part of a grid while the rest is in transit:
 * ghosted [n][5][12^3] receives patch p0+i in row i; interior [np][5][8^3]
 * is the whole grid (read wherever the ghost zones reach);
 * 0 <= p0, n >= 0, p0 + n <= npx*npy*npz. */
srhd_status srhd_fill_ghosts_uniform_range(srhd_ctx* ctx, srhd_prec prec, const void* interior,
                                           void* ghosted, int32_t npx, int32_t npy, int32_t npz,
                                           const int32_t* bc, int32_t p0, int32_t n,
                                           void* stream);

/* srhd_fill_ghosts_uniform with three ghost cells per side: ghosted
 * [np][5][14^3] for srhd_advance_patches_vl. */
srhd_status srhd_fill_ghosts_uniform3(srhd_ctx* ctx, srhd_prec prec, const void* interior,
                                      void* ghosted, int32_t npx, int32_t npy, int32_t npz,
                                      const int32_t* bc, void* stream);

/* One MUSCL-Hancock step (the fused update of srhd_advance_patches, with
 * the CFL bound of the result) of a uniform grid whose state lives in HOST
 * memory, tiled as in srhd_fill_ghosts_uniform. Only interiors cross the
 * host link: the grid is cut into chunks of whole z slabs of patches; the
 * copies in, the step of each chunk (srhd_advance_uniform, which gathers
 * the ghost zones from the copied slabs) and the copies out run on streams
 * of the context (one for each copy direction, two for the chunks' steps,
 * taken in turn), so the copies of one chunk overlap the step of another. (Not part of the paper's solver: the host-resident
 * driver of a uniform-grid run.) The call is synchronous: it starts after
 * the work already queued on `stream` and returns when the outputs are
 * written; work queued on `stream` afterwards follows it.
 *   host_in  [np][5][8^3] host array, the state at t^n (np = npx*npy*npz);
 *   host_out [np][5][8^3] host array, the state at t^n + dt; it may be
 *            host_in itself, otherwise it must not overlap it. Page-locked
 *            (pinned) host memory lets the copies overlap; pageable memory
 *            gives the same result, serialised;
 *   bc[3]: srhd_bc of x, y, z; dt >= 0 and dh > 0 for every patch;
 *   dt_next (nullable, HOST double): min over all cells of C_CFL dh / S_max
 *            of the result, NaN if some updated cell is unphysical;
 *   patch_status (nullable) [np] HOST int32, see SRHD_PATCH_*;
 *   chunks in [1, 64]: chunk k holds slabs npz*k/K .. npz*(k+1)/K - 1,
 *            K = min(chunks, npz); one slab per chunk overlaps best.
 * Device memory: the first call allocates the stage (two interior copies of
 * the grid, per-patch scratch) and keeps it
 * in the context for later calls; a larger grid or a wider storage type
 * reallocates it. On an error the call waits for its queued work and
 * returns the status; host_out is then undefined. */
srhd_status srhd_advance_uniform_host(srhd_ctx* ctx, srhd_prec prec, const void* host_in,
                                      void* host_out, int32_t npx, int32_t npy, int32_t npz,
                                      const int32_t* bc, double dt, double dh, double* dt_next,
                                      int32_t* patch_status, int32_t chunks, void* stream);

/* The double-precision reciprocal that the FP64 arithmetic of the kernels
 * uses for its quotients (the paper has no counterpart: it fixes the
 * precision of the arithmetic, not how a division is evaluated): the
 * hardware approximation refined by two Newton-Raphson steps, within about
 * one ulp of the IEEE reciprocal; zero, subnormal, |x| >= 2^1021 and
 * non-finite x give the IEEE result exactly. Exported so that its error can
 * be checked on the device.
 *   x, y: device arrays of n >= 0 doubles (y may be x); no context, no
 *   allocation; asynchronous on stream. */
srhd_status srhd_reciprocal_f64(const double* x, double* y, int64_t n, void* stream);

/* CFL time step of a batch of interior patches, like srhd_cfl_dt, for
 * callers that cannot allocate device memory. (The paper has no counterpart:
 * this is a deployment variant of srhd_cfl_dt.) Some callers cannot call
 * cudaMalloc: an application whose device memory all comes from its own pool
 * allocator, or a time-step loop that must not let an allocation synchronise
 * the device. srhd_cfl_dt needs a context and srhd_create allocates, so this
 * entry point takes no context and allocates nothing.
 *   cons [npatch][5][8^3]; 0 <= npatch <= 131072 (larger batches are refused
 *   with SRHD_ERR_ARG); dh > 0; params (nullable: defaults) supplies cfl,
 *   cfl_mode, ndim, newton_max_iter, scheme (SRHD_SCHEME_TOTAL converts the
 *   total-energy form), eos and gamma (the polytropic EoS), all validated as
 *   in srhd_create; its other fields are ignored; dt_out: one device double receiving
 *   min over cells of C_CFL dh / S_max, NaN if a cell is unphysical, +inf if
 *   npatch == 0.
 * Its scratch is a fixed 1.5 MB static device array that every GPU loading
 * the library holds until the process exits. The first call on each device
 * looks up that array's device address (cudaGetSymbolAddress) with the
 * device current, so make that first call before any stream capture begins.
 * All calls share the array and leave their per-patch results in it: calls
 * whose work overlaps on the GPU race and must be ordered by the caller. */
srhd_status srhd_cfl_dt_noalloc(srhd_prec prec, const void* cons, int32_t npatch, double dh,
                                const srhd_params* params, double* dt_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SRHD_H */
