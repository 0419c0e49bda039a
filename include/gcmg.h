/*
 * gcmg.h -- C ABI of the GB300 ghost-cell multigrid library (libgcmg.so).
 *
 * Solves the Poisson problem with mixed boundary conditions on an arbitrary
 * domain given by a level set (Coco & Russo, "A Finite Difference Ghost-cell
 * Multigrid approach for Poisson Equation with mixed Boundary Conditions in
 * Arbitrary Domain", arXiv 1111.0983, Sec. 2, Eq. (mainpr)):
 *
 *     -Lap u = f  in Omega = {phi < 0},   u = g_D on Gamma_D,   du/dn = g_N on Gamma_N,
 *
 * discretised on a vertex grid with n = N+1 nodes per axis, spacing h and
 * node j at origin + j h (Sec. 2.3); by default the box D = [-1,1]^d
 * (d = 2 or 3), h = 2/N, origin -1.  The unknowns are
 * the inside nodes Omega_h (phi < 0) and the ghost nodes Gamma_h (outside
 * nodes with an axis neighbour inside).  Each ghost G carries the boundary
 * condition at its closest boundary point B (Eq. clpt), interpolated on an
 * upwind 3^d stencil (Eqs. St_G, dir2d, neu2d; reduced stencils of Remark 3).
 * The system (Eq. discr) is solved by multigrid V- or W-cycles (TGCS of
 * Sec. 2.4 applied recursively) with the boundary restriction of Sec. 2.5,
 * the defect extension of Sec. 2.6 and the extra boundary sweeps of Sec. 3.2.
 *
 * Conventions for every call:
 *  - Grid arrays are dense, C ordered, axis 0 (x) slowest: element
 *    ((j0 * n) + j1) * n + j2 for node (j0, j1, j2); n^d elements.
 *  - Per-ghost arrays of a level follow the ghost order of that level, which
 *    is increasing node index.
 *  - "_dev" pointers are device memory on the context's device, "_host"
 *    pointers host memory.  All buffers stay owned by the caller and are only
 *    borrowed for the duration of the call; the library copies what it keeps.
 *  - Work is enqueued on the stream given at creation (cudaStream_t passed as
 *    void*, NULL = legacy default stream).  Calls that return values to the
 *    host synchronise that stream before returning.
 *  - Every call returns a status; no call aborts or throws.  The message of
 *    the last failure is kept per context (gcmg_last_error).
 *  - A context is not thread safe: use one context per host thread.
 */
#ifndef GCMG_H
#define GCMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gcmg_ctx gcmg_ctx;

typedef enum {
    GCMG_OK = 0,
    GCMG_E_ARG = 1,      /* invalid argument (sizes, pointers, level index) */
    GCMG_E_CUDA = 2,     /* a CUDA call failed; see gcmg_last_error */
    GCMG_E_OOM = 3,      /* device or host allocation failed */
    GCMG_E_GEOM = 4,     /* geometry unusable: an unknown, ghost stencil or extension
                            node on the box boundary, no usable ghost stencil, a
                            degenerate normal, or a singular coarsest system */
    GCMG_E_NOCONV = 5,   /* max_cycles reached, a NaN/Inf defect, or a defect that grew
                            in diverge_cycles consecutive cycles (rho > 1) */
    GCMG_E_STATE = 6,    /* call out of order (e.g. solve before set_rhs) */
    GCMG_E_SIZE = 7,     /* problem larger than a fixed-capacity entry point accepts */
    GCMG_E_TIMEOUT = 8   /* a bounded device-side wait ran out (the context stays usable) */
} gcmg_status;

/* Cycle parameters (Sec. 2.4, Sec. 3.2).  gcmg_default_params fills the
 * paper's values: nu1 = 2, nu2 = 1, lambda = 5, delta = 3h, mu_D dt = 0.9,
 * mu_N dt = 0.9 * 2h / (3 sqrt(d)), V-cycle; plus the junction relaxation
 * that this library adds for mixed boundaries (2D: an exact solve of the
 * zone within R_J = 20 h; 3D: mu_J = 10 sweeps within R_J = 2 h; the paper
 * has no counterpart -- without it the V-cycle factor of a mixed problem
 * grows as h shrinks). */
typedef struct {
    int dim;                 /* 2 or 3 */
    int n;                   /* fine nodes per axis: (n - 1) = (n_coarse - 1) * 2^k, k >= 1 */
    int n_coarse;            /* nodes per axis of the coarsest grid (exact solve there) */
    int nu1, nu2;            /* pre / post relaxations */
    int lambda;              /* extra sweeps on the band and the ghosts after each relaxation */
    int gamma;               /* 1 = V-cycle, 2 = W-cycle */
    double delta_over_h;     /* band half-width delta / h of the extra sweeps */
    double c_dirichlet;      /* mu_D dt of Eq. dir2d */
    double c_neumann_factor; /* mu_N dt = c_neumann_factor * 2h / (3 sqrt(d)) (Eq. neu2d) */
    int precision;           /* 0: FP64 cycles; 1: FP32 cycles inside FP64 iterative refinement */
    int max_cycles;          /* limit of cycles (plain) or refinement steps (mixed) */
    double rtol;             /* stop when ||r||_inf <= rtol * ||r0||_inf, r0 = (f, g) */
    int junction_sweeps;     /* mu_J: local sweeps near Dirichlet/Neumann junctions after every
                                relaxation on every level (0: the paper's smoother alone) */
    double junction_radius;  /* R_J: zone = unknowns within R_J h of a ghost whose 3^d
                                neighbourhood holds a ghost of the other boundary type */
    int junction_solve;      /* 1: after every relaxation solve the zone's equations exactly
                                (values outside held fixed) instead of mu_J sweeps; the zone
                                is first grown by its ghosts' stencils, then stripped of
                                ghosts whose stencil leaves it; components of at most 4096
                                unknowns (larger: GCMG_E_GEOM at the solve) */
    int fused_coarse_n;      /* 2D FP32 V-cycles: the levels with at most this many nodes a side
                                run as one launch (a cluster of CTAs with barriers between the
                                steps; same results); 0: one launch per step */
    int smoother;            /* 0: the paper's relaxation (ghost relaxation + lambda band sweeps);
                                1: its Kaczmarz comparison (Sec. 3.3, "Comparison with the
                                Kaczmarz and the block relaxations"): a Gauss-Seidel sweep over
                                the inside nodes, then lambda Kaczmarz sweeps over the ghost
                                equations and the band's inside equations, rows ordered by the
                                colour sum_a (j_a mod 5) 5^a of their node.  2D, plain FP64
                                (precision 0), junction relaxation off; else GCMG_E_ARG */
    double h;                /* fine grid spacing (Sec. 2.3); 0: 2 / (n - 1), the box [-1,1]^d */
    double origin[3];        /* coordinates of node 0 on each axis (the first dim used); the
                                defaults are -1; B of gcmg_ghost_geometry is given in them */
    int diverge_cycles;      /* stop with GCMG_E_NOCONV once the defect has grown in this many
                                consecutive cycles (rho > 1); 0: only NaN/Inf and max_cycles */
} gcmg_params;

/* Grid of the problem statement (Sec. 2.1, Eq. mainpr; Sec. 2.3): n[a] nodes on
 * axis a (all equal: the hierarchy halves every axis), spacing h, node j of
 * axis a at origin[a] + j h. */
typedef struct {
    int dim;
    int64_t n[3];
    double h;
    double origin[3];
} gcmg_grid;

/* Per-solve report.  rel[m] = ||r^(m)||_inf / ||r^(0)||_inf for m = 0..cycles
 * (max 256 kept), over Omega_h u Gamma_h, in FP64; the ratio of consecutive
 * entries is the convergence factor rho^(m) of Sec. 3. */
typedef struct {
    int cycles;
    int converged;
    double rel_residual;
    double r0_norm;
    double rel[257];
    int diverged;    /* 1: stopped because the defect grew diverge_cycles cycles in a row */
} gcmg_stats;

/* Fills p with the defaults above for (dim, n, n_coarse). */
gcmg_status gcmg_default_params(gcmg_params *p, int dim, int n, int n_coarse);

/* Builds the hierarchy from the fine level set phi_dev (device, n^d doubles):
 * classification, ghost equations, bands and extension lists of every level
 * (coarse levels use phi at their nodes; coarse operators are rediscretised,
 * Sec. 1.3 Remark 3), and the coarsest dense inverse with all ghosts
 * Dirichlet until gcmg_set_bc_types is called for that level.  stream is a
 * cudaStream_t (NULL: default).  On failure *out is NULL unless a context
 * exists to read the message from; destroy it with gcmg_destroy. */
gcmg_status gcmg_create(const gcmg_params *p, const double *phi_dev, void *stream, gcmg_ctx **out);

/* gcmg_create on an explicit grid: grid->dim, n[0] (= n[1] = n[2] for the axes
 * used), h and origin replace the corresponding fields of p (p's other
 * fields, n_coarse included, are used as given).  phi_dev holds the level set
 * at the grid's nodes.  GCMG_E_ARG: unequal n, h <= 0 or not finite. */
gcmg_status gcmg_create_grid(const gcmg_grid *grid, const double *phi_dev, const gcmg_params *p, void *stream,
                             gcmg_ctx **out);

/* Reinitialisation of a level set (Eq. sdf, Sec. 2.1), for a phi0 that is not
 * a signed distance function, before gcmg_create: phi_dev (device, n^dim
 * doubles of the box [-1,1]^dim) receives the result of `steps` explicit steps
 * of phi_t = sgn(phi0)(1 - |grad phi|) from phi0_dev, with dt = h / dim, the
 * Godunov upwind form of |grad phi| and, at nodes next to the zero set of
 * phi0, the subcell fix that keeps the zero set in place.  phi0_dev and
 * phi_dev must not alias; one scratch grid is allocated for the call; runs on
 * `stream` and synchronises it.  GCMG_E_ARG: dim not 2 or 3, n < 3, steps < 0
 * or bad pointers; GCMG_E_OOM, GCMG_E_CUDA. */
gcmg_status gcmg_reinit(int dim, int n, const double *phi0_dev, int steps, double *phi_dev, void *stream);

void gcmg_destroy(gcmg_ctx *ctx);
const char *gcmg_last_error(const gcmg_ctx *ctx);

int gcmg_num_levels(const gcmg_ctx *ctx);
int gcmg_level_n(const gcmg_ctx *ctx, int level);

/* Number of ghost points of a level, and the number of unknowns
 * |Omega_h| + |Gamma_h| (the unit of the throughput metric). */
gcmg_status gcmg_num_ghosts(const gcmg_ctx *ctx, int level, int64_t *count);
gcmg_status gcmg_num_unknowns(const gcmg_ctx *ctx, int level, int64_t *count);

/* Ghost geometry of a level (host outputs, any may be NULL):
 * node_host[count]  linear node index of each ghost G,
 * B_host[count*dim] closest boundary point B (Eq. clpt),
 * nu_host[count*dim] discrete outward normal at B used by the Neumann row,
 * case_host[count]  stencil: 0 quadratic 3^d, 1 linear 2^d, 2 corner, 3 two-point. */
gcmg_status gcmg_ghost_geometry(const gcmg_ctx *ctx, int level, int64_t *node_host, double *B_host,
                                double *nu_host, uint8_t *case_host);

/* Full ghost equations of a level for inspection (host outputs, any may be
 * NULL): stencil nodes stn_host[count*27] and Dirichlet / Neumann weights
 * wD_host, wN_host[count*27] (unused slots: node = G, weight 0). */
gcmg_status gcmg_ghost_equations(const gcmg_ctx *ctx, int level, int64_t *stn_host, double *wD_host,
                                 double *wN_host);

/* Node types of a level (host, n^d bytes): 0 outside, 1 inside (Omega_h),
 * 2 ghost (Gamma_h); bit 2 (value 4) marks inside nodes of the extra-sweep
 * band (distance -phi/|grad phi| <= delta, Sec. 3.2). */
gcmg_status gcmg_node_types(const gcmg_ctx *ctx, int level, uint8_t *types_host);

/* Junction zone of a level under its current boundary types (host, n^d
 * bytes): 1 for the unknowns within R_J h of a junction ghost, else 0. */
gcmg_status gcmg_junction_zone(const gcmg_ctx *ctx, int level, uint8_t *mask_host);

/* The unknowns whose equations the exact junction solve of a level solves
 * (host, n^d bytes, 1 / 0) under its current boundary types; all 0 unless
 * junction_solve is set.  Builds the zone's inverses if they are out of date
 * (GCMG_E_GEOM: singular or too large a component). */
gcmg_status gcmg_junction_solve_set(gcmg_ctx *ctx, int level, uint8_t *mask_host);

/* Boundary type per ghost of a level (host, count bytes): 0 Dirichlet, 1
 * Neumann -- whether the ghost's B lies on Gamma_D or Gamma_N.  Must be given
 * for every level whose ghosts are not all Dirichlet; sets the relaxation
 * coefficient mu dt of each ghost and, for the coarsest level, refactors the
 * dense inverse. */
gcmg_status gcmg_set_bc_types(gcmg_ctx *ctx, int level, const uint8_t *types_host);

/* The boundary types a level's ghosts carry now (host, count bytes, 0
 * Dirichlet, 1 Neumann): those of gcmg_set_bc_types or of the mask below. */
gcmg_status gcmg_bc_types(const gcmg_ctx *ctx, int level, uint8_t *types_host);

/* Boundary types of every level from a Dirichlet/Neumann mask on the fine
 * grid (Sec. 2.1: Gamma = Gamma_D u Gamma_N; a ghost's type is that of the
 * part its B lies on, Sec. 2.3): mask_dev (device, n^d bytes, 0 Dirichlet,
 * nonzero Neumann).  For each ghost of each level the mask is read at the
 * fine node nearest B (per axis round((B_a - origin_a) / h); a tie goes to the
 * side of the ghost G itself), on the device; the types then take effect as
 * with gcmg_set_bc_types on every level.  Synchronises the stream. */
gcmg_status gcmg_set_bc_types_from_mask(gcmg_ctx *ctx, const uint8_t *mask_dev);

/* Right-hand side: f_dev (device, n^d doubles; values at inside nodes are
 * used) and g_dev (device, one double per fine ghost: g_D(B) or g_N(B)). */
gcmg_status gcmg_set_rhs(gcmg_ctx *ctx, const double *f_dev, const double *g_dev);

/* Multigrid solve: u_dev (device, n^d doubles) holds the initial guess on
 * entry and the solution on exit (0 off Omega_h u Gamma_h).  Stops at
 * rel <= rtol, after max_cycles, at a NaN/Inf defect or once the defect has
 * grown in diverge_cycles consecutive cycles (stats->diverged = 1); returns
 * GCMG_E_NOCONV if not converged.  stats may be NULL. */
gcmg_status gcmg_solve(gcmg_ctx *ctx, double *u_dev, gcmg_stats *stats);

/* Replaces the cycle limit of the next solves (params.max_cycles, 1..256; the
 * paper runs a fixed number of cycles or stops on the defect, Sec. 3).  The
 * limit lives in device memory, so a captured solve graph is kept (e.g. one
 * cycle from a given start, to see the defect it leaves, then the rest of the
 * solve from its result).  GCMG_E_ARG outside [1, 256]. */
gcmg_status gcmg_set_max_cycles(gcmg_ctx *ctx, int max_cycles);

/* FP64 defect of a fine-grid function (TGCS step 3, Eq. discr): r_dev
 * (device, n^d doubles) = f + Lap_h u on Omega_h, g - L_h u on Gamma_h (stored
 * at the ghost node), 0 elsewhere, with the f and g of gcmg_set_rhs; u_dev
 * (device, n^d doubles) is read at Omega_h u Gamma_h.  rel_norm (host, may
 * be NULL) = ||r||_inf / ||(f, g)||_inf over Omega_h u Gamma_h (the solve's
 * relative residual; 0 if f = g = 0).  GCMG_E_STATE before gcmg_set_rhs. */
gcmg_status gcmg_residual(gcmg_ctx *ctx, const double *u_dev, double *r_dev, double *rel_norm);

/* Same solve with host buffers: f_host (n^d) and g_host (fine ghosts) to the
 * device, a solve from u = 0, the solution copied to u_host (n^d).  When
 * f_host is page-locked (device-addressable host memory) the device reads it
 * at the inside nodes only, the only nodes where the solver uses f, and a
 * page-locked u_host is stored by the device; other host memory is copied
 * whole.  The buffers are read and written before the call returns. */
gcmg_status gcmg_solve_host(gcmg_ctx *ctx, const double *f_host, const double *g_host, double *u_host,
                            gcmg_stats *stats);

/* f and g of level `level` (device: n_l^d doubles, and one double per ghost
 * of that level in the order of gcmg_ghosts): the problem's data sampled on
 * that level, as gcmg_fmg needs it.  Plain FP64 contexts (precision 0) only:
 * GCMG_E_STATE otherwise. */
gcmg_status gcmg_set_rhs_level(gcmg_ctx *ctx, int level, const double *f_dev, const double *g_dev);

/* Full multigrid (nested iteration; the paper notes it derives from the
 * cycle, Sec. 2.4): the coarsest level's problem solved exactly, then on each
 * finer level the interpolation (Sec. 2.6) of the coarser level's solution
 * improved by nu >= 0 cycles with that level as the finest.  Needs f and g on
 * every level (gcmg_set_rhs for level 0, gcmg_set_rhs_level for the others);
 * the cycles overwrite the coarser levels' f and g with restricted defects,
 * so they must be set again before another call.  u_dev (device, n^d
 * doubles) receives the fine-grid result.  Plain FP64 contexts only. */
gcmg_status gcmg_fmg(gcmg_ctx *ctx, int nu, double *u_dev);

/* ---- single steps of the cycle on caller buffers, for tests and tools.
 * Each works on level `level` of the hierarchy, in FP64, on device grid
 * arrays of that level's size (n_l^d doubles) and per-ghost arrays. */

/* Defect (TGCS step 3): r = f + Lap_h u on Omega_h, r = g - L_h u on Gamma_h,
 * 0 elsewhere; *norm = ||r||_inf over Omega_h u Gamma_h (may be NULL). */
gcmg_status gcmg_defect(gcmg_ctx *ctx, int level, const double *u_dev, const double *f_dev,
                        const double *g_dev, double *r_dev, double *norm);

/* One relaxation R_h in place: red-black Gauss-Seidel on Omega_h (red =
 * even index sum first), then a simultaneous (Jacobi) update of all ghosts
 * (Eqs. jac2d, dir2d, neu2d); with_extra adds the lambda band sweeps of
 * Sec. 3.2. */
gcmg_status gcmg_relax(gcmg_ctx *ctx, int level, double *u_dev, const double *f_dev, const double *g_dev,
                       int with_extra);

/* Defect extension along normals (Sec. 2.6) in place on r_dev (level grid);
 * writes the extension nodes only. */
gcmg_status gcmg_extend(gcmg_ctx *ctx, int level, double *r_dev);

/* Composite restriction (Sec. 2.5) of the fine grid function r_dev (level
 * `level`) to level + 1: fc_dev (coarse grid; inside nodes written, others 0)
 * and gc_dev (one value per coarse ghost). */
gcmg_status gcmg_restrict(gcmg_ctx *ctx, int level, const double *r_dev, double *fc_dev, double *gc_dev);

/* Interpolation (Sec. 2.6) of ec_dev (level + 1 grid) to level `level`:
 * out_dev = I e on Omega_h u Gamma_h, 0 elsewhere. */
gcmg_status gcmg_prolong(gcmg_ctx *ctx, int level, const double *ec_dev, double *out_dev);

/* ---- measurement */

/* Kernel classes whose launches can be timed: the fine-level launches of
 * classes 0-3, the launches of every level of class 4. */
enum {
    GCMG_KERNEL_SMOOTH = 0,   /* red-black interior half-sweep (Eq. jac2d) */
    GCMG_KERNEL_DEFECT = 1,   /* defect (TGCS step 3) */
    GCMG_KERNEL_PROLONG = 2,  /* interpolation and correction (Sec. 2.6) */
    GCMG_KERNEL_RESTRICT = 3, /* composite restriction (Sec. 2.5) */
    GCMG_KERNEL_BOUNDARY = 4  /* 2D boundary blocks: ghost sweep + lambda band sweeps (Sec. 3.2)
                                 of one relaxation in shared memory, every level */
};

/* With kind >= 0, later solves bracket every timed launch of that kernel
 * class with CUDA events on the context's stream (kind = -1: off); graph
 * capture is off meanwhile.  gcmg_kernel_timing synchronises the stream and
 * returns the number of timed launches and their summed device time since
 * the last call or enable. */
gcmg_status gcmg_set_kernel_timing(gcmg_ctx *ctx, int kind);
gcmg_status gcmg_kernel_timing(gcmg_ctx *ctx, int64_t *launches, double *total_ms);
/* As gcmg_kernel_timing, plus the algorithmic bytes of the timed launches
 * that carry the boundary blocks (else 0): per launch each distinct staged
 * node's u read, each distinct inside node's f read, each distinct ghost's
 * 3^d weights, g and mu dt read, each written-back node's u write, in the
 * cycle precision; for the FP32 2D relaxation in one launch (interior sweep
 * and boundary blocks together; timed under class 0 or 4) also the interior
 * sweep's u and f read and u written once per inside node. */
gcmg_status gcmg_kernel_timing_ex(gcmg_ctx *ctx, int64_t *launches, double *total_ms, double *alg_bytes);

/* How the 3D boundary relaxation (the ghost sweep, the lambda band sweeps
 * of Sec. 3.2 and the junction sweeps) is launched; every mode gives the same
 * results bitwise.  mode 0 (default): one launch per phase, the store of
 * each Jacobi ghost sweep merged into the launch of the next red band or
 * junction-zone sweep; 1: on levels whose ghost, band and junction lists
 * hold at most 65,536 entries all phases as one thread-block cluster of 16
 * CTAs with hardware barriers between them, mode 0 on the other levels; 2:
 * all phases as one grid with software barriers.  Modes 1 and 2 measured
 * slower on GB300 (the per-phase launches overlap inside the solve's graph
 * and spread each phase's gathers over every SM).  Not in the paper. */
gcmg_status gcmg_set_boundary3d(gcmg_ctx *ctx, int mode);

/* Mode 2 of gcmg_set_boundary3d with test controls: every software barrier
 * wait gives up after spin_limit polls (default 4,194,304, about a second)
 * and the solve then returns GCMG_E_TIMEOUT with the context still usable;
 * phantom_blocks > 0 makes every barrier wait for that many CTAs that do not
 * exist, so that a test can make the waits run out.  enable = 0 returns to
 * mode 0.  Not in the paper. */
gcmg_status gcmg_debug_barrier(gcmg_ctx *ctx, int enable, int phantom_blocks, unsigned spin_limit);

/* Kernel of the 3D interior sweep (red and black in one pass over the active
 * tiles, Eq. jac2d): 0 tiles of 16 x 64 nodes with the planes staged in
 * shared memory; 1 tiles of 12 x 28 nodes with the planes in registers, a
 * warp a row; 2 blocks of 12 rows whose window along the
 * contiguous axis covers the rows' unknowns, reading and writing only the
 * spans of unknowns of each row (FP32 cycles; FP64 cycles and levels whose
 * rows hold more than one interval of inside nodes use 1); 3 (default)
 * the red and the black half-sweeps as two launches in place over segments
 * of up to 64 inside nodes of a row (both precisions, any domain).  Same
 * results bitwise.  Not in the paper. */
gcmg_status gcmg_set_sweep3d(gcmg_ctx *ctx, int variant);

/* Rebuilds the work items of sweep 2 on every 3D level: `columns` nodes a
 * lane along the contiguous axis (2..5; a window of 32 columns nodes, 0 =
 * chosen per level by a work model) and items of at most `planes` planes
 * (1..32; 0 = 32).  Blocks until done; results are unchanged (tuning only).
 * GCMG_E_ARG for values out of range.  Not in the paper. */
gcmg_status gcmg_set_span3d(gcmg_ctx *ctx, int columns, int planes);

/* 3D junction zone (the mu junction sweeps; not in the paper): enable = 1
 * splits a zone component of more than 1,500 nodes into blocks of 8^3 nodes
 * relaxed in shared memory, each updating the zone within 4 mu nodes of its
 * block and writing back only its own nodes (two launches a relaxation
 * instead of three a sweep; the same results bitwise); 0 (default) keeps
 * whole components (a large one then runs on global lists; measured faster
 * on GB300: the blocks redo about ten times the zone's work).  Rebuilds the
 * junction programs of every level; GCMG_E_ARG for a null context. */
gcmg_status gcmg_set_junction_blocks(gcmg_ctx *ctx, int enable);

/* 2D FP32 relaxation of a level with at least min_strips sweep strips as
 * two launches side by side -- the boundary blocks and the strips' interior
 * nodes, which store disjoint nodes -- instead of one merged launch whose
 * strips share the blocks' shared-memory reservation; 0 (default): always
 * merged (on GB300 the blocks' chain of phases sets the time either way:
 * 4097^2 finest level 26.6 us split, 25.5 us merged).  Same results
 * bitwise.  GCMG_E_ARG for a negative count.  Not in the paper. */
gcmg_status gcmg_set_split2d(gcmg_ctx *ctx, int min_strips);

/* How level l's junction sweeps run in the context's cycle precision (3D
 * mixed form: the FP32 programs, which need less shared memory): 0 on global
 * lists (or no junction zone), 1 whole components in shared memory, 2 blocks
 * in shared memory; -1 for a bad context or level.  Not in the paper. */
int gcmg_junction_mode(const gcmg_ctx *ctx, int l);

/* Sweep 2's work on level l: number of items (0: the level uses sweep 1)
 * and nodes a lane holds.  Not in the paper. */
gcmg_status gcmg_span3d_info(const gcmg_ctx *ctx, int l, int *items, int *columns);

/* Number of CUDA kernels this library has launched in the process so far. */
int64_t gcmg_launch_counter(void);

/* ---- batched solves of many domains (not in the paper).
 * Independent 2D domains of uneven grid sizes are solved together: each step
 * of the cycle is one kernel launch over all domains and the whole solve --
 * FP32 V-cycles inside FP64 iterative refinement until every domain reaches
 * rtol -- is one CUDA-graph launch with a device-side loop. */
typedef struct gcmg_batch gcmg_batch;

/* Creates `count` domains: params[i] (dim 2, precision 1; gamma (V or W cycles),
 * nu1, nu2, lambda, junction_sweeps and junction_solve equal across domains; with
 * gamma = 2 every domain must have the same number of levels; rtol and max_cycles of
 * params[0] apply to the batch) and phi_dev[i] (device, n_i^2 doubles).  The
 * host geometry of the domains is built in parallel threads. */
gcmg_status gcmg_batch_create(int count, const gcmg_params *params, const double *const *phi_dev, void *stream,
                              gcmg_batch **out);
void gcmg_batch_destroy(gcmg_batch *batch);
const char *gcmg_batch_last_error(const gcmg_batch *batch);
int gcmg_batch_size(const gcmg_batch *batch);

/* The context of domain i, owned by the batch: use it for the ghost
 * geometry, gcmg_set_bc_types and gcmg_set_rhs of that domain (do not destroy
 * it, and do not call gcmg_solve on it while the batch is in use). */
gcmg_ctx *gcmg_batch_domain(gcmg_batch *batch, int i);

/* Solves every domain from u = 0.  stats (may be NULL) receives one entry per
 * domain; *steps (may be NULL) the number of refinement steps the batch ran
 * (all domains run the same number).  GCMG_E_NOCONV if a domain missed rtol. */
gcmg_status gcmg_batch_solve(gcmg_batch *batch, gcmg_stats *stats, int *steps);

/* Copies the solution of domain i to u_dev (device, n_i^2 doubles). */
gcmg_status gcmg_batch_get_solution(gcmg_batch *batch, int i, double *u_dev);

/* on = 0: later solves run their steps as plain kernel launches from a host
 * loop that reads the stop condition after each step (the same kernels and
 * results; for profilers, which cannot look inside the graph's while node);
 * on = 1 (default): one graph launch per solve. */
gcmg_status gcmg_batch_set_graph(gcmg_batch *batch, int on);

/* Height of the strips of the interior sweep (each strip: 60 owned columns,
 * one warp): 0 = 8 rows, 1 = 16 rows, 2 = 32 rows. */
gcmg_status gcmg_batch_set_tiles(gcmg_batch *batch, int variant);

/* Autotuner: times the batched interior sweeps of one cycle with every strip
 * height, selects the fastest (*best) and reports each time in ms[0..2]. */
gcmg_status gcmg_batch_autotune(gcmg_batch *batch, int *best, double *ms);

/* ---- allocation-free defect (no counterpart in the paper: a service for
 * callers that cannot allocate device memory -- code whose device memory is
 * all owned by another allocator, such as a framework's caching pool or an
 * arena reserved under a fixed budget, and latency-critical loops that must
 * not pay the device-wide synchronisation of cudaMalloc / cudaFree).
 *
 * Same result as gcmg_defect without a context: the caller passes every input
 * and output.  type_dev: node types (n^dim bytes, 0 outside, 1 inside, 2
 * ghost; higher bits ignored), u_dev, f_dev, r_dev: n^dim doubles, h = 2/(n-1);
 * ng ghosts with gnode_dev[ng] (node index), stn_dev[ng*27] and w_dev[ng*27]
 * (the ghost's stencil nodes and the weights of its boundary type, as
 * returned by gcmg_ghost_equations; unused slots weight 0) and g_dev[ng].
 * Writes r on the whole grid and, if norm_host is not NULL, ||r||_inf over
 * inside nodes and ghosts (after synchronising the stream).
 *
 * It allocates nothing: its scratch is a fixed array of 65,537 doubles
 * (512 KiB) in the library's device image, held by every device that loads
 * the library until the process exits.  Capacity: n^dim + ng <= 67,108,864;
 * larger problems return GCMG_E_SIZE.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  All calls on a device share the array: calls
 * that overlap on the GPU race and must be serialised by the caller. */
gcmg_status gcmg_defect_noalloc(int dim, int n, double h, const uint8_t *type_dev, const double *u_dev,
                                const double *f_dev, int64_t ng, const int32_t *gnode_dev, const int32_t *stn_dev,
                                const double *w_dev, const double *g_dev, double *r_dev, double *norm_host,
                                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GCMG_H */
