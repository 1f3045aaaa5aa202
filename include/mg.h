/*
 * mg.h -- C ABI of the GB300 nested-grid multigrid Poisson solver
 * (Wang & Yen, "Self-gravitational Force Calculation of Second Order Accuracy
 * Using Multigrid Method on Nested Grids").
 *
 * The problem (Eq. 1): lap(Phi) = 4 pi G rho, F = -grad(Phi), on a nested
 * hierarchy of square (2D) or cubic (3D) patches Omega^0 superset Omega^1 ...
 * with refinement ratio 2 (Sec. 2.1).  Densities are point values at cell
 * centres.  Levels are solved one at a time from coarse to fine (the one-way
 * scheme, Sec. 2.1): each finer level gets its Dirichlet potential (outer
 * buffer ring) and the density of its inner buffer ring by linear
 * interpolation from its parent, then is solved by multigrid V-cycles
 * (Sec. 2.3) with red-black Gauss-Seidel smoothing, averaging restriction,
 * bi/trilinear prolongation and the anti-symmetric ghost rule of Sec. 2.4 on
 * the coarse multigrid levels.  Forces come from the fourth-order difference
 * of Eq. 2.
 *
 * Conventions common to every call
 *   - Arrays are C order with x fastest: 3D index (k*n + j)*n + i, 2D j*n + i.
 *   - Array pointers may be host or device memory; the library inspects each
 *     pointer (cudaPointerGetAttributes).  Page-locked host memory that CUDA
 *     maps into the device address space (cudaMallocHost, cudaHostAlloc,
 *     cudaHostRegister; torch pin_memory) is read and written by the kernels
 *     in place over the host link; other host memory is copied through a
 *     library staging area on the hierarchy's stream.  The library never keeps
 *     a caller pointer after a call returns.  Host pointers make the call
 *     synchronous with respect to that stream.
 *   - The library owns all its device memory (allocated in
 *     mg_create_hierarchy, freed in mg_destroy) and runs on one GPU, the
 *     current device at creation.
 *   - Calls on one handle are not thread-safe.  Errors are returned, never
 *     raised; after MG_ECUDA or MG_ETIMEOUT the handle answers MG_ESTATE to
 *     everything but mg_destroy.  mg_error_message() gives the detail.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_MAX_LEVELS 8   /* refinement levels per hierarchy */

typedef struct mg_hierarchy mg_hierarchy;   /* opaque; owns all device state */

typedef enum {
    MG_OK = 0,
    MG_EINVAL = 1,      /* bad argument (message says which) */
    MG_ENOMEM = 2,      /* device or host allocation failed */
    MG_ECUDA = 3,       /* a CUDA call failed; handle poisoned */
    MG_ESTATE = 4,      /* call out of order, or handle poisoned */
    MG_ENOCONV = 5,     /* max_cycles reached above rel_tol (results are valid, unconverged) */
    MG_EDIVERGED = 6,   /* the right-hand side or the residual is NaN/Inf */
    MG_ETIMEOUT = 7     /* a bounded device-side wait gave up */
} mg_status;

enum { MG_FP64 = 0,        /* every step in FP64 */
       MG_MIXED = 1 };     /* FP32 V-cycles inside FP64 defect correction */

enum { MG_GUESS_INTERP = 0,  /* initial potential interpolated from the parent (Sec. 2.4) */
       MG_GUESS_ZERO = 1,    /* zero initial potential */
       MG_GUESS_USER = 2,    /* initial potential supplied by mg_set_guess */
       MG_GUESS_LEARNED = 3 };  /* interpolated potential corrected by the network of mg_set_unet
                                   (levels whose n is a power of two <= the network's nmax;
                                   others use the interpolated potential) */

enum { MG_FORCE_EQ2 = 0,     /* fourth-order difference of Eq. 2 (default) */
       MG_FORCE_CD2 = 1 };   /* two-point central difference */

/* When a level stops iterating (besides max_cycles). */
enum { MG_STOP_RESIDUAL = 0, /* ||b - A Phi||_2 / ||b||_2 < rel_tol over Gamma (default) */
       MG_STOP_FORCE = 1 };  /* the test of Sec. 3.1 / 3.2: the acceleration on Omega
                                (force_stencil) changes by less than rel_tol between
                                two iterations, measured as the largest length of the
                                change vector over the cells; at least one iteration.
                                mg_level_stats.rel_res then holds that change.  Only
                                with MG_IFACE_BUFFER. */

/* Treatment of the buffer rings of levels l > 0. */
enum { MG_IFACE_BUFFER = 0,  /* Sec. 2.1 (default): the outer ring holds potential
                                interpolated from level l-1, the inner ring holds
                                interpolated density and its potential is solved
                                together with the patch (M = n + 2 active cells) */
       MG_IFACE_FROZEN = 1 };/* the scheme Sec. 4 and Fig. 4 compare against, as an
                                ablation: both rings hold interpolated potential and
                                multigrid solves Omega alone with the inner ring as
                                its Dirichlet boundary (M = n active cells) */

/* Geometry of one hierarchy (Sec. 2.1): num_levels patches, patch 0 the
 * base.  Patch l has n[l] cells per edge (>= 2; even for l > 0; at most 1286
 * in 3D) and lower corner lo[l].  Its parent is patch l-1 (tree = 0: a chain
 * of nested levels, one patch per refinement level) or patch parent[l] <
 * l (tree = 1: several patches may share a parent, the patch-based refinement
 * of Sec. 5); a patch's cell size is h0 / 2^depth, depth = the number of
 * steps to the base.  Every "level" argument of the calls below is a patch
 * index.  A child must sit on parent cell faces, its lower corner o[a] whole
 * parent cells above the parent's, with 1 <= o[a] <= n[parent] - n[l]/2 - 1
 * so that every buffer cell interpolates from cells the parent solves for.
 * Sibling patches are solved independently (each from its parent); their
 * overlap, if any, is not reconciled. */
typedef struct {
    int dim;                          /* 2 or 3 */
    int num_levels;                   /* 1..MG_MAX_LEVELS patches, patch 0 is the base */
    int n[MG_MAX_LEVELS];
    double lo[MG_MAX_LEVELS][3];
    double h0;                        /* cell size of patch 0 (> 0) */
    double G;                         /* gravitational constant of Eq. 1 */
    int tree;                         /* 0: parent of patch l is l-1; 1: parent[l] */
    int parent[MG_MAX_LEVELS];        /* tree = 1: parent patch of l > 0, < l */
} mg_hierarchy_desc;

#define MG_INNER_MAX 32   /* largest mg_options.inner_max */

/* Solver options; mg_default_options fills the paper's choices. */
typedef struct {
    int nu_pre;          /* Gauss-Seidel sweeps before restriction (paper: 2, Sec. 3) */
    int nu_post;         /* sweeps after prolongation (paper: 1) */
    int max_cycles;      /* V-cycle limit per level (FP64: V-cycles; MIXED: FP32 V-cycles) */
    double rel_tol;      /* stop when ||f - lap Phi||_2 / ||f - lap Phi_0||_2 < rel_tol over
                            the solved cells, Phi_0 being zero inside with the same boundary;
                            0 runs exactly max_cycles cycles */
    int precision;       /* MG_FP64 | MG_MIXED */
    int inner_cycles;    /* MIXED: FP32 V-cycles per FP64 defect-correction step (>= 1) */
    int guess;           /* MG_GUESS_* for levels > 0 (level 0 starts from zero, or USER) */
    int force_stencil;   /* MG_FORCE_EQ2 | MG_FORCE_CD2 */
    int interface;       /* MG_IFACE_BUFFER | MG_IFACE_FROZEN */
    int stop;            /* MG_STOP_RESIDUAL | MG_STOP_FORCE */
    void *stream;        /* cudaStream_t to run on; NULL = the legacy default stream */
    int inner_max;       /* MIXED under MG_STOP_RESIDUAL, 0..MG_INNER_MAX: 0 runs inner_cycles
                            FP32 V-cycles in every defect-correction step; > 0 runs inner_cycles in
                            the first step and lets each later step choose its count, 1..inner_max:
                            the cycles that the per-cycle residual contraction of the step before
                            predicts for reaching rel_tol, one more after a step of fewer than four
                            cycles (decided on the device, in the graph; a batch then runs as graph
                            branches or the persistent launch, not the opt-in batched kernels).
                            Not part of the paper's method, whose V-cycles are all FP64. */
} mg_options;

/* Per (hierarchy, level) result of mg_solve. */
typedef struct {
    int cycles;          /* V-cycles run (FP32 V-cycles in MIXED mode) */
    int outer_steps;     /* MIXED: FP64 defect-correction steps; FP64: equal to cycles */
    double rel_res;      /* final ||r||_2 / ||b||_2 (FP64) */
    double b_norm;       /* ||b||_2 */
    int status;          /* MG_OK, MG_ENOCONV or MG_EDIVERGED */
} mg_level_stats;

/* Fill *opt with nu_pre = 2, nu_post = 1 (Sec. 3), max_cycles = 50,
 * rel_tol = 1e-10, MG_FP64, inner_cycles = 3, MG_GUESS_INTERP, MG_FORCE_EQ2,
 * stream NULL, inner_max = 0.  Returns MG_EINVAL if opt is NULL. */
mg_status mg_default_options(mg_options *opt);

/* Create `batch` independent hierarchies (Sec. 2.1 data structure) with
 * descriptions descs[0..batch-1], allocate all their device memory and build
 * the multigrid level sizes of every refinement level (Sec. 2.2: the solved
 * region of n+2 cells per edge, halved until one active cell remains, sizes
 * rounded half up).  opt may be NULL (defaults).  On success *out owns the
 * memory; on failure *out is NULL.  Errors: MG_EINVAL (geometry violates the
 * nesting rules above, batch < 1, bad options), MG_ENOMEM, MG_ECUDA. */
mg_status mg_create_hierarchy(const mg_hierarchy_desc *descs, int batch, const mg_options *opt,
                              mg_hierarchy **out);

/* Give hierarchy b its density on level `level` (Sec. 2.1: point values at
 * the cell centres of Omega^level).
 *   rho     n^d values on Omega^level.
 *   bc_rho  level 0 only: (n+2)^d density at the centres of Omega^0 plus one
 *           ring; only the ring (the inner buffer layer) is read.
 *   bc_phi  level 0 only: (n+4)^d potential at the centres of Omega^0 plus two
 *           rings; only the outer ring (the Dirichlet layer) is read.
 * For level > 0 both must be NULL: the interface of Sec. 2.1 fills them from
 * the parent during mg_solve.  Every level of a hierarchy must be set before
 * mg_solve.  Errors: MG_EINVAL, MG_ESTATE, MG_ECUDA. */
mg_status mg_set_density(mg_hierarchy *h, int b, int level, const double *rho, const double *bc_rho,
                         const double *bc_phi);

/* Optional initial potential of hierarchy b on `level`: (n+2)^d values on
 * the solved region (Omega plus the inner ring), used when opt.guess is
 * MG_GUESS_USER (for level 0 it replaces the zero start whatever the guess
 * mode).  Must follow mg_set_density for that level.  The call only records
 * the values; they are copied in when the level's solve starts. */
mg_status mg_set_guess(mg_hierarchy *h, int b, int level, const double *phi0);

/* Solve every hierarchy, every level, coarse to fine (Sec. 2.1 one-way
 * scheme; Sec. 2.3 multigrid iteration).  stats, if not NULL, receives
 * batch * MG_MAX_LEVELS entries (entry b*MG_MAX_LEVELS + level).
 * Returns MG_OK when every level reached rel_tol, MG_ENOCONV if some level
 * stopped at max_cycles (results still usable), MG_EDIVERGED on a non-finite
 * residual, MG_ESTATE if a density is missing, MG_ECUDA. */
mg_status mg_solve(mg_hierarchy *h, mg_level_stats *stats);

/* Results of hierarchy b on `level` after mg_solve.
 *   phi_out  n^d potential on Omega^level, or NULL.
 *   F_out    dim * n^d force F = -grad(Phi) (Eq. 1) by Eq. 2 (or the two-point
 *            difference), component a at F_out[a * n^d + cell]; or NULL.
 * Errors: MG_EINVAL, MG_ESTATE (no solve yet), MG_ECUDA. */
mg_status mg_forces(mg_hierarchy *h, int b, int level, double *phi_out, double *F_out);

/* Register where mg_solve itself writes the results of hierarchy b on
 * `level` (the values mg_forces would give, same layouts): F_out (required
 * for phi_out) and phi_out, each device memory or page-locked host memory
 * (written in place); NULL, NULL unregisters.  mg_solve then computes them
 * after the solves, inside its own graph launch, and returns with them
 * complete (no synchronisation per level, as mg_forces needs for host
 * arrays).  The pointers are kept until changed
 * (a change rebuilds the solve graph once).  Not part of the paper: the
 * results of Sec. 2 (Eq. 2) without a call per level.  Errors: MG_EINVAL
 * (range, phi without F, pageable host memory). */
mg_status mg_set_outputs(mg_hierarchy *h, int b, int level, double *phi_out, double *F_out);

/* How many hierarchies of the batch the solve graph gives to the persistent
 * launch (one launch, one thread block per hierarchy at a time, solving its
 * levels with block-wide phases; chosen when a cost model of the two puts it
 * ahead of one graph branch per hierarchy, which suits many small
 * hierarchies), 0 when every hierarchy runs as graph branches, -1 before the
 * first mg_solve builds the graph or with a NULL handle.  Not part of the
 * paper. */
int mg_persistent_count(const mg_hierarchy *h);

/* Release everything; NULL-safe; always MG_OK. */
mg_status mg_destroy(mg_hierarchy *h);

/* Static description of a status code. */
const char *mg_status_str(mg_status s);

/* Detail of the last error on h (empty string if none); valid until the next
 * call on h.  h may be NULL (reports the last creation error). */
const char *mg_error_message(const mg_hierarchy *h);

/* Per-kernel timing, for measurement (not part of the method).  While
 * enabled, every kernel launch of the handle is bracketed by CUDA events on
 * its stream; mg_profile_read synchronises that stream and reports, per
 * kernel kind, the launch count, the summed event time and the summed
 * algorithmic bytes (the minimal DRAM traffic each launch must move).
 * mg_profile(h, 0/1) also clears the totals. */
typedef struct {
    char name[32];
    long launches;
    double ms;
    double bytes;
} mg_kernel_stat;
mg_status mg_profile(mg_hierarchy *h, int enable);
/* Fills up to cap entries; returns how many kernel kinds ran, or -1. */
int mg_profile_read(mg_hierarchy *h, mg_kernel_stat *out, int cap);

/* Attach the learned initial guess (include/unet.h) used by MG_GUESS_LEARNED;
 * the solver runs it on its stream inside mg_solve.  net may be NULL
 * (detach).  The network must outlive its use by h. */
struct mg_unet;
mg_status mg_set_unet(mg_hierarchy *h, struct mg_unet *net);

/* After mg_solve: the initial potential level `level` (> 0) of hierarchy b
 * started from under MG_GUESS_INTERP -- the parent's solution interpolated
 * onto the level (Sec. 2.4) -- on Omega, n^d values into out, and (resid_out
 * not NULL) its h^2-scaled residual h^2 (4 pi G rho - lap_h Phi) there (device
 * or host pointers).  Used to build training data for the learned guess. */
mg_status mg_interp_guess(mg_hierarchy *h, int b, int level, double *out, double *resid_out);

/* Autotuner of the mixed-precision V-cycle (not part of the method; it picks
 * among equivalent launch plans).  For each distinct level size it times, on
 * the level's own FP32 correction arrays, (1) the size limit of the one-block
 * kernel for the coarse multigrid levels (4, 8 or 17 cells per edge) and
 * (2) for every multigrid level above it, how its smoothing runs: one
 * kernel per colour and phase (0), the temporally blocked legs (tile 8, 12 or
 * 16), or the plane-marching sweeps (3D, 1-2 sweeps per stint: every stint one
 * launch, two tile shapes and three splits of z each).
 * Every choice computes the same result.  cache_path (may be NULL) is a text
 * file of earlier choices keyed by (dim, n, nu_pre, nu_post); new choices are
 * appended.  No-op for MG_FP64.  Call after mg_create_hierarchy, before
 * mg_solve.  Errors: MG_EINVAL, MG_ESTATE, MG_ECUDA. */
mg_status mg_autotune(mg_hierarchy *h, const char *cache_path);

/* The current FP32 plan of hierarchy b's level: writes the plan of each
 * multigrid level into tiles[0..cap) (0 = one kernel per phase, > 0 the
 * blocked legs' tile, < 0 the plane-marching sweeps: -(256 * tile shape +
 * z-chunks), tile shape 0 = 56 x 10, 1 = 56 x 6) and returns
 * the edge of the first level run by the one-block kernel (-1 on bad
 * arguments). */
int mg_tuning(const mg_hierarchy *h, int b, int level, int *tiles, int cap);

/* Time multigrid level L of hierarchy b's refinement level `level` as the
 * solve graph launches it (measurement, not part of the method; MG_MIXED
 * only, L above the one-block kernel).  `launches` smoothing launches of the
 * level's current FP32 plan are captured back to back into one CUDA graph with
 * programmatic dependent launch, as in mg_solve, and the graph is replayed on
 * the handle's stream between CUDA events (one warm-up replay, then five;
 * with MG_SOLVE_GRAPH=0 the launches run and are timed without a graph).
 * Plane-marching plan: one launch = nu_pre complete red-black sweeps, the FP32
 * correction arrays ping-ponged; one-kernel-per-phase plan: one launch = one
 * colour in place.  Writes the mean time per launch in microseconds and the
 * algorithmic bytes per launch, the least DRAM traffic the launch must move:
 * 3 words per active cell for a plane-marching launch (Phi and f read once,
 * Phi written once), 1.5 for one colour (Phi read, half of f read, half of
 * Phi written).  Overwrites the level's FP32 correction arrays, which the next
 * mg_solve rewrites.  Errors: MG_EINVAL, MG_ESTATE, MG_ECUDA. */
mg_status mg_time_smoothing(mg_hierarchy *h, int b, int level, int L, int launches, double *us_per_launch,
                            double *bytes_per_launch);

/* Allocation-free solve of one refinement level, for callers that cannot
 * allocate device memory: codes that give all of the GPU's memory to their
 * own pool, or call the Poisson solve inside a time step where cudaMalloc and
 * cudaFree (and the device-wide synchronisation they imply) are not allowed.
 * The paper has no counterpart; the arithmetic is that of mg_solve for a
 * single level (FP64 V-cycles, zero ghost rule on coarse levels), with the
 * same kernels in the same order.
 *   rho   device, (n+4)^d block: density on the solved region (Omega and the
 *         inner buffer ring, storage indices 1..n+2); other cells unread.
 *   phi   device, (n+4)^d block: on entry the outer ring holds the Dirichlet
 *         potential and the solved region the initial guess; on return the
 *         solved region holds the solution.
 *   h, G  cell size and gravitational constant; opt as for mg_solve (NULL =
 *         defaults); precision must be MG_FP64 and stop MG_STOP_RESIDUAL;
 *         opt->stream is used.
 *   stats host, may be NULL.
 * Working memory is one library-owned device array of 4 MiB (every GPU that
 * loads the library holds it until the process exits): n <= 69 in 3D and
 * n <= 554 in 2D; larger n is rejected with MG_EINVAL before any GPU work.
 * The array is shared by every call and keeps the previous call's contents
 * (the call clears the part it uses): calls whose GPU work overlaps race and
 * must not be issued concurrently.  The first call on each device looks the
 * array's device address up once (cudaGetSymbolAddress with that device
 * current).  Every call waits on the host for its residual norms, so it must
 * never be issued on a stream that is capturing a graph: such a stream is
 * refused with MG_EINVAL before any work.  Errors: MG_EINVAL (message on
 * stderr), MG_ECUDA (the call first waits for the work it queued, so that
 * nothing of it runs on when it returns), and MG_ENOCONV / MG_EDIVERGED as
 * for mg_solve.  The call returns after the solve has finished. */
mg_status mg_solve_level_noalloc(int dim, int n, double h, double G, const double *rho, double *phi,
                                 const mg_options *opt, mg_level_stats *stats);

/* Multigrid level sizes of Sec. 2.2 for a solved region of M cells per edge:
 * writes up to cap sizes into N and returns how many levels there are. */
int mg_level_sizes(int M, int *N, int cap);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
