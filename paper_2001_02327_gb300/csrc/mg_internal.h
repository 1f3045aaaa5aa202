// mg_internal.h -- declarations shared by the host driver and the kernels of
// the nested-grid multigrid solver.  Not part of the public ABI (include/mg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cmath>
#include <cstdlib>

#define MG_MAX_MG 16          // multigrid levels per refinement level (n+2 <= 2^15)

// One multigrid level L of one refinement level (Sec. 2.2).  Active cells use
// 1-based indices 1..N per axis inside an (N+2)^d array with one ghost layer.
// At L = 0 the ghost layer is the outer buffer ring of the refinement level
// and holds Dirichlet data; at L > 0 it is never read: the ghost rule of
// Sec. 2.4 is folded into the boundary cells' stencil coefficients.
struct MgGeom {
    int N;          // active cells per edge
    int E;          // N + 2, storage edge
    int L;          // multigrid level, 0 = finest
    int tie;        // centre of cell N sits exactly at x_MG = 1
    double cR;      // right ghost = cR * Phi_N when !tie
    double h2;      // squared physical cell size of this multigrid level
    double inv_h2;  // 1 / h2
    // the same constants rounded to FP32 for the FP32 kernels (a conversion
    // from double runs on the FP64 pipe, which this part has little of)
    float cRf, h2f, inv_h2f;
    // Optional device tables of the ghost-folded diagonal of boundary cells
    // (L > 0), indexed by the per-axis boundary class c_x + 4 c_y + 16 c_z
    // (class: bit 0 = first active cell, bit 1 = last): entries 0..63 hold
    // the diagonal, 64..127 its negated reciprocal.  NULL: computed in place.
    const double *tab64;
    const float *tab32;
    // FP32 storage of this level: sH = 0 plain; sH > 0 colour-split -- cell
    // (i, j, k) of colour (i + j + k) & 1 at colour * shalf + (k E + j) sH + i / 2,
    // sH = mg_split_H(E) words per row of one colour, shalf = sH E^(d-1)
    int sH;
    long long shalf;
};

// Words per row of one colour in colour-split FP32 storage: half the row,
// rounded up to a multiple of 4 so that every row starts 16-byte aligned.
__host__ __device__ inline int mg_split_H(int E) { return ((E + 1) / 2 + 3) & ~3; }

// Index of cell (i, j, k) (storage indices) in an FP32 array of level g
__host__ __device__ inline long long mg_idx32(const MgGeom &g, int dim, int i, int j, int k)
{
    if (g.sH > 0)
        return ((i + j + k) & 1) * g.shalf + ((long long)k * g.E + j) * g.sH + (i >> 1);
    return dim == 3 ? ((long long)k * g.E + j) * g.E + i : (long long)j * g.E + i;
}

// Diagonal contribution of one axis for boundary class c (Sec. 2.4 ghost
// rule folded in): left ghost -Phi_1 adds -1; right ghost cR Phi_N adds cR,
// or, when x_N = 1, -Phi_{N-1} cancels the left neighbour instead.
__host__ __device__ inline double mg_axis_diag(int c, const MgGeom &g)
{
    double d = -2.0;
    if (c & 1)
        d -= 1.0;
    if (c & 2) {
        if (g.tie) {
            if (g.N < 2)
                d += 1.0;   // -Phi_0 = +Phi_1
        } else {
            d += g.cR;
        }
    }
    return d;
}

// Fill tab[0..127] (diagonal, then -1/diagonal) for a level of dimension dim.
inline void mg_fill_diag_table(const MgGeom &g, int dim, double *tab)
{
    for (int c = 0; c < 64; c++) {
        const int cx = c & 3, cy = (c >> 2) & 3, cz = (c >> 4) & 3;
        double d = mg_axis_diag(cx, g);
        d += mg_axis_diag(cy, g);
        if (dim == 3)
            d += mg_axis_diag(cz, g);
        tab[c] = d;
        tab[64 + c] = 1.0 / (-d);
    }
}

// ---------------------------------------------------------------------------
// kernel launchers (mg_kernels.cu).  `fp32` selects float arrays; the
// geometry is the same.  All launches go to stream s and return the launch
// error (cudaGetLastError).
// ---------------------------------------------------------------------------
struct MgSolveCtl;
// One colour (0 = red, (i+j[+k]) even; 1 = black) of a Gauss-Seidel sweep;
// ctl != NULL: the launch also counts one V-cycle of an adaptive step's
// nested loop (ctl->cycles, ctl->left) and sets that loop's condition hi.
cudaError_t mg_launch_smooth(int dim, bool fp32, void *phi, const void *f, const MgGeom &g, int colour,
                             cudaStream_t s, MgSolveCtl *ctl = nullptr, cudaGraphConditionalHandle hi = 0);
// The levels at and below a multigrid level Ls, run by one thread block with
// all their arrays in shared memory (k_bottom).
#define MG_BOTTOM_MAX 12
#define MG_BOTTOM_SMEM_MAX (200 * 1024)
struct MgBottom {
    int nlev;                   // levels Ls .. Ls+nlev-1 (the last one has one cell)
    MgGeom g[MG_BOTTOM_MAX];
    // device image of the kernel's per-cell plan for exactly these levels
    // (mg_launch_bottom_plan), or NULL: the kernel then builds it itself
    const void *plan = nullptr;
};

// One thread-block cluster running the V-cycle from a multigrid level Lc down
// (levels Lc + q, q = 0..nlev-1) with every array in the shared memory of the
// cluster's CTAs (3D): levels q < nclu are split by z-planes over the CTAs
// (CTA r owns planes [ceil(r E / C), ceil((r+1) E / C))), level nclu lives in
// CTA 0, and the levels below it are the one-block path (plan `bt`) of CTA 0.
// In every CTA, level q's Phi planes start at element off[q] and its f planes
// pmax[q] planes later; the one-block scratch starts at byte `scratch`.
// phi[0] / f[0]: the global arrays of level Lc, loaded at the start (both)
// and stored at the end (Phi).  nclu >= 1, nclu < nlev.
#define MG_CLUSTER_THREADS 512
#define MG_CLUSTER_PLANES 256
#define MG_CLUSTER_SMEM_MAX (220 * 1024)
struct MgClusterPlan {
    int nlev, nclu, cycles, nu_pre, nu_post;
    MgGeom g[MG_MAX_MG];
    void *phi0;
    const void *f0;
    int pmax[MG_MAX_MG];
    int off[MG_MAX_MG + 1];
    int scratch;
    MgBottom bt;
};

size_t mg_bottom_smem(int dim, bool fp32, const MgBottom &bt);
size_t mg_bottom_plan_bytes(int dim, bool fp32, const MgBottom &bt);
// writes the per-cell plan of bt's levels to `img` (mg_bottom_plan_bytes)
cudaError_t mg_launch_bottom_plan(int dim, bool fp32, const MgBottom &bt, void *img, cudaStream_t s);
cudaError_t mg_bottom_prepare();   // once per device before the first launch
cudaError_t mg_launch_bottom(int dim, bool fp32, void *phi, const void *f, const MgBottom &bt, int nu_pre,
                             int nu_post, cudaStream_t s);

// Temporally blocked FP32 legs of the V-cycle (tile^d fine cells per block,
// tile even): pre = nu red-black sweeps, residual and restriction to the
// next level (phi_in -> phi_out, f_c, phi_c = 0); post = prolongation of
// phi_c, correction and nu sweeps (phi_in -> phi_out).
#define MG_TB_SMEM_MAX (200 * 1024)
size_t mg_tb_smem(int dim, bool fp32, int tile, int halo);
cudaError_t mg_tb_prepare();
cudaError_t mg_launch_tb_pre(int dim, const float *phi_in, float *phi_out, const float *f, const MgGeom &g,
                             float *phi_c, float *f_c, const MgGeom &gc, int tile, int nu, cudaStream_t s);
cudaError_t mg_launch_tb_post(int dim, const float *phi_in, float *phi_out, const float *f, const MgGeom &g,
                              const float *phi_c, const MgGeom &gc, int tile, int nu, cudaStream_t s);

// Plane-marching red-black sweeps of an FP32 3D level (mg_wave.cu): nsw (1 or
// 2) complete sweeps phi_in -> phi_out (distinct arrays whose ghost layers
// hold the same values), bit-identical to 2 nsw mg_launch_smooth colours in
// place.  variant 0: 56 x 10 tiles, 1: 56 x 6 tiles; the z extent is split
// into zchunks ranges.  ctl != NULL: as mg_launch_smooth.  A load wait that
// runs out of its clock budget (about 2 s) writes MG_ETIMEOUT to *err (if
// err is not NULL) and ends the block; fault != 0 leaves one load group of
// every block unissued with a budget of about 1 ms (a test of that path).
// Colour-split FP32 levels (MgGeom::sH > 0) of the cubic engine, run by the
// box-patch kernels of mg_box.cu: one red-black colour pass (the level must
// be split), and the residual restriction / prolongation between two levels
// of which either may be split.
cudaError_t mg_split_colour(int dim, float *phi, const float *f, const MgGeom &g, int colour, cudaStream_t s);
cudaError_t mg_split_resid_restrict(int dim, const float *phi, const float *f, const MgGeom &gf, float *phic,
                                    float *fc, const MgGeom &gc, cudaStream_t s);
cudaError_t mg_split_prolong(int dim, const float *phic, const MgGeom &gc, float *phif, const MgGeom &gf,
                             cudaStream_t s);
// FP32 array size (floats) of a level of storage edge E: room for both layouts
inline size_t mg_fp32_cells(int E, int dim)
{
    const size_t plain = dim == 3 ? (size_t)E * E * E : (size_t)E * E;
    const size_t split = 2 * (size_t)mg_split_H(E) * (dim == 3 ? (size_t)E * E : (size_t)E) + 16;
    return plain > split ? plain : split;
}

cudaError_t mg_wave_prepare();   // once per device before the first launch
bool mg_wave_applies(int dim, int nsw, int N);
cudaError_t mg_launch_wave(const float *phi_in, float *phi_out, const float *f, const MgGeom &g, int nsw, int variant,
                           int zchunks, cudaStream_t s, MgSolveCtl *ctl = nullptr, cudaGraphConditionalHandle hi = 0,
                           int *err = nullptr, int fault = 0);

// red_first: also the coarse level's first red half-sweep (the V-cycle then
// starts that level's pre-smoothing with black; nu_pre >= 1 only)
cudaError_t mg_launch_resid_restrict(int dim, bool fp32, const void *phi_f, const void *f_f, const MgGeom &gf,
                                     void *phi_c, void *f_c, const MgGeom &gc, cudaStream_t s,
                                     bool red_first = false);
cudaError_t mg_launch_prolong(int dim, bool fp32, const void *phi_c, const MgGeom &gc, void *phi_f, const MgGeom &gf,
                              cudaStream_t s);

// ||f - lap(Phi)||^2 over the active cells of a finest multigrid level
// (zero_inside: Phi taken as zero on the active cells, ring kept), written to
// *out after a fixed-order two-pass reduction through `partials`
// (MG_NORM_BLOCKS doubles).
#define MG_NORM_BLOCKS 304
// Single-launch form: out2[0] = ||b||^2 if (which & 1), out2[1] = ||r||^2 if
// (which & 2); the last block to finish reduces the per-block partials
// (MG_NORM_BLOCKS_MAX doubles) in a fixed order; counter (one unsigned, zero
// between launches) tracks finished blocks.
#define MG_NORM_BLOCKS_MAX 1216
// ||b||^2 / ||r||^2 of a finest level; with r32 set, also the FP32 right-hand
// side r32 = f - A Phi and a zero correction e32 of the next defect-correction
// step (what mg_launch_defect writes), from the same residual values.
cudaError_t mg_launch_norms2(int dim, const double *phi, const double *f, const MgGeom &g, int which,
                             double *partials, unsigned *counter, double *out2, cudaStream_t s,
                             float *r32 = nullptr, float *e32 = nullptr);
cudaError_t mg_launch_resid_norm2(int dim, const double *phi, const double *f, const MgGeom &g, bool zero_inside,
                                  double *partials, double *out, cudaStream_t s);

// Mixed precision: r32 = float(f - lap(Phi)) on the active cells of the
// finest level (ring of r32 and e32 untouched), and Phi += double(e32).
cudaError_t mg_launch_defect(int dim, const double *phi, const double *f, const MgGeom &g, float *r32, float *e32,
                             cudaStream_t s);
cudaError_t mg_launch_accumulate(int dim, double *phi, const float *e32, const MgGeom &g, cudaStream_t s);

// Level data copy-in: rho (n^d) into the Omega part of rho_blk/f_blk
// ((n+4)^d); for level 0 also bc_rho's ring ((n+2)^d) and bc_phi's outer
// ring ((n+4)^d), and a zero start on Gamma.  fourpiG = 4 pi G.
cudaError_t mg_launch_set_density(int dim, int n, const double *rho, const double *bc_rho, const double *bc_phi,
                                  double *rho_blk, double *f_blk, double *phi_blk, double fourpiG, cudaStream_t s);

// Interface of Sec. 2.1 / 2.4: from the parent's (np+4)^d potential and
// density fill the child's outer-ring potential, inner-ring density (and
// f = 4 pi G rho there) and the initial potential on Gamma (guess 0: parent
// interpolation, 1: zero, 2: copy of guess_src ((nc+2)^d)).
cudaError_t mg_launch_interface(int dim, int np, const double *phi_p, const double *rho_p, int nc, int ox, int oy,
                                int oz, double *phi_c, double *rho_c, double *f_c, double fourpiG, int guess,
                                const double *guess_src, int frozen, cudaStream_t s);
cudaError_t mg_launch_copy_guess(int dim, int n, const double *guess_src, double *phi_blk, cudaStream_t s);

// Forces F = -grad(Phi) on Omega ((n+4)^d block in, dim * n^d out) and the
// potential on Omega (n^d, optional).
cudaError_t mg_launch_forces(int dim, int n, double h, const double *phi_blk, double *F, double *phi_out,
                             int stencil, cudaStream_t s);

cudaError_t mg_launch_zero(void *p, size_t bytes, cudaStream_t s);
cudaError_t mg_launch_extract(int dim, int n, const double *blk, double *out, cudaStream_t s);
// Force-change stopping test (Sec. 3): phase 0 before the first iteration,
// 1 before each iteration (save phi), 2 after it (scal[1] from the change).
cudaError_t mg_launch_force_stop(int phase, int dim, int n, double h, const double *phi_blk, double *prev,
                                 int stencil, unsigned long long *cmax, double *scal, cudaStream_t s);
// Cluster V-cycle: mg_cluster_prepare picks the cluster size (16 CTAs where
// the device can co-schedule them, else 8; 0 if neither) once per process;
// mg_cluster_layout fills the shared-memory layout of a plan (false if it
// does not fit) and returns its dynamic shared memory in *smem.
int mg_cluster_prepare();
bool mg_cluster_layout(bool fp32, int csize, MgClusterPlan &p, size_t *smem);
cudaError_t mg_launch_cluster(bool fp32, const MgClusterPlan &p, int csize, size_t smem, cudaStream_t s);
cudaError_t mg_launch_copy_box(int dim, int e, const double *src, int Es, int os, double *dst, int Ed, int od,
                              cudaStream_t s);
cudaError_t mg_launch_resid_h2(int dim, int n, const double *phi_blk, const double *rho_blk, double frho,
                               double *out, cudaStream_t s);

// Device-side state of one level solve, updated by the control kernels that
// close every iteration of the solve graph.
struct MgSolveCtl {
    int cycles;      // V-cycles run (FP32 V-cycles in mixed mode)
    int outer;       // iterations of the loop body
    int status;      // 0 ok, 6 (MG_EDIVERGED) on a non-finite residual
    int go;          // last value given to the loop condition
    double rel;      // ||r|| / ||b||
    double bnorm;    // ||b||
    int inner;       // adaptive mixed mode: FP32 V-cycles of the current step
    int left;        //   of them not run yet
    int cyc0;        //   cycles when the current step began
};

// Adaptive mixed mode: FP32 V-cycles of the next defect-correction step.
// The last step took the relative residual from rel_before to rel_after in
// `ran` V-cycles; at that per-cycle contraction, the cycles still needed to
// reach tol (one more after a step of fewer than four cycles), between 1 and
// inner_max (inner_max when the step did not contract or there is no
// tolerance to aim at).
__host__ __device__ inline int mg_next_inner(double rel_before, double rel_after, int ran, double tol, int inner_max)
{
    if (!(tol > 0.0) || !(rel_after > 0.0) || !(rel_after < rel_before) || ran < 1)
        return inner_max;
    if (rel_after < tol)
        return 1;
    const double per_cycle = log(rel_after / rel_before) / ran;   // < 0
    const double need = log(tol / rel_after) / per_cycle;          // > 0
    if (!(need < inner_max))
        return inner_max;
    int k = (int)ceil(need - 1e-9);   // a whole number of cycles stays whole under rounding
    if (ran < 4)   // a contraction read off fewer than four cycles (the first step's, from the
        k += 1;    // initial guess) is faster than the steps after it: one cycle spare
    k = k < inner_max ? k : inner_max;
    return k < 1 ? 1 : k;
}

#ifdef __CUDACC__
// Programmatic dependent launch: every kernel first waits until the kernel
// before it in the stream has completed and its writes are visible, then
// lets the next kernel start launching, so that launch latency overlaps the
// running kernel.  Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One FP32 V-cycle of an adaptive defect-correction step done (the step's
// nested graph loop): count it and let the loop go on while cycles are left.
// One thread.
__device__ __forceinline__ void inner_step_count(MgSolveCtl *ctl, cudaGraphConditionalHandle hi)
{
    MgSolveCtl c = *ctl;
    c.cycles += 1;
    c.left -= 1;
    *ctl = c;
    cudaGraphSetConditional(hi, c.left > 0);
}

// Every kernel is launched with programmatic dependent launch (the kernels
// begin with pdl_begin) unless MG_PDL=0.  Errors are left for
// cudaGetLastError, as with the triple-chevron launch.
inline bool mg_pdl_enabled()
{
    static const bool on = [] {
        const char *v = std::getenv("MG_PDL");
        return !(v && v[0] == '0');
    }();
    return on;
}

template <typename... KArgs, typename... Args>
inline void mg_launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = mg_pdl_enabled() ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}
#endif

// ctl_init: from scal = {||b||^2, ||r||^2} start the counters and set the
// loop condition (handle) to 1 iff another iteration is needed.
// ctl_step: after one iteration of `inc` V-cycles, with scal[1] = ||r||^2.
// inner0 / inner_max: first step's FP32 V-cycles and the adaptive cap
// (inner_max 0: fixed steps of `inc` cycles, counted by ctl_step; > 0: the
// nested loop of the step counts its cycles in inner_step, ctl_step sets the
// next step's count and re-arms that loop's condition hi).
cudaError_t mg_launch_ctl_init(MgSolveCtl *ctl, const double *scal, double tol, int max_cycles, int inner0,
                               cudaGraphConditionalHandle hc, cudaStream_t s);
cudaError_t mg_launch_ctl_step(MgSolveCtl *ctl, const double *scal, int inc, double tol, int max_cycles,
                               int inner_max, cudaGraphConditionalHandle hc, cudaGraphConditionalHandle hi,
                               cudaStream_t s);
cudaError_t mg_launch_inner_step(MgSolveCtl *ctl, cudaGraphConditionalHandle hi, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched mixed-precision solve: one launch per phase over every hierarchy
// of a batch that has refinement level l.  A part is one hierarchy's level;
// tile tasks and cell-chunk tasks say which part and which piece a block
// works on; active[p] masks the parts that have converged.
// ---------------------------------------------------------------------------
struct MgBPart {
    int b, l;                      // hierarchy and refinement level
    int nmg, Ls;                   // multigrid levels; first level of the one-block kernel
    MgGeom g[MG_MAX_MG];
    int tile[MG_MAX_MG];
    float *phi32[MG_MAX_MG], *phi32b[MG_MAX_MG], *f32[MG_MAX_MG];
    double *phi, *f, *rho;         // (n+4)^d finest blocks
    double *scal;                  // ||b||^2, ||r||^2
    MgSolveCtl *ctl;
    double *partials;              // 2 * MG_NORM_BLOCKS_MAX
    unsigned *counter;
    int nblk_lvl[MG_MAX_MG];       // cell chunks of the one-kernel-per-phase launches per level
    int nblk_act;                  // cell chunks over the active finest cells
    int nblk_blk;                  // cell chunks over the (n+4)^d block
    MgBottom bt;
    // interface from the parent (l > 0), initial guess
    int n, np, off[3], gmode;      // gmode: 0 interpolate, 1 zero, 2 copy guess, -1 none (level 0)
    const double *phi_p, *rho_p, *guess;
    double fourpiG;
    // persistent solve: the level's registered outputs (or NULL) and cell size
    double *out_F, *out_phi;
    double h;
};
struct MgPTask {                   // persistent solve: one hierarchy, its parts in level order
    int first, count;
};
struct MgBTask {                   // tile task
    int part, bx, by, bz;
};
struct MgBCell {                   // cell-chunk task
    int part, chunk;
};

cudaError_t mg_batch_prepare();
// Persistent batched mixed-precision solve (one launch for the whole batch):
// `grid` blocks of mg_persist_threads() threads take hierarchies from
// tasks[0..ntasks-1] in order through the counter *next (zero at launch) and
// solve each one's levels coarse to fine, every phase by the block alone
// (interface, norms with the fused FP32 defect, the FP32 V-cycles of each
// defect-correction step with the one-block bottom, accumulation, control,
// registered outputs).  Every level above the bottom must use the plain FP32
// layout and one kernel per phase.  smem: the largest bottom plan's shared
// memory.  inner_max > 0: adaptive steps (mg_next_inner), else inner0 cycles
// per step.
int mg_persist_threads();
cudaError_t mg_persist_prepare(int dim, size_t smem, int *blocks_per_sm);
cudaError_t mg_launch_persist(int dim, const MgBPart *parts, const MgPTask *tasks, int ntasks, unsigned *next,
                              int grid, size_t smem, int nu_pre, int nu_post, double tol, int max_cycles, int inner0,
                              int inner_max, int stencil, cudaStream_t s);
cudaError_t mg_launch_b_tb_pre(int dim, const MgBPart *parts, const MgBTask *tasks, int ntasks, const int *active,
                               int depth, int nu, size_t smem, cudaStream_t s);
cudaError_t mg_launch_b_tb_post(int dim, const MgBPart *parts, const MgBTask *tasks, int ntasks, const int *active,
                                int depth, int nu, size_t smem, cudaStream_t s);
// one-kernel-per-phase legs over parts: cells = (part, chunk) tasks of level L
// (chunks over that level's colour cells / coarse cells / fine cells)
cudaError_t mg_launch_b_smooth(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                               int L, int colour, cudaStream_t s);
cudaError_t mg_launch_b_restrict(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                                 int L, cudaStream_t s);
cudaError_t mg_launch_b_prolong(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                                int L, cudaStream_t s);
cudaError_t mg_launch_b_bottom(int dim, const MgBPart *parts, int nparts, const int *active, int nu_pre, int nu_post,
                               size_t smem, cudaStream_t s);
cudaError_t mg_launch_b_defect(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                               cudaStream_t s);
cudaError_t mg_launch_b_accumulate(int dim, const MgBPart *parts, const MgBCell *cells, int ncells,
                                   const int *active, cudaStream_t s);
cudaError_t mg_launch_b_norms2(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                               int which, cudaStream_t s);
cudaError_t mg_launch_b_interface(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, cudaStream_t s);
// init = 1: start every part's loop from its norms; else account `inc`
// cycles to the active parts.  Sets active[] and the loop condition.
cudaError_t mg_launch_b_ctl(const MgBPart *parts, int nparts, int *active, int init, int inc, double tol,
                            int max_cycles, cudaGraphConditionalHandle hc, cudaStream_t s);
