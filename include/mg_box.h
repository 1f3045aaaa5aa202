/*
 * mg_box.h -- C ABI of the nested-grid multigrid solver on box (non-cubic)
 * patches: n_x x n_y (x n_z) cells per patch, each axis with its own
 * multigrid sizes.
 *
 * Sec. 2.2 builds the multigrid sizes along one axis (normalise the solved
 * region Gamma of M = n + 2 cells to [0, 1], double the cell size per level,
 * round the cell count half up, stop at one cell) and applies the same rule to
 * the other axes.  For a patch whose axes differ this library reads it per
 * axis: an axis that has reached one cell stops coarsening while the others go
 * on (semi-coarsening), so multigrid level L has N_a = N_a^{min(L, stop_a)}
 * cells of size h 2^{min(L, stop_a)} along axis a, and the multigrid
 * hierarchy ends when every axis has one cell.  On every level:
 *   - the Laplacian is the sum over axes of the second difference divided by
 *     that axis's squared cell size (the 5- or 7-point stencil of Sec. 2.3);
 *   - red-black Gauss-Seidel (red: i + j (+ k) even, 1-based, first) solves
 *     each cell's own equation, the ghost rule of Sec. 2.4 folded in per axis
 *     on the coarse levels (left ghost -Phi_1; right ghost linear through zero
 *     at x_MG = 1 from Phi_N, or -Phi_{N-1} when the centre of cell N sits at
 *     x_MG = 1), each axis with its own normalised geometry;
 *   - restriction averages the children: two along an axis that coarsened,
 *     one along an axis that did not (weight 2^-k, k the coarsened axes;
 *     children beyond the fine level's last cell count zero; Sec. 2.3 step 5,
 *     Appendix A);
 *   - prolongation and correction use the 3/4 - 1/4 weights along coarsened
 *     axes (coarse ghosts by the rule of Sec. 2.4) and copy along the others
 *     (Sec. 2.3 step 10, Appendix A).
 * With every axis equal this is the method of mg.h.  The nesting (Sec. 2.1),
 * the interface (buffer rings by bi/trilinear interpolation from the parent,
 * Appendix A), the stopping rule on ||b - A Phi||_2 / ||b||_2 and the forces
 * of Eq. 2 are those of mg.h, per axis.
 *
 * Conventions: those of mg.h (arrays C order with x fastest, host or device
 * pointers, errors returned, a handle poisoned after MG_ECUDA).  A patch of
 * n = (n_x, n_y, n_z) cells stores its Omega values as [n_z][n_y][n_x] (2D
 * [n_y][n_x]); "the (n+2) block" is Omega plus one ring, [n_z+2][n_y+2][n_x+2],
 * and "the (n+4) block" Omega plus two rings.
 */
#ifndef MG_BOX_H
#define MG_BOX_H

#include "mg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_box mg_box;   /* opaque; owns all device state of one hierarchy of box patches */

/* A hierarchy of box patches (Sec. 2.1 nesting).  Patch 0 is the base; patch
 * l > 0 lies inside its parent with cells half the parent's size, its lower
 * corner on a parent cell face at an offset o_a (parent cells, per axis) with
 * 1 <= o_a <= n_a(parent) - n_a/2 - 1, and n_a even.  All cells are cubes of
 * edge h0 / 2^depth. */
typedef struct {
    int dim;                          /* 2 or 3 */
    int num_patches;                  /* 1..MG_MAX_LEVELS */
    int n[MG_MAX_LEVELS][3];          /* cells per axis (x, y, z) of each patch, >= 2; n[l][2] ignored in 2D */
    double lo[MG_MAX_LEVELS][3];      /* lower corner of each patch */
    double h0;                        /* cell size of patch 0 (> 0) */
    double G;                         /* gravitational constant of Eq. 1 */
    int tree;                         /* 0: the parent of patch l is l - 1; 1: parent[l] */
    int parent[MG_MAX_LEVELS];        /* tree = 1: parent patch of l > 0, < l */
} mg_box_desc;

/* Create the hierarchy and allocate all its device memory.  opt as in mg.h
 * (NULL: defaults), restricted to what box patches support: precision FP64 or
 * MIXED (fixed inner_cycles, or adaptive with inner_max > 0), guess INTERP or
 * ZERO, interface BUFFER, stop RESIDUAL, either force stencil.  On failure
 * *out is NULL.  Errors: MG_EINVAL (geometry, options), MG_ENOMEM, MG_ECUDA. */
mg_status mg_box_create(const mg_box_desc *desc, const mg_options *opt, mg_box **out);

/* Density of patch p (Sec. 2.1: point values at the cell centres).
 *   rho     Omega values of patch p.
 *   bc_rho  patch 0 only: the (n+2) block; only its outer ring is read (the
 *           density of the inner buffer layer).
 *   bc_phi  patch 0 only: the (n+4) block; only its outer ring is read (the
 *           Dirichlet potential).
 * Patches above 0 take NULL for both (the interface fills them).  Errors:
 * MG_EINVAL, MG_ESTATE, MG_ECUDA. */
mg_status mg_box_set_density(mg_box *b, int patch, const double *rho, const double *bc_rho, const double *bc_phi);

/* Solve every patch in index order (parents first; Sec. 2.1 one-way scheme,
 * Sec. 2.3 iteration).  stats, if not NULL, receives num_patches entries.
 * Returns MG_OK, MG_ENOCONV (some patch stopped at max_cycles; results
 * usable), MG_EDIVERGED, MG_ESTATE (a density missing), MG_ECUDA. */
mg_status mg_box_solve(mg_box *b, mg_level_stats *stats);

/* Results of patch p after mg_box_solve: phi_out (Omega values) and/or F_out
 * (dim x Omega values, component a at F_out[a * cells + cell]; Eq. 2 or the
 * two-point difference).  Either may be NULL.  Errors: MG_EINVAL, MG_ESTATE,
 * MG_ECUDA. */
mg_status mg_box_forces(mg_box *b, int patch, double *phi_out, double *F_out);

/* Multigrid sizes of patch p: writes up to cap rows of three ints
 * (N_x, N_y, N_z) -- N_z = 1 in 2D -- for multigrid levels 0, 1, ... (level 0
 * is Gamma, n + 2 cells per axis); returns the number of levels, or -1 for a
 * bad argument. */
int mg_box_level_sizes(const mg_box *b, int patch, int *N, int cap);

/* Mean device time of one red-black Gauss-Seidel colour pass over multigrid
 * level L of patch p, in the precision the solve's V-cycles use, over
 * `launches` back-to-back launches, and the algorithmic bytes of one pass
 * (the potential read once and its colour written, the right-hand side of
 * that colour read: 1.5 words per cell).  Changes the potential stored on
 * that level; call it outside a solve.  Errors: MG_EINVAL, MG_ESTATE,
 * MG_ECUDA. */
mg_status mg_box_time_smoothing(mg_box *b, int patch, int L, int launches, double *us_per_launch,
                                double *bytes_per_launch);

/* Detail of the last error on this handle (or of the last failed create). */
const char *mg_box_error_message(const mg_box *b);

/* Release everything; NULL-safe; always MG_OK. */
mg_status mg_box_destroy(mg_box *b);

#ifdef __cplusplus
}
#endif

#endif /* MG_BOX_H */
