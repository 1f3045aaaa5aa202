/*
 * mg_oracle.c -- plain, slow CPU FP64 oracle of the nested-grid multigrid
 * Poisson solver of Wang & Yen, "Self-gravitational Force Calculation of
 * Second Order Accuracy Using Multigrid Method on Nested Grids".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that tests, the package smoke check and the
 * CPU baseline of the benchmark have an independent, obviously-correct
 * statement of what the method computes.  It shares no code with the CUDA
 * path.  Compile with -O2 -ffp-contract=off (no FMA contraction).
 *
 * Conventions (all arrays are C order, x fastest; 2D arrays are (y,x)):
 *   A refinement level with n patch cells per edge is stored as an
 *   (n+4)^d block.  Storage index s = 0 and s = n+3 is the outer buffer ring
 *   (Dirichlet potential), s = 1 and s = n+2 the inner buffer ring, s = 2..n+1
 *   the patch Omega (Sec. 2.1, Fig. 1b/c).  Gamma = s in 1..n+2 is the region
 *   the multigrid solves on, M = n+2 cells per edge.
 *   A multigrid level L with N active cells per edge is stored as (N+2)^d
 *   with one ghost layer; active cells use 1-based indices 1..N (Sec. 2.4).
 *
 * Readings of points the paper leaves open (each is stated where used):
 *   R1  defect form: r = f - lap(Phi), f^{L+1} = R(r^L), lap(e) = f^{L+1}.
 *   R2  Gauss-Seidel ordering: red-black, red = (i+j[+k]) even, red first.
 *   R4  coarse corrections start from zero in every cycle.
 *   R7  right multigrid ghost: linear extrapolation through zero at
 *       x_MG = 1 (the printed ratio is garbled), -Phi_{N-1} when x_N = 1.
 *   R8  round() of Sec. 2.2 item 3 rounds halves up.
 *   R9  coarse cell I covers fine cells 2I-1 and 2I; fine cells beyond N
 *       contribute zero to the restriction (weights stay 1/2^d).
 *   R10 the buffer-zone interpolation of Sec. 2.1 is bi/trilinear from the
 *       2^d enclosing parent centres (Appendix A weights).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_MG 40

typedef struct {
    int N;         /* active cells per edge */
    int L;         /* multigrid level index, 0 = finest */
    double h;      /* physical cell size of this multigrid level */
    int tie;       /* right-most active centre sits exactly at x_MG = 1 */
    double cR;     /* right-ghost extrapolation factor when !tie */
} or_mglev;

static long lin(int dim, int E, const int *c)
{
    return dim == 3 ? ((long)c[2] * E + c[1]) * E + c[0] : (long)c[1] * E + c[0];
}

static long cells(int dim, int E) { return dim == 3 ? (long)E * E * E : (long)E * E; }

/* ---------------------------------------------------------------------------
 * Sec. 2.2, items 1-4: normalise Gamma to [0,1], h^0 = 1/M, h^L = 2 h^{L-1},
 * N^L = round(1/h^L) (halves rounded up, R8), stop once N^L = 1.
 * Returns the number of multigrid levels; N[L] receives N^L.
 * ------------------------------------------------------------------------- */
int or_mg_sizes(int M, int *N, int cap)
{
    /* 1/h^L = M / 2^L is evaluated exactly (a division by a power of two),
     * so that halves are recognised and rounded up */
    int L = 0;
    N[0] = M;
    while (N[L] > 1 && L + 1 < cap) {
        L++;
        N[L] = (int)floor((double)M / (double)(1 << L) + 0.5);
    }
    return L + 1;
}

static void make_levels(int M, double h_fine, or_mglev *lv, int *nL)
{
    int N[OR_MAX_MG];
    int n = or_mg_sizes(M, N, OR_MAX_MG);
    for (int L = 0; L < n; L++) {
        /* in units of 1/(2M): x_N = (2N-1) 2^L and h^L = 2 * 2^L, so both
         * the tie test x_N = 1 and the ratio (1 - x_N - h)/(1 - x_N) are
         * formed from exact integers */
        double twoM = 2.0 * (double)M;
        double xN2 = (2.0 * (double)N[L] - 1.0) * (double)(1 << L);
        double hL2 = 2.0 * (double)(1 << L);
        lv[L].N = N[L];
        lv[L].L = L;
        lv[L].h = h_fine * (double)(1 << L);
        lv[L].tie = (xN2 == twoM);
        lv[L].cR = lv[L].tie ? 0.0 : (twoM - xN2 - hL2) / (twoM - xN2);
    }
    *nL = n;
}

/* ---------------------------------------------------------------------------
 * Neighbour sum of one active cell for the 5/7-point Laplacian
 * (Eqs. for the 2D/3D Laplacian in Sec. 2.3).  At L = 0 the neighbours are read
 * directly (the outer ring holds the Dirichlet potential).  At L > 0 a
 * neighbour outside the active region is a ghost given by the rule of
 * Sec. 2.4 in terms of the current potential: left ghost = -Phi_1; right
 * ghost = -Phi_{N-1} if x_N = 1, else Phi_N (1 - x_N - h)/(1 - x_N) (R7).
 * Ghost terms that equal the cell's own value are returned in *self so that
 * the caller can solve the cell's own equation ("the boundary value should
 * be updated according to the updated Phi", Sec. 2.4).
 * ------------------------------------------------------------------------- */
static double neighbour_sum(int dim, const or_mglev *lv, const double *phi, const int *c, double *self)
{
    int E = lv->N + 2;
    double other = 0.0;
    *self = 0.0;
    for (int a = 0; a < dim; a++) {
        for (int side = -1; side <= 1; side += 2) {
            int q[3] = {c[0], c[1], dim == 3 ? c[2] : 0};
            q[a] += side;
            if (lv->L == 0 || (q[a] >= 1 && q[a] <= lv->N)) {
                other += phi[lin(dim, E, q)];
            } else if (q[a] == 0) {
                *self += -1.0;                          /* Phi_0 = -Phi_1, and c[a] == 1 */
            } else if (lv->tie) {                       /* q[a] == N+1, x_N = 1 */
                if (lv->N >= 2) {
                    q[a] = lv->N - 1;
                    other += -phi[lin(dim, E, q)];
                } else {
                    *self += 1.0;                       /* -Phi_0 = +Phi_1 */
                }
            } else {
                *self += lv->cR;                        /* Phi_{N+1} = cR Phi_N, c[a] == N */
            }
        }
    }
    return other;
}

/* Gauss-Seidel smoothing, N_pre / N_post sweeps (Sec. 2.3 steps 2, 6, 11),
 * red-black ordering (R2).  Each update solves the cell's own equation
 * lap(Phi)_c = f_c for Phi_c. */
static void smooth(int dim, const or_mglev *lv, double *phi, const double *f, int sweeps)
{
    int N = lv->N, E = N + 2;
    double h2 = lv->h * lv->h;
    int kmax = dim == 3 ? N : 1;
    for (int s = 0; s < sweeps; s++) {
        for (int colour = 0; colour < 2; colour++) {
            for (int k = 1; k <= kmax; k++)
                for (int j = 1; j <= N; j++)
                    for (int i = 1; i <= N; i++) {
                        int c[3] = {i, j, dim == 3 ? k : 0};
                        int par = (i + j + (dim == 3 ? k : 0)) & 1;
                        if (par != colour)
                            continue;
                        double self;
                        double other = neighbour_sum(dim, lv, phi, c, &self);
                        long p = lin(dim, E, c);
                        phi[p] = (other - h2 * f[p]) / (2.0 * dim - self);
                    }
        }
    }
}

/* Residual r = f - lap(Phi) on the active cells (Sec. 2.3 step 4, R1). */
static void residual(int dim, const or_mglev *lv, const double *phi, const double *f, double *r)
{
    int N = lv->N, E = N + 2;
    double h2 = lv->h * lv->h;
    int kmax = dim == 3 ? N : 1;
    for (int k = 1; k <= kmax; k++)
        for (int j = 1; j <= N; j++)
            for (int i = 1; i <= N; i++) {
                int c[3] = {i, j, dim == 3 ? k : 0};
                double self;
                double other = neighbour_sum(dim, lv, phi, c, &self);
                long p = lin(dim, E, c);
                r[p] = f[p] - (other + (self - 2.0 * dim) * phi[p]) / h2;
            }
}

static double norm2_active(int dim, int N, const double *r)
{
    int E = N + 2, kmax = dim == 3 ? N : 1;
    double s = 0.0;
    for (int k = 1; k <= kmax; k++)
        for (int j = 1; j <= N; j++)
            for (int i = 1; i <= N; i++) {
                int c[3] = {i, j, dim == 3 ? k : 0};
                double v = r[lin(dim, E, c)];
                s += v * v;
            }
    return sqrt(s);
}

/* Restriction (Sec. 2.3 step 5; 2D: E = (a+b+c+d)/4, 3D: A = (a+...+h)/8):
 * f_c(I) = 2^-d sum over children 2I-1, 2I per axis, children beyond the
 * fine active range count as zero (R9). */
static void restrict_avg(int dim, const or_mglev *fine, const double *rf, const or_mglev *coarse, double *fc)
{
    int Nf = fine->N, Nc = coarse->N, Ef = Nf + 2, Ec = Nc + 2;
    int kmax = dim == 3 ? Nc : 1;
    double w = dim == 3 ? 0.125 : 0.25;
    for (int K = 1; K <= kmax; K++)
        for (int J = 1; J <= Nc; J++)
            for (int I = 1; I <= Nc; I++) {
                double s = 0.0;
                int dkmax = dim == 3 ? 1 : 0;
                for (int dk = 0; dk <= dkmax; dk++)
                    for (int dj = 0; dj <= 1; dj++)
                        for (int di = 0; di <= 1; di++) {
                            int q[3] = {2 * I - 1 + di, 2 * J - 1 + dj, dim == 3 ? 2 * K - 1 + dk : 0};
                            if (q[0] > Nf || q[1] > Nf || (dim == 3 && q[2] > Nf))
                                continue;
                            s += rf[lin(dim, Ef, q)];
                        }
                int C[3] = {I, J, dim == 3 ? K : 0};
                fc[lin(dim, Ec, C)] = w * s;
            }
}

/* Fill the ghost layer of a coarse multigrid level (L > 0) from the rule of
 * Sec. 2.4, one axis after another so that edge and corner ghosts follow the
 * same rule along each axis in turn. */
static void fill_ghosts(int dim, const or_mglev *lv, double *phi)
{
    int N = lv->N, E = N + 2;
    long tot = cells(dim, E);
    for (int a = 0; a < dim; a++) {
        for (int pass = 0; pass < 2; pass++) {          /* left ghosts, then right */
            for (long p = 0; p < tot; p++) {
                int c[3];
                c[0] = (int)(p % E);
                c[1] = (int)((p / E) % E);
                c[2] = dim == 3 ? (int)(p / ((long)E * E)) : 0;
                int q[3] = {c[0], c[1], c[2]};
                if (pass == 0 && c[a] == 0) {
                    q[a] = 1;
                    phi[p] = -phi[lin(dim, E, q)];
                } else if (pass == 1 && c[a] == N + 1) {
                    if (lv->tie) {
                        q[a] = N - 1;
                        phi[p] = -phi[lin(dim, E, q)];
                    } else {
                        q[a] = N;
                        phi[p] = lv->cR * phi[lin(dim, E, q)];
                    }
                }
            }
        }
    }
}

/* Prolongation and correction (Sec. 2.3 step 10; 2D e = (9A+3B+C+3D)/16,
 * 3D a = (27E+9A+9H+9F+3G+3D+3B+C)/64): the fine centre of cell i lies a
 * quarter coarse cell from the centre of coarse cell I = ceil(i/2), towards
 * coarse cell I-1 (i odd) or I+1 (i even); weights 3/4 and 1/4 per axis. */
static void prolong_add(int dim, const or_mglev *coarse, double *phic, const or_mglev *fine, double *phif)
{
    int Nf = fine->N, Ef = Nf + 2, Ec = coarse->N + 2;
    int kmax = dim == 3 ? Nf : 1;
    fill_ghosts(dim, coarse, phic);
    for (int k = 1; k <= kmax; k++)
        for (int j = 1; j <= Nf; j++)
            for (int i = 1; i <= Nf; i++) {
                int f[3] = {i, j, k};
                int near[3], far[3];
                for (int a = 0; a < 3; a++) {
                    near[a] = (f[a] + 1) / 2;
                    far[a] = (f[a] & 1) ? near[a] - 1 : near[a] + 1;
                }
                double v = 0.0;
                int dkmax = dim == 3 ? 1 : 0;
                for (int tk = 0; tk <= dkmax; tk++)
                    for (int tj = 0; tj <= 1; tj++)
                        for (int ti = 0; ti <= 1; ti++) {
                            int q[3] = {ti ? far[0] : near[0], tj ? far[1] : near[1], tk ? far[2] : near[2]};
                            double w = (ti ? 0.25 : 0.75) * (tj ? 0.25 : 0.75);
                            if (dim == 3)
                                w *= tk ? 0.25 : 0.75;
                            else
                                q[2] = 0;
                            v += w * phic[lin(dim, Ec, q)];
                        }
                int F[3] = {i, j, dim == 3 ? k : 0};
                phif[lin(dim, Ef, F)] += v;
            }
}

/* One multigrid iteration (Sec. 2.3 steps 2-13). */
static void vcycle(int dim, int nL, const or_mglev *lv, double **phi, double **f, double *r, int nu_pre, int nu_post)
{
    smooth(dim, &lv[0], phi[0], f[0], nu_pre);                                /* step 2 */
    int L = 0;
    do {
        residual(dim, &lv[L], phi[L], f[L], r);                               /* step 4 */
        restrict_avg(dim, &lv[L], r, &lv[L + 1], f[L + 1]);                   /* step 5 */
        memset(phi[L + 1], 0, sizeof(double) * cells(dim, lv[L + 1].N + 2));  /* R4 */
        smooth(dim, &lv[L + 1], phi[L + 1], f[L + 1], nu_pre);                /* step 6 */
        L++;                                                                  /* step 7 */
    } while (lv[L].N > 1 && L + 1 < nL);                                      /* step 8 */
    do {
        prolong_add(dim, &lv[L], phi[L], &lv[L - 1], phi[L - 1]);             /* step 10 */
        smooth(dim, &lv[L - 1], phi[L - 1], f[L - 1], nu_post);               /* step 11 */
        L--;                                                                  /* step 12 */
    } while (L > 0);                                                          /* step 13 */
}

/* ---------------------------------------------------------------------------
 * Solve one refinement level (Sec. 2.2-2.4).
 *   phi  (n+4)^d: on entry the outer ring holds the Dirichlet potential and
 *        Gamma holds the initial guess; on exit Gamma holds the solution.
 *   rho  (n+4)^d: density on Gamma (patch and inner ring); other cells unread.
 *   fourpiG = 4 pi G (Eq. 1); h = cell size of the level.
 *   Stops when ||f - lap(Phi)||_2 / ||f - lap(Phi_zero)||_2 < rel_tol over
 *   the active cells (Phi_zero: zero on Gamma, same outer ring), or after
 *   max_cycles.  hist[c] receives that ratio after c cycles (hist[0] for the
 *   initial guess; max_cycles+1 entries).  Returns the cycles performed.
 * ------------------------------------------------------------------------- */
void or_forces(int dim, int n, double h, const double *phi, double *F, int stencil);

/* max over Omega of |F_a - F_b| (Euclidean length of the difference vector) */
static double max_force_change(int dim, long nd, const double *Fa, const double *Fb)
{
    double m = 0.0;
    for (long p = 0; p < nd; p++) {
        double s = 0.0;
        for (int a = 0; a < dim; a++) {
            double d = Fa[(long)a * nd + p] - Fb[(long)a * nd + p];
            s += d * d;
        }
        if (s > m)
            m = s;
    }
    return sqrt(m);
}

/* Stopping rules: stop = 0 -- ||b - A Phi||_2 / ||b||_2 < tol over Gamma;
 * stop = 1 -- the convergence test of Sec. 3.1/3.2: the acceleration on Omega
 * (force stencil `stencil`) changes by less than tol between two cycles,
 * measured as the largest length of the change vector over the cells. */
int or_level_solve(int dim, int n, double h, double *phi, const double *rho, double fourpiG,
                   int nu_pre, int nu_post, int max_cycles, double rel_tol, double *hist, int stop, int stencil)
{
    or_mglev lv[OR_MAX_MG];
    int nL;
    int M = n + 2;
    make_levels(M, h, lv, &nL);
    double *phis[OR_MAX_MG], *fs[OR_MAX_MG];
    long tot0 = cells(dim, M + 2);
    phis[0] = phi;
    fs[0] = (double *)calloc(tot0, sizeof(double));
    for (long p = 0; p < tot0; p++)
        fs[0][p] = fourpiG * rho[p];
    for (int L = 1; L < nL; L++) {
        phis[L] = (double *)calloc(cells(dim, lv[L].N + 2), sizeof(double));
        fs[L] = (double *)calloc(cells(dim, lv[L].N + 2), sizeof(double));
    }
    double *r = (double *)calloc(tot0, sizeof(double));

    /* ||b||: residual of the zero guess with the same Dirichlet ring */
    double *z = (double *)malloc(sizeof(double) * tot0);
    memcpy(z, phi, sizeof(double) * tot0);
    {
        int E = M + 2, kmax = dim == 3 ? M : 1;
        for (int k = 1; k <= kmax; k++)
            for (int j = 1; j <= M; j++)
                for (int i = 1; i <= M; i++) {
                    int c[3] = {i, j, dim == 3 ? k : 0};
                    z[lin(dim, E, c)] = 0.0;
                }
    }
    residual(dim, &lv[0], z, fs[0], r);
    double bnorm = norm2_active(dim, M, r);
    free(z);

    residual(dim, &lv[0], phi, fs[0], r);
    double rel = bnorm > 0.0 ? norm2_active(dim, M, r) / bnorm : 0.0;
    const long nd = cells(dim, n);
    double *Fp = 0, *Fc = 0;
    if (stop == 1) {
        Fp = (double *)calloc((size_t)dim * nd, sizeof(double));
        Fc = (double *)calloc((size_t)dim * nd, sizeof(double));
        or_forces(dim, n, h, phi, Fp, stencil);
        rel = HUGE_VAL;                 /* no previous iterate: at least one cycle */
    }
    if (hist)
        hist[0] = rel;
    int c = 0;
    while (c < max_cycles && !(rel < rel_tol) && bnorm > 0.0) {
        if (nL > 1)
            vcycle(dim, nL, lv, phis, fs, r, nu_pre, nu_post);
        else
            smooth(dim, &lv[0], phis[0], fs[0], nu_pre + nu_post);
        c++;
        if (stop == 1) {
            or_forces(dim, n, h, phi, Fc, stencil);
            rel = max_force_change(dim, nd, Fc, Fp);
            double *t = Fp;
            Fp = Fc;
            Fc = t;
        } else {
            residual(dim, &lv[0], phi, fs[0], r);
            rel = norm2_active(dim, M, r) / bnorm;
        }
        if (hist)
            hist[c] = rel;
    }
    free(Fp);
    free(Fc);
    free(r);
    free(fs[0]);
    for (int L = 1; L < nL; L++) {
        free(phis[L]);
        free(fs[L]);
    }
    return c;
}

/* Residual 2-norm over Gamma of a given potential (diagnostic). */
double or_residual_norm(int dim, int n, double h, const double *phi, const double *rho, double fourpiG)
{
    or_mglev lv[OR_MAX_MG];
    int nL, M = n + 2;
    make_levels(M, h, lv, &nL);
    long tot = cells(dim, M + 2);
    double *f = (double *)calloc(tot, sizeof(double));
    double *r = (double *)calloc(tot, sizeof(double));
    for (long p = 0; p < tot; p++)
        f[p] = fourpiG * rho[p];
    residual(dim, &lv[0], phi, f, r);
    double s = norm2_active(dim, M, r);
    free(f);
    free(r);
    return s;
}

/* ---------------------------------------------------------------------------
 * One-way coarse-to-fine interface (Sec. 2.1, Fig. 1c; Sec. 2.4 first
 * sentences; R10).  The child patch has nc cells per edge and its lower
 * corner lies off[a] parent cells above the parent patch's lower corner.
 * Each child cell centre is interpolated bi/trilinearly (Appendix A) from the
 * 2^d parent centres that enclose it:
 *   outer ring of phi_c  <- parent potential phi_p   (Dirichlet data)
 *   inner ring of rho_c  <- parent density   rho_p
 *   Gamma of phi_c       <- parent potential (initial guess) if guess,
 *                           else zero.
 * Parent and child arrays are (n+4)^d blocks.
 * ------------------------------------------------------------------------- */
void or_interface_fill(int dim, int np, const double *phi_p, const double *rho_p, int nc, const int *off,
                       double *phi_c, double *rho_c, int guess)
{
    int Ep = np + 4, Ec = nc + 4;
    int kmax = dim == 3 ? Ec : 1;
    for (int k = 0; k < kmax; k++)
        for (int j = 0; j < Ec; j++)
            for (int i = 0; i < Ec; i++) {
                int s[3] = {i, j, k};
                int outer = 0, inner = 0;
                for (int a = 0; a < dim; a++) {
                    if (s[a] == 0 || s[a] == nc + 3)
                        outer = 1;
                    else if (s[a] == 1 || s[a] == nc + 2)
                        inner = 1;
                }
                /* child centre in parent storage coordinates: the parent
                 * centre of storage index p sits at coordinate p */
                int p0[3] = {0, 0, 0};
                double t[3] = {0, 0, 0};
                for (int a = 0; a < dim; a++) {
                    double q = (double)off[a] + 1.5 + ((double)s[a] - 1.5) * 0.5;
                    p0[a] = (int)floor(q);
                    t[a] = q - (double)p0[a];
                }
                const double *src = outer ? phi_p : rho_p;
                double v = 0.0;
                int dkmax = dim == 3 ? 1 : 0;
                for (int dk = 0; dk <= dkmax; dk++)
                    for (int dj = 0; dj <= 1; dj++)
                        for (int di = 0; di <= 1; di++) {
                            double w = (di ? t[0] : 1.0 - t[0]) * (dj ? t[1] : 1.0 - t[1]);
                            if (dim == 3)
                                w *= dk ? t[2] : 1.0 - t[2];
                            int q[3] = {p0[0] + di, p0[1] + dj, dim == 3 ? p0[2] + dk : 0};
                            v += w * src[lin(dim, Ep, q)];
                        }
                long c = lin(dim, Ec, s);
                if (outer) {
                    phi_c[c] = v;
                } else {
                    if (inner)
                        rho_c[c] = v;
                    if (guess) {
                        double g = 0.0;
                        for (int dk = 0; dk <= dkmax; dk++)
                            for (int dj = 0; dj <= 1; dj++)
                                for (int di = 0; di <= 1; di++) {
                                    double w = (di ? t[0] : 1.0 - t[0]) * (dj ? t[1] : 1.0 - t[1]);
                                    if (dim == 3)
                                        w *= dk ? t[2] : 1.0 - t[2];
                                    int q[3] = {p0[0] + di, p0[1] + dj, dim == 3 ? p0[2] + dk : 0};
                                    g += w * phi_p[lin(dim, Ep, q)];
                                }
                        phi_c[c] = g;
                    } else {
                        phi_c[c] = 0.0;
                    }
                }
            }
}

/* ---------------------------------------------------------------------------
 * Force F = -grad(Phi) (Eq. 1) on the patch cells s = 2..n+1, per axis by the
 * fourth-order difference of Eq. 2 (stencil 0) or by the two-point central
 * difference (stencil 1).  F is (dim, n^d): component a at F[a*n^d + cell].
 * ------------------------------------------------------------------------- */
void or_forces(int dim, int n, double h, const double *phi, double *F, int stencil)
{
    int E = n + 4;
    long nd = cells(dim, n);
    int kmax = dim == 3 ? n : 1;
    for (int k = 0; k < kmax; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                int s[3] = {i + 2, j + 2, dim == 3 ? k + 2 : 0};
                int o[3] = {i, j, k};
                long out = lin(dim, n, o);
                for (int a = 0; a < dim; a++) {
                    int p1[3] = {s[0], s[1], s[2]}, m1[3] = {s[0], s[1], s[2]};
                    int p2[3] = {s[0], s[1], s[2]}, m2[3] = {s[0], s[1], s[2]};
                    p1[a] += 1;
                    m1[a] -= 1;
                    p2[a] += 2;
                    m2[a] -= 2;
                    double d1 = phi[lin(dim, E, p1)] - phi[lin(dim, E, m1)];
                    double d2 = phi[lin(dim, E, p2)] - phi[lin(dim, E, m2)];
                    double g;
                    if (stencil == 0)
                        g = (4.0 / 3.0) * d1 / (2.0 * h) - (1.0 / 3.0) * d2 / (4.0 * h);
                    else
                        g = d1 / (2.0 * h);
                    F[(long)a * nd + out] = -g;
                }
            }
}

/* Test hook: fill the ghost layer of multigrid level L of a Gamma of M cells
 * per edge by the rule of Sec. 2.4 (phi is (N^L+2)^d).  Returns N^L, or -1 if
 * the hierarchy has no level L. */
int or_fill_ghosts(int dim, int M, int L, double *phi)
{
    or_mglev lv[OR_MAX_MG];
    int nL;
    make_levels(M, 1.0, lv, &nL);
    if (L < 1 || L >= nL)
        return -1;
    fill_ghosts(dim, &lv[L], phi);
    return lv[L].N;
}

/* Test hook: residual r = f - lap(Phi) at multigrid level L (L >= 1 uses the
 * ghost rule of Sec. 2.4) for a Gamma of M cells per edge with unit fine cell
 * size; arrays are (N^L+2)^d.  Returns N^L, or -1 if there is no level L. */
int or_mg_residual(int dim, int M, int L, const double *phi, const double *f, double *r)
{
    or_mglev lv[OR_MAX_MG];
    int nL;
    make_levels(M, 1.0, lv, &nL);
    if (L < 0 || L >= nL)
        return -1;
    residual(dim, &lv[L], phi, f, r);
    return lv[L].N;
}

/* Test hook: the restriction of Sec. 2.3 step 5 from multigrid level L to
 * L + 1 of a Gamma of M cells per edge: rf is (N^L+2)^d, fc (N^{L+1}+2)^d (its
 * active cells are written).  Returns N^{L+1}, or -1 if there is no level
 * L + 1. */
int or_mg_restrict(int dim, int M, int L, const double *rf, double *fc)
{
    or_mglev lv[OR_MAX_MG];
    int nL;
    make_levels(M, 1.0, lv, &nL);
    if (L < 0 || L + 1 >= nL)
        return -1;
    restrict_avg(dim, &lv[L], rf, &lv[L + 1], fc);
    return lv[L + 1].N;
}

/* Test hook: the prolongation and correction of Sec. 2.3 step 10 from
 * multigrid level L + 1 to L: the ghost layer of phic ((N^{L+1}+2)^d) is
 * filled by the rule of Sec. 2.4, then P(phic) is added to the active cells of
 * phif ((N^L+2)^d).  Returns N^{L+1}, or -1 if there is no level L + 1. */
int or_mg_prolong(int dim, int M, int L, double *phic, double *phif)
{
    or_mglev lv[OR_MAX_MG];
    int nL;
    make_levels(M, 1.0, lv, &nL);
    if (L < 0 || L + 1 >= nL)
        return -1;
    prolong_add(dim, &lv[L + 1], phic, &lv[L], phif);
    return lv[L + 1].N;
}
