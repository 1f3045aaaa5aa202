// mg_kernels.cu -- CUDA kernels of the nested-grid multigrid Poisson solver
// for sm_103a: red-black Gauss-Seidel smoothing, fused residual+restriction,
// prolongation+correction, the one-block bottom of the V-cycle, residual
// norms, mixed-precision defect correction, the coarse-to-fine interface and
// the force stencil.  Arrays are C order, x fastest.
//
// The part runs FP64 at two FMA per clock per SM, so the FP64 kernels are
// written to minimise double-precision operations per cell: no device
// divisions (host tables of the boundary diagonals), neighbour folding by
// selects rather than multiplies, separable interpolation.  Index arithmetic
// is 32-bit.
#include <algorithm>
#include <cstdlib>

#include <math_constants.h>

#include "mg_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBottomThreads = 512;

inline int grid_for(long work, int cap = 152 * 16)
{
    long b = (work + kThreads - 1) / kThreads;
    if (b < 1)
        b = 1;
    if (b > cap)
        b = cap;
    return (int)b;
}

inline long cube(int e, int dim) { return dim == 3 ? (long)e * e * e : (long)e * e; }

template <int DIM>
__device__ __forceinline__ int lin(int i, int j, int k, int E)
{
    return DIM == 3 ? (k * E + j) * E + i : j * E + i;
}

// floor(x / d) for 0 <= x < 2^31, d >= 1 and a quotient below 2^21 (every
// index here: at most (1286 + 4)^2): the FP32 value of x, the reciprocal of d
// and their product, each rounded toward zero, underestimate x/d by less than
// 3 * 2^-23 relative, i.e. by less than 1, so truncation gives floor(x/d) or
// one less, and one exact remainder test corrects it.  A few instructions
// instead of the long dependent sequence of a general integer division --
// this sits at the start of every phase of every kernel, where it is latency.
__device__ __forceinline__ int div_small(int x, int d)
{
    int q = __float2int_rz(__fmul_rz(__int2float_rz(x), __frcp_rz(__int2float_rz(d))));
    if (x - q * d >= d)
        q++;
    return q;
}

// Walk t = t0, t0 + S, t0 + 2S, ... over an nx * ny * nz box (x fastest) with
// the coordinates advanced incrementally: the divisions happen once, not per
// cell.
struct Walk3 {
    int x, y, z, dx, dy, dz, nx, ny;
    __device__ __forceinline__ Walk3(int t0, int S, int nx_, int ny_) : nx(nx_), ny(ny_)
    {
        const int r = div_small(t0, nx);
        x = t0 - r * nx;
        z = div_small(r, ny);
        y = r - z * ny;
        const int q = div_small(S, nx);
        dx = S - q * nx;
        dz = div_small(q, ny);
        dy = q - dz * ny;
    }
    __device__ __forceinline__ void next()
    {
        x += dx;
        int c = 0;
        if (x >= nx) {
            x -= nx;
            c = 1;
        }
        y += dy + c;
        c = 0;
        if (y >= ny) {
            y -= ny;
            c = 1;
        }
        z += dz + c;
    }
};

// level constants in the working precision
template <typename T>
__device__ __forceinline__ T geo_h2(const MgGeom &g);
template <>
__device__ __forceinline__ double geo_h2<double>(const MgGeom &g) { return g.h2; }
template <>
__device__ __forceinline__ float geo_h2<float>(const MgGeom &g) { return g.h2f; }
template <typename T>
__device__ __forceinline__ T geo_inv_h2(const MgGeom &g);
template <>
__device__ __forceinline__ double geo_inv_h2<double>(const MgGeom &g) { return g.inv_h2; }
template <>
__device__ __forceinline__ float geo_inv_h2<float>(const MgGeom &g) { return g.inv_h2f; }
template <typename T>
__device__ __forceinline__ T geo_cR(const MgGeom &g);
template <>
__device__ __forceinline__ double geo_cR<double>(const MgGeom &g) { return g.cR; }
template <>
__device__ __forceinline__ float geo_cR<float>(const MgGeom &g) { return g.cRf; }

template <typename T>
__device__ __forceinline__ const T *tab_of(const MgGeom &g);
template <>
__device__ __forceinline__ const double *tab_of<double>(const MgGeom &g) { return g.tab64; }
template <>
__device__ __forceinline__ const float *tab_of<float>(const MgGeom &g) { return g.tab32; }

// Ghost-folded neighbour sum of the 5/7-point Laplacian (Sec. 2.3 item 1) at
// active cell (i,j,k) of index p, and the cell's boundary class (0 if it
// touches no multigrid boundary, always 0 on the finest level where the outer
// ring holds Dirichlet data).
template <typename T, int DIM>
__device__ __forceinline__ T neighbour_sum_ptr(const T *c, const T *d, const T *u, const MgGeom &g, int i, int j,
                                              int k, int sy, int &cls)
{
    // c: the cell; d, u: the same cell in the planes k-1 and k+1 (3D)
    const int N = g.N;
    const bool coarse = g.L > 0;
    const bool inner = !coarse || (i > 1 && i < N && j > 1 && j < N && (DIM == 2 || (k > 1 && k < N)));
    if (inner) {
        cls = 0;
        T s = (c[-1] + c[1]) + (c[-sy] + c[sy]);
        if (DIM == 3)
            s += d[0] + u[0];
        return s;
    }
    // left neighbour dropped at index 1 (ghost = -self: goes to the diagonal)
    // and at index N when x_N = 1 (ghost = -Phi_{N-1} cancels it); right
    // neighbour dropped at index N (ghost cR Phi_N: diagonal)
    const bool tieN = g.tie && N >= 2;
    cls = 0;
    auto axis = [&](int a, const T *lp, const T *rp, int shift) -> T {
        const bool lo = a == 1, hi = a == N;
        cls |= ((lo ? 1 : 0) | (hi ? 2 : 0)) << shift;
        const T l = (!lo && !(hi && tieN)) ? *lp : T(0);
        const T r = !hi ? *rp : T(0);
        return l + r;
    };
    T s = axis(i, c - 1, c + 1, 0) + axis(j, c - sy, c + sy, 2);
    if (DIM == 3)
        s += axis(k, d, u, 4);
    return s;
}

// Ghost-folded neighbour sum at index p of an array with strides (1, sy, sz)
template <typename T, int DIM>
__device__ __forceinline__ T neighbour_sum_s(const T *__restrict__ phi, const MgGeom &g, int i, int j, int k, int p,
                                            int sy, int sz, int &cls)
{
    return neighbour_sum_ptr<T, DIM>(phi + p, phi + p - (DIM == 3 ? sz : 0), phi + p + (DIM == 3 ? sz : 0), g, i, j,
                                     k, sy, cls);
}

// the same on a level array of edge g.E
template <typename T, int DIM>
__device__ __forceinline__ T neighbour_sum(const T *__restrict__ phi, const MgGeom &g, int i, int j, int k, int p,
                                          int &cls)
{
    return neighbour_sum_s<T, DIM>(phi, g, i, j, k, p, g.E, g.E * g.E, cls);
}

template <typename T, int DIM>
__device__ __forceinline__ T diag_of(const MgGeom &g, int cls)
{
    if (cls == 0)
        return T(-2 * DIM);
    const T *tab = tab_of<T>(g);
    if (tab)
        return tab[cls];
    double d = mg_axis_diag(cls & 3, g) + mg_axis_diag((cls >> 2) & 3, g);
    if (DIM == 3)
        d += mg_axis_diag((cls >> 4) & 3, g);
    return T(d);
}

template <typename T, int DIM>
__device__ __forceinline__ T neg_inv_diag(const MgGeom &g, int cls)
{
    if (cls == 0)
        return T(1.0 / (2 * DIM));
    const T *tab = tab_of<T>(g);
    if (tab)
        return tab[64 + cls];
    return T(1) / (-diag_of<T, DIM>(g, cls));
}

// One colour of a red-black Gauss-Seidel sweep (Sec. 2.3 steps 2, 6, 11)
// over work items t0, t0+stride, ...  Red cells have (i+j[+k]) even and are
// updated first.  Each update solves the cell's own equation.
template <typename T, int DIM>
__device__ __forceinline__ void op_smooth_colour(T *__restrict__ phi, const T *__restrict__ f, const MgGeom &g,
                                                 int colour, int t0, int stride)
{
    const int N = g.N;
    const int half = (N + 1) >> 1;
    const int total = half * N * (DIM == 3 ? N : 1);
    const T h2 = geo_h2<T>(g);
    Walk3 w(t0, stride, half, DIM == 3 ? N : total);
    for (int t = t0; t < total; t += stride, w.next()) {
        const int j = w.y + 1;
        const int k = DIM == 3 ? w.z + 1 : 0;
        const int i = ((((1 + j + k) & 1) == colour) ? 1 : 2) + 2 * w.x;
        if (i > N)
            continue;
        const int p = lin<DIM>(i, j, k, g.E);
        int cls;
        const T other = neighbour_sum<T, DIM>(phi, g, i, j, k, p, cls);
        phi[p] = (other - h2 * f[p]) * neg_inv_diag<T, DIM>(g, cls);
    }
}

// f - lap(Phi) at a cell given by pointers to it and to it in the planes k-1, k+1
template <typename T, int DIM>
__device__ __forceinline__ T residual_ptr(const T *c, const T *d, const T *u, T fv, const MgGeom &g, int i, int j,
                                          int k)
{
    int cls;
    const T other = neighbour_sum_ptr<T, DIM>(c, d, u, g, i, j, k, g.E, cls);
    return fv - (other + diag_of<T, DIM>(g, cls) * c[0]) * geo_inv_h2<T>(g);
}

template <typename T, int DIM>
__device__ __forceinline__ T residual_at(const T *__restrict__ phi, const T *__restrict__ f, const MgGeom &g, int i,
                                         int j, int k)
{
    const int p = lin<DIM>(i, j, k, g.E);
    const int sz = DIM == 3 ? g.E * g.E : 0;
    return residual_ptr<T, DIM>(phi + p, phi + p - sz, phi + p + sz, f[p], g, i, j, k);
}

// Residual (Sec. 2.3 step 4) restricted to the next coarser level by the
// 2^d-child average (step 5; fine cells beyond N contribute zero); the
// coarse correction starts from zero.  Generic form (one coarse cell per work
// item) for the one-block kernel.
template <typename T, int DIM>
__device__ __forceinline__ void op_resid_restrict(const T *__restrict__ phi_f, const T *__restrict__ f_f,
                                                  const MgGeom &gf, T *__restrict__ phi_c, T *__restrict__ f_c,
                                                  const MgGeom &gc, int t0, int stride)
{
    const int Nc = gc.N, Nf = gf.N;
    const int total = Nc * Nc * (DIM == 3 ? Nc : 1);
    const T w = DIM == 3 ? T(0.125) : T(0.25);
    Walk3 wk(t0, stride, Nc, DIM == 3 ? Nc : total);
    for (int t = t0; t < total; t += stride, wk.next()) {
        const int I = wk.x + 1, J = wk.y + 1, K = DIM == 3 ? wk.z + 1 : 0;
        T s = T(0);
        for (int dk = 0; dk < (DIM == 3 ? 2 : 1); dk++) {
            const int k = DIM == 3 ? 2 * K - 1 + dk : 0;
            if (DIM == 3 && k > Nf)
                continue;
            for (int dj = 0; dj < 2; dj++) {
                const int j = 2 * J - 1 + dj;
                if (j > Nf)
                    continue;
                for (int di = 0; di < 2; di++) {
                    const int i = 2 * I - 1 + di;
                    if (i > Nf)
                        continue;
                    s += residual_at<T, DIM>(phi_f, f_f, gf, i, j, k);
                }
            }
        }
        const int pc = lin<DIM>(I, J, K, gc.E);
        f_c[pc] = w * s;
        phi_c[pc] = T(0);
    }
}

// Coarse index q along one axis of level gc (ghosts included) written as
// coefficient * active value (Sec. 2.4 ghost rule).
template <typename T>
__device__ __forceinline__ void ghost_map(int q, const MgGeom &gc, int &idx, T &c)
{
    if (q >= 1 && q <= gc.N) {
        idx = q;
        c = T(1);
    } else if (q == 0) {
        idx = 1;
        c = T(-1);
    } else if (gc.tie) {
        if (gc.N >= 2) {
            idx = gc.N - 1;
            c = T(-1);
        } else {
            idx = 1;
            c = T(1);
        }
    } else {
        idx = gc.N;
        c = geo_cR<T>(gc);
    }
}

// Prolongation (Sec. 2.3 step 10; bi/trilinear 3/4-1/4 weights per axis,
// i.e. 9/3/3/1 in 2D and 27/9/9/9/3/3/3/1 in 3D), coarse ghosts by the rule,
// evaluated one axis at a time: the interpolation from per-axis coarse
// indices and weights; plane(kz) returns the coarse plane kz (the whole
// array in 2D)
template <typename T, int DIM, typename Planes>
__device__ __forceinline__ T prolong_combine(const Planes &plane, int Ec, const int (&idx)[3][2], const T (&w)[3][2])
{
    if (DIM == 3) {
        T zsum = T(0);
        for (int c = 0; c < 2; c++) {
            const T *pl = plane(idx[2][c]);
            T ysum = T(0);
            for (int b = 0; b < 2; b++) {
                const int row = idx[1][b] * Ec;
                const T xv = w[0][0] * pl[row + idx[0][0]] + w[0][1] * pl[row + idx[0][1]];
                ysum += w[1][b] * xv;
            }
            zsum += w[2][c] * ysum;
        }
        return zsum;
    }
    const T *pl = plane(0);
    T ysum = T(0);
    for (int b = 0; b < 2; b++) {
        const int row = idx[1][b] * Ec;
        const T xv = w[0][0] * pl[row + idx[0][0]] + w[0][1] * pl[row + idx[0][1]];
        ysum += w[1][b] * xv;
    }
    return ysum;
}

// the two coarse indices and weights along one axis for fine index v
template <typename T>
__device__ __forceinline__ void prolong_axis(int v, const MgGeom &gc, int &i0, int &i1, T &w0, T &w1)
{
    const int near = (v + 1) >> 1;
    const int far = (v & 1) ? near - 1 : near + 1;
    T c0, c1;
    ghost_map<T>(near, gc, i0, c0);
    ghost_map<T>(far, gc, i1, c1);
    w0 = T(0.75) * c0;
    w1 = T(0.25) * c1;
}

// P(Phi_c) at fine active cell f
template <typename T, int DIM, typename Planes>
__device__ __forceinline__ T prolong_value_pl(const Planes &plane, const MgGeom &gc, const int *f)
{
    int idx[3][2] = {};
    T w[3][2] = {};
    for (int a = 0; a < DIM; a++)
        prolong_axis<T>(f[a], gc, idx[a][0], idx[a][1], w[a][0], w[a][1]);
    return prolong_combine<T, DIM>(plane, gc.E, idx, w);
}

template <typename T, int DIM>
__device__ __forceinline__ T prolong_value(const T *__restrict__ phi_c, const MgGeom &gc, const int *f)
{
    const int E2 = gc.E * gc.E;
    return prolong_value_pl<T, DIM>([&](int kz) { return phi_c + (DIM == 3 ? kz * E2 : 0); }, gc, f);
}

// Prolongation and correction (Sec. 2.3 step 10; bi/trilinear 3/4-1/4
// weights per axis, i.e. 9/3/3/1 in 2D and 27/9/9/9/3/3/3/1 in 3D), coarse
// ghosts by the rule, evaluated one axis at a time.
template <typename T, int DIM>
__device__ __forceinline__ void op_prolong(const T *__restrict__ phi_c, const MgGeom &gc, T *__restrict__ phi_f,
                                           const MgGeom &gf, int t0, int stride)
{
    const int Nf = gf.N;
    const int total = Nf * Nf * (DIM == 3 ? Nf : 1);
    Walk3 wk(t0, stride, Nf, DIM == 3 ? Nf : total);
    for (int t = t0; t < total; t += stride, wk.next()) {
        const int f[3] = {wk.x + 1, wk.y + 1, DIM == 3 ? wk.z + 1 : 0};
        phi_f[lin<DIM>(f[0], f[1], f[2], gf.E)] += prolong_value<T, DIM>(phi_c, gc, f);
    }
}

__device__ __forceinline__ int gtid() { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int gstride() { return gridDim.x * blockDim.x; }

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) k_smooth_colour(T *__restrict__ phi, const T *__restrict__ f, MgGeom g,
                                                            int colour)
{
    pdl_begin();
    op_smooth_colour<T, DIM>(phi, f, g, colour, gtid(), gstride());
}

// The same colour, when it is the last launch of a V-cycle in an adaptive
// step's nested loop: one thread also counts the cycle (inner_step_count).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) k_smooth_colour_counted(T *__restrict__ phi, const T *__restrict__ f,
                                                                    MgGeom g, int colour, MgSolveCtl *ctl,
                                                                    cudaGraphConditionalHandle hi)
{
    pdl_begin();
    if (blockIdx.x == 0 && threadIdx.x == 0)
        inner_step_count(ctl, hi);
    op_smooth_colour<T, DIM>(phi, f, g, colour, gtid(), gstride());
}

// Ghost-rule class of cell (i, j, k) of a coarse multigrid level, as
// neighbour_sum_ptr forms it: per axis bit 0 at index 1, bit 1 at index N.
template <int DIM>
__device__ __forceinline__ int cell_class(const MgGeom &g, int i, int j, int k)
{
    const int N = g.N;
    auto bits = [N](int a) { return (a == 1 ? 1 : 0) | (a == N ? 2 : 0); };
    return bits(i) | (bits(j) << 2) | (DIM == 3 ? bits(k) << 4 : 0);
}

// Residual and restriction with one fine cell per thread: 256 threads compute
// the residuals of a fine tile (16x8x2 in 3D, 32x8 in 2D) into shared memory
// `r` and the first of them average the children of the coarse cells of the
// tile (8x4x1 in 3D, 16x4 in 2D).  Tile (bx, by, bz) of the level; `lt` the
// thread's index in the tile; contains a __syncthreads (every thread of the
// block must call it, `ok` false for threads without a tile).
// The coarse correction starts from zero (Sec. 2.3 step 6).  With red_first
// the first red half-sweep on the coarse level is done here as well: with
// every black cell zero, a red cell's update is its own right-hand side times
// the update factor, (0 - h^2 f) * neg_inv_diag, exactly what op_smooth_colour
// computes there (its neighbour sum is +0.0), so the V-cycle skips that
// launch and the results do not change in any bit.
template <typename T, int DIM>
__device__ __forceinline__ void resid_restrict_tile(const T *__restrict__ phi_f, const T *__restrict__ f_f,
                                                    const MgGeom &gf, T *__restrict__ phi_c, T *__restrict__ f_c,
                                                    const MgGeom &gc, int bx, int by, int bz, int lt, bool ok,
                                                    T *__restrict__ r, bool red_first = false)
{
    const int Nf = gf.N, Nc = gc.N;
    constexpr int FX = DIM == 3 ? 16 : 32, FY = 8;
    const int tx = lt % FX, ty = (lt / FX) % FY, tz = DIM == 3 ? lt / (FX * FY) : 0;
    const int i = 1 + FX * bx + tx, j = 1 + FY * by + ty;
    const int k = DIM == 3 ? 1 + 2 * bz + tz : 0;
    T v = T(0);
    if (ok && i <= Nf && j <= Nf && (DIM == 2 || k <= Nf))
        v = residual_at<T, DIM>(phi_f, f_f, gf, i, j, k);
    r[lt] = v;
    __syncthreads();
    constexpr int CX = FX / 2, CY = FY / 2;
    if (ok && lt < CX * CY) {
        const int cx = lt % CX, cy = lt / CX;
        const int I = 1 + CX * bx + cx, J = 1 + CY * by + cy;
        const int K = DIM == 3 ? 1 + bz : 0;
        if (I <= Nc && J <= Nc && (DIM == 2 || K <= Nc)) {
            T s = T(0);
            for (int dz = 0; dz < (DIM == 3 ? 2 : 1); dz++)
                for (int dy = 0; dy < 2; dy++)
                    for (int dx = 0; dx < 2; dx++)
                        s += r[(dz * FY + 2 * cy + dy) * FX + 2 * cx + dx];
            const int pc = lin<DIM>(I, J, K, gc.E);
            const T fv = (DIM == 3 ? T(0.125) : T(0.25)) * s;
            f_c[pc] = fv;
            T pv = T(0);
            if (red_first && ((I + J + K) & 1) == 0)
                pv = (T(0) - geo_h2<T>(gc) * fv) * neg_inv_diag<T, DIM>(gc, cell_class<DIM>(gc, I, J, K));
            phi_c[pc] = pv;
        }
    }
}

// tiles of a restriction from a level of Nc coarse cells per edge
__host__ __device__ inline void resid_restrict_tiles(int dim, int Nc, int &nx, int &ny, int &nz)
{
    nx = dim == 3 ? (Nc + 7) / 8 : (Nc + 15) / 16;
    ny = (Nc + 3) / 4;
    nz = dim == 3 ? Nc : 1;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) k_resid_restrict(const T *__restrict__ phi_f, const T *__restrict__ f_f,
                                                             MgGeom gf, T *__restrict__ phi_c, T *__restrict__ f_c,
                                                             MgGeom gc, int red_first)
{
    pdl_begin();
    __shared__ T r[kThreads];
    resid_restrict_tile<T, DIM>(phi_f, f_f, gf, phi_c, f_c, gc, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, true,
                                r, red_first != 0);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) k_prolong(const T *__restrict__ phi_c, MgGeom gc, T *__restrict__ phi_f,
                                                      MgGeom gf)
{
    pdl_begin();
    op_prolong<T, DIM>(phi_c, gc, phi_f, gf, gtid(), gstride());
}

// Residual and restriction inside one block in two stages: every thread takes
// fine cells (residual into the dense scratch `r`), then every thread takes
// coarse cells (sum of the children in the order of op_resid_restrict, so the
// result is the same).  Spreads the FP64 work over all warps instead of 2^d
// serial residuals per coarse cell.
template <typename T, int DIM>
__device__ __forceinline__ void op_resid_restrict_staged(const T *__restrict__ phi_f, const T *__restrict__ f_f,
                                                         const MgGeom &gf, T *__restrict__ phi_c, T *__restrict__ f_c,
                                                         const MgGeom &gc, T *__restrict__ r, int t0, int stride)
{
    const int Nc = gc.N, Nf = gf.N;
    const int totf = Nf * Nf * (DIM == 3 ? Nf : 1);
    Walk3 wf(t0, stride, Nf, DIM == 3 ? Nf : totf);
    for (int t = t0; t < totf; t += stride, wf.next())
        r[t] = residual_at<T, DIM>(phi_f, f_f, gf, wf.x + 1, wf.y + 1, DIM == 3 ? wf.z + 1 : 0);
    __syncthreads();
    const int total = Nc * Nc * (DIM == 3 ? Nc : 1);
    const T w = DIM == 3 ? T(0.125) : T(0.25);
    Walk3 wk(t0, stride, Nc, DIM == 3 ? Nc : total);
    for (int t = t0; t < total; t += stride, wk.next()) {
        const int I = wk.x + 1, J = wk.y + 1, K = DIM == 3 ? wk.z + 1 : 0;
        T s = T(0);
        for (int dk = 0; dk < (DIM == 3 ? 2 : 1); dk++) {
            const int k = DIM == 3 ? 2 * K - 1 + dk : 0;
            if (DIM == 3 && k > Nf)
                continue;
            for (int dj = 0; dj < 2; dj++) {
                const int j = 2 * J - 1 + dj;
                if (j > Nf)
                    continue;
                for (int di = 0; di < 2; di++) {
                    const int i = 2 * I - 1 + di;
                    if (i > Nf)
                        continue;
                    s += r[((DIM == 3 ? (k - 1) * Nf : 0) + (j - 1)) * Nf + (i - 1)];
                }
            }
        }
        const int pc = lin<DIM>(I, J, K, gc.E);
        f_c[pc] = w * s;
        phi_c[pc] = T(0);
    }
}

// Per-cell plan of the one-block kernel, built once per launch so that its
// phases are loads, the arithmetic and a barrier.  Entry t of colour c of a
// level (t over the half-rows of op_smooth_colour's walk: the same cells in
// the same order; the two colours together cover every active cell once)
// holds in `idx` the cell's index in the level array (bits 0-19) and which of
// its six neighbours the ghost rule drops (bits 20-25: x-, x+, y-, y+, z-, z+),
// or -1 when the half-row has no cell of that colour; in `ijk` its indices
// (i | j << 8 | k << 16); in `nid` and `dg` its negated reciprocal diagonal and
// its diagonal.  Per fine level, for each index v = 1..N along an axis, the
// prolongation's two coarse indices and weights (ghost rule applied).
constexpr int kPlanCellBits = 20;

template <int DIM>
__host__ __device__ __forceinline__ int bottom_plan_count(int N)
{
    return ((N + 1) >> 1) * N * (DIM == 3 ? N : 1);   // entries per colour
}

template <typename T>
struct BottomPlan {
    int *idx, *ijk;
    T *nid, *dg;
};

template <typename T, int DIM>
__device__ __forceinline__ void bottom_plan_build(const MgGeom &g, const BottomPlan<T> &P, const T *stab, int t0,
                                                  int stride)
{
    const int N = g.N, half = (N + 1) >> 1, cnt = bottom_plan_count<DIM>(N);
    const bool coarse = g.L > 0, tieN = g.tie && N >= 2;
    for (int t = t0; t < 2 * cnt; t += stride) {
        const int c = t >= cnt ? 1 : 0, r = t - c * cnt;
        const int x = r % half, y = (r / half) % N, z = DIM == 3 ? r / (half * N) : 0;
        const int j = y + 1, k = DIM == 3 ? z + 1 : 0;
        const int i = ((((1 + j + k) & 1) == c) ? 1 : 2) + 2 * x;
        if (i > N) {
            P.idx[t] = -1;
            P.ijk[t] = 0;
            P.nid[t] = T(0);
            P.dg[t] = T(0);
            continue;
        }
        int e = lin<DIM>(i, j, k, g.E), cls = 0;
        if (coarse) {
            // the drops and boundary classes of neighbour_sum_ptr
            auto axis = [&](int a, int shift, int bit) {
                const bool lo = a == 1, hi = a == N;
                cls |= ((lo ? 1 : 0) | (hi ? 2 : 0)) << shift;
                if (lo || (hi && tieN))
                    e |= 1 << bit;
                if (hi)
                    e |= 1 << (bit + 1);
            };
            axis(i, 0, kPlanCellBits);
            axis(j, 2, kPlanCellBits + 2);
            if (DIM == 3)
                axis(k, 4, kPlanCellBits + 4);
        }
        P.idx[t] = e;
        P.ijk[t] = i | (j << 8) | (k << 16);
        // the values of neg_inv_diag and diag_of, the level's table read from
        // its copy in shared memory
        if (cls == 0 || !stab) {
            P.nid[t] = neg_inv_diag<T, DIM>(g, cls);
            P.dg[t] = diag_of<T, DIM>(g, cls);
        } else {
            P.nid[t] = stab[64 + cls];
            P.dg[t] = stab[cls];
        }
    }
}

// the ghost-folded neighbour sum of neighbour_sum_ptr (same association) of
// the cell of plan entry e at c, dropped neighbours read from `zero`
template <typename T, int DIM>
__device__ __forceinline__ T bottom_plan_nsum(const T *c, int e, int sy, int sz, const T *zero)
{
    constexpr int B = kPlanCellBits;
    const T *a0 = (e >> B) & 1 ? zero : c - 1;
    const T *a1 = (e >> (B + 1)) & 1 ? zero : c + 1;
    const T *a2 = (e >> (B + 2)) & 1 ? zero : c - sy;
    const T *a3 = (e >> (B + 3)) & 1 ? zero : c + sy;
    T s = (*a0 + *a1) + (*a2 + *a3);
    if (DIM == 3) {
        const T *a4 = (e >> (B + 4)) & 1 ? zero : c - sz;
        const T *a5 = (e >> (B + 5)) & 1 ? zero : c + sz;
        s += *a4 + *a5;
    }
    return s;
}

// one colour of a red-black sweep (the arithmetic of op_smooth_colour)
template <typename T, int DIM>
__device__ __forceinline__ void bottom_plan_smooth(T *__restrict__ phi, const T *__restrict__ f, const MgGeom &g,
                                                   const int *__restrict__ pidx, const T *__restrict__ pnid,
                                                   const T *zero, int t0, int stride)
{
    const int cnt = bottom_plan_count<DIM>(g.N);
    const int sy = g.E, sz = DIM == 3 ? g.E * g.E : 0;
    const T h2 = geo_h2<T>(g);
    for (int t = t0; t < cnt; t += stride) {
        const int e = pidx[t];
        if (e < 0)
            continue;
        const int p = e & ((1 << kPlanCellBits) - 1);
        T *c = phi + p;
        const T s = bottom_plan_nsum<T, DIM>(c, e, sy, sz, zero);
        if (sizeof(T) < sizeof(double) && g.N == 1) {
            // the coarsest level's one unknown (Sec. 2.3 step 8, an exact
            // solve) in FP64 even inside an FP32 V-cycle: its diagonal from
            // the ghost rule on every axis (first and last cell at once)
            double d = mg_axis_diag(3, g) + mg_axis_diag(3, g);
            if (DIM == 3)
                d += mg_axis_diag(3, g);
            *c = T(((double)s - g.h2 * (double)f[p]) / (-d));
        } else {
            *c = (s - h2 * f[p]) * pnid[t];
        }
    }
}

// Residual (Sec. 2.3 step 4) of every active cell of level gf into r at the
// cell's own index (r's ghost positions stay zero), then the 2^d-child
// average into level gc (step 5): the arithmetic and order of
// op_resid_restrict_staged, children beyond N read as a zero.  Contains a
// __syncthreads.
template <typename T, int DIM>
__device__ __forceinline__ void bottom_plan_restrict(const T *__restrict__ phi_f, const T *__restrict__ f_f,
                                                     const MgGeom &gf, const BottomPlan<T> &Pf,
                                                     T *__restrict__ phi_c, T *__restrict__ f_c, const MgGeom &gc,
                                                     const BottomPlan<T> &Pc, T *__restrict__ r, const T *zero,
                                                     int t0, int stride)
{
    constexpr int M = (1 << kPlanCellBits) - 1;
    const int Ef = gf.E, sz = DIM == 3 ? Ef * Ef : 0;
    const int nf = 2 * bottom_plan_count<DIM>(gf.N);
    const T ih2 = geo_inv_h2<T>(gf);
    for (int t = t0; t < nf; t += stride) {
        const int e = Pf.idx[t];
        if (e < 0)
            continue;
        const int p = e & M;
        const T *c = phi_f + p;
        const T other = bottom_plan_nsum<T, DIM>(c, e, Ef, sz, zero);
        r[p] = f_f[p] - (other + Pf.dg[t] * c[0]) * ih2;
    }
    __syncthreads();
    const int nc = 2 * bottom_plan_count<DIM>(gc.N);
    const T w = DIM == 3 ? T(0.125) : T(0.25);
    for (int t = t0; t < nc; t += stride) {
        const int e = Pc.idx[t];
        if (e < 0)
            continue;
        const int ijk = Pc.ijk[t];
        const int I = ijk & 255, J = (ijk >> 8) & 255, K = ijk >> 16;
        const T *b = r + lin<DIM>(2 * I - 1, 2 * J - 1, DIM == 3 ? 2 * K - 1 : 0, Ef);
        T s = T(0);
        for (int dk = 0; dk < (DIM == 3 ? 2 : 1); dk++)
            for (int dj = 0; dj < 2; dj++)
                for (int di = 0; di < 2; di++)
                    s += b[dk * sz + dj * Ef + di];
        f_c[e & M] = w * s;
        phi_c[e & M] = T(0);
    }
}

// Prolongation and correction (Sec. 2.3 step 10) into every active cell of
// level gf, the per-axis indices and weights from the tables ix, wt (entries
// 2(v-1), 2(v-1)+1 for fine index v): the arithmetic of op_prolong.
template <typename T, int DIM>
__device__ __forceinline__ void bottom_plan_prolong(const T *__restrict__ phi_c, const MgGeom &gc,
                                                    T *__restrict__ phi_f, const MgGeom &gf,
                                                    const BottomPlan<T> &Pf, const int *__restrict__ ix,
                                                    const T *__restrict__ wt, int t0, int stride)
{
    constexpr int M = (1 << kPlanCellBits) - 1;
    const int nf = 2 * bottom_plan_count<DIM>(gf.N);
    const int E2 = gc.E * gc.E;
    for (int t = t0; t < nf; t += stride) {
        const int e = Pf.idx[t];
        if (e < 0)
            continue;
        const int ijk = Pf.ijk[t];
        const int f[3] = {ijk & 255, (ijk >> 8) & 255, ijk >> 16};
        int idx[3][2] = {};
        T w[3][2] = {};
        for (int a = 0; a < DIM; a++) {
            const int v = 2 * (f[a] - 1);
            idx[a][0] = ix[v];
            idx[a][1] = ix[v + 1];
            w[a][0] = wt[v];
            w[a][1] = wt[v + 1];
        }
        phi_f[e & M] += prolong_combine<T, DIM>([&](int kz) { return phi_c + (DIM == 3 ? kz * E2 : 0); }, gc.E,
                                                idx, w);
    }
}

// Shared-memory layout of the one-block kernel, in elements: T region - Phi
// and f of every level, each level's residual (in its own layout), the
// plans' nid and dg, the prolongation weights, a copy of each level's
// boundary-diagonal table (128 entries), one zero; int region - the plans'
// idx and ijk, the prolongation indices.
struct BottomLayout {
    int lev[MG_BOTTOM_MAX + 1], res[MG_BOTTOM_MAX + 1], plan[MG_BOTTOM_MAX + 1], tab[MG_BOTTOM_MAX + 1];
    __host__ __device__ BottomLayout(const MgBottom &bt, int dim)
    {
        lev[0] = res[0] = plan[0] = tab[0] = 0;
        for (int q = 0; q < bt.nlev; q++) {
            const int E = bt.g[q].E, N = bt.g[q].N;
            const int vol = dim == 3 ? E * E * E : E * E;
            lev[q + 1] = lev[q] + 2 * vol;
            res[q + 1] = res[q] + vol;
            plan[q + 1] = plan[q] + 2 * (dim == 3 ? bottom_plan_count<3>(N) : bottom_plan_count<2>(N));
            tab[q + 1] = tab[q] + 2 * N;
        }
    }
    __host__ __device__ size_t t_elems(int n) const
    {
        return (size_t)lev[n] + res[n] + 2 * plan[n] + tab[n] + 128 * (size_t)n + 1;
    }
    __host__ __device__ size_t i_elems(int n) const { return 2 * (size_t)plan[n] + tab[n]; }
};

// The part of the V-cycle at and below multigrid level Ls (Sec. 2.3 steps
// 6-11 restricted to those levels) in one thread block, every array of those
// levels in shared memory: pre-smoothing at Ls, restriction and smoothing
// down to the one-cell level, prolongation and post-smoothing back up to Ls.
// Phi and f of level Ls come from global memory (f written by the
// restriction from Ls-1, Phi zero; or the finest level itself when Ls = 0);
// the smoothed Phi of level Ls goes back.  Same per-cell arithmetic and the
// same order of phases as the one-kernel-per-phase path, every phase from
// the per-cell plan.
template <typename T, int DIM>
__device__ __forceinline__ void bottom_body(T *__restrict__ phi_g, const T *__restrict__ f_g, const MgBottom &bt,
                                            int nu_pre, int nu_post, unsigned char *smem_raw)
{
    const int n = bt.nlev;
    const BottomLayout lay(bt, DIM);
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *res = sm + lay.lev[n];
    T *nid = res + lay.res[n];
    T *dg = nid + lay.plan[n];
    T *wt = dg + lay.plan[n];
    T *stab = wt + lay.tab[n];
    T *zero = stab + 128 * n;
    int *idx = reinterpret_cast<int *>(zero + 1);
    int *ijk = idx + lay.plan[n];
    int *ix = ijk + lay.plan[n];
    auto PHI = [&](int q) { return sm + lay.lev[q]; };
    auto F = [&](int q) { return sm + lay.lev[q] + (lay.lev[q + 1] - lay.lev[q]) / 2; };
    auto plan = [&](int q) {
        return BottomPlan<T>{idx + lay.plan[q], ijk + lay.plan[q], nid + lay.plan[q], dg + lay.plan[q]};
    };
    const int tid = threadIdx.x, nth = blockDim.x;
    // 1. level Ls from global memory, every other array to zero, the plan's
    // image (or the boundary-diagonal tables to build it from) to shared
    // memory: the global loads in one phase
    const int c0 = (lay.lev[1] - lay.lev[0]) / 2;
    for (int t = tid; t < c0; t += nth) {
        PHI(0)[t] = phi_g[t];
        F(0)[t] = f_g[t];
    }
    for (int t = lay.lev[1] + tid; t < lay.lev[n] + lay.res[n]; t += nth)
        sm[t] = T(0);
    if (bt.plan) {
        const int nimg = 2 * lay.plan[n] + lay.tab[n];   // nid, dg, wt and idx, ijk, ix are contiguous
        const T *imgT = static_cast<const T *>(bt.plan);
        const int *imgI = reinterpret_cast<const int *>(imgT + nimg);
        for (int t = tid; t < nimg; t += nth) {
            nid[t] = imgT[t];
            idx[t] = imgI[t];
        }
    } else {
        for (int t = tid; t < 128 * n; t += nth) {
            const T *tb = tab_of<T>(bt.g[t >> 7]);
            stab[t] = tb ? tb[t & 127] : T(0);
        }
    }
    if (tid == 0)
        *zero = T(0);
    __syncthreads();
    // 2. the plans, when there is no image (bt.plan is the same for the block)
    if (!bt.plan) {
        for (int q = 0; q < n; q++)
            bottom_plan_build<T, DIM>(bt.g[q], plan(q), tab_of<T>(bt.g[q]) ? stab + 128 * q : nullptr, tid, nth);
        for (int q = 0; q + 1 < n; q++)
            for (int v = 1 + tid; v <= bt.g[q].N; v += nth) {
                const int o = lay.tab[q] + 2 * (v - 1);
                prolong_axis<T>(v, bt.g[q + 1], ix[o], ix[o + 1], wt[o], wt[o + 1]);
            }
        __syncthreads();
    }
    auto smooth = [&](int q, int sweeps) {
        const int cnt = bottom_plan_count<DIM>(bt.g[q].N);
        const BottomPlan<T> P = plan(q);
        for (int sw = 0; sw < sweeps; sw++)
            for (int c = 0; c < 2; c++) {
                bottom_plan_smooth<T, DIM>(PHI(q), F(q), bt.g[q], P.idx + c * cnt, P.nid + c * cnt, zero, tid, nth);
                __syncthreads();
            }
    };
    smooth(0, bt.g[0].N == 1 ? (nu_pre > 0 ? 1 : 0) : nu_pre);
    int q = 0;
    while (bt.g[q].N > 1 && q + 1 < n) {
        bottom_plan_restrict<T, DIM>(PHI(q), F(q), bt.g[q], plan(q), PHI(q + 1), F(q + 1), bt.g[q + 1], plan(q + 1),
                                     res + lay.res[q], zero, tid, nth);
        __syncthreads();
        smooth(q + 1, bt.g[q + 1].N == 1 ? (nu_pre > 0 ? 1 : 0) : nu_pre);
        q++;
    }
    while (q > 0) {
        bottom_plan_prolong<T, DIM>(PHI(q), bt.g[q], PHI(q - 1), bt.g[q - 1], plan(q - 1), ix + lay.tab[q - 1],
                                    wt + lay.tab[q - 1], tid, nth);
        __syncthreads();
        smooth(q - 1, nu_post);
        q--;
    }
    for (int t = tid; t < c0; t += nth)
        phi_g[t] = PHI(0)[t];
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(T *__restrict__ phi_g, const T *__restrict__ f_g,
                                                           MgBottom bt, int nu_pre, int nu_post)
{
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bottom_body<T, DIM>(phi_g, f_g, bt, nu_pre, nu_post, smem_raw);
}

// The plan image of the one-block kernel (one block, global memory): the
// values bottom_body builds itself, in its shared-memory order - T part nid,
// dg, wt, then int part idx, ijk, ix.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBottomThreads) k_bottom_plan(MgBottom bt, T *__restrict__ img)
{
    pdl_begin();
    const int n = bt.nlev;
    const BottomLayout lay(bt, DIM);
    T *nid = img, *dg = nid + lay.plan[n], *wt = dg + lay.plan[n];
    int *idx = reinterpret_cast<int *>(wt + lay.tab[n]);
    int *ijk = idx + lay.plan[n], *ix = ijk + lay.plan[n];
    for (int q = 0; q < n; q++)
        bottom_plan_build<T, DIM>(bt.g[q],
                                  BottomPlan<T>{idx + lay.plan[q], ijk + lay.plan[q], nid + lay.plan[q],
                                                dg + lay.plan[q]},
                                  nullptr, threadIdx.x, blockDim.x);
    for (int q = 0; q + 1 < n; q++)
        for (int v = 1 + (int)threadIdx.x; v <= bt.g[q].N; v += blockDim.x) {
            const int o = lay.tab[q] + 2 * (v - 1);
            prolong_axis<T>(v, bt.g[q + 1], ix[o], ix[o + 1], wt[o], wt[o + 1]);
        }
}

// ---------------------------------------------------------------------------
// Cluster V-cycle with the levels in distributed shared memory (3D).  One
// thread-block cluster holds the multigrid levels from Lc down: each of the
// larger ones split by z-planes over the CTAs, read across CTAs through
// shared::cluster addresses, the smallest in CTA 0.  Phases are separated by
// cluster barriers (release/acquire at cluster scope); no phase touches global
// memory except the load of level Lc at the start and the store of its Phi at
// the end.  Same per-cell arithmetic and order of phases as the
// one-kernel-per-phase path.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_ctas()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// every thread of every CTA of the cluster, from converged code
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// generic address of the same shared-memory location in CTA `rank` of the cluster
template <typename T>
__device__ __forceinline__ T *cluster_map(T *p, unsigned rank)
{
    unsigned long long out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"((unsigned long long)p), "r"(rank));
    return reinterpret_cast<T *>(out);
}

// first z-plane of CTA r when E planes are split over C CTAs
__host__ __device__ __forceinline__ int cluster_first_plane(int r, int E, int C) { return (r * E + C - 1) / C; }

template <typename T>
__global__ void __launch_bounds__(MG_CLUSTER_THREADS, 1) k_cluster_vcycle(const __grid_constant__ MgClusterPlan P)
{
    pdl_begin();
    constexpr int DIM = 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T *tabP[MG_CLUSTER_PLANES];
    __shared__ T *tabF[MG_CLUSTER_PLANES];
    __shared__ int tbo[MG_MAX_MG + 1];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int rank = (int)cluster_rank(), C = (int)cluster_ctas();
    const int tid = threadIdx.x, nth = blockDim.x;
    const int nl = P.nclu + 1;                       // levels held as planes (the last one in CTA 0)
    auto owner = [&](int q, int k) { return q < P.nclu ? (k * C) / P.g[q].E : 0; };
    auto first = [&](int q, int r) { return q < P.nclu ? cluster_first_plane(r, P.g[q].E, C) : (r == 0 ? 0 : P.g[q].E); };
    if (tid == 0) {
        tbo[0] = 0;
        for (int q = 0; q < nl; q++)
            tbo[q + 1] = tbo[q] + P.g[q].E;
    }
    __syncthreads();
    // plane pointer tables (shared::cluster addresses as generic pointers)
    for (int q = 0; q < nl; q++) {
        const int E = P.g[q].E, E2 = E * E;
        for (int k = tid; k < E; k += nth) {
            const int o = owner(q, k), lk = k - first(q, o);
            tabP[tbo[q] + k] = cluster_map(sm + P.off[q] + lk * E2, o);
            tabF[tbo[q] + k] = cluster_map(sm + P.off[q] + (P.pmax[q] + lk) * E2, o);
        }
    }
    // own planes start at zero (ghost layers and rings stay zero); level Lc from global
    for (int t = tid; t < P.off[nl]; t += nth)
        sm[t] = T(0);
    __syncthreads();
    {
        const int E = P.g[0].E, E2 = E * E;
        const int z0 = first(0, rank), z1 = first(0, rank + 1);
        const T *gp = static_cast<const T *>(P.phi0), *gf = static_cast<const T *>(P.f0);
        for (int t = tid; t < (z1 - z0) * E2; t += nth) {
            sm[P.off[0] + t] = gp[z0 * E2 + t];
            sm[P.off[0] + P.pmax[0] * E2 + t] = gf[z0 * E2 + t];
        }
    }
    cluster_barrier();
    auto PL = [&](int q, int k) { return tabP[tbo[q] + k]; };
    auto FL = [&](int q, int k) { return tabF[tbo[q] + k]; };
    // interior planes [kl, kh) of level q owned by this CTA
    auto own = [&](int q, int &kl, int &kh) {
        kl = max(first(q, rank), 1);
        kh = min(first(q, rank + 1), P.g[q].N + 1);
    };
    auto smooth = [&](int q, int sweeps) {
        const MgGeom &g = P.g[q];
        const int N = g.N, E = g.E, half = (N + 1) >> 1;
        const T h2 = geo_h2<T>(g);
        int kl, kh;
        own(q, kl, kh);
        const int total = half * N * max(kh - kl, 0);
        for (int sw = 0; sw < sweeps; sw++)
            for (int colour = 0; colour < 2; colour++) {
                Walk3 w(tid, nth, half, N);
                for (int t = tid; t < total; t += nth, w.next()) {
                    const int j = w.y + 1, k = w.z + kl;
                    const int i = ((((1 + j + k) & 1) == colour) ? 1 : 2) + 2 * w.x;
                    if (i > N)
                        continue;
                    const int p = j * E + i;
                    T *c = PL(q, k) + p;
                    int cls;
                    const T other = neighbour_sum_ptr<T, DIM>(c, PL(q, k - 1) + p, PL(q, k + 1) + p, g, i, j, k, E, cls);
                    c[0] = (other - h2 * FL(q, k)[p]) * neg_inv_diag<T, DIM>(g, cls);
                }
                cluster_barrier();
            }
    };
    for (int cyc = 0; cyc < P.cycles; cyc++) {
        for (int q = 0; q < P.nclu; q++) {
            smooth(q, P.nu_pre);
            // residual and restriction into level q + 1: coarse cells of own planes
            const MgGeom &gf = P.g[q], &gc = P.g[q + 1];
            const int Nf = gf.N, Ef = gf.E, Nc = gc.N, Ec = gc.E;
            const T wgt = T(0.125);
            int kl, kh;
            own(q + 1, kl, kh);
            const int total = Nc * Nc * max(kh - kl, 0);
            Walk3 w(tid, nth, Nc, Nc);
            for (int t = tid; t < total; t += nth, w.next()) {
                const int I = w.x + 1, J = w.y + 1, K = w.z + kl;
                T s = T(0);
                for (int dk = 0; dk < 2; dk++) {
                    const int k = 2 * K - 1 + dk;
                    if (k > Nf)
                        continue;
                    for (int dj = 0; dj < 2; dj++) {
                        const int j = 2 * J - 1 + dj;
                        if (j > Nf)
                            continue;
                        for (int di = 0; di < 2; di++) {
                            const int i = 2 * I - 1 + di;
                            if (i > Nf)
                                continue;
                            const int p = j * Ef + i;
                            s += residual_ptr<T, DIM>(PL(q, k) + p, PL(q, k - 1) + p, PL(q, k + 1) + p, FL(q, k)[p],
                                                      gf, i, j, k);
                        }
                    }
                }
                const int pc = J * Ec + I;
                FL(q + 1, K)[pc] = wgt * s;
                PL(q + 1, K)[pc] = T(0);
            }
            cluster_barrier();
        }
        if (rank == 0) {
            const int E = P.g[P.nclu].E;
            T *pb = sm + P.off[P.nclu];
            bottom_body<T, DIM>(pb, pb + E * E * E, P.bt, P.nu_pre, P.nu_post, smem_raw + P.scratch);
        }
        cluster_barrier();
        for (int q = P.nclu - 1; q >= 0; q--) {
            const MgGeom &gf = P.g[q], &gc = P.g[q + 1];
            const int Nf = gf.N, Ef = gf.E;
            int kl, kh;
            own(q, kl, kh);
            const int total = Nf * Nf * max(kh - kl, 0);
            Walk3 w(tid, nth, Nf, Nf);
            for (int t = tid; t < total; t += nth, w.next()) {
                const int f[3] = {w.x + 1, w.y + 1, w.z + kl};
                const T v = prolong_value_pl<T, DIM>([&](int kz) { return (const T *)PL(q + 1, kz); }, gc, f);
                PL(q, f[2])[f[1] * Ef + f[0]] += v;
            }
            cluster_barrier();
            smooth(q, P.nu_post);
        }
    }
    {
        const int E = P.g[0].E, E2 = E * E;
        const int z0 = first(0, rank), z1 = first(0, rank + 1);
        T *gp = static_cast<T *>(P.phi0);
        for (int t = tid; t < (z1 - z0) * E2; t += nth)
            gp[z0 * E2 + t] = sm[P.off[0] + t];
    }
    cluster_barrier();   // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// Temporally blocked FP32 V-cycle legs.  A block owns a tile of `tile`^d
// fine active cells (origin at an odd 1-based index, tile even, so the tile
// holds whole restriction families) and keeps the tile plus a halo in shared
// memory.  Each half-sweep updates a region one cell narrower than the one
// before, so the halo's values -- recomputed identically by the neighbouring
// blocks -- stay exact for the next half-sweep; only the tile is written
// back, into the other Phi buffer (the neighbours still read the input).
// The arithmetic per cell and the order of the phases are those of the
// one-kernel-per-phase path.
// ---------------------------------------------------------------------------
struct TbBox {
    int b0[3];   // storage coordinates of the Phi box origin
    int P;       // Phi box edge (tile + 2 halo)
};

// Visit the cells of colour `colour` in the storage box [lo, hi] (inclusive).
template <int DIM, class Fn>
__device__ __forceinline__ void for_colour_cells(const int *lo, const int *hi, int colour, Fn &&fn)
{
    if (hi[0] < lo[0] || hi[1] < lo[1] || (DIM == 3 && hi[2] < lo[2]))
        return;
    const int W = hi[0] - lo[0] + 1, hw = (W + 1) >> 1;
    const int ny = hi[1] - lo[1] + 1, nz = DIM == 3 ? hi[2] - lo[2] + 1 : 1;
    const int total = hw * ny * nz;
    Walk3 w(threadIdx.x, blockDim.x, hw, ny);
    for (int t = threadIdx.x; t < total; t += blockDim.x, w.next()) {
        const int j = lo[1] + w.y;
        const int k = DIM == 3 ? lo[2] + w.z : 0;
        const int i0 = lo[0] + (((lo[0] + j + k + colour) & 1) ? 1 : 0);
        const int i = i0 + 2 * w.x;
        if (i <= hi[0])
            fn(i, j, k);
    }
}

// Visit every cell of the storage box [lo, hi].
template <int DIM, class Fn>
__device__ __forceinline__ void for_box_cells(const int *lo, const int *hi, Fn &&fn)
{
    if (hi[0] < lo[0] || hi[1] < lo[1] || (DIM == 3 && hi[2] < lo[2]))
        return;
    const int W = hi[0] - lo[0] + 1, ny = hi[1] - lo[1] + 1, nz = DIM == 3 ? hi[2] - lo[2] + 1 : 1;
    const int total = W * ny * nz;
    Walk3 w(threadIdx.x, blockDim.x, W, ny);
    for (int t = threadIdx.x; t < total; t += blockDim.x, w.next())
        fn(lo[0] + w.x, lo[1] + w.y, DIM == 3 ? lo[2] + w.z : 0);
}

template <int DIM>
__device__ __forceinline__ int box_index(const TbBox &b, int i, int j, int k)
{
    return DIM == 3 ? ((k - b.b0[2]) * b.P + (j - b.b0[1])) * b.P + (i - b.b0[0]) : (j - b.b0[1]) * b.P + (i - b.b0[0]);
}

// Load the Phi box (cells outside the level's storage read as zero) and f
// (active cells only) of a tile.  Each thread keeps kLoadBatch loads in
// flight: the box comes from L2/HBM and one load at a time would leave the
// kernel bound by memory latency.
constexpr int kLoadBatch = 8;

template <typename T, int DIM>
__device__ __forceinline__ void tb_load(const T *__restrict__ phi, const T *__restrict__ f, const MgGeom &g,
                                        const TbBox &b, T *sPhi, T *sF)
{
    const int N = g.N;
    const int P = b.P;
    const int nP = P * P * (DIM == 3 ? P : 1);
    const int step = blockDim.x * kLoadBatch;
    Walk3 w(threadIdx.x, blockDim.x, P, DIM == 3 ? P : nP);
    for (int t0 = threadIdx.x; t0 < nP; t0 += step) {
        T vp[kLoadBatch], vf[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; u++) {
            const int t = t0 + u * blockDim.x;
            vp[u] = T(0);
            vf[u] = T(0);
            if (t < nP) {
                const int i = b.b0[0] + w.x, j = b.b0[1] + w.y, k = DIM == 3 ? b.b0[2] + w.z : 0;
                const bool in = i >= 0 && i <= N + 1 && j >= 0 && j <= N + 1 && (DIM == 2 || (k >= 0 && k <= N + 1));
                const bool act = i >= 1 && i <= N && j >= 1 && j <= N && (DIM == 2 || (k >= 1 && k <= N));
                const int gq = in ? lin<DIM>(i, j, k, g.E) : 0;
                if (in)
                    vp[u] = phi[gq];
                if (act)
                    vf[u] = f[gq];
            }
            w.next();
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; u++) {
            const int t = t0 + u * blockDim.x;
            if (t < nP) {
                sPhi[t] = vp[u];
                sF[t] = vf[u];
            }
        }
    }
}

// Half-sweeps s = 0 .. nhalf-1 over regions [o - (H-1-s), o + tile - 1 + (H-1-s)]
template <typename T, int DIM>
__device__ __forceinline__ void tb_sweeps(T *sPhi, const T *sF, const MgGeom &g, const TbBox &b, const int *o,
                                          int tile, int H, int nhalf)
{
    const int N = g.N;
    const T h2 = geo_h2<T>(g);
    const int sy = b.P, sz = b.P * b.P;
    for (int s = 0; s < nhalf; s++) {
        const int w = H - 1 - s;
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = max(o[a] - w, 1);
            hi[a] = min(o[a] + tile - 1 + w, N);
        }
        for_colour_cells<DIM>(lo, hi, s & 1, [&](int i, int j, int k) {
            const int q = box_index<DIM>(b, i, j, k);
            int cls;
            const T other = neighbour_sum_s<T, DIM>(sPhi, g, i, j, k, q, sy, sz, cls);
            sPhi[q] = (other - h2 * sF[q]) * neg_inv_diag<T, DIM>(g, cls);
        });
        __syncthreads();
    }
}

// P(Phi_c) at fine cell f with the coarse values read from a shared-memory box
template <typename T, int DIM>
__device__ __forceinline__ T prolong_value_box(const T *sC, const TbBox &cb, const MgGeom &gc, const int *f)
{
    int idx[3][2];
    T w[3][2];
    for (int a = 0; a < DIM; a++) {
        const int near = (f[a] + 1) >> 1;
        const int far = (f[a] & 1) ? near - 1 : near + 1;
        T c0, c1;
        ghost_map<T>(near, gc, idx[a][0], c0);
        ghost_map<T>(far, gc, idx[a][1], c1);
        w[a][0] = T(0.75) * c0;
        w[a][1] = T(0.25) * c1;
    }
    if (DIM == 3) {
        T zsum = T(0);
        for (int c = 0; c < 2; c++) {
            T ysum = T(0);
            for (int b = 0; b < 2; b++) {
                const int row = ((idx[2][c] - cb.b0[2]) * cb.P + (idx[1][b] - cb.b0[1])) * cb.P - cb.b0[0];
                const T xv = w[0][0] * sC[row + idx[0][0]] + w[0][1] * sC[row + idx[0][1]];
                ysum += w[1][b] * xv;
            }
            zsum += w[2][c] * ysum;
        }
        return zsum;
    }
    T ysum = T(0);
    for (int b = 0; b < 2; b++) {
        const int row = (idx[1][b] - cb.b0[1]) * cb.P - cb.b0[0];
        const T xv = w[0][0] * sC[row + idx[0][0]] + w[0][1] * sC[row + idx[0][1]];
        ysum += w[1][b] * xv;
    }
    return ysum;
}

template <typename T, int DIM>
__device__ __forceinline__ void tb_store(T *__restrict__ phi, const MgGeom &g, const T *sPhi, const TbBox &b,
                                         const int *o, int tile)
{
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = o[a];
        hi[a] = min(o[a] + tile - 1, g.N);
    }
    for_box_cells<DIM>(lo, hi, [&](int i, int j, int k) { phi[lin<DIM>(i, j, k, g.E)] = sPhi[box_index<DIM>(b, i, j, k)]; });
}

// Pre-smoothing (nu sweeps), residual and restriction of the tile at block
// coordinates blk.
template <typename T, int DIM>
__device__ __forceinline__ void tb_pre_body(const T *__restrict__ phi_in, T *__restrict__ phi_out,
                                            const T *__restrict__ f, const MgGeom &g, T *__restrict__ phi_c,
                                            T *__restrict__ f_c, const MgGeom &gc, int tile, int nu, const int *blk,
                                            unsigned char *smem_raw)
{
    const int H = 2 * nu + 1;
    TbBox b;
    b.P = tile + 2 * H;
    const int o[3] = {1 + tile * blk[0], 1 + tile * blk[1], DIM == 3 ? 1 + tile * blk[2] : 0};
    for (int a = 0; a < 3; a++)
        b.b0[a] = (DIM == 2 && a == 2) ? 0 : o[a] - H;
    const int nP = b.P * b.P * (DIM == 3 ? b.P : 1);
    T *sPhi = reinterpret_cast<T *>(smem_raw);
    T *sF = sPhi + nP;
    tb_load<T, DIM>(phi_in, f, g, b, sPhi, sF);
    __syncthreads();
    tb_sweeps<T, DIM>(sPhi, sF, g, b, o, tile, H, 2 * nu);
    // residual on the tile and the 2^d-child averages (fine cells beyond N count zero)
    const int Nf = g.N, Nc = gc.N;
    const int ch = tile / 2;
    int clo[3], chi[3];
    for (int a = 0; a < 3; a++) {
        clo[a] = (o[a] + 1) / 2;
        chi[a] = min(clo[a] + ch - 1, Nc);
    }
    if (DIM == 2) {
        clo[2] = chi[2] = 0;
    }
    const T w = DIM == 3 ? T(0.125) : T(0.25);
    const T ih2 = geo_inv_h2<T>(g);
    const int sy = b.P, sz = b.P * b.P;
    for_box_cells<DIM>(clo, chi, [&](int I, int J, int K) {
        T s = T(0);
        for (int dk = 0; dk < (DIM == 3 ? 2 : 1); dk++) {
            const int k = DIM == 3 ? 2 * K - 1 + dk : 0;
            if (DIM == 3 && k > Nf)
                continue;
            for (int dj = 0; dj < 2; dj++) {
                const int j = 2 * J - 1 + dj;
                if (j > Nf)
                    continue;
                for (int di = 0; di < 2; di++) {
                    const int i = 2 * I - 1 + di;
                    if (i > Nf)
                        continue;
                    const int q = box_index<DIM>(b, i, j, k);
                    int cls;
                    const T other = neighbour_sum_s<T, DIM>(sPhi, g, i, j, k, q, sy, sz, cls);
                    s += sF[q] - (other + diag_of<T, DIM>(g, cls) * sPhi[q]) * ih2;
                }
            }
        }
        const int pc = lin<DIM>(I, J, K, gc.E);
        f_c[pc] = w * s;
        phi_c[pc] = T(0);
    });
    tb_store<T, DIM>(phi_out, g, sPhi, b, o, tile);
}

// Prolongation + correction and post-smoothing (nu sweeps) of the tile at
// block coordinates blk.
template <typename T, int DIM>
__device__ __forceinline__ void tb_post_body(const T *__restrict__ phi_in, T *__restrict__ phi_out,
                                             const T *__restrict__ f, const MgGeom &g, const T *__restrict__ phi_c,
                                             const MgGeom &gc, int tile, int nu, const int *blk,
                                             unsigned char *smem_raw)
{
    const int H = 2 * nu;
    TbBox b;
    b.P = tile + 2 * H;
    const int o[3] = {1 + tile * blk[0], 1 + tile * blk[1], DIM == 3 ? 1 + tile * blk[2] : 0};
    for (int a = 0; a < 3; a++)
        b.b0[a] = (DIM == 2 && a == 2) ? 0 : o[a] - H;
    const int nP = b.P * b.P * (DIM == 3 ? b.P : 1);
    T *sPhi = reinterpret_cast<T *>(smem_raw);
    T *sF = sPhi + nP;
    tb_load<T, DIM>(phi_in, f, g, b, sPhi, sF);
    __syncthreads();
    // correct every active cell of the box from the coarse cells around it,
    // staged in shared memory behind the fine box
    {
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = max(b.b0[a], 1);
            hi[a] = min(b.b0[a] + b.P - 1, g.N);
        }
        if (DIM == 2)
            lo[2] = hi[2] = 0;
        TbBox cb;
        cb.P = 0;
        int cl[3] = {0, 0, 0}, chh[3] = {0, 0, 0};
        for (int a = 0; a < DIM; a++) {
            cl[a] = max(((lo[a] + 1) >> 1) - 1, 0);
            chh[a] = min(((hi[a] + 1) >> 1) + 1, gc.N + 1);
            cb.b0[a] = cl[a];
            cb.P = max(cb.P, chh[a] - cl[a] + 1);
        }
        if (DIM == 2)
            cb.b0[2] = 0;
        T *sC = sF + nP;
        const int nC = cb.P * cb.P * (DIM == 3 ? cb.P : 1);
        const int step = blockDim.x * kLoadBatch;
        Walk3 wc(threadIdx.x, blockDim.x, cb.P, DIM == 3 ? cb.P : nC);
        for (int t0 = threadIdx.x; t0 < nC; t0 += step) {
            T v[kLoadBatch];
#pragma unroll
            for (int u = 0; u < kLoadBatch; u++) {
                const int t = t0 + u * blockDim.x;
                v[u] = T(0);
                if (t < nC) {
                    const int i = cb.b0[0] + wc.x, j = cb.b0[1] + wc.y, k = DIM == 3 ? cb.b0[2] + wc.z : 0;
                    if (i <= gc.N + 1 && j <= gc.N + 1 && (DIM == 2 || k <= gc.N + 1))
                        v[u] = phi_c[lin<DIM>(i, j, k, gc.E)];
                }
                wc.next();
            }
#pragma unroll
            for (int u = 0; u < kLoadBatch; u++) {
                const int t = t0 + u * blockDim.x;
                if (t < nC)
                    sC[t] = v[u];
            }
        }
        __syncthreads();
        for_box_cells<DIM>(lo, hi, [&](int i, int j, int k) {
            const int fc[3] = {i, j, k};
            sPhi[box_index<DIM>(b, i, j, k)] += prolong_value_box<T, DIM>(sC, cb, gc, fc);
        });
    }
    __syncthreads();
    tb_sweeps<T, DIM>(sPhi, sF, g, b, o, tile, H, 2 * nu);
    tb_store<T, DIM>(phi_out, g, sPhi, b, o, tile);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(512) k_tb_pre(const T *__restrict__ phi_in, T *__restrict__ phi_out,
                                                const T *__restrict__ f, MgGeom g, T *__restrict__ phi_c,
                                                T *__restrict__ f_c, MgGeom gc, int tile, int nu)
{
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int blk[3] = {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z};
    tb_pre_body<T, DIM>(phi_in, phi_out, f, g, phi_c, f_c, gc, tile, nu, blk, smem_raw);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(512) k_tb_post(const T *__restrict__ phi_in, T *__restrict__ phi_out,
                                                 const T *__restrict__ f, MgGeom g, const T *__restrict__ phi_c,
                                                 MgGeom gc, int tile, int nu)
{
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int blk[3] = {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z};
    tb_post_body<T, DIM>(phi_in, phi_out, f, g, phi_c, gc, tile, nu, blk, smem_raw);
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sm)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
        sm[w] = v;
    __syncthreads();
    v = threadIdx.x < kThreads / 32 ? sm[threadIdx.x] : 0.0;
    if (w == 0)
        v = warp_sum(v);
    return v;
}

// r^2 and b^2 at active cell t of a finest level: b is the residual of the
// zero potential inside (only the outer-ring neighbours count).
template <int DIM>
__device__ __forceinline__ void norm_terms(const double *__restrict__ phi, const double *__restrict__ f,
                                           const MgGeom &g, int t, int which, double &b2, double &r2,
                                           float *__restrict__ r32, float *__restrict__ e32)
{
    const int N = g.N, E = g.E;
    const int r = div_small(t, N);
    const int i = t - r * N + 1;
    int j, k;
    if (DIM == 3) {
        k = div_small(r, N);
        j = r - k * N + 1;
        k += 1;
    } else {
        j = r + 1;
        k = 0;
    }
    const int p = lin<DIM>(i, j, k, E);
    if (which & 1) {
        double o = 0.0;
        if (i == 1) o += phi[p - 1];
        if (i == N) o += phi[p + 1];
        if (j == 1) o += phi[p - E];
        if (j == N) o += phi[p + E];
        if (DIM == 3) {
            if (k == 1) o += phi[p - E * E];
            if (k == N) o += phi[p + E * E];
        }
        const double v = f[p] - o * g.inv_h2;
        b2 += v * v;
    }
    if (which & 2) {
        const double v = residual_at<double, DIM>(phi, f, g, i, j, k);
        r2 += v * v;
        if (r32) {   // the next defect-correction step's right-hand side (k_defect's values)
            const long long q = mg_idx32(g, DIM, i, j, k);
            r32[q] = (float)v;
            e32[q] = 0.0f;
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_norms2(const double *__restrict__ phi, const double *__restrict__ f,
                                                     MgGeom g, int which, double *__restrict__ partials,
                                                     unsigned *__restrict__ counter, double *__restrict__ out2,
                                                     float *__restrict__ r32, float *__restrict__ e32)
{
    pdl_begin();
    __shared__ double sm[kThreads / 32];
    __shared__ bool last;
    const int N = g.N;
    const int total = N * N * (DIM == 3 ? N : 1);
    double b2 = 0.0, r2 = 0.0;
    for (int t = gtid(); t < total; t += gstride())
        norm_terms<DIM>(phi, f, g, t, which, b2, r2, r32, e32);
    // FP64 reductions cost FP64-pipe time: reduce only what was asked for
    if (which & 1)
        b2 = block_sum(b2, sm);
    if (which & 2)
        r2 = block_sum(r2, sm);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = b2;
        partials[2 * blockIdx.x + 1] = r2;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    double sb = 0.0, sr = 0.0;
    for (int t = threadIdx.x; t < (int)gridDim.x; t += blockDim.x) {
        sb += partials[2 * t];
        sr += partials[2 * t + 1];
    }
    if (which & 1)
        sb = block_sum(sb, sm);
    if (which & 2)
        sr = block_sum(sr, sm);
    if (threadIdx.x == 0) {
        if (which & 1)
            out2[0] = sb;
        if (which & 2)
            out2[1] = sr;
        *counter = 0u;
    }
}

// Two-launch form kept for the allocation-free entry point.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_resid_norm2(const double *__restrict__ phi, const double *__restrict__ f,
                                                          MgGeom g, int zero_inside, double *__restrict__ partials)
{
    pdl_begin();
    __shared__ double sm[kThreads / 32];
    const int N = g.N;
    const int total = N * N * (DIM == 3 ? N : 1);
    double b2 = 0.0, r2 = 0.0;
    for (int t = gtid(); t < total; t += gstride())
        norm_terms<DIM>(phi, f, g, t, zero_inside ? 1 : 2, b2, r2, nullptr, nullptr);
    const double acc = block_sum(zero_inside ? b2 : r2, sm);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) k_sum_partials(const double *__restrict__ partials, int n,
                                                           double *__restrict__ out)
{
    pdl_begin();
    __shared__ double sm[kThreads / 32];
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x)
        acc += partials[t];
    acc = block_sum(acc, sm);
    if (threadIdx.x == 0)
        *out = acc;
}

// Mixed precision defect: r32 = (float)(f - lap Phi) in FP64 on the finest
// level; the FP32 correction restarts from zero.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_defect(const double *__restrict__ phi, const double *__restrict__ f,
                                                     MgGeom g, float *__restrict__ r32, float *__restrict__ e32)
{
    pdl_begin();
    const int N = g.N;
    const int total = N * N * (DIM == 3 ? N : 1);
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, N);
        const int i = t - r * N + 1;
        int j, k;
        if (DIM == 3) {
            k = div_small(r, N);
            j = r - k * N + 1;
            k += 1;
        } else {
            j = r + 1;
            k = 0;
        }
        const long long q = mg_idx32(g, DIM, i, j, k);
        r32[q] = (float)residual_at<double, DIM>(phi, f, g, i, j, k);
        e32[q] = 0.0f;
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_accumulate(double *__restrict__ phi, const float *__restrict__ e32,
                                                         MgGeom g)
{
    pdl_begin();
    const int N = g.N;
    const int total = N * N * (DIM == 3 ? N : 1);
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, N);
        const int i = t - r * N + 1;
        int j, k;
        if (DIM == 3) {
            k = div_small(r, N);
            j = r - k * N + 1;
            k += 1;
        } else {
            j = r + 1;
            k = 0;
        }
        const int p = lin<DIM>(i, j, k, g.E);
        phi[p] += (double)e32[mg_idx32(g, DIM, i, j, k)];
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_set_density(int n, const double *__restrict__ rho,
                                                          const double *__restrict__ bc_rho,
                                                          const double *__restrict__ bc_phi, double *__restrict__ rho_blk,
                                                          double *__restrict__ f_blk, double *__restrict__ phi_blk,
                                                          double fourpiG)
{
    pdl_begin();
    const int E = n + 4;
    const int total = E * E * (DIM == 3 ? E : 1);
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, E);
        const int i = t - r * E;
        const int rq = DIM == 3 ? div_small(r, E) : 0;
        const int j = DIM == 3 ? r - rq * E : r;
        const int k = DIM == 3 ? rq : 2;
        const bool outer = i == 0 || i == n + 3 || j == 0 || j == n + 3 || (DIM == 3 && (k == 0 || k == n + 3));
        const bool omega = i >= 2 && i <= n + 1 && j >= 2 && j <= n + 1 && (DIM == 2 || (k >= 2 && k <= n + 1));
        if (omega) {
            const double v = rho[lin<DIM>(i - 2, j - 2, k - 2, n)];
            rho_blk[t] = v;
            f_blk[t] = fourpiG * v;
            if (bc_phi)
                phi_blk[t] = 0.0;
        } else if (bc_phi) {          // level 0: caller-owned buffer data
            if (outer) {
                phi_blk[t] = bc_phi[t];
            } else {
                const double v = bc_rho[lin<DIM>(i - 1, j - 1, DIM == 3 ? k - 1 : 0, n + 2)];
                rho_blk[t] = v;
                f_blk[t] = fourpiG * v;
                phi_blk[t] = 0.0;
            }
        }
    }
}

// Child storage index s -> parent storage index p0 and weight t of p0+1
// (child centre at parent coordinate off + 3/4 + s/2).
__device__ __forceinline__ void iface_axis(int s, int off, int &p0, double &t)
{
    if ((s & 1) == 0) {
        p0 = off + (s >> 1);
        t = 0.75;
    } else {
        p0 = off + ((s + 1) >> 1);
        t = 0.25;
    }
}

// Bilinear / trilinear interpolation (Appendix A) from the 2^d enclosing
// parent centres, one axis at a time.
template <int DIM>
__device__ __forceinline__ double interp(const double *__restrict__ src, int Ep, const int *p0, const double *t)
{
    double zs = 0.0;
    for (int dk = 0; dk < (DIM == 3 ? 2 : 1); dk++) {
        double ys = 0.0;
        for (int dj = 0; dj < 2; dj++) {
            const int row = DIM == 3 ? ((p0[2] + dk) * Ep + p0[1] + dj) * Ep : (p0[1] + dj) * Ep;
            const double xv = (1.0 - t[0]) * src[row + p0[0]] + t[0] * src[row + p0[0] + 1];
            ys += (dj ? t[1] : 1.0 - t[1]) * xv;
        }
        zs += DIM == 3 ? (dk ? t[2] : 1.0 - t[2]) * ys : ys;
    }
    return zs;
}

// Storage index of the r-th cell of the two outer rings of a block of edge E
// (E >= 5), rings enumerated so that consecutive r are consecutive ring cells:
// first the planes k = 0, 1, E-2, E-1 (3D), then per plane between them the
// rows j = 0, 1, E-2, E-1 and, per row between those, the four cells
// i = 0, 1, E-2, E-1.
template <int DIM>
__device__ __forceinline__ void ring_cell(int r, int E, int *s)
{
    auto edge = [E](int q) { return q < 2 ? q : E - 4 + q; };   // 0, 1, E-2, E-1
    int k = 0;
    if (DIM == 3) {
        const int P = E * E;
        if (r < 4 * P) {
            const int q = div_small(r, P), rem = r - q * P;
            const int j = div_small(rem, E);
            s[0] = rem - j * E;
            s[1] = j;
            s[2] = edge(q);
            return;
        }
        r -= 4 * P;
        const int M = 4 * E + 4 * (E - 4);   // ring cells of one plane between
        const int q = div_small(r, M);
        k = 2 + q;
        r -= q * M;
    }
    s[2] = k;
    if (r < 4 * E) {
        const int q = div_small(r, E);
        s[0] = r - q * E;
        s[1] = edge(q);
        return;
    }
    r -= 4 * E;
    s[1] = 2 + (r >> 2);
    s[0] = edge(r & 3);
}

// One-way interface (Sec. 2.1; Sec. 2.4).  With omega_done the interpolated
// guess on Omega is k_iface_guess's and this kernel walks the rings only
// (ring_cell), whole warps of ring cells.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_interface(int np, const double *__restrict__ phi_p,
                                                        const double *__restrict__ rho_p, int nc, int ox, int oy, int oz,
                                                        double *__restrict__ phi_c, double *__restrict__ rho_c,
                                                        double *__restrict__ f_c, double fourpiG, int guess,
                                                        const double *__restrict__ guess_src, int frozen,
                                                        int omega_done)
{
    pdl_begin();
    const int E = nc + 4, Ep = np + 4;
    const int all = E * E * (DIM == 3 ? E : 1);
    const int inside = DIM == 3 ? nc * nc * nc : nc * nc;
    const int total = omega_done ? all - inside : all;
    for (int u = gtid(); u < total; u += gstride()) {
        int s[3];
        int t;
        if (omega_done) {
            ring_cell<DIM>(u, E, s);
            if (DIM == 2)
                s[2] = 2;
            t = lin<DIM>(s[0], s[1], s[2], E);
        } else {
            t = u;
            const int r = div_small(t, E);
            s[0] = t - r * E;
            const int rq = DIM == 3 ? div_small(r, E) : 0;
            s[1] = DIM == 3 ? r - rq * E : r;
            s[2] = DIM == 3 ? rq : 2;
        }
        bool outer = false, inner = false;
        for (int a = 0; a < DIM; a++) {
            if (s[a] == 0 || s[a] == nc + 3)
                outer = true;
            else if (s[a] == 1 || s[a] == nc + 2)
                inner = true;
        }
        int p0[3] = {0, 0, 0};
        double w[3] = {0, 0, 0};
        const int off[3] = {ox, oy, oz};
        for (int a = 0; a < DIM; a++)
            iface_axis(s[a], off[a], p0[a], w[a]);
        if (outer) {
            phi_c[t] = interp<DIM>(phi_p, Ep, p0, w);
            continue;
        }
        if (inner) {
            const double rv = interp<DIM>(rho_p, Ep, p0, w);
            rho_c[t] = rv;
            f_c[t] = fourpiG * rv;
            if (frozen) {
                // frozen-interface ablation: interpolated potential held fixed
                phi_c[t] = interp<DIM>(phi_p, Ep, p0, w);
                continue;
            }
        }
        if (guess == 0)
            phi_c[t] = interp<DIM>(phi_p, Ep, p0, w);
        else if (guess == 1)
            phi_c[t] = 0.0;
        else
            phi_c[t] = guess_src[lin<DIM>(s[0] - 1, s[1] - 1, DIM == 3 ? s[2] - 1 : 0, nc + 2)];
    }
}

// The interpolated initial guess (Sec. 2.4; Appendix A) on Omega of a child
// level: per work item the 2^d children s = 2 sigma, 2 sigma + 1 along each
// axis, which share 3^d parent centres (off + sigma .. off + sigma + 2).  The
// x interpolation of each parent row serves both children planes, the y
// combination both child z planes -- about half of interp's FP64 operations
// per cell, with interp's arithmetic per cell (x, then y, then z).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_iface_guess(int np, const double *__restrict__ phi_p, int nc, int ox,
                                                          int oy, int oz, double *__restrict__ phi_c)
{
    pdl_begin();
    const int E = nc + 4, Ep = np + 4, hc = nc / 2;
    const int total = hc * hc * (DIM == 3 ? hc : 1);
    constexpr int NZ = DIM == 3 ? 3 : 1;
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, hc);
        const int sx = t - r * hc;
        const int rq = DIM == 3 ? div_small(r, hc) : 0;
        const int sy = DIM == 3 ? r - rq * hc : r, sz = DIM == 3 ? rq : 0;
        // parent cells off + sigma .. off + sigma + 2, sigma = s + 1
        const int bx = ox + sx + 1, by = oy + sy + 1, bz = DIM == 3 ? oz + sz + 1 : 0;
        double xv[NZ][3][2];   // [parent z row][parent y row][child x: even, odd]
#pragma unroll
        for (int pz = 0; pz < NZ; pz++)
#pragma unroll
            for (int py = 0; py < 3; py++) {
                const int row = DIM == 3 ? ((bz + pz) * Ep + by + py) * Ep : (by + py) * Ep;
                const double a = phi_p[row + bx], b = phi_p[row + bx + 1], c = phi_p[row + bx + 2];
                const double te = 0.75, to = 0.25;   // weight of the second parent: even child, odd child
                xv[pz][py][0] = (1.0 - te) * a + te * b;
                xv[pz][py][1] = (1.0 - to) * b + to * c;
            }
#pragma unroll
        for (int cx = 0; cx < 2; cx++)
#pragma unroll
            for (int cy = 0; cy < 2; cy++) {
                const double t1 = cy ? 0.25 : 0.75;
                double ys[NZ];
#pragma unroll
                for (int pz = 0; pz < NZ; pz++) {
                    double v = 0.0;
                    v += (1.0 - t1) * xv[pz][cy][cx];
                    v += t1 * xv[pz][cy + 1][cx];
                    ys[pz] = v;
                }
#pragma unroll
                for (int cz = 0; cz < (DIM == 3 ? 2 : 1); cz++) {
                    double zs = 0.0;
                    if (DIM == 3) {
                        const double t2 = cz ? 0.25 : 0.75;
                        zs += (1.0 - t2) * ys[cz];
                        zs += t2 * ys[cz + 1];
                    } else {
                        zs += ys[0];
                    }
                    const int i = 2 * (sx + 1) + cx, j = 2 * (sy + 1) + cy, k = DIM == 3 ? 2 * (sz + 1) + cz : 0;
                    phi_c[lin<DIM>(i, j, k, E)] = zs;
                }
            }
    }
}

// dst[c + od] = src[c + os] for the c-box [0, e)^d, arrays of edges Es / Ed
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_copy_box(int e, const double *__restrict__ src, int Es, int os,
                                                       double *__restrict__ dst, int Ed, int od)
{
    pdl_begin();
    const int total = e * e * (DIM == 3 ? e : 1);
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, e);
        const int i = t - r * e;
        const int rq = DIM == 3 ? div_small(r, e) : 0;
        const int j = DIM == 3 ? r - rq * e : r;
        const int k = DIM == 3 ? rq : 0;
        dst[lin<DIM>(i + od, j + od, DIM == 3 ? k + od : 0, Ed)] = src[lin<DIM>(i + os, j + os, DIM == 3 ? k + os : 0, Es)];
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_copy_guess(int n, const double *__restrict__ src,
                                                         double *__restrict__ phi_blk)
{
    pdl_begin();
    const int M = n + 2;
    const int total = M * M * (DIM == 3 ? M : 1);
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, M);
        const int i = t - r * M;
        const int rq = DIM == 3 ? div_small(r, M) : 0;
        const int j = DIM == 3 ? r - rq * M : r;
        const int k = DIM == 3 ? rq : 0;
        phi_blk[lin<DIM>(i + 1, j + 1, DIM == 3 ? k + 1 : 0, n + 4)] = src[t];
    }
}

// F = -grad(Phi) on Omega: Eq. 2 (stencil 0) or the two-point difference.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_forces(int n, double h, const double *__restrict__ phi,
                                                     double *__restrict__ F, double *__restrict__ phi_out, int stencil)
{
    pdl_begin();
    const int E = n + 4;
    const int total = n * n * (DIM == 3 ? n : 1);
    const double c1 = stencil == 0 ? (4.0 / 3.0) / (2.0 * h) : 1.0 / (2.0 * h);
    const double c2 = stencil == 0 ? (1.0 / 3.0) / (4.0 * h) : 0.0;
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, n);
        const int i = t - r * n + 2;
        const int rq = DIM == 3 ? div_small(r, n) : 0;
        const int j = DIM == 3 ? r - rq * n + 2 : r + 2;
        const int k = DIM == 3 ? rq + 2 : 0;
        const int p = lin<DIM>(i, j, k, E);
        const int st[3] = {1, E, E * E};
        for (int a = 0; a < DIM; a++) {
            const double d1 = phi[p + st[a]] - phi[p - st[a]];
            const double d2 = phi[p + 2 * st[a]] - phi[p - 2 * st[a]];
            F[(long)a * total + t] = -(c1 * d1 - c2 * d2);
        }
        if (phi_out)
            phi_out[t] = phi[p];
    }
}

// Stopping test of Sec. 3: max over Omega of |F(phi) - F(prev)|^2 into *cmax
// (non-negative doubles order like their bit patterns, so the atomic maximum
// is exact and independent of the order of the blocks).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_force_change(int n, double h, const double *__restrict__ phi,
                                                           const double *__restrict__ prev, int stencil,
                                                           unsigned long long *__restrict__ cmax)
{
    pdl_begin();
    const int E = n + 4;
    const int total = n * n * (DIM == 3 ? n : 1);
    const double c1 = stencil == 0 ? (4.0 / 3.0) / (2.0 * h) : 1.0 / (2.0 * h);
    const double c2 = stencil == 0 ? (1.0 / 3.0) / (4.0 * h) : 0.0;
    double m = 0.0;
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, n);
        const int i = t - r * n + 2;
        const int rq = DIM == 3 ? div_small(r, n) : 0;
        const int j = DIM == 3 ? r - rq * n + 2 : r + 2;
        const int k = DIM == 3 ? rq + 2 : 0;
        const int p = lin<DIM>(i, j, k, E);
        const int st[3] = {1, E, E * E};
        double s2 = 0.0;
        for (int a = 0; a < DIM; a++) {
            const double ga = c1 * (phi[p + st[a]] - phi[p - st[a]]) - c2 * (phi[p + 2 * st[a]] - phi[p - 2 * st[a]]);
            const double gb =
                c1 * (prev[p + st[a]] - prev[p - st[a]]) - c2 * (prev[p + 2 * st[a]] - prev[p - 2 * st[a]]);
            const double d = ga - gb;
            s2 += d * d;
        }
        m = fmax(m, s2);
    }
    for (int o = 16; o > 0; o >>= 1)
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(cmax, (unsigned long long)__double_as_longlong(m));
}

// prev = phi over the whole (n+4)^d block; resets the maximum of k_force_change
__global__ void k_save_prev(long total, const double *__restrict__ phi, double *__restrict__ prev,
                            unsigned long long *__restrict__ cmax)
{
    pdl_begin();
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *cmax = 0ull;
    for (long t = gtid(); t < total; t += gstride())
        prev[t] = phi[t];
}

// scal[1] = max|dF|^2 ||b||^2, so that the control kernels' sqrt(scal[1]) / ||b||
// is the change of the acceleration
__global__ void k_force_finish(double *scal, const unsigned long long *cmax)
{
    pdl_begin();
    scal[1] = __longlong_as_double((long long)*cmax) * scal[0];
}

// before the first iteration under the force test: an infinite change
__global__ void k_force_start(double *scal)
{
    pdl_begin();
    if (scal[0] > 0.0)
        scal[1] = CUDART_INF;
}

// copy Omega of an (n+4)^d block into a dense n^d array
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_extract(int n, const double *__restrict__ blk, double *__restrict__ out)
{
    pdl_begin();
    const int E = n + 4;
    const int total = n * n * (DIM == 3 ? n : 1);
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, n);
        const int i = t - r * n + 2;
        const int rq = DIM == 3 ? div_small(r, n) : 0;
        const int j = DIM == 3 ? r - rq * n + 2 : r + 2;
        const int k = DIM == 3 ? rq + 2 : 0;
        out[t] = blk[lin<DIM>(i, j, k, E)];
    }
}

// h^2 r = frho rho - (sum of the 2d neighbours - 2d Phi) on Omega of (n+4)^d blocks
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_resid_h2(int n, const double *__restrict__ phi,
                                                       const double *__restrict__ rho, double frho,
                                                       double *__restrict__ out)
{
    pdl_begin();
    const int E = n + 4;
    const int total = n * n * (DIM == 3 ? n : 1);
    for (int t = gtid(); t < total; t += gstride()) {
        const int r = div_small(t, n);
        const int i = t - r * n + 2;
        const int rq = DIM == 3 ? div_small(r, n) : 0;
        const int j = DIM == 3 ? r - rq * n + 2 : r + 2;
        const int k = DIM == 3 ? rq + 2 : 0;
        const int p = lin<DIM>(i, j, k, E);
        double nb = phi[p - 1] + phi[p + 1] + phi[p - E] + phi[p + E];
        if (DIM == 3)
            nb += phi[p - E * E] + phi[p + E * E];
        out[t] = frho * rho[p] - (nb - 2.0 * DIM * phi[p]);
    }
}

__global__ void k_zero(uint4 *p, size_t n16)
{
    pdl_begin();
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n16; t += (size_t)gridDim.x * blockDim.x)
        p[t] = make_uint4(0, 0, 0, 0);
}

__device__ __forceinline__ int keep_going(const MgSolveCtl &c, double tol, int max_cycles)
{
    return c.bnorm > 0.0 && c.status == 0 && c.cycles < max_cycles && !(c.rel < tol);
}

__global__ void k_ctl_init(MgSolveCtl *ctl, const double *scal, double tol, int max_cycles, int inner0,
                           cudaGraphConditionalHandle hc)
{
    pdl_begin();
    MgSolveCtl c;
    c.bnorm = sqrt(scal[0]);
    c.rel = c.bnorm > 0.0 ? sqrt(scal[1]) / c.bnorm : 0.0;
    c.cycles = 0;
    c.outer = 0;
    c.status = isfinite(c.bnorm) ? 0 : 6;   // non-finite input: diverged, not "nothing to do"
    c.inner = inner0;
    c.left = min(inner0, max_cycles);
    c.cyc0 = 0;
    c.go = keep_going(c, tol, max_cycles);
    *ctl = c;
    cudaGraphSetConditional(hc, c.go);
}

__global__ void k_ctl_step(MgSolveCtl *ctl, const double *scal, int inc, double tol, int max_cycles, int inner_max,
                           cudaGraphConditionalHandle hc, cudaGraphConditionalHandle hi)
{
    pdl_begin();
    MgSolveCtl c = *ctl;
    const double before = c.rel;
    c.cycles += inc;
    c.outer += 1;
    c.rel = sqrt(scal[1]) / c.bnorm;
    if (!isfinite(c.rel))
        c.status = 6;
    if (inner_max > 0) {
        c.inner = mg_next_inner(before, c.rel, c.cycles - c.cyc0, tol, inner_max);
        c.left = min(c.inner, max_cycles - c.cycles);
        c.cyc0 = c.cycles;
    }
    c.go = keep_going(c, tol, max_cycles);
    *ctl = c;
    cudaGraphSetConditional(hc, c.go);
    if (inner_max > 0)
        cudaGraphSetConditional(hi, 1);   // the next step's nested loop runs at least once
}

// end of one FP32 V-cycle of an adaptive step's nested loop (when the
// V-cycle's last launch is not a smoothing colour that counts it)
__global__ void k_inner_step(MgSolveCtl *ctl, cudaGraphConditionalHandle hi)
{
    pdl_begin();
    inner_step_count(ctl, hi);
}


// ---------------------------------------------------------------------------
// batched kernels (one launch per phase over all parts)
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(512) kb_tb_pre(const MgBPart *__restrict__ parts, const MgBTask *__restrict__ tasks,
                                                 const int *__restrict__ active, int L, int nu)
{
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MgBTask tk = tasks[blockIdx.x];
    if (!active[tk.part])
        return;
    const MgBPart &P = parts[tk.part];
    const int blk[3] = {tk.bx, tk.by, tk.bz};
    tb_pre_body<float, DIM>(P.phi32[L], P.phi32b[L], P.f32[L], P.g[L], P.phi32[L + 1], P.f32[L + 1], P.g[L + 1],
                            P.tile[L], nu, blk, smem_raw);
}

template <int DIM>
__global__ void __launch_bounds__(512) kb_tb_post(const MgBPart *__restrict__ parts, const MgBTask *__restrict__ tasks,
                                                  const int *__restrict__ active, int L, int nu)
{
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MgBTask tk = tasks[blockIdx.x];
    if (!active[tk.part])
        return;
    const MgBPart &P = parts[tk.part];
    const int blk[3] = {tk.bx, tk.by, tk.bz};
    tb_post_body<float, DIM>(P.phi32b[L], P.phi32[L], P.f32[L], P.g[L], P.phi32[L + 1], P.g[L + 1], P.tile[L], nu,
                             blk, smem_raw);
}

template <int DIM>
__global__ void __launch_bounds__(kBottomThreads) kb_bottom(const MgBPart *__restrict__ parts,
                                                            const int *__restrict__ active, int nu_pre, int nu_post)
{
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (!active[blockIdx.x])
        return;
    const MgBPart &P = parts[blockIdx.x];
    bottom_body<float, DIM>(P.phi32[P.Ls], P.f32[P.Ls], P.bt, nu_pre, nu_post, smem_raw);
}

// level L of a part in one-kernel-per-phase form: chunk c of nblk_lvl[L]
template <int DIM>
__global__ void __launch_bounds__(kThreads) kb_smooth(const MgBPart *__restrict__ parts,
                                                      const MgBCell *__restrict__ cells, const int *__restrict__ active,
                                                      int L, int colour)
{
    pdl_begin();
    const MgBCell c = cells[blockIdx.x];
    if (!active[c.part])
        return;
    const MgBPart &P = parts[c.part];
    op_smooth_colour<float, DIM>(P.phi32[L], P.f32[L], P.g[L], colour, c.chunk * kThreads + threadIdx.x,
                                 P.nblk_lvl[L] * kThreads);
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) kb_restrict(const MgBPart *__restrict__ parts,
                                                        const MgBCell *__restrict__ cells,
                                                        const int *__restrict__ active, int L)
{
    pdl_begin();
    const MgBCell c = cells[blockIdx.x];
    if (!active[c.part])
        return;
    const MgBPart &P = parts[c.part];
    op_resid_restrict<float, DIM>(P.phi32[L], P.f32[L], P.g[L], P.phi32[L + 1], P.f32[L + 1], P.g[L + 1],
                                  c.chunk * kThreads + threadIdx.x, P.nblk_lvl[L] * kThreads);
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) kb_prolong(const MgBPart *__restrict__ parts,
                                                       const MgBCell *__restrict__ cells,
                                                       const int *__restrict__ active, int L)
{
    pdl_begin();
    const MgBCell c = cells[blockIdx.x];
    if (!active[c.part])
        return;
    const MgBPart &P = parts[c.part];
    op_prolong<float, DIM>(P.phi32[L + 1], P.g[L + 1], P.phi32[L], P.g[L], c.chunk * kThreads + threadIdx.x,
                           P.nblk_lvl[L] * kThreads);
}

template <int DIM>
__device__ __forceinline__ void active_cell(const MgGeom &g, int t, int &i, int &j, int &k)
{
    const int N = g.N;
    const int r = div_small(t, N);
    i = t - r * N + 1;
    if (DIM == 3) {
        k = div_small(r, N);
        j = r - k * N + 1;
        k += 1;
    } else {
        j = r + 1;
        k = 0;
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) kb_defect(const MgBPart *__restrict__ parts,
                                                      const MgBCell *__restrict__ cells, const int *__restrict__ active)
{
    pdl_begin();
    const MgBCell c = cells[blockIdx.x];
    if (!active[c.part])
        return;
    const MgBPart &P = parts[c.part];
    const MgGeom &g = P.g[0];
    const int total = g.N * g.N * (DIM == 3 ? g.N : 1);
    for (int t = c.chunk * kThreads + threadIdx.x; t < total; t += P.nblk_act * kThreads) {
        int i, j, k;
        active_cell<DIM>(g, t, i, j, k);
        const long long q = mg_idx32(g, DIM, i, j, k);
        P.f32[0][q] = (float)residual_at<double, DIM>(P.phi, P.f, g, i, j, k);
        P.phi32[0][q] = 0.0f;
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) kb_accumulate(const MgBPart *__restrict__ parts,
                                                          const MgBCell *__restrict__ cells,
                                                          const int *__restrict__ active)
{
    pdl_begin();
    const MgBCell c = cells[blockIdx.x];
    if (!active[c.part])
        return;
    const MgBPart &P = parts[c.part];
    const MgGeom &g = P.g[0];
    const int total = g.N * g.N * (DIM == 3 ? g.N : 1);
    for (int t = c.chunk * kThreads + threadIdx.x; t < total; t += P.nblk_act * kThreads) {
        int i, j, k;
        active_cell<DIM>(g, t, i, j, k);
        const int p = lin<DIM>(i, j, k, g.E);
        P.phi[p] += (double)P.phi32[0][mg_idx32(g, DIM, i, j, k)];
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) kb_norms2(const MgBPart *__restrict__ parts,
                                                      const MgBCell *__restrict__ cells, const int *__restrict__ active,
                                                      int which)
{
    pdl_begin();
    __shared__ double sm[kThreads / 32];
    __shared__ bool last;
    const MgBCell c = cells[blockIdx.x];
    if (!active[c.part])
        return;
    const MgBPart &P = parts[c.part];
    const MgGeom &g = P.g[0];
    const int total = g.N * g.N * (DIM == 3 ? g.N : 1);
    double b2 = 0.0, r2 = 0.0;
    for (int t = c.chunk * kThreads + threadIdx.x; t < total; t += P.nblk_act * kThreads)
        norm_terms<DIM>(P.phi, P.f, g, t, which, b2, r2, nullptr, nullptr);
    if (which & 1)
        b2 = block_sum(b2, sm);
    if (which & 2)
        r2 = block_sum(r2, sm);
    if (threadIdx.x == 0) {
        P.partials[2 * c.chunk] = b2;
        P.partials[2 * c.chunk + 1] = r2;
        __threadfence();
        last = atomicAdd(P.counter, 1u) == (unsigned)P.nblk_act - 1;
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    double sb = 0.0, sr = 0.0;
    for (int t = threadIdx.x; t < P.nblk_act; t += blockDim.x) {
        sb += P.partials[2 * t];
        sr += P.partials[2 * t + 1];
    }
    if (which & 1)
        sb = block_sum(sb, sm);
    if (which & 2)
        sr = block_sum(sr, sm);
    if (threadIdx.x == 0) {
        if (which & 1)
            P.scal[0] = sb;
        if (which & 2)
            P.scal[1] = sr;
        *P.counter = 0u;
    }
}

// Interface of part P at cell t of its (n+4)^d block (Sec. 2.1, Appendix A):
// the outer ring's potential and the inner ring's density (and f) by
// interpolation from the parent, the initial guess inside (gmode 0
// interpolated, 1 zero, 2 the caller's); on level 0 only a caller's start.
template <int DIM>
__device__ __forceinline__ void iface_cell(const MgBPart &P, int t)
{
    const int nc = P.n, E = nc + 4, Ep = P.np + 4;
    int s[3];
    const int r = div_small(t, E);
    s[0] = t - r * E;
    const int rq = DIM == 3 ? div_small(r, E) : 0;
    s[1] = DIM == 3 ? r - rq * E : r;
    s[2] = DIM == 3 ? rq : 2;
    bool outer = false, inner = false;
    for (int a = 0; a < DIM; a++) {
        if (s[a] == 0 || s[a] == nc + 3)
            outer = true;
        else if (s[a] == 1 || s[a] == nc + 2)
            inner = true;
    }
    if (P.l == 0) {            // level 0: only a caller-supplied start inside
        if (!outer && P.gmode == 2)
            P.phi[t] = P.guess[lin<DIM>(s[0] - 1, s[1] - 1, DIM == 3 ? s[2] - 1 : 0, nc + 2)];
        return;
    }
    int p0[3] = {0, 0, 0};
    double w[3] = {0, 0, 0};
    for (int a = 0; a < DIM; a++)
        iface_axis(s[a], P.off[a], p0[a], w[a]);
    if (outer) {
        P.phi[t] = interp<DIM>(P.phi_p, Ep, p0, w);
        return;
    }
    if (inner) {
        const double rv = interp<DIM>(P.rho_p, Ep, p0, w);
        P.rho[t] = rv;
        P.f[t] = P.fourpiG * rv;
    }
    if (P.gmode == 0)
        P.phi[t] = interp<DIM>(P.phi_p, Ep, p0, w);
    else if (P.gmode == 1)
        P.phi[t] = 0.0;
    else
        P.phi[t] = P.guess[lin<DIM>(s[0] - 1, s[1] - 1, DIM == 3 ? s[2] - 1 : 0, nc + 2)];
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) kb_interface(const MgBPart *__restrict__ parts,
                                                         const MgBCell *__restrict__ cells)
{
    pdl_begin();
    const MgBCell c = cells[blockIdx.x];
    const MgBPart &P = parts[c.part];
    if (P.gmode < 0)
        return;
    const int E = P.n + 4;
    const int total = E * E * (DIM == 3 ? E : 1);
    for (int t = c.chunk * kThreads + threadIdx.x; t < total; t += P.nblk_blk * kThreads)
        iface_cell<DIM>(P, t);
}

__global__ void __launch_bounds__(1024) kb_ctl(const MgBPart *__restrict__ parts, int nparts, int *__restrict__ active,
                                               int init, int inc, double tol, int max_cycles,
                                               cudaGraphConditionalHandle hc)
{
    pdl_begin();
    int any = 0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
        const MgBPart &P = parts[p];
        MgSolveCtl c;
        if (init) {
            c.bnorm = sqrt(P.scal[0]);
            c.rel = c.bnorm > 0.0 ? sqrt(P.scal[1]) / c.bnorm : 0.0;
            c.cycles = 0;
            c.outer = 0;
            c.status = isfinite(c.bnorm) ? 0 : 6;
        } else {
            c = *P.ctl;
            if (!active[p])
                continue;
            c.cycles += inc;
            c.outer += 1;
            c.rel = sqrt(P.scal[1]) / c.bnorm;
            if (!isfinite(c.rel))
                c.status = 6;
        }
        c.go = keep_going(c, tol, max_cycles);
        *P.ctl = c;
        active[p] = c.go;
        any |= c.go;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0)
        cudaGraphSetConditional(hc, any ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// persistent batched solve: one block per hierarchy at a time
// ---------------------------------------------------------------------------
constexpr int kPersistThreads = 512;

// Fixed-order sum over the block (up to 1024 threads); valid in thread 0.
__device__ __forceinline__ double block_sum_all(double v, double *sm)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
        sm[w] = v;
    __syncthreads();
    v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    if (w == 0)
        v = warp_sum(v);
    return v;
}

// One FP32 V-cycle (Sec. 2.3 steps 2-13) of part P by this block: per level
// above the bottom, nu_pre sweeps and the residual restriction, the bottom
// levels from the one-block plan, then prolongation and nu_post sweeps back
// up.  The same per-cell functions as the one-kernel-per-phase launches.
template <int DIM>
__device__ void persist_vcycle(const MgBPart &P, int nu_pre, int nu_post, unsigned char *smem)
{
    const int tid = threadIdx.x, nth = blockDim.x, Ls = P.Ls;
    for (int L = 0; L < Ls; L++) {
        for (int sw = 0; sw < nu_pre; sw++)
            for (int col = 0; col < 2; col++) {
                op_smooth_colour<float, DIM>(P.phi32[L], P.f32[L], P.g[L], col, tid, nth);
                __syncthreads();
            }
        op_resid_restrict<float, DIM>(P.phi32[L], P.f32[L], P.g[L], P.phi32[L + 1], P.f32[L + 1], P.g[L + 1], tid,
                                      nth);
        __syncthreads();
    }
    bottom_body<float, DIM>(P.phi32[Ls], P.f32[Ls], P.bt, nu_pre, nu_post, smem);
    __syncthreads();
    for (int L = Ls; L > 0; L--) {
        op_prolong<float, DIM>(P.phi32[L], P.g[L], P.phi32[L - 1], P.g[L - 1], tid, nth);
        __syncthreads();
        for (int sw = 0; sw < nu_post; sw++)
            for (int col = 0; col < 2; col++) {
                op_smooth_colour<float, DIM>(P.phi32[L - 1], P.f32[L - 1], P.g[L - 1], col, tid, nth);
                __syncthreads();
            }
    }
}

// ||b||^2 and / or ||r||^2 of part P's finest level (which as in
// norm_terms), writing the next step's FP32 defect with it; the sums land in
// red[0..1] for every thread.
template <int DIM>
__device__ void persist_norms(const MgBPart &P, int which, double *sm, double *red)
{
    const MgGeom &g = P.g[0];
    const int total = g.N * g.N * (DIM == 3 ? g.N : 1);
    double b2 = 0.0, r2 = 0.0;
    for (int t = threadIdx.x; t < total; t += blockDim.x)
        norm_terms<DIM>(P.phi, P.f, g, t, which, b2, r2, P.f32[0], P.phi32[0]);
    b2 = block_sum_all(b2, sm);
    r2 = block_sum_all(r2, sm);
    if (threadIdx.x == 0) {
        red[0] = b2;
        red[1] = r2;
    }
    __syncthreads();
}

// The solve of one refinement level (part P) by this block, with the loop
// control of the graph path (k_ctl_init / k_ctl_step, nested adaptive steps)
// taken by thread 0.
template <int DIM>
__device__ void persist_level(const MgBPart &P, int nu_pre, int nu_post, double tol, int max_cycles, int inner0,
                              int inner_max, int stencil, unsigned char *smem)
{
    __shared__ double sm[32];
    __shared__ double red[2];
    __shared__ MgSolveCtl cs;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int E = P.n + 4;
    if (P.gmode >= 0) {
        const int total = E * E * (DIM == 3 ? E : 1);
        for (int t = tid; t < total; t += nth)
            iface_cell<DIM>(P, t);
        __syncthreads();
    }
    persist_norms<DIM>(P, 3, sm, red);
    if (tid == 0) {
        MgSolveCtl c;
        c.bnorm = sqrt(red[0]);
        c.rel = c.bnorm > 0.0 ? sqrt(red[1]) / c.bnorm : 0.0;
        c.cycles = 0;
        c.outer = 0;
        c.status = isfinite(c.bnorm) ? 0 : 6;
        c.inner = inner0;
        c.left = min(inner0, max_cycles);
        c.cyc0 = 0;
        c.go = keep_going(c, tol, max_cycles);
        cs = c;
    }
    __syncthreads();
    const MgGeom &g0 = P.g[0];
    const int nact = g0.N * g0.N * (DIM == 3 ? g0.N : 1);
    while (cs.go) {
        const int ncyc = inner_max > 0 ? cs.left : inner0;
        for (int v = 0; v < ncyc; v++)
            persist_vcycle<DIM>(P, nu_pre, nu_post, smem);
        for (int t = tid; t < nact; t += nth) {   // Phi += e in FP64
            int i, j, k;
            active_cell<DIM>(g0, t, i, j, k);
            P.phi[lin<DIM>(i, j, k, g0.E)] += (double)P.phi32[0][mg_idx32(g0, DIM, i, j, k)];
        }
        __syncthreads();
        persist_norms<DIM>(P, 2, sm, red);
        if (tid == 0) {
            MgSolveCtl c = cs;
            const double before = c.rel;
            c.cycles += ncyc;
            c.outer += 1;
            c.rel = sqrt(red[1]) / c.bnorm;
            if (!isfinite(c.rel))
                c.status = 6;
            if (inner_max > 0) {
                c.inner = mg_next_inner(before, c.rel, c.cycles - c.cyc0, tol, inner_max);
                c.left = min(c.inner, max_cycles - c.cycles);
                c.cyc0 = c.cycles;
            }
            c.go = keep_going(c, tol, max_cycles);
            cs = c;
        }
        __syncthreads();
    }
    if (P.out_F) {   // registered outputs: potential and forces of Eq. 2 (or the two-point difference)
        const int n = P.n;
        const int total = n * n * (DIM == 3 ? n : 1);
        const double c1 = stencil == 0 ? (4.0 / 3.0) / (2.0 * P.h) : 1.0 / (2.0 * P.h);
        const double c2 = stencil == 0 ? (1.0 / 3.0) / (4.0 * P.h) : 0.0;
        for (int t = tid; t < total; t += nth) {
            const int r = div_small(t, n);
            const int i = t - r * n + 2;
            const int rq = DIM == 3 ? div_small(r, n) : 0;
            const int j = DIM == 3 ? r - rq * n + 2 : r + 2;
            const int k = DIM == 3 ? rq + 2 : 0;
            const int p = lin<DIM>(i, j, k, E);
            const int st[3] = {1, E, E * E};
            for (int a = 0; a < DIM; a++) {
                const double d1 = P.phi[p + st[a]] - P.phi[p - st[a]];
                const double d2 = P.phi[p + 2 * st[a]] - P.phi[p - 2 * st[a]];
                P.out_F[(long)a * total + t] = -(c1 * d1 - c2 * d2);
            }
            if (P.out_phi)
                P.out_phi[t] = P.phi[p];
        }
    }
    if (tid == 0)
        *P.ctl = cs;
    __syncthreads();
}

// The whole batch in one launch: each block takes the next hierarchy from
// the counter (hierarchies ordered largest first on the host) and solves its
// levels in order; no block waits for another.
template <int DIM>
__global__ void __launch_bounds__(kPersistThreads, 2) k_persist(const MgBPart *__restrict__ parts,
                                                               const MgPTask *__restrict__ tasks, int ntasks,
                                                               unsigned *__restrict__ next, int nu_pre, int nu_post,
                                                               double tol, int max_cycles, int inner0, int inner_max,
                                                               int stencil)
{
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int task;
    for (;;) {
        if (threadIdx.x == 0)
            task = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int q = task;
        if (q >= ntasks)
            return;
        const MgPTask T = tasks[q];
        for (int l = 0; l < T.count; l++)
            persist_level<DIM>(parts[T.first + l], nu_pre, nu_post, tol, max_cycles, inner0, inner_max, stencil,
                               smem_raw);
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t mg_launch_smooth(int dim, bool fp32, void *phi, const void *f, const MgGeom &g, int c, cudaStream_t s,
                             MgSolveCtl *ctl, cudaGraphConditionalHandle hi)
{
    const long work = (long)((g.N + 1) / 2) * g.N * (dim == 3 ? g.N : 1);
    const int grid = grid_for(work);
    if (ctl) {
        if (dim == 3 && fp32)
            mg_launch_kernel(k_smooth_colour_counted<float, 3>, grid, kThreads, 0, s, (float *)phi, (const float *)f, g, c, ctl, hi);
        else if (dim == 3)
            mg_launch_kernel(k_smooth_colour_counted<double, 3>, grid, kThreads, 0, s, (double *)phi, (const double *)f, g, c, ctl,
                   hi);
        else if (fp32)
            mg_launch_kernel(k_smooth_colour_counted<float, 2>, grid, kThreads, 0, s, (float *)phi, (const float *)f, g, c, ctl, hi);
        else
            mg_launch_kernel(k_smooth_colour_counted<double, 2>, grid, kThreads, 0, s, (double *)phi, (const double *)f, g, c, ctl,
                   hi);
        return cudaGetLastError();
    }
    if (dim == 3) {
        if (fp32)
            mg_launch_kernel(k_smooth_colour<float, 3>, grid, kThreads, 0, s, (float *)phi, (const float *)f, g, c);
        else
            mg_launch_kernel(k_smooth_colour<double, 3>, grid, kThreads, 0, s, (double *)phi, (const double *)f, g, c);
    } else {
        if (fp32)
            mg_launch_kernel(k_smooth_colour<float, 2>, grid, kThreads, 0, s, (float *)phi, (const float *)f, g, c);
        else
            mg_launch_kernel(k_smooth_colour<double, 2>, grid, kThreads, 0, s, (double *)phi, (const double *)f, g, c);
    }
    return cudaGetLastError();
}

size_t mg_bottom_smem(int dim, bool fp32, const MgBottom &bt)
{
    const BottomLayout lay(bt, dim);
    return lay.t_elems(bt.nlev) * (fp32 ? 4 : 8) + lay.i_elems(bt.nlev) * sizeof(int);
}

size_t mg_bottom_plan_bytes(int dim, bool fp32, const MgBottom &bt)
{
    const BottomLayout lay(bt, dim);
    const size_t nimg = 2 * (size_t)lay.plan[bt.nlev] + lay.tab[bt.nlev];
    return nimg * ((fp32 ? 4 : 8) + sizeof(int));
}

cudaError_t mg_launch_bottom_plan(int dim, bool fp32, const MgBottom &bt, void *img, cudaStream_t s)
{
    if (dim == 3) {
        if (fp32)
            mg_launch_kernel(k_bottom_plan<float, 3>, 1, kBottomThreads, 0, s, bt, (float *)img);
        else
            mg_launch_kernel(k_bottom_plan<double, 3>, 1, kBottomThreads, 0, s, bt, (double *)img);
    } else {
        if (fp32)
            mg_launch_kernel(k_bottom_plan<float, 2>, 1, kBottomThreads, 0, s, bt, (float *)img);
        else
            mg_launch_kernel(k_bottom_plan<double, 2>, 1, kBottomThreads, 0, s, bt, (double *)img);
    }
    return cudaGetLastError();
}

cudaError_t mg_bottom_prepare()
{
    // allow the bottom kernel the dynamic shared memory it may ask for (current device)
    const int lim = MG_BOTTOM_SMEM_MAX;
    cudaError_t e = cudaFuncSetAttribute(k_bottom<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(k_bottom<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(k_bottom<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(k_bottom<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    return e;
}

cudaError_t mg_launch_bottom(int dim, bool fp32, void *phi, const void *f, const MgBottom &bt, int nu_pre,
                             int nu_post, cudaStream_t s)
{
    const size_t smem = mg_bottom_smem(dim, fp32, bt);
    if (dim == 3) {
        if (fp32)
            mg_launch_kernel(k_bottom<float, 3>, 1, kBottomThreads, smem, s, (float *)phi, (const float *)f, bt, nu_pre, nu_post);
        else
            mg_launch_kernel(k_bottom<double, 3>, 1, kBottomThreads, smem, s, (double *)phi, (const double *)f, bt, nu_pre, nu_post);
    } else {
        if (fp32)
            mg_launch_kernel(k_bottom<float, 2>, 1, kBottomThreads, smem, s, (float *)phi, (const float *)f, bt, nu_pre, nu_post);
        else
            mg_launch_kernel(k_bottom<double, 2>, 1, kBottomThreads, smem, s, (double *)phi, (const double *)f, bt, nu_pre, nu_post);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t cluster_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_cluster_vcycle<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (!e)
        e = cudaFuncSetAttribute(k_cluster_vcycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MG_CLUSTER_SMEM_MAX);
    return e;
}

static cudaLaunchConfig_t cluster_config(int csize, size_t smem, cudaStream_t s, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize, 1, 1);
    cfg.blockDim = dim3(MG_CLUSTER_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

int mg_cluster_prepare()
{
    static int dev_done = -1, chosen = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dev_done == dev)
        return chosen;
    dev_done = dev;
    chosen = 0;
    if (cluster_attrs<float>() || cluster_attrs<double>()) {
        cudaGetLastError();
        return 0;
    }
    for (int cs : {16, 8}) {
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg = cluster_config(cs, MG_CLUSTER_SMEM_MAX, nullptr, at);
        int n64 = 0, n32 = 0;
        if (cudaOccupancyMaxActiveClusters(&n64, k_cluster_vcycle<double>, &cfg) == cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&n32, k_cluster_vcycle<float>, &cfg) == cudaSuccess && n64 > 0 && n32 > 0) {
            chosen = cs;
            break;
        }
        cudaGetLastError();
    }
    return chosen;
}

bool mg_cluster_layout(bool fp32, int csize, MgClusterPlan &p, size_t *smem)
{
    if (csize <= 0 || p.nclu < 1 || p.nclu >= p.nlev)
        return false;
    const size_t w = fp32 ? 4 : 8;
    long planes = 0, off = 0;
    for (int q = 0; q <= p.nclu; q++) {
        const int E = p.g[q].E;
        p.pmax[q] = q < p.nclu ? (E + csize - 1) / csize : E;
        p.off[q] = (int)off;
        off += 2L * p.pmax[q] * E * E;
        planes += E;
    }
    p.off[p.nclu + 1] = (int)off;
    const size_t sb = (off * w + 15) / 16 * 16;
    p.scratch = (int)sb;
    const size_t total = sb + mg_bottom_smem(3, fp32, p.bt);
    if (planes > MG_CLUSTER_PLANES || total > MG_CLUSTER_SMEM_MAX)
        return false;
    *smem = total;
    return true;
}

cudaError_t mg_launch_cluster(bool fp32, const MgClusterPlan &p, int csize, size_t smem, cudaStream_t s)
{
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = cluster_config(csize, smem, s, at);
    return fp32 ? cudaLaunchKernelEx(&cfg, k_cluster_vcycle<float>, p) : cudaLaunchKernelEx(&cfg, k_cluster_vcycle<double>, p);
}

size_t mg_tb_smem(int dim, bool fp32, int tile, int halo)
{
    const size_t P = tile + 2 * halo;
    const size_t C = P / 2 + 3;   // coarse box of the post leg
    return (2 * (dim == 3 ? P * P * P : P * P) + (dim == 3 ? C * C * C : C * C)) * (fp32 ? 4 : 8);
}

cudaError_t mg_tb_prepare()
{
    const int lim = MG_TB_SMEM_MAX;
    cudaError_t e = cudaFuncSetAttribute(k_tb_pre<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(k_tb_post<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(k_tb_pre<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(k_tb_post<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    return e;
}

cudaError_t mg_launch_tb_pre(int dim, const float *phi_in, float *phi_out, const float *f, const MgGeom &g,
                             float *phi_c, float *f_c, const MgGeom &gc, int tile, int nu, cudaStream_t s)
{
    const int nb = (g.N + tile - 1) / tile;
    const size_t smem = mg_tb_smem(dim, true, tile, 2 * nu + 1);
    if (dim == 3)
        mg_launch_kernel(k_tb_pre<float, 3>, dim3(nb, nb, nb), 512, smem, s, phi_in, phi_out, f, g, phi_c, f_c, gc, tile, nu);
    else
        mg_launch_kernel(k_tb_pre<float, 2>, dim3(nb, nb, 1), 512, smem, s, phi_in, phi_out, f, g, phi_c, f_c, gc, tile, nu);
    return cudaGetLastError();
}

cudaError_t mg_launch_tb_post(int dim, const float *phi_in, float *phi_out, const float *f, const MgGeom &g,
                              const float *phi_c, const MgGeom &gc, int tile, int nu, cudaStream_t s)
{
    const int nb = (g.N + tile - 1) / tile;
    const size_t smem = mg_tb_smem(dim, true, tile, 2 * nu);
    if (dim == 3)
        mg_launch_kernel(k_tb_post<float, 3>, dim3(nb, nb, nb), 512, smem, s, phi_in, phi_out, f, g, phi_c, gc, tile, nu);
    else
        mg_launch_kernel(k_tb_post<float, 2>, dim3(nb, nb, 1), 512, smem, s, phi_in, phi_out, f, g, phi_c, gc, tile, nu);
    return cudaGetLastError();
}

cudaError_t mg_launch_resid_restrict(int dim, bool fp32, const void *phi_f, const void *f_f, const MgGeom &gf,
                                     void *phi_c, void *f_c, const MgGeom &gc, cudaStream_t s, bool red_first)
{
    const int rf = red_first ? 1 : 0;
    int nx, ny, nz;
    resid_restrict_tiles(dim, gc.N, nx, ny, nz);
    const dim3 grid(nx, ny, nz);
    if (dim == 3) {
        if (fp32)
            mg_launch_kernel(k_resid_restrict<float, 3>, grid, kThreads, 0, s, (const float *)phi_f, (const float *)f_f, gf,
                                                                 (float *)phi_c, (float *)f_c, gc, rf);
        else
            mg_launch_kernel(k_resid_restrict<double, 3>, grid, kThreads, 0, s, (const double *)phi_f, (const double *)f_f, gf,
                                                                  (double *)phi_c, (double *)f_c, gc, rf);
    } else {
        if (fp32)
            mg_launch_kernel(k_resid_restrict<float, 2>, grid, kThreads, 0, s, (const float *)phi_f, (const float *)f_f, gf,
                                                                 (float *)phi_c, (float *)f_c, gc, rf);
        else
            mg_launch_kernel(k_resid_restrict<double, 2>, grid, kThreads, 0, s, (const double *)phi_f, (const double *)f_f, gf,
                                                                  (double *)phi_c, (double *)f_c, gc, rf);
    }
    return cudaGetLastError();
}

cudaError_t mg_launch_prolong(int dim, bool fp32, const void *phi_c, const MgGeom &gc, void *phi_f, const MgGeom &gf,
                              cudaStream_t s)
{
    const int grid = grid_for(cube(gf.N, dim));
    if (dim == 3) {
        if (fp32)
            mg_launch_kernel(k_prolong<float, 3>, grid, kThreads, 0, s, (const float *)phi_c, gc, (float *)phi_f, gf);
        else
            mg_launch_kernel(k_prolong<double, 3>, grid, kThreads, 0, s, (const double *)phi_c, gc, (double *)phi_f, gf);
    } else {
        if (fp32)
            mg_launch_kernel(k_prolong<float, 2>, grid, kThreads, 0, s, (const float *)phi_c, gc, (float *)phi_f, gf);
        else
            mg_launch_kernel(k_prolong<double, 2>, grid, kThreads, 0, s, (const double *)phi_c, gc, (double *)phi_f, gf);
    }
    return cudaGetLastError();
}

cudaError_t mg_launch_norms2(int dim, const double *phi, const double *f, const MgGeom &g, int which,
                             double *partials, unsigned *counter, double *out2, cudaStream_t s, float *r32, float *e32)
{
    // about four cells per thread: fewer block reductions on the FP64 pipe
    const int grid = std::max(1, std::min<int>((int)((cube(g.N, dim) + 4 * kThreads - 1) / (4 * kThreads)), MG_NORM_BLOCKS_MAX));
    if (dim == 3)
        mg_launch_kernel(k_norms2<3>, grid, kThreads, 0, s, phi, f, g, which, partials, counter, out2, r32, e32);
    else
        mg_launch_kernel(k_norms2<2>, grid, kThreads, 0, s, phi, f, g, which, partials, counter, out2, r32, e32);
    return cudaGetLastError();
}

cudaError_t mg_launch_resid_norm2(int dim, const double *phi, const double *f, const MgGeom &g, bool zero_inside,
                                  double *partials, double *out, cudaStream_t s)
{
    if (dim == 3)
        mg_launch_kernel(k_resid_norm2<3>, MG_NORM_BLOCKS, kThreads, 0, s, phi, f, g, zero_inside ? 1 : 0, partials);
    else
        mg_launch_kernel(k_resid_norm2<2>, MG_NORM_BLOCKS, kThreads, 0, s, phi, f, g, zero_inside ? 1 : 0, partials);
    mg_launch_kernel(k_sum_partials, 1, kThreads, 0, s, partials, MG_NORM_BLOCKS, out);
    return cudaGetLastError();
}

cudaError_t mg_launch_defect(int dim, const double *phi, const double *f, const MgGeom &g, float *r32, float *e32,
                             cudaStream_t s)
{
    const int grid = grid_for(cube(g.N, dim));
    if (dim == 3)
        mg_launch_kernel(k_defect<3>, grid, kThreads, 0, s, phi, f, g, r32, e32);
    else
        mg_launch_kernel(k_defect<2>, grid, kThreads, 0, s, phi, f, g, r32, e32);
    return cudaGetLastError();
}

cudaError_t mg_launch_accumulate(int dim, double *phi, const float *e32, const MgGeom &g, cudaStream_t s)
{
    const int grid = grid_for(cube(g.N, dim));
    if (dim == 3)
        mg_launch_kernel(k_accumulate<3>, grid, kThreads, 0, s, phi, e32, g);
    else
        mg_launch_kernel(k_accumulate<2>, grid, kThreads, 0, s, phi, e32, g);
    return cudaGetLastError();
}

cudaError_t mg_launch_set_density(int dim, int n, const double *rho, const double *bc_rho, const double *bc_phi,
                                  double *rho_blk, double *f_blk, double *phi_blk, double fourpiG, cudaStream_t s)
{
    const int grid = grid_for(cube(n + 4, dim));
    if (dim == 3)
        mg_launch_kernel(k_set_density<3>, grid, kThreads, 0, s, n, rho, bc_rho, bc_phi, rho_blk, f_blk, phi_blk, fourpiG);
    else
        mg_launch_kernel(k_set_density<2>, grid, kThreads, 0, s, n, rho, bc_rho, bc_phi, rho_blk, f_blk, phi_blk, fourpiG);
    return cudaGetLastError();
}

cudaError_t mg_launch_interface(int dim, int np, const double *phi_p, const double *rho_p, int nc, int ox, int oy,
                                int oz, double *phi_c, double *rho_c, double *f_c, double fourpiG, int guess,
                                const double *guess_src, int frozen, cudaStream_t s)
{
    const int grid = grid_for(cube(nc + 4, dim));
    const int split = guess == 0;   // Omega by k_iface_guess, the rings here
    if (dim == 3)
        mg_launch_kernel(k_interface<3>, grid, kThreads, 0, s, np, phi_p, rho_p, nc, ox, oy, oz, phi_c, rho_c, f_c, fourpiG, guess,
                                                 guess_src, frozen, split);
    else
        mg_launch_kernel(k_interface<2>, grid, kThreads, 0, s, np, phi_p, rho_p, nc, ox, oy, 0, phi_c, rho_c, f_c, fourpiG, guess,
                                                 guess_src, frozen, split);
    if (cudaError_t e = cudaGetLastError())
        return e;
    if (split) {
        const int g2 = grid_for(cube(nc / 2, dim));
        if (dim == 3)
            mg_launch_kernel(k_iface_guess<3>, g2, kThreads, 0, s, np, phi_p, nc, ox, oy, oz, phi_c);
        else
            mg_launch_kernel(k_iface_guess<2>, g2, kThreads, 0, s, np, phi_p, nc, ox, oy, 0, phi_c);
    }
    return cudaGetLastError();
}

cudaError_t mg_launch_copy_guess(int dim, int n, const double *guess_src, double *phi_blk, cudaStream_t s)
{
    const int grid = grid_for(cube(n + 2, dim));
    if (dim == 3)
        mg_launch_kernel(k_copy_guess<3>, grid, kThreads, 0, s, n, guess_src, phi_blk);
    else
        mg_launch_kernel(k_copy_guess<2>, grid, kThreads, 0, s, n, guess_src, phi_blk);
    return cudaGetLastError();
}

cudaError_t mg_launch_forces(int dim, int n, double h, const double *phi_blk, double *F, double *phi_out, int stencil,
                             cudaStream_t s)
{
    const int grid = grid_for(cube(n, dim));
    if (dim == 3)
        mg_launch_kernel(k_forces<3>, grid, kThreads, 0, s, n, h, phi_blk, F, phi_out, stencil);
    else
        mg_launch_kernel(k_forces<2>, grid, kThreads, 0, s, n, h, phi_blk, F, phi_out, stencil);
    return cudaGetLastError();
}

cudaError_t mg_launch_force_stop(int phase, int dim, int n, double h, const double *phi_blk, double *prev,
                                 int stencil, unsigned long long *cmax, double *scal, cudaStream_t s)
{
    if (phase == 0) {
        mg_launch_kernel(k_force_start, 1, 1, 0, s, scal);
    } else if (phase == 1) {
        const long total = cube(n + 4, dim);
        mg_launch_kernel(k_save_prev, grid_for(total), kThreads, 0, s, total, phi_blk, prev, cmax);
    } else {
        const int grid = grid_for(cube(n, dim));
        if (dim == 3)
            mg_launch_kernel(k_force_change<3>, grid, kThreads, 0, s, n, h, phi_blk, prev, stencil, cmax);
        else
            mg_launch_kernel(k_force_change<2>, grid, kThreads, 0, s, n, h, phi_blk, prev, stencil, cmax);
        mg_launch_kernel(k_force_finish, 1, 1, 0, s, scal, cmax);
    }
    return cudaGetLastError();
}

cudaError_t mg_launch_ctl_init(MgSolveCtl *ctl, const double *scal, double tol, int max_cycles, int inner0,
                               cudaGraphConditionalHandle hc, cudaStream_t s)
{
    mg_launch_kernel(k_ctl_init, 1, 1, 0, s, ctl, scal, tol, max_cycles, inner0, hc);
    return cudaGetLastError();
}

cudaError_t mg_launch_ctl_step(MgSolveCtl *ctl, const double *scal, int inc, double tol, int max_cycles,
                               int inner_max, cudaGraphConditionalHandle hc, cudaGraphConditionalHandle hi,
                               cudaStream_t s)
{
    mg_launch_kernel(k_ctl_step, 1, 1, 0, s, ctl, scal, inc, tol, max_cycles, inner_max, hc, hi);
    return cudaGetLastError();
}

cudaError_t mg_launch_inner_step(MgSolveCtl *ctl, cudaGraphConditionalHandle hi, cudaStream_t s)
{
    mg_launch_kernel(k_inner_step, 1, 1, 0, s, ctl, hi);
    return cudaGetLastError();
}

cudaError_t mg_launch_extract(int dim, int n, const double *blk, double *out, cudaStream_t s)
{
    const int grid = grid_for(cube(n, dim));
    if (dim == 3)
        mg_launch_kernel(k_extract<3>, grid, kThreads, 0, s, n, blk, out);
    else
        mg_launch_kernel(k_extract<2>, grid, kThreads, 0, s, n, blk, out);
    return cudaGetLastError();
}

cudaError_t mg_launch_copy_box(int dim, int e, const double *src, int Es, int os, double *dst, int Ed, int od,
                              cudaStream_t s)
{
    const int grid = grid_for(cube(e, dim));
    if (dim == 3)
        mg_launch_kernel(k_copy_box<3>, grid, kThreads, 0, s, e, src, Es, os, dst, Ed, od);
    else
        mg_launch_kernel(k_copy_box<2>, grid, kThreads, 0, s, e, src, Es, os, dst, Ed, od);
    return cudaGetLastError();
}

cudaError_t mg_launch_resid_h2(int dim, int n, const double *phi_blk, const double *rho_blk, double frho,
                               double *out, cudaStream_t s)
{
    const int grid = grid_for(cube(n, dim));
    if (dim == 3)
        mg_launch_kernel(k_resid_h2<3>, grid, kThreads, 0, s, n, phi_blk, rho_blk, frho, out);
    else
        mg_launch_kernel(k_resid_h2<2>, grid, kThreads, 0, s, n, phi_blk, rho_blk, frho, out);
    return cudaGetLastError();
}

cudaError_t mg_launch_zero(void *p, size_t bytes, cudaStream_t s)
{
    // callers pass 256-byte aligned sub-allocations whose sizes are multiples of 16
    const size_t n16 = bytes / 16;
    if (n16)
        mg_launch_kernel(k_zero, grid_for((long)n16), kThreads, 0, s, (uint4 *)p, n16);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// batched launchers
// ---------------------------------------------------------------------------
cudaError_t mg_batch_prepare()
{
    const int lim = MG_TB_SMEM_MAX;
    cudaError_t e = cudaFuncSetAttribute(kb_tb_pre<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(kb_tb_post<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(kb_tb_pre<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(kb_tb_post<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (!e)
        e = cudaFuncSetAttribute(kb_bottom<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, MG_BOTTOM_SMEM_MAX);
    if (!e)
        e = cudaFuncSetAttribute(kb_bottom<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, MG_BOTTOM_SMEM_MAX);
    return e;
}

int mg_persist_threads() { return kPersistThreads; }

cudaError_t mg_persist_prepare(int dim, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = dim == 3 ? cudaFuncSetAttribute(k_persist<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    MG_BOTTOM_SMEM_MAX)
                             : cudaFuncSetAttribute(k_persist<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    MG_BOTTOM_SMEM_MAX);
    if (e)
        return e;
    return dim == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_persist<3>, kPersistThreads, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_persist<2>, kPersistThreads, smem);
}

cudaError_t mg_launch_persist(int dim, const MgBPart *parts, const MgPTask *tasks, int ntasks, unsigned *next,
                              int grid, size_t smem, int nu_pre, int nu_post, double tol, int max_cycles, int inner0,
                              int inner_max, int stencil, cudaStream_t s)
{
    if (ntasks <= 0 || grid <= 0)
        return cudaSuccess;
    if (dim == 3)
        mg_launch_kernel(k_persist<3>, grid, kPersistThreads, smem, s, parts, tasks, ntasks, next, nu_pre, nu_post,
                         tol, max_cycles, inner0, inner_max, stencil);
    else
        mg_launch_kernel(k_persist<2>, grid, kPersistThreads, smem, s, parts, tasks, ntasks, next, nu_pre, nu_post,
                         tol, max_cycles, inner0, inner_max, stencil);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_tb_pre(int dim, const MgBPart *parts, const MgBTask *tasks, int ntasks, const int *active,
                               int depth, int nu, size_t smem, cudaStream_t s)
{
    if (ntasks <= 0)
        return cudaSuccess;
    if (dim == 3)
        mg_launch_kernel(kb_tb_pre<3>, ntasks, 512, smem, s, parts, tasks, active, depth, nu);
    else
        mg_launch_kernel(kb_tb_pre<2>, ntasks, 512, smem, s, parts, tasks, active, depth, nu);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_tb_post(int dim, const MgBPart *parts, const MgBTask *tasks, int ntasks, const int *active,
                                int depth, int nu, size_t smem, cudaStream_t s)
{
    if (ntasks <= 0)
        return cudaSuccess;
    if (dim == 3)
        mg_launch_kernel(kb_tb_post<3>, ntasks, 512, smem, s, parts, tasks, active, depth, nu);
    else
        mg_launch_kernel(kb_tb_post<2>, ntasks, 512, smem, s, parts, tasks, active, depth, nu);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_smooth(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                               int L, int colour, cudaStream_t s)
{
    if (ncells <= 0)
        return cudaSuccess;
    if (dim == 3)
        mg_launch_kernel(kb_smooth<3>, ncells, kThreads, 0, s, parts, cells, active, L, colour);
    else
        mg_launch_kernel(kb_smooth<2>, ncells, kThreads, 0, s, parts, cells, active, L, colour);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_restrict(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                                 int L, cudaStream_t s)
{
    if (ncells <= 0)
        return cudaSuccess;
    if (dim == 3)
        mg_launch_kernel(kb_restrict<3>, ncells, kThreads, 0, s, parts, cells, active, L);
    else
        mg_launch_kernel(kb_restrict<2>, ncells, kThreads, 0, s, parts, cells, active, L);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_prolong(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                                int L, cudaStream_t s)
{
    if (ncells <= 0)
        return cudaSuccess;
    if (dim == 3)
        mg_launch_kernel(kb_prolong<3>, ncells, kThreads, 0, s, parts, cells, active, L);
    else
        mg_launch_kernel(kb_prolong<2>, ncells, kThreads, 0, s, parts, cells, active, L);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_bottom(int dim, const MgBPart *parts, int nparts, const int *active, int nu_pre, int nu_post,
                               size_t smem, cudaStream_t s)
{
    if (dim == 3)
        mg_launch_kernel(kb_bottom<3>, nparts, kBottomThreads, smem, s, parts, active, nu_pre, nu_post);
    else
        mg_launch_kernel(kb_bottom<2>, nparts, kBottomThreads, smem, s, parts, active, nu_pre, nu_post);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_defect(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                               cudaStream_t s)
{
    if (dim == 3)
        mg_launch_kernel(kb_defect<3>, ncells, kThreads, 0, s, parts, cells, active);
    else
        mg_launch_kernel(kb_defect<2>, ncells, kThreads, 0, s, parts, cells, active);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_accumulate(int dim, const MgBPart *parts, const MgBCell *cells, int ncells,
                                   const int *active, cudaStream_t s)
{
    if (dim == 3)
        mg_launch_kernel(kb_accumulate<3>, ncells, kThreads, 0, s, parts, cells, active);
    else
        mg_launch_kernel(kb_accumulate<2>, ncells, kThreads, 0, s, parts, cells, active);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_norms2(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, const int *active,
                               int which, cudaStream_t s)
{
    if (dim == 3)
        mg_launch_kernel(kb_norms2<3>, ncells, kThreads, 0, s, parts, cells, active, which);
    else
        mg_launch_kernel(kb_norms2<2>, ncells, kThreads, 0, s, parts, cells, active, which);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_interface(int dim, const MgBPart *parts, const MgBCell *cells, int ncells, cudaStream_t s)
{
    if (dim == 3)
        mg_launch_kernel(kb_interface<3>, ncells, kThreads, 0, s, parts, cells);
    else
        mg_launch_kernel(kb_interface<2>, ncells, kThreads, 0, s, parts, cells);
    return cudaGetLastError();
}

cudaError_t mg_launch_b_ctl(const MgBPart *parts, int nparts, int *active, int init, int inc, double tol,
                            int max_cycles, cudaGraphConditionalHandle hc, cudaStream_t s)
{
    mg_launch_kernel(kb_ctl, 1, 1024, 0, s, parts, nparts, active, init, inc, tol, max_cycles, hc);
    return cudaGetLastError();
}
