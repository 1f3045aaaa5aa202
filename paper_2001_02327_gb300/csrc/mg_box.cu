// mg_box.cu -- the nested-grid multigrid solve on box (non-cubic) patches:
// per-axis multigrid sizes with semi-coarsening (Sec. 2.2 applied to each
// axis), the per-axis ghost rule of Sec. 2.4, the child-average restriction
// and the 3/4-1/4 prolongation of Appendix A along the axes that coarsened,
// the interface of Sec. 2.1 and the forces of Eq. 2.  The C ABI is in
// include/mg_box.h; this file holds the kernels and the host engine.
//
// Storage: every array of a multigrid level is one block of
// (N_z+2) x (N_y+2) x (N_x+2) cells (2D: no z), x fastest, one ghost layer per
// side.  Multigrid level 0 of a patch is its solved region Gamma (n_a + 2
// cells) with the outer buffer ring as the ghost layer, so its potential is
// the patch's (n+4) block itself.
//
// Launches: every per-cell kernel runs on a 3D grid -- x along the row (in
// blocks of up to 256 threads), y over rows (several per block when rows are
// short), z over planes -- so no thread divides to find its cell.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mg_box.h"
#include "mg_internal.h"

namespace {

// Geometry of one multigrid level of a box patch, per axis (x, y, z).
struct BoxGeom {
    int N[3];         // active cells (z: 1 in 2D)
    int E[3];         // storage extent N + 2 (z: 1 in 2D)
    int L;            // multigrid level; 0: the ghost layer holds boundary data
    int tie[3];       // centre of cell N at x_MG = 1 along this axis
    double cR[3];     // right ghost = cR Phi_N when !tie (Sec. 2.4)
    double ih2[3];    // 1 / h_a^2, h_a this axis's cell size on this level
    double d0, inv0;  // diagonal of a cell with no ghost folded in (-2 sum ih2) and its reciprocal
    int H;            // FP32 colour-split storage: cells of one colour per row, (E_x + 1) / 2
    long long half;   //   and per colour array, H E_y E_z
    float cRf[3], ih2f[3], d0f, inv0f;
};

template <typename T> __device__ __forceinline__ T gsel(double d, float f);
template <> __device__ __forceinline__ double gsel<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float gsel<float>(double, float f) { return f; }

__device__ __forceinline__ long long box_index(const BoxGeom &g, int i, int j, int k)
{
    return ((long long)k * g.E[1] + j) * g.E[0] + i;
}

// Index of cell (i, j, k) (storage indices, ghost layer included) in a level
// array of precision T.  FP64 arrays are plain blocks.  FP32 arrays are
// colour-split: colour (i + j + k) & 1 -- red 0, black 1, as the 1-based
// active indices give them -- selects one of two arrays of H cells per row,
// the cell at position i / 2 of its row.  A red cell's six neighbours are all
// black, so a colour pass reads the other colour's array, writes its own, and
// consecutive threads touch consecutive words.
template <bool SPLIT>
__device__ __forceinline__ long long lidx(const BoxGeom &g, int i, int j, int k)
{
    if (SPLIT)
        return ((i + j + k) & 1) * g.half + ((long long)k * g.E[1] + j) * g.H + (i >> 1);
    return box_index(g, i, j, k);
}

// Division of an unsigned 32-bit n by an invariant d with one multiply-high,
// an add and shifts (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994, round-up method): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (t + ((n - t) >> min(l, 1))) >>
// max(l - 1, 0) with t = mulhi(m, n); exact for every n and d >= 1.
struct FastDiv {
    unsigned m;
    int s1, s2;
};

inline FastDiv fast_div(unsigned d)
{
    int l = 0;
    while ((1ull << l) < d)
        l++;
    FastDiv f;
    f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = std::min(l, 1);
    f.s2 = std::max(l - 1, 0);
    return f;
}

__device__ __forceinline__ unsigned fdiv(const FastDiv &f, unsigned n)
{
    const unsigned t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// thread coordinates of a 3D launch: x along the row, y over rows, z planes
__device__ __forceinline__ int gx() { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int gy() { return blockIdx.y * blockDim.y + threadIdx.y; }
__device__ __forceinline__ int gz() { return blockIdx.z; }

// The off-diagonal sum of cell (i, j, k)'s equation and what ghosts add to
// its diagonal (Sec. 2.3 stencil, per-axis cell sizes): per axis the two
// neighbours, except on coarse levels where a neighbour in the ghost layer is
// replaced by the ghost rule of Sec. 2.4 folded into the cell's own
// coefficient (left ghost -Phi_1: -1; right ghost cR Phi_N: +cR; at a tie
// -Phi_{N-1}, which cancels the left neighbour, or +Phi_1 when N = 1).  The
// diagonal is d0 + fold.  Axis order x, y, z.  Returns whether the cell has a
// ghost neighbour on a coarse level.
template <typename T, int DIM, bool S>
__device__ __forceinline__ bool box_terms(const T *__restrict__ phi, const BoxGeom &g, int i, int j, int k, T &other,
                                          T &fold)
{
    const int id[3] = {i, j, k};
    other = T(0);
    fold = T(0);
    bool folded = false;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const T left = phi[lidx<S>(g, i - (a == 0), j - (a == 1), k - (a == 2))];
        const T right = phi[lidx<S>(g, i + (a == 0), j + (a == 1), k + (a == 2))];
        const T ih2 = gsel<T>(g.ih2[a], g.ih2f[a]);
        T o;
        if (g.L == 0) {
            o = left + right;
        } else {
            const bool lo = id[a] == 1, hi = id[a] == g.N[a];
            T self = lo ? T(-1) : T(0);
            o = lo ? T(0) : left;
            if (hi) {
                if (g.tie[a]) {
                    if (g.N[a] >= 2)
                        o = o + (-left);
                    else
                        self = self + T(1);
                } else {
                    self = self + gsel<T>(g.cR[a], g.cRf[a]);
                }
            } else {
                o = o + right;
            }
            if (lo || hi) {
                folded = true;
                fold = fold + self * ih2;
            }
        }
        other = other + o * ih2;
    }
    return folded;
}

// Red-black Gauss-Seidel, one colour (Sec. 2.3 steps 2, 6, 11): each cell
// with (i + j + k) & 1 == colour (2D: i + j; 1-based) solves its own equation
// for the current neighbours.  Thread x takes the x-th cell of its colour in
// row (j, k).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) kx_smooth(T *__restrict__ phi, const T *__restrict__ f, BoxGeom g, int colour)
{
    pdl_begin();
    const int j = gy() + 1, k = DIM == 3 ? gz() + 1 : 0;
    if (j > g.N[1])
        return;
    const int i = 2 * gx() + (((colour - j - k) & 1) ? 1 : 2);
    if (i > g.N[0])
        return;
    T other, fold;
    const bool folded = box_terms<T, DIM, false>(phi, g, i, j, k, other, fold);
    const long long p = box_index(g, i, j, k);
    const T rhs = f[p] - other;
    phi[p] = folded ? rhs / (gsel<T>(g.d0, g.d0f) + fold) : rhs * gsel<T>(g.inv0, g.inv0f);
}

// The same colour pass on colour-split FP32 storage, four cells of the
// colour per thread: row (j, k) of this colour holds cell i = 2m + p at
// position m (p = the colour's parity of i in this row), so cells m0..m0+3
// need the other colour's positions m0-1..m0+4 of the same row and m0..m0+3
// of the rows and planes around it -- aligned float4 loads (H is a multiple
// of 4) and one more word.  Cells next to a ghost on a coarse level take the
// per-cell form with the ghost rule folded in.
// Threads run over (row, group of four) linearly -- q groups per row, no
// idle threads at row ends -- the row and plane found by FastDiv.
// Loads that a colour pass makes of data it does not touch again before
// other data has passed through L2 (the other colour's potential, this
// colour's right-hand side): streaming, evict-first, so that the colour this
// pass writes -- the next pass's input -- stays in L2.
__device__ __forceinline__ float4 ld_stream4(const float *p)
{
    return __ldcs(reinterpret_cast<const float4 *>(p));
}
template <int DIM>
__global__ void __launch_bounds__(256) kx_smooth32(float *__restrict__ phi, const float *__restrict__ f, BoxGeom g,
                                                   int colour, unsigned total, int q, FastDiv dq, FastDiv dny)
{
    pdl_begin();
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const unsigned r = fdiv(dq, t);
    const unsigned kz = DIM == 3 ? fdiv(dny, r) : 0u;
    const int j = (int)(r - kz * (unsigned)g.N[1]) + 1, k = DIM == 3 ? (int)kz + 1 : 0;
    const int par = (colour - j - k) & 1;
    const int m0 = 4 * (int)(t - r * (unsigned)q);
    if (2 * m0 + par > g.N[0])
        return;
    const int row = (k * g.E[1] + j) * g.H;
    const float *o = phi + (colour ^ 1) * g.half + row;
    float *own = phi + colour * g.half + row;
    const float *fr = f + colour * g.half + row;
    const float4 c = ld_stream4(o + m0);
    const float s = __ldcs(par ? o + m0 + 4 : o + m0 - 1);
    const float4 yd = ld_stream4(o + m0 - g.H);
    const float4 yu = ld_stream4(o + m0 + g.H);
    float4 zd = make_float4(0.f, 0.f, 0.f, 0.f), zu = zd;
    if (DIM == 3) {
        const int pl = g.E[1] * g.H;
        zd = ld_stream4(o + m0 - pl);
        zu = ld_stream4(o + m0 + pl);
    }
    const float4 fv = ld_stream4(fr + m0);
    const float xl[4] = {par ? c.x : s, par ? c.y : c.x, par ? c.z : c.y, par ? c.w : c.z};
    const float xr[4] = {par ? c.y : c.x, par ? c.z : c.y, par ? c.w : c.z, par ? s : c.w};
    const float ydv[4] = {yd.x, yd.y, yd.z, yd.w}, yuv[4] = {yu.x, yu.y, yu.z, yu.w};
    const float zdv[4] = {zd.x, zd.y, zd.z, zd.w}, zuv[4] = {zu.x, zu.y, zu.z, zu.w};
    const float fvv[4] = {fv.x, fv.y, fv.z, fv.w};
    float nv[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
        float other = (xl[e] + xr[e]) * g.ih2f[0];
        other = other + (ydv[e] + yuv[e]) * g.ih2f[1];
        if (DIM == 3)
            other = other + (zdv[e] + zuv[e]) * g.ih2f[2];
        nv[e] = (fvv[e] - other) * g.inv0f;
    }
    const int i0 = 2 * m0 + par;
    const bool row_edge = g.L > 0 && (j == 1 || j == g.N[1] || (DIM == 3 && (k == 1 || k == g.N[2])));
    const bool plain = i0 >= 1 && i0 + 6 <= g.N[0] && (g.L == 0 || (!row_edge && i0 > 1 && i0 + 6 < g.N[0]));
    if (plain) {
        *reinterpret_cast<float4 *>(own + m0) = make_float4(nv[0], nv[1], nv[2], nv[3]);
        return;
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const int i = i0 + 2 * e;
        if (i < 1 || i > g.N[0])
            continue;
        if (g.L > 0 && (row_edge || i == 1 || i == g.N[0])) {
            float other, fold;
            const bool folded = box_terms<float, DIM, true>(phi, g, i, j, k, other, fold);
            const float rhs = fr[m0 + e] - other;
            own[m0 + e] = folded ? rhs / (g.d0f + fold) : rhs * g.inv0f;
        } else {
            own[m0 + e] = nv[e];
        }
    }
}

// r = f - A Phi at cell (i, j, k), storage layout S
template <typename T, int DIM, bool S>
__device__ __forceinline__ T box_resid(const T *__restrict__ phi, const T *__restrict__ f, const BoxGeom &g, int i,
                                       int j, int k)
{
    T other, fold;
    box_terms<T, DIM, S>(phi, g, i, j, k, other, fold);
    const long long p = lidx<S>(g, i, j, k);
    return f[p] - (other + (gsel<T>(g.d0, g.d0f) + fold) * phi[p]);
}

// Residual of the fine level restricted to the coarse right-hand side (Sec.
// 2.3 steps 4-5; Appendix A): coarse cell I sums the residuals of fine cells
// 2I-1 and 2I along each axis that coarsened (a child past the fine level's
// last cell counts zero) and of cell I along the others, x pairs first, then
// y, then z, times 2^-k (k the coarsened axes, bit a of cmask).  Also starts
// the coarse potential at zero (Sec. 2.3 step 6).  One thread per coarse cell.
// FS / CS: the fine / coarse arrays colour-split (FP32) or plain.
template <typename T, int DIM, bool FS, bool CS>
__global__ void __launch_bounds__(256) kx_resid_restrict(const T *__restrict__ phi, const T *__restrict__ f,
                                                         BoxGeom gf, T *__restrict__ fc, T *__restrict__ phic,
                                                         BoxGeom gc, int cmask, T wk)
{
    pdl_begin();
    const int I = gx() + 1, J = gy() + 1, K = DIM == 3 ? gz() + 1 : 0;
    if (I > gc.N[0] || J > gc.N[1])
        return;
    // first child and child count per axis
    const bool cx = cmask & 1, cy = (cmask >> 1) & 1, cz = DIM == 3 && ((cmask >> 2) & 1);
    const int x0 = cx ? 2 * I - 1 : I, y0 = cy ? 2 * J - 1 : J, z0 = cz ? 2 * K - 1 : K;
    const int nx = cx && 2 * I <= gf.N[0] ? 2 : 1, ny = cy && 2 * J <= gf.N[1] ? 2 : 1,
              nz = cz && 2 * K <= gf.N[2] ? 2 : 1;
    T sz = T(0);
#pragma unroll
    for (int dz = 0; dz < (DIM == 3 ? 2 : 1); dz++) {
        if (dz < nz) {
            T sy = T(0);
#pragma unroll
            for (int dy = 0; dy < 2; dy++) {
                if (dy < ny) {
                    T sx = T(0);
#pragma unroll
                    for (int dx = 0; dx < 2; dx++)
                        if (dx < nx)
                            sx = sx + box_resid<T, DIM, FS>(phi, f, gf, x0 + dx, y0 + dy, z0 + dz);
                    sy = sy + sx;
                }
            }
            sz = sz + sy;
        }
    }
    const long long pc = lidx<CS>(gc, I, J, K);
    fc[pc] = sz * wk;
    phic[pc] = T(0);
}

// The same residual and restriction from a colour-split FP32 level 0 (its
// ghost layer holds data: no ghost rule) whose every axis halves exactly
// (N_a = 2 N_a^c), four coarse cells along x per thread: coarse cells
// I0..I0+3 (I0 = 4u + 1) have fine children x = 8u+1 .. 8u+8, which with
// their x neighbours 8u and 8u+9 are positions 4u..4u+4 of the two colour
// arrays of each fine row -- two aligned float4 loads and two words per row
// instead of one word per cell and neighbour.  Per cell the arithmetic is
// that of kx_resid_restrict (per-axis pair sums times 1/h_a^2 in x, y, z
// order, then f - (other + d0 Phi)), the child sums x pairs first, then y,
// then z, times 2^-d.  Threads run over (coarse row, group of four) linearly.
// Positions past a row's end read the next row (or the arrays' 16-word
// tail); they feed only cells of coarse indices past N^c, which are not
// stored.
struct Row8 {     // fine cells 8u+1 .. 8u+8 of one row, in x order
    float v[8];
};

// odd-x cells from array `od` (positions m..m+3), even-x cells from `ev`
// (positions m+1..m+4)
__device__ __forceinline__ Row8 load_row8(const float *od, const float *ev)
{
    const float4 a = ld_stream4(od), b = ld_stream4(ev);
    const float e4 = __ldcs(ev + 4);
    Row8 r;
    r.v[0] = a.x; r.v[1] = b.y; r.v[2] = a.y; r.v[3] = b.z;
    r.v[4] = a.z; r.v[5] = b.w; r.v[6] = a.w; r.v[7] = e4;
    return r;
}

template <int DIM, bool CS>
__global__ void __launch_bounds__(256) kx_restrict32(const float *__restrict__ phi, const float *__restrict__ f,
                                                     BoxGeom gf, float *__restrict__ fc, float *__restrict__ phic,
                                                     BoxGeom gc, float wk, unsigned total, int q, FastDiv dq,
                                                     FastDiv dny)
{
    pdl_begin();
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const unsigned r = fdiv(dq, t);
    const unsigned kz = DIM == 3 ? fdiv(dny, r) : 0u;
    const int J = (int)(r - kz * (unsigned)gc.N[1]) + 1, K = DIM == 3 ? (int)kz + 1 : 0;
    const int u = (int)(t - r * (unsigned)q);
    const int m = 4 * u, I0 = m + 1;
    // the array holding the odd-x cells of fine row (j, k), and the other
    auto odd = [&](const float *a, int j, int k) {
        return a + ((1 + j + k) & 1) * gf.half + ((long long)k * gf.E[1] + j) * gf.H + m;
    };
    auto even = [&](const float *a, int j, int k) {
        return a + ((j + k) & 1) * gf.half + ((long long)k * gf.E[1] + j) * gf.H + m;
    };
    float sz[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int dz = 0; dz < (DIM == 3 ? 2 : 1); dz++) {
        const int k = DIM == 3 ? 2 * K - 1 + dz : 0;
        float sy[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const int j = 2 * J - 1 + dy;
            const float *po = odd(phi, j, k), *pe = even(phi, j, k);
            const float4 a = ld_stream4(po), b = ld_stream4(pe);
            const float a4 = __ldcs(po + 4), b4 = __ldcs(pe + 4);
            // x = 8u .. 8u+9
            const float xr[10] = {b.x, a.x, b.y, a.y, b.z, a.z, b.w, a.w, b4, a4};
            const Row8 yd = load_row8(odd(phi, j - 1, k), even(phi, j - 1, k));
            const Row8 yu = load_row8(odd(phi, j + 1, k), even(phi, j + 1, k));
            Row8 zd, zu;
            if (DIM == 3) {
                zd = load_row8(odd(phi, j, k - 1), even(phi, j, k - 1));
                zu = load_row8(odd(phi, j, k + 1), even(phi, j, k + 1));
            }
            const Row8 fv = load_row8(odd(f, j, k), even(f, j, k));
            float res[8];
#pragma unroll
            for (int d = 0; d < 8; d++) {
                float other = 0.f;
                other = other + (xr[d] + xr[d + 2]) * gf.ih2f[0];
                other = other + (yd.v[d] + yu.v[d]) * gf.ih2f[1];
                if (DIM == 3)
                    other = other + (zd.v[d] + zu.v[d]) * gf.ih2f[2];
                res[d] = fv.v[d] - (other + gf.d0f * xr[d + 1]);
            }
#pragma unroll
            for (int c = 0; c < 4; c++) {
                float sx = 0.f;
                sx = sx + res[2 * c];
                sx = sx + res[2 * c + 1];
                sy[c] = sy[c] + sx;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++)
            sz[c] = sz[c] + sy[c];
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        if (I0 + c > gc.N[0])
            break;
        const long long pc = lidx<CS>(gc, I0 + c, J, K);
        fc[pc] = sz[c] * wk;
        phic[pc] = 0.f;
    }
}

// A coarse value read through the ghost rule of Sec. 2.4, applied axis after
// axis (x, y, z) as a ghost fill would: index 0 -> -Phi_1; N+1 -> cR Phi_N,
// or at a tie -Phi_{N-1} (+Phi_1 when N = 1).
template <typename T, int DIM, bool S>
__device__ __forceinline__ T ghost_read(const T *__restrict__ phic, const BoxGeom &g, int i, int j, int k)
{
    int id[3] = {i, j, k};
    T c[3] = {T(1), T(1), T(1)};
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const int N = g.N[a];
        if (id[a] == 0) {
            id[a] = 1;
            c[a] = T(-1);
        } else if (id[a] == N + 1) {
            if (g.tie[a]) {
                id[a] = N >= 2 ? N - 1 : 1;
                c[a] = N >= 2 ? T(-1) : T(1);
            } else {
                id[a] = N;
                c[a] = gsel<T>(g.cR[a], g.cRf[a]);
            }
        }
    }
    T v = phic[lidx<S>(g, id[0], id[1], id[2])];
#pragma unroll
    for (int a = 0; a < DIM; a++)
        v = v * c[a];
    return v;
}

// Phi_fine += P Phi_coarse (Sec. 2.3 step 10; Appendix A): along an axis that
// coarsened, fine cell i lies a quarter coarse cell from coarse cell
// ceil(i/2) towards ceil(i/2) - 1 (i odd) or + 1 (i even): weights 3/4 and
// 1/4; along the others it takes coarse cell i.  Interpolated x first, then
// y, then z.  This is the correction at fine cell (i, j, k), coarse layout CS.
template <typename T, int DIM, bool CS>
__device__ __forceinline__ T prolong_value(const BoxGeom &gf, const T *__restrict__ phic, const BoxGeom &gc, int cmask,
                                           int i, int j, int k)
{
    (void)gf;
    // per axis: the near and far coarse cells and their weights (one tap of
    // weight 1 along an axis that did not coarsen)
    const bool cx = cmask & 1, cy = (cmask >> 1) & 1, cz = DIM == 3 && ((cmask >> 2) & 1);
    const int ax0 = cx ? (i + 1) >> 1 : i, ay0 = cy ? (j + 1) >> 1 : j, az0 = cz ? (k + 1) >> 1 : k;
    const int ax1 = (i & 1) ? ax0 - 1 : ax0 + 1, ay1 = (j & 1) ? ay0 - 1 : ay0 + 1, az1 = (k & 1) ? az0 - 1 : az0 + 1;
    const T w0 = T(0.75), w1 = T(0.25);
    auto row = [&](int y, int z) {   // interpolated along x
        if (!cx)
            return T(0) + T(1) * ghost_read<T, DIM, CS>(phic, gc, ax0, y, z);
        T v = T(0) + w0 * ghost_read<T, DIM, CS>(phic, gc, ax0, y, z);
        return v + w1 * ghost_read<T, DIM, CS>(phic, gc, ax1, y, z);
    };
    auto plane = [&](int z) {        // then along y
        if (!cy)
            return T(0) + row(ay0, z);
        T v = T(0) + w0 * row(ay0, z);
        return v + w1 * row(ay1, z);
    };
    T vz;                            // then along z
    if (!cz) {
        vz = T(0) + plane(az0);
    } else {
        vz = T(0) + w0 * plane(az0);
        vz = vz + w1 * plane(az1);
    }
    return vz;
}

// One thread per fine cell; CS / FS: the coarse / fine arrays colour-split
// (FP32) or plain.
template <typename T, int DIM, bool CS, bool FS>
__global__ void __launch_bounds__(256) kx_prolong(T *__restrict__ phif, BoxGeom gf, const T *__restrict__ phic,
                                                  BoxGeom gc, int cmask)
{
    pdl_begin();
    const int i = gx() + 1, j = gy() + 1, k = DIM == 3 ? gz() + 1 : 0;
    if (i > gf.N[0] || j > gf.N[1])
        return;
    phif[lidx<FS>(gf, i, j, k)] += prolong_value<T, DIM, CS>(gf, phic, gc, cmask, i, j, k);
}

// The same on a colour-split FP32 fine level whose x axis coarsened, eight
// fine cells of a row per thread, both colours (threads over (row, group of
// eight) linearly, as in kx_smooth32): cells x = 8u .. 8u+7 of row (j, k) --
// the odd ones at positions 4u..4u+3 of one colour array, the even ones at
// positions 4u..4u+3 of the other, one aligned float4 each -- take their x
// taps from coarse cells 4u .. 4u+4 of each of the (up to four) coarse rows
// (cell 8u+e: near 4u + (e+1)/2, far the other x neighbour), read once per
// thread.  Coarse indices go through the ghost rule as (cell, factor) pairs,
// so no thread leaves the common path; threads at a row's ends store cell by
// cell.
template <int DIM, bool CS>
__global__ void __launch_bounds__(256, 4) kx_prolong8(float *__restrict__ phif, BoxGeom gf, const float *__restrict__ phic,
                                                   BoxGeom gc, int cmask, unsigned total, int q, FastDiv dq,
                                                   FastDiv dny)
{
    pdl_begin();
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const unsigned r = fdiv(dq, t);
    const unsigned kz = DIM == 3 ? fdiv(dny, r) : 0u;
    const int j = (int)(r - kz * (unsigned)gf.N[1]) + 1, k = DIM == 3 ? (int)kz + 1 : 0;
    const int u = (int)(t - r * (unsigned)q);
    const int x0 = 8 * u;
    const long long rowf = ((long long)k * gf.E[1] + j) * gf.H + 4 * u;
    float *po = phif + ((1 + j + k) & 1) * gf.half + rowf;   // cells x0+1, x0+3, x0+5, x0+7
    float *pe = phif + ((j + k) & 1) * gf.half + rowf;       // cells x0, x0+2, x0+4, x0+6
    const bool cy = (cmask >> 1) & 1, cz = DIM == 3 && ((cmask >> 2) & 1);
    const int J0 = cy ? (j + 1) >> 1 : j, J1 = cy ? ((j & 1) ? J0 - 1 : J0 + 1) : J0;
    const int K0 = cz ? (k + 1) >> 1 : k, K1 = cz ? ((k & 1) ? K0 - 1 : K0 + 1) : K0;
    // every coarse index through the ghost rule of Sec. 2.4 as a (cell,
    // factor) pair -- factor 1 inside, so the products below are exact there
    // and equal ghost_read's at the ghosts
    auto gmap = [&](int a, int I, int &m) -> float {   // selects, no branches
        const int N = gc.N[a];
        const bool lo = I <= 0, in = I <= N, gh = I == N + 1, tie = gc.tie[a] != 0;
        const int mg = tie ? (N >= 2 ? N - 1 : 1) : N;                 // the ghost's cell
        const float fg = tie ? (N >= 2 ? -1.0f : 1.0f) : gc.cRf[a];   // and its factor
        m = lo ? 1 : (in ? I : (gh ? mg : N));
        return lo ? -1.0f : (in ? 1.0f : (gh ? fg : 0.0f));   // past the ghost: only cells outside use it
    };
    int jm[2], km[2], im[5];
    float cj[2], ck[2], ci[5];
    cj[0] = gmap(1, J0, jm[0]);
    cj[1] = gmap(1, J1, jm[1]);
    if (DIM == 3) {
        ck[0] = gmap(2, K0, km[0]);
        ck[1] = gmap(2, K1, km[1]);
    } else {
        km[0] = km[1] = 0;
        ck[0] = ck[1] = 1.0f;
    }
#pragma unroll
    for (int x = 0; x < 5; x++)
        ci[x] = gmap(0, 4 * u + x, im[x]);
    float w[4][5];
    const int nr = DIM == 3 ? 4 : 2;
#pragma unroll
    for (int rr = 0; rr < nr; rr++) {
        const int Jm = jm[rr & 1], Km = km[rr >> 1];
        const long long rb = (long long)Km * gc.E[1] + Jm;
#pragma unroll
        for (int x = 0; x < 5; x++) {
            const int I = im[x];
            float v = CS ? phic[((I + Jm + Km) & 1) * gc.half + rb * gc.H + (I >> 1)] : phic[rb * gc.E[0] + I];
            v = v * ci[x];
            v = v * cj[rr & 1];
            if (DIM == 3)
                v = v * ck[rr >> 1];
            w[rr][x] = v;
        }
    }
    const float wn = 0.75f, wf = 0.25f;
    float nv[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int near = (e + 1) >> 1, far = (e & 1) ? near - 1 : near + 1;
        float vx[4];
#pragma unroll
        for (int rr = 0; rr < nr; rr++) {
            const float a = 0.0f + wn * w[rr][near];
            vx[rr] = a + wf * w[rr][far];
        }
        float vy0, vy1 = 0.0f;
        if (cy) {
            vy0 = (0.0f + wn * vx[0]) + wf * vx[1];
            if (DIM == 3)
                vy1 = (0.0f + wn * vx[2]) + wf * vx[3];
        } else {
            vy0 = 0.0f + vx[0];
            if (DIM == 3)
                vy1 = 0.0f + vx[2];
        }
        float vz;
        if (DIM == 3 && cz)
            vz = (0.0f + wn * vy0) + wf * vy1;
        else
            vz = 0.0f + vy0;
        nv[e] = vz;
    }
    if (x0 >= 1 && x0 + 7 <= gf.N[0]) {
        float4 a = *reinterpret_cast<float4 *>(pe), b = *reinterpret_cast<float4 *>(po);
        a.x += nv[0];
        b.x += nv[1];
        a.y += nv[2];
        b.y += nv[3];
        a.z += nv[4];
        b.z += nv[5];
        a.w += nv[6];
        b.w += nv[7];
        *reinterpret_cast<float4 *>(pe) = a;
        *reinterpret_cast<float4 *>(po) = b;
        return;
    }
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int i = x0 + e;
        if (i >= 1 && i <= gf.N[0])
            ((e & 1) ? po : pe)[e >> 1] += nv[e];
    }
}

constexpr int kNormBlocks = 152 * 4;   // fixed grid of the norm reduction: the same partial sums every call
constexpr int kNormThreads = 256;

// block sum in a fixed order (warp shuffles, then the warps in order)
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double ws[kNormThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0)
        ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kNormThreads / 32; w++)
            s += ws[w];
    return s;
}

// ||f - A Phi||^2 over the active cells of multigrid level 0 in FP64 (Sec.
// 2.3 step 14), per block into part[blockIdx.x]; block b takes rows b,
// b + gridDim.x, ...  zero_inside: the potential taken as zero on the active
// cells (the ghost layer as stored), for ||b||.  Mixed precision (f32 !=
// NULL): the residual is also the next defect, written as FP32 into f32, with
// the FP32 correction e32 cleared.
template <int DIM>
__global__ void __launch_bounds__(kNormThreads) kx_resid_norm(const double *__restrict__ phi,
                                                               const double *__restrict__ f, BoxGeom g, int zero_inside,
                                                               double *__restrict__ part, float *__restrict__ f32,
                                                               float *__restrict__ e32)
{
    pdl_begin();
    const int rows = g.N[1] * (DIM == 3 ? g.N[2] : 1);
    double acc = 0.0;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = row % g.N[1] + 1;
        const int k = DIM == 3 ? row / g.N[1] + 1 : 0;
        for (int i = threadIdx.x + 1; i <= g.N[0]; i += blockDim.x) {
            const long long p = box_index(g, i, j, k);
            double res;
            if (zero_inside) {
                // only the ghost-layer neighbours (level 0: boundary data) remain
                const long long st[3] = {1, g.E[0], (long long)g.E[0] * g.E[1]};
                const int id[3] = {i, j, k};
                double other = 0.0;
                for (int a = 0; a < DIM; a++) {
                    const double left = id[a] == 1 ? phi[p - st[a]] : 0.0;
                    const double right = id[a] == g.N[a] ? phi[p + st[a]] : 0.0;
                    other = other + (left + right) * g.ih2[a];
                }
                res = f[p] - other;
            } else {
                res = box_resid<double, DIM, false>(phi, f, g, i, j, k);
            }
            if (f32) {
                const long long q = lidx<true>(g, i, j, k);
                f32[q] = (float)res;
                e32[q] = 0.0f;
            }
            acc += res * res;
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0)
        part[blockIdx.x] = s;
}

// out = sum of part[0..n-1] in a fixed order; one block
__global__ void __launch_bounds__(kNormThreads) kx_sum(const double *__restrict__ part, int n, double *out)
{
    pdl_begin();
    double v = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x)
        v += part[q];
    const double s = block_sum(v);
    if (threadIdx.x == 0)
        *out = s;
}

// Phi += e on the active cells of level 0 (mixed precision: the FP32
// correction accumulated in FP64)
template <int DIM>
__global__ void __launch_bounds__(256) kx_accumulate(double *__restrict__ phi, const float *__restrict__ e32, BoxGeom g)
{
    pdl_begin();
    const int i = gx() + 1, j = gy() + 1, k = DIM == 3 ? gz() + 1 : 0;
    if (i > g.N[0] || j > g.N[1])
        return;
    phi[box_index(g, i, j, k)] += (double)e32[lidx<true>(g, i, j, k)];
}

// Patch geometry for the kernels that work on the (n+4) blocks.
struct PatchDims {
    int n[3];     // Omega cells per axis (z: 1 in 2D)
    int B[3];     // (n+4) block extents (z: 1 in 2D)
};

// ring of a storage index of the (n+4) block: 2 for Omega, 1 for the inner
// buffer ring (Gamma minus Omega), 0 for the outer ring
__device__ __forceinline__ int block_ring(const PatchDims &d, int dim, const int s[3])
{
    int ring = 2;
    for (int a = 0; a < dim; a++) {
        const int m = min(s[a], d.n[a] + 3 - s[a]);
        ring = min(ring, m);
    }
    return ring;
}

// block coordinates of this thread (x, y, z over the (n+4) block); false
// outside it
__device__ __forceinline__ bool block_cell(const PatchDims &d, int s[3], long long &t)
{
    s[0] = gx();
    s[1] = gy();
    s[2] = gz();
    if (s[0] >= d.B[0] || s[1] >= d.B[1])
        return false;
    t = ((long long)s[2] * d.B[1] + s[1]) * d.B[0] + s[0];
    return true;
}

// mg_box_set_density: Omega density into the patch's density block; patch 0
// also the inner-ring density (from the (n+2) block bc_rho) and the outer-ring
// potential (from the (n+4) block bc_phi), the outer ring's density zero.
__global__ void __launch_bounds__(256) kx_place(PatchDims d, int dim, const double *__restrict__ rho,
                                                const double *__restrict__ bc_rho, const double *__restrict__ bc_phi,
                                                double *__restrict__ rho_blk, double *__restrict__ phi_blk)
{
    pdl_begin();
    int s[3];
    long long t;
    if (!block_cell(d, s, t))
        return;
    const int ring = block_ring(d, dim, s);
    if (ring == 2) {
        const long long q = dim == 3 ? (((long long)(s[2] - 2) * d.n[1] + (s[1] - 2)) * d.n[0] + (s[0] - 2))
                                     : ((long long)(s[1] - 2) * d.n[0] + (s[0] - 2));
        rho_blk[t] = rho[q];
    } else if (ring == 1) {
        if (bc_rho) {
            const int e0 = d.n[0] + 2, e1 = d.n[1] + 2;
            const long long q = dim == 3 ? (((long long)(s[2] - 1) * e1 + (s[1] - 1)) * e0 + (s[0] - 1))
                                         : ((long long)(s[1] - 1) * e0 + (s[0] - 1));
            rho_blk[t] = bc_rho[q];
        }
    } else if (bc_phi) {
        phi_blk[t] = bc_phi[t];
        rho_blk[t] = 0.0;
    }
}

// Buffer rings of a child patch from its parent (Sec. 2.1; Appendix A
// weights): bi/trilinear interpolation from the 2^d parent centres around
// each child centre.  The parent's centre of block index p sits at
// coordinate p, the child's block index s at off + 1.5 + (s - 1.5) / 2.
// mode 0: potential of the outer ring, density of the inner ring, and zero
// on Gamma (the start from which ||b|| is taken); mode 1: the interpolated
// potential on Gamma only (the initial guess of Sec. 2.4).
__global__ void __launch_bounds__(256) kx_interface(PatchDims dc, PatchDims dp, int dim, int o0, int o1, int o2,
                                                    const double *__restrict__ phi_p, const double *__restrict__ rho_p,
                                                    double *__restrict__ phi_c, double *__restrict__ rho_c, int mode)
{
    pdl_begin();
    int s[3];
    long long t;
    if (!block_cell(dc, s, t))
        return;
    const int ring = block_ring(dc, dim, s);
    if (mode == 1 && ring == 0)
        return;
    const int off[3] = {o0, o1, o2};
    int p0[3];
    double tw[3];
    for (int a = 0; a < 3; a++) {
        if (a < dim) {
            const double q = off[a] + 1.5 + (s[a] - 1.5) * 0.5;
            p0[a] = (int)floor(q);
            tw[a] = q - p0[a];
        } else {
            p0[a] = 0;
            tw[a] = 0.0;
        }
    }
    auto interp = [&](const double *src) {
        double v = 0.0;
        const int nz = dim == 3 ? 2 : 1;
        for (int cx = 0; cx < 2; cx++)
            for (int cy = 0; cy < 2; cy++)
                for (int cz = 0; cz < nz; cz++) {
                    double w = 1.0;
                    w = w * (cx ? tw[0] : 1.0 - tw[0]);
                    w = w * (cy ? tw[1] : 1.0 - tw[1]);
                    if (dim == 3)
                        w = w * (cz ? tw[2] : 1.0 - tw[2]);
                    const long long q = ((long long)(p0[2] + cz) * dp.B[1] + (p0[1] + cy)) * dp.B[0] + (p0[0] + cx);
                    v += w * src[q];
                }
        return v;
    };
    if (mode == 1) {
        phi_c[t] = interp(phi_p);
        return;
    }
    if (ring == 0)
        phi_c[t] = interp(phi_p);
    else
        phi_c[t] = 0.0;
    if (ring == 1)
        rho_c[t] = interp(rho_p);
}

// The right-hand side of multigrid level 0: 4 pi G rho on Gamma (Eq. 1)
__global__ void __launch_bounds__(256) kx_rhs(PatchDims d, int dim, const double *__restrict__ rho,
                                              double *__restrict__ f, double fourpiG)
{
    pdl_begin();
    int s[3];
    long long t;
    if (!block_cell(d, s, t))
        return;
    f[t] = block_ring(d, dim, s) >= 1 ? fourpiG * rho[t] : 0.0;
}

// Potential zero on Gamma (patch 0's start), the outer ring kept
__global__ void __launch_bounds__(256) kx_zero_gamma(PatchDims d, int dim, double *__restrict__ phi)
{
    pdl_begin();
    int s[3];
    long long t;
    if (!block_cell(d, s, t))
        return;
    if (block_ring(d, dim, s) >= 1)
        phi[t] = 0.0;
}

// F = -grad Phi on Omega (Eq. 2: 4/3 of the centred difference over 2h minus
// 1/3 of the one over 4h, i2h = 1/(2h), i4h = 1/(4h); stencil 1: the
// two-point centred difference), and the potential on Omega.  Component a at
// F[a * cells + cell].
__global__ void __launch_bounds__(256) kx_forces(PatchDims d, int dim, double i2h, double i4h,
                                                 const double *__restrict__ phi, double *__restrict__ F,
                                                 double *__restrict__ phi_out, int stencil)
{
    pdl_begin();
    const int x = gx(), y = gy(), z = gz();
    if (x >= d.n[0] || y >= d.n[1])
        return;
    const long long cells = (long long)d.n[0] * d.n[1] * (dim == 3 ? d.n[2] : 1);
    const long long t = ((long long)z * d.n[1] + y) * d.n[0] + x;
    const int i = x + 2, j = y + 2, k = dim == 3 ? z + 2 : 0;
    const long long st[3] = {1, d.B[0], (long long)d.B[0] * d.B[1]};
    const long long p = ((long long)k * d.B[1] + j) * d.B[0] + i;
    for (int a = 0; a < dim; a++) {
        const double d1 = phi[p + st[a]] - phi[p - st[a]];
        double gr;
        if (stencil == 0) {
            const double d2 = phi[p + 2 * st[a]] - phi[p - 2 * st[a]];
            gr = (4.0 / 3.0) * d1 * i2h - (1.0 / 3.0) * d2 * i4h;
        } else {
            gr = d1 * i2h;
        }
        if (F)
            F[a * cells + t] = -gr;
    }
    if (phi_out)
        phi_out[t] = phi[p];
}

}  // namespace

// ==========================================================================
// Host engine
// ==========================================================================
namespace {

// One multigrid level of a patch.
struct BoxLevel {
    BoxGeom g;
    size_t cells = 0;            // storage cells
    double *phi64 = nullptr;     // FP64 potential and right-hand side (level 0: the patch's blocks)
    double *f64 = nullptr;
    float *phi32 = nullptr;      // mixed precision: FP32 correction and defect
    float *f32 = nullptr;
    int cmask = 0;               // axes (bit a) that coarsen from this level to the next
    int ncoars = 0;
};

struct BoxPatch {
    int n[3] = {1, 1, 1};
    int off[3] = {0, 0, 0};      // lower corner in parent cells
    int parent = -1;
    double h = 0.0;              // cell size
    PatchDims d{};
    std::vector<BoxLevel> lv;
    double *phi = nullptr, *rho = nullptr, *f0 = nullptr;   // (n+4) blocks
    double *scal = nullptr;      // device: ||b||^2, ||r||^2
    bool density_set = false;
    std::map<int, cudaGraphExec_t> step;   // one iteration, keyed by its FP32 V-cycles (FP64: 1)
};

std::vector<int> axis_sizes(int M)
{
    // Sec. 2.2: N^L = M / 2^L rounded half up, until one cell
    std::vector<int> N{M};
    for (int L = 1; N.back() > 1; L++)
        N.push_back((M + (1 << (L - 1))) >> L);
    return N;
}

BoxGeom level_geom(const int n[3], int dim, double h, int L)
{
    BoxGeom g{};
    g.L = L;
    for (int a = 0; a < 3; a++) {
        if (a >= dim) {
            g.N[a] = 1;
            g.E[a] = 1;
            continue;
        }
        const int M = n[a] + 2;
        const std::vector<int> seq = axis_sizes(M);
        const int la = std::min(L, (int)seq.size() - 1);
        const int N = seq[la];
        g.N[a] = N;
        g.E[a] = N + 2;
        const long long twoM = 2LL * M, xN2 = (2LL * N - 1) << la, hL2 = 2LL << la;
        g.tie[a] = xN2 == twoM;
        g.cR[a] = g.tie[a] ? 0.0 : (double)(twoM - xN2 - hL2) / (double)(twoM - xN2);
        const double ha = std::ldexp(h, la);
        g.ih2[a] = 1.0 / (ha * ha);
        g.cRf[a] = (float)g.cR[a];
        g.ih2f[a] = (float)g.ih2[a];
    }
    double d = 0.0;
    for (int a = 0; a < dim; a++)
        d += -2.0 * g.ih2[a];
    g.d0 = d;
    g.inv0 = 1.0 / d;
    g.d0f = (float)g.d0;
    g.inv0f = (float)g.inv0;
    g.H = mg_split_H(g.E[0]);   // a multiple of 4: rows start 16-byte aligned
    g.half = (long long)g.H * g.E[1] * g.E[2];
    return g;
}

int level_count(const int n[3], int dim)
{
    int depth = 1;
    for (int a = 0; a < dim; a++)
        depth = std::max(depth, (int)axis_sizes(n[a] + 2).size());
    return depth;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

bool device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

thread_local std::string g_create_msg;

}  // namespace

struct mg_box {
    mg_box_desc desc{};
    mg_options opt{};
    int dim = 3;
    int device = 0;
    std::vector<BoxPatch> p;
    cudaStream_t stream = nullptr;    // the caller's stream (NULL: legacy default)
    cudaStream_t cap = nullptr;       // capture stream of the iteration graphs
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    char *arena = nullptr;
    double *part = nullptr;           // norm partial sums
    double *stage = nullptr;          // staging for host arrays
    size_t stage_doubles = 0;
    double *hscal = nullptr;          // page-locked: 2 per patch
    bool solved = false;
    bool poisoned = false;
    std::string msg;
};

namespace {

mg_status bfail(mg_box *b, mg_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    (b ? b->msg : g_create_msg) = buf;
    return s;
}

mg_status bfail_cuda(mg_box *b, cudaError_t e, const char *what)
{
    if (b)
        b->poisoned = true;
    return bfail(b, MG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BCK(b, call)                                   \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess)                         \
            return bfail_cuda((b), e_, #call);         \
    } while (0)

// A 3D launch over nx x ny x nz threads: blocks of 256 threads, 32..256 of
// them along x (the width that leaves the fewest idle threads at the row's
// end, the wider on a tie), the rest of the block over rows.
template <typename... KArgs, typename... Args>
cudaError_t launch3(void (*kernel)(KArgs...), long long nx, long long ny, long long nz, cudaStream_t s, Args... args)
{
    if (nx <= 0 || ny <= 0 || nz <= 0)
        return cudaSuccess;
    int bx = 256;
    for (int w = 128; w >= 32; w /= 2)
        if ((nx + w - 1) / w * w < (nx + bx - 1) / bx * bx)
            bx = w;
    const int by = 256 / bx;
    mg_launch_kernel(kernel, dim3((unsigned)((nx + bx - 1) / bx), (unsigned)((ny + by - 1) / by), (unsigned)nz),
                     dim3(bx, by, 1), 0, s, args...);
    return cudaGetLastError();
}

long long block_cells(const PatchDims &d) { return (long long)d.B[0] * d.B[1] * d.B[2]; }

// a launch over the active cells of a level, or over a patch's (n+4) block
template <typename... KArgs, typename... Args>
cudaError_t launch_cells(void (*kernel)(KArgs...), const BoxGeom &g, cudaStream_t s, Args... args)
{
    return launch3(kernel, g.N[0], g.N[1], g.N[2], s, args...);
}
template <typename... KArgs, typename... Args>
cudaError_t launch_block(void (*kernel)(KArgs...), const PatchDims &d, cudaStream_t s, Args... args)
{
    return launch3(kernel, d.B[0], d.B[1], d.B[2], s, args...);
}

template <typename T> T *lphi(const BoxLevel &l);
template <typename T> T *lf(const BoxLevel &l);
template <> double *lphi<double>(const BoxLevel &l) { return l.phi64; }
template <> double *lf<double>(const BoxLevel &l) { return l.f64; }
template <> float *lphi<float>(const BoxLevel &l) { return l.phi32; }
template <> float *lf<float>(const BoxLevel &l) { return l.f32; }

// one colour pass: FP64 one cell per thread, FP32 (colour-split) four
cudaError_t colour_pass(int dim, double *phi, const double *f, const BoxGeom &g, int c, cudaStream_t s)
{
    const int half = (g.N[0] + 1) >> 1;
    return dim == 3 ? launch3(kx_smooth<double, 3>, half, g.N[1], g.N[2], s, phi, f, g, c)
                    : launch3(kx_smooth<double, 2>, half, g.N[1], 1, s, phi, f, g, c);
}
cudaError_t colour_pass(int dim, float *phi, const float *f, const BoxGeom &g, int c, cudaStream_t s)
{
    const int q = ((g.N[0] >> 1) + 4) / 4;   // positions 0..N_x/2 in fours
    const unsigned total = (unsigned)q * (unsigned)g.N[1] * (unsigned)(dim == 3 ? g.N[2] : 1);
    const dim3 grid((total + 255) / 256);
    if (dim == 3)
        mg_launch_kernel(kx_smooth32<3>, grid, dim3(256), 0, s, phi, f, g, c, total, q, fast_div(q),
                         fast_div(g.N[1]));
    else
        mg_launch_kernel(kx_smooth32<2>, grid, dim3(256), 0, s, phi, f, g, c, total, q, fast_div(q),
                         fast_div(g.N[1]));
    return cudaGetLastError();
}

// kx_restrict32 applies: fine level 0 colour-split, every axis halving exactly
bool restrict32_applies(int dim, const BoxGeom &gf, const BoxGeom &gc, int cmask)
{
    if (gf.L != 0 || cmask != (1 << dim) - 1)
        return false;
    for (int a = 0; a < dim; a++)
        if (gf.N[a] != 2 * gc.N[a])
            return false;
    return true;
}

template <bool CS>
cudaError_t restrict32(int dim, const float *phi, const float *f, const BoxGeom &gf, float *fc, float *phic,
                       const BoxGeom &gc, float wk, cudaStream_t s)
{
    const int q = (gc.N[0] + 3) / 4;
    const unsigned total = (unsigned)q * (unsigned)gc.N[1] * (unsigned)(dim == 3 ? gc.N[2] : 1);
    const dim3 grid((total + 255) / 256);
    if (dim == 3)
        mg_launch_kernel(kx_restrict32<3, CS>, grid, dim3(256), 0, s, phi, f, gf, fc, phic, gc, wk, total, q,
                         fast_div(q), fast_div(gc.N[1]));
    else
        mg_launch_kernel(kx_restrict32<2, CS>, grid, dim3(256), 0, s, phi, f, gf, fc, phic, gc, wk, total, q,
                         fast_div(q), fast_div(gc.N[1]));
    return cudaGetLastError();
}

// Prolongation into a colour-split FP32 fine level: four fine cells per
// thread where the x axis coarsened, else one
template <bool CS>
cudaError_t prolong32(int dim, float *phif, const BoxGeom &gf, const float *phic, const BoxGeom &gc, int cmask,
                      cudaStream_t s)
{
    if (!(cmask & 1))
        return dim == 3 ? launch_cells(kx_prolong<float, 3, CS, true>, gf, s, phif, gf, phic, gc, cmask)
                        : launch_cells(kx_prolong<float, 2, CS, true>, gf, s, phif, gf, phic, gc, cmask);
    const int q = gf.N[0] / 8 + 1;   // groups x = 8u .. 8u+7 with 8u <= N_x
    const unsigned total = (unsigned)q * (unsigned)gf.N[1] * (unsigned)(dim == 3 ? gf.N[2] : 1);
    const dim3 grid((total + 255) / 256);
    if (dim == 3)
        mg_launch_kernel(kx_prolong8<3, CS>, grid, dim3(256), 0, s, phif, gf, phic, gc, cmask, total, q, fast_div(q),
                         fast_div(gf.N[1]));
    else
        mg_launch_kernel(kx_prolong8<2, CS>, grid, dim3(256), 0, s, phif, gf, phic, gc, cmask, total, q, fast_div(q),
                         fast_div(gf.N[1]));
    return cudaGetLastError();
}

template <typename T>
cudaError_t smooth(const mg_box *b, const BoxLevel &l, int sweeps, cudaStream_t s)
{
    for (int sw = 0; sw < sweeps; sw++)
        for (int c = 0; c < 2; c++) {
            cudaError_t e = colour_pass(b->dim, lphi<T>(l), (const T *)lf<T>(l), l.g, c, s);
            if (e)
                return e;
        }
    return cudaSuccess;
}

// One V-cycle (Sec. 2.3 steps 2-13) over every multigrid level of patch P in
// precision T: pre-smoothing and restriction down to the level where every
// axis has one cell (smoothed nu_pre times there), then prolongation,
// correction and post-smoothing back up.
template <typename T>
cudaError_t vcycle(const mg_box *b, const BoxPatch &P, cudaStream_t s)
{
    const int dim = b->dim;
    const int Lc = (int)P.lv.size() - 1;
    cudaError_t e = smooth<T>(b, P.lv[0], b->opt.nu_pre, s);
    for (int L = 0; L < Lc && !e; L++) {
        const BoxLevel &fl = P.lv[L], &cl = P.lv[L + 1];
        const T wk = (T)std::ldexp(1.0, -fl.ncoars);
        constexpr bool S = sizeof(T) == 4;   // FP32 levels colour-split, FP64 plain
        if constexpr (S)
            if (restrict32_applies(dim, fl.g, cl.g, fl.cmask)) {
                e = restrict32<true>(dim, (const float *)lphi<T>(fl), (const float *)lf<T>(fl), fl.g,
                                     (float *)lf<T>(cl), (float *)lphi<T>(cl), cl.g, (float)wk, s);
                if (!e)
                    e = smooth<T>(b, cl, b->opt.nu_pre, s);
                continue;
            }
        e = dim == 3 ? launch_cells(kx_resid_restrict<T, 3, S, S>, cl.g, s, (const T *)lphi<T>(fl),
                                    (const T *)lf<T>(fl), fl.g, lf<T>(cl), lphi<T>(cl), cl.g, fl.cmask, wk)
                     : launch_cells(kx_resid_restrict<T, 2, S, S>, cl.g, s, (const T *)lphi<T>(fl),
                                    (const T *)lf<T>(fl), fl.g, lf<T>(cl), lphi<T>(cl), cl.g, fl.cmask, wk);
        if (!e)
            e = smooth<T>(b, cl, b->opt.nu_pre, s);
    }
    for (int L = Lc; L > 0 && !e; L--) {
        const BoxLevel &cl = P.lv[L], &fl = P.lv[L - 1];
        if constexpr (sizeof(T) == 4)   // FP32 levels colour-split
            e = prolong32<true>(dim, fl.phi32, fl.g, cl.phi32, cl.g, fl.cmask, s);
        else
            e = dim == 3 ? launch_cells(kx_prolong<double, 3, false, false>, fl.g, s, fl.phi64, fl.g,
                                        (const double *)cl.phi64, cl.g, fl.cmask)
                         : launch_cells(kx_prolong<double, 2, false, false>, fl.g, s, fl.phi64, fl.g,
                                        (const double *)cl.phi64, cl.g, fl.cmask);
        if (!e)
            e = smooth<T>(b, fl, b->opt.nu_post, s);
    }
    return e;
}

// ||f - A Phi||^2 of level 0 into *out (zero_inside: Phi zero on Gamma);
// mixed precision with write32: the residual also becomes the FP32 defect
cudaError_t resid_norm(const mg_box *b, const BoxPatch &P, int zero_inside, bool write32, double *out, cudaStream_t s)
{
    const BoxLevel &l = P.lv[0];
    float *f32 = write32 ? l.f32 : nullptr, *e32 = write32 ? l.phi32 : nullptr;
    const int blocks = std::min(kNormBlocks, l.g.N[1] * l.g.N[2]);
    if (b->dim == 3)
        mg_launch_kernel(kx_resid_norm<3>, dim3(blocks), dim3(kNormThreads), 0, s, (const double *)l.phi64,
                         (const double *)l.f64, l.g, zero_inside, b->part, f32, e32);
    else
        mg_launch_kernel(kx_resid_norm<2>, dim3(blocks), dim3(kNormThreads), 0, s, (const double *)l.phi64,
                         (const double *)l.f64, l.g, zero_inside, b->part, f32, e32);
    cudaError_t e = cudaGetLastError();
    if (e)
        return e;
    mg_launch_kernel(kx_sum, dim3(1), dim3(kNormThreads), 0, s, (const double *)b->part, blocks, out);
    return cudaGetLastError();
}

bool mixed(const mg_box *b) { return b->opt.precision == MG_MIXED; }

// One iteration of patch pi's loop (Sec. 2.3 step 14): an FP64 V-cycle, or
// ncyc FP32 V-cycles on the correction of the stored defect and their FP64
// accumulation; then ||r||^2 (in mixed precision also the next defect), copied
// to the page-locked host slot.
cudaError_t iteration(mg_box *b, int pi, int ncyc, cudaStream_t s)
{
    BoxPatch &P = b->p[pi];
    cudaError_t e;
    if (!mixed(b)) {
        e = vcycle<double>(b, P, s);
    } else {
        e = cudaSuccess;
        for (int c = 0; c < ncyc && !e; c++)
            e = vcycle<float>(b, P, s);
        if (!e)
            e = launch_cells(b->dim == 3 ? kx_accumulate<3> : kx_accumulate<2>, P.lv[0].g, s, P.lv[0].phi64,
                             (const float *)P.lv[0].phi32, P.lv[0].g);
    }
    if (!e)
        e = resid_norm(b, P, 0, mixed(b), P.scal + 1, s);
    if (!e)
        e = cudaMemcpyAsync(b->hscal + 2 * pi + 1, P.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
    return e;
}

// The iteration as a CUDA graph (captured once per FP32 V-cycle count)
cudaError_t iteration_graph(mg_box *b, int pi, int ncyc, cudaGraphExec_t *out)
{
    BoxPatch &P = b->p[pi];
    auto it = P.step.find(ncyc);
    if (it != P.step.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e)
        return e;
    const cudaError_t eb = iteration(b, pi, ncyc, b->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (eb || e) {
        if (g)
            cudaGraphDestroy(g);
        return eb ? eb : e;
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e)
        return e;
    P.step[ncyc] = x;
    *out = x;
    return cudaSuccess;
}

// The start of patch pi's solve: its buffer rings (from the parent, or the
// caller's boundary data), the right-hand side, ||b|| from a zero Gamma, the
// initial guess and the starting residual
cudaError_t prelude(mg_box *b, int pi, cudaStream_t s)
{
    BoxPatch &P = b->p[pi];
    const int dim = b->dim;
    cudaError_t e;
    if (pi == 0) {
        e = launch_block(kx_zero_gamma, P.d, s, P.d, dim, P.phi);
    } else {
        const BoxPatch &Q = b->p[P.parent];
        e = launch_block(kx_interface, P.d, s, P.d, Q.d, dim, P.off[0], P.off[1], P.off[2], (const double *)Q.phi,
                         (const double *)Q.rho, P.phi, P.rho, 0);
    }
    if (!e)
        e = launch_block(kx_rhs, P.d, s, P.d, dim, (const double *)P.rho, P.f0, 4.0 * M_PI * b->desc.G);
    if (!e)
        e = resid_norm(b, P, 1, false, P.scal, s);
    if (!e && pi > 0 && b->opt.guess == MG_GUESS_INTERP) {
        const BoxPatch &Q = b->p[P.parent];
        e = launch_block(kx_interface, P.d, s, P.d, Q.d, dim, P.off[0], P.off[1], P.off[2], (const double *)Q.phi,
                         (const double *)Q.rho, P.phi, P.rho, 1);
    }
    if (!e)
        e = resid_norm(b, P, 0, mixed(b), P.scal + 1, s);
    if (!e)
        e = cudaMemcpyAsync(b->hscal + 2 * pi, P.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    return e;
}

mg_status check_box_options(const mg_options &o)
{
    if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre + o.nu_post < 1 || o.max_cycles < 0 || !(o.rel_tol >= 0.0) ||
        (o.precision != MG_FP64 && o.precision != MG_MIXED) || o.inner_cycles < 1 || o.inner_max < 0 ||
        o.inner_max > MG_INNER_MAX || (o.guess != MG_GUESS_INTERP && o.guess != MG_GUESS_ZERO) ||
        (o.force_stencil != MG_FORCE_EQ2 && o.force_stencil != MG_FORCE_CD2) || o.interface != MG_IFACE_BUFFER ||
        o.stop != MG_STOP_RESIDUAL)
        return MG_EINVAL;
    return MG_OK;
}

int box_parent(const mg_box_desc &d, int l) { return d.tree ? d.parent[l] : l - 1; }

mg_status check_box_desc(const mg_box_desc &d)
{
    if (d.dim != 2 && d.dim != 3)
        return bfail(nullptr, MG_EINVAL, "dim must be 2 or 3");
    if (d.num_patches < 1 || d.num_patches > MG_MAX_LEVELS)
        return bfail(nullptr, MG_EINVAL, "num_patches %d out of range", d.num_patches);
    if (!(d.h0 > 0.0) || !std::isfinite(d.h0) || !std::isfinite(d.G))
        return bfail(nullptr, MG_EINVAL, "h0 must be positive and G finite");
    if (d.tree != 0 && d.tree != 1)
        return bfail(nullptr, MG_EINVAL, "tree must be 0 or 1");
    for (int l = 1; l < d.num_patches; l++)
        if (d.tree && (d.parent[l] < 0 || d.parent[l] >= l))
            return bfail(nullptr, MG_EINVAL, "patch %d: parent %d not in [0, %d)", l, d.parent[l], l);
    for (int l = 0; l < d.num_patches; l++) {
        double cells = 1.0;
        for (int a = 0; a < d.dim; a++) {
            const int n = d.n[l][a];
            if (n < 2 || n > 65000 || (l > 0 && (n & 1)))   // launch grids: y and z extents below 2^16
                return bfail(nullptr, MG_EINVAL, "patch %d axis %d: n=%d (need 2..65000, even above patch 0)", l, a,
                             n);
            cells *= (double)(n + 4);
        }
        if (cells > 2147483647.0)
            return bfail(nullptr, MG_EINVAL, "patch %d: (n+4) block of %.0f cells exceeds 2^31", l, cells);
        if (l == 0)
            continue;
        const int pl = box_parent(d, l);
        int depth = 0;
        for (int q = pl; q > 0; q = box_parent(d, q))
            depth++;
        const double hp = std::ldexp(d.h0, -depth);
        for (int a = 0; a < d.dim; a++) {
            const double o = (d.lo[l][a] - d.lo[pl][a]) / hp;
            const double r = std::floor(o + 0.5);
            if (std::fabs(o - r) > 1e-6)
                return bfail(nullptr, MG_EINVAL, "patch %d axis %d: not on parent cell faces", l, a);
            const int hi = d.n[pl][a] - d.n[l][a] / 2 - 1;
            if (r < 1.0 || r > (double)hi)
                return bfail(nullptr, MG_EINVAL, "patch %d axis %d: offset %g outside [1, %d] parent cells", l, a, r, hi);
        }
    }
    return MG_OK;
}

void destroy_box(mg_box *b)
{
    if (!b)
        return;
    for (auto &P : b->p)
        for (auto &kv : P.step)
            cudaGraphExecDestroy(kv.second);
    if (b->arena)
        cudaFree(b->arena);
    if (b->hscal)
        cudaFreeHost(b->hscal);
    if (b->ev0)
        cudaEventDestroy(b->ev0);
    if (b->ev1)
        cudaEventDestroy(b->ev1);
    if (b->cap)
        cudaStreamDestroy(b->cap);
    delete b;
}

}  // namespace

// --------------------------------------------------------------------------
// The cubic engine's colour-split FP32 levels (declared in mg_internal.h)
// --------------------------------------------------------------------------
namespace {

BoxGeom box_from_mg(const MgGeom &g, int dim)
{
    BoxGeom b{};
    b.L = g.L;
    for (int a = 0; a < 3; a++) {
        if (a >= dim) {
            b.N[a] = 1;
            b.E[a] = 1;
            continue;
        }
        b.N[a] = g.N;
        b.E[a] = g.E;
        b.tie[a] = g.tie;
        b.cR[a] = g.cR;
        b.ih2[a] = g.inv_h2;
        b.cRf[a] = g.cRf;
        b.ih2f[a] = g.inv_h2f;
    }
    b.d0 = -2.0 * dim * g.inv_h2;
    b.inv0 = 1.0 / b.d0;
    b.d0f = (float)b.d0;
    b.inv0f = (float)b.inv0;
    b.H = g.sH > 0 ? g.sH : mg_split_H(g.E);
    b.half = (long long)b.H * g.E * (dim == 3 ? g.E : 1);
    return b;
}

template <bool FS, bool CS>
cudaError_t split_restrict(int dim, const float *phi, const float *f, const BoxGeom &bf, float *phic, float *fc,
                           const BoxGeom &bc, cudaStream_t s)
{
    const int cmask = (1 << dim) - 1;
    const float wk = dim == 3 ? 0.125f : 0.25f;
    if (FS && restrict32_applies(dim, bf, bc, cmask))
        return restrict32<CS>(dim, phi, f, bf, fc, phic, bc, wk, s);
    return dim == 3 ? launch_cells(kx_resid_restrict<float, 3, FS, CS>, bc, s, phi, f, bf, fc, phic, bc, cmask, wk)
                    : launch_cells(kx_resid_restrict<float, 2, FS, CS>, bc, s, phi, f, bf, fc, phic, bc, cmask, wk);
}

template <bool CS, bool FS>
cudaError_t split_prolong(int dim, const float *phic, const BoxGeom &bc, float *phif, const BoxGeom &bf, cudaStream_t s)
{
    const int cmask = (1 << dim) - 1;
    return dim == 3 ? launch_cells(kx_prolong<float, 3, CS, FS>, bf, s, phif, bf, phic, bc, cmask)
                    : launch_cells(kx_prolong<float, 2, CS, FS>, bf, s, phif, bf, phic, bc, cmask);
}

}  // namespace

cudaError_t mg_split_colour(int dim, float *phi, const float *f, const MgGeom &g, int colour, cudaStream_t s)
{
    if (g.sH <= 0)
        return cudaErrorInvalidValue;
    return colour_pass(dim, phi, f, box_from_mg(g, dim), colour, s);
}

cudaError_t mg_split_resid_restrict(int dim, const float *phi, const float *f, const MgGeom &gf, float *phic,
                                    float *fc, const MgGeom &gc, cudaStream_t s)
{
    const BoxGeom bf = box_from_mg(gf, dim), bc = box_from_mg(gc, dim);
    const bool fs = gf.sH > 0, cs = gc.sH > 0;
    if (fs && cs)
        return split_restrict<true, true>(dim, phi, f, bf, phic, fc, bc, s);
    if (fs)
        return split_restrict<true, false>(dim, phi, f, bf, phic, fc, bc, s);
    if (cs)
        return split_restrict<false, true>(dim, phi, f, bf, phic, fc, bc, s);
    return split_restrict<false, false>(dim, phi, f, bf, phic, fc, bc, s);
}

cudaError_t mg_split_prolong(int dim, const float *phic, const MgGeom &gc, float *phif, const MgGeom &gf,
                             cudaStream_t s)
{
    const BoxGeom bf = box_from_mg(gf, dim), bc = box_from_mg(gc, dim);
    const bool fs = gf.sH > 0, cs = gc.sH > 0;
    const int cmask = (1 << dim) - 1;
    if (fs && cs)
        return prolong32<true>(dim, phif, bf, phic, bc, cmask, s);
    if (fs)
        return prolong32<false>(dim, phif, bf, phic, bc, cmask, s);
    if (cs)
        return split_prolong<true, false>(dim, phic, bc, phif, bf, s);
    return split_prolong<false, false>(dim, phic, bc, phif, bf, s);
}

extern "C" {

mg_status mg_box_create(const mg_box_desc *desc, const mg_options *opt, mg_box **out)
{
    if (!out)
        return bfail(nullptr, MG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!desc)
        return bfail(nullptr, MG_EINVAL, "desc is NULL");
    mg_options o;
    mg_default_options(&o);
    if (opt)
        o = *opt;
    if (check_box_options(o) != MG_OK)
        return bfail(nullptr, MG_EINVAL,
                     "options: box patches take FP64 or MIXED, guess INTERP or ZERO, interface BUFFER, stop RESIDUAL");
    mg_status st = check_box_desc(*desc);
    if (st != MG_OK)
        return st;
    mg_box *b = new mg_box;
    b->desc = *desc;
    b->opt = o;
    b->dim = desc->dim;
    b->stream = (cudaStream_t)o.stream;
    cudaError_t e = cudaGetDevice(&b->device);
    const int dim = b->dim;
    b->p.resize(desc->num_patches);
    // layout of the arena
    size_t bytes = up256(kNormBlocks * sizeof(double));
    size_t stage = 0;
    std::vector<std::vector<size_t>> offs(desc->num_patches);
    for (int l = 0; l < desc->num_patches; l++) {
        BoxPatch &P = b->p[l];
        for (int a = 0; a < 3; a++)
            P.n[a] = a < dim ? desc->n[l][a] : 1;
        P.parent = l > 0 ? box_parent(*desc, l) : -1;
        int depth = 0;
        for (int q = l; q > 0; q = box_parent(*desc, q))
            depth++;
        P.h = std::ldexp(desc->h0, -depth);
        for (int a = 0; a < 3; a++) {
            P.d.n[a] = P.n[a];
            P.d.B[a] = a < dim ? P.n[a] + 4 : 1;
            if (l > 0 && a < dim) {
                const double hp = 2.0 * P.h;
                P.off[a] = (int)std::floor((desc->lo[l][a] - desc->lo[P.parent][a]) / hp + 0.5);
            }
        }
        const int depthL = level_count(P.n, dim);
        P.lv.resize(depthL);
        for (int L = 0; L < depthL; L++) {
            BoxLevel &v = P.lv[L];
            v.g = level_geom(P.n, dim, P.h, L);
            v.cells = (size_t)v.g.E[0] * v.g.E[1] * v.g.E[2];
        }
        for (int L = 0; L + 1 < depthL; L++) {
            const BoxGeom &f = P.lv[L].g, &c = P.lv[L + 1].g;
            int m = 0, k = 0;
            for (int a = 0; a < dim; a++) {
                // an axis coarsens when its own level index grows: its cell count changes, or
                // it stays at one cell (then la is capped and nothing changes)
                const std::vector<int> seq = axis_sizes(P.n[a] + 2);
                const int laf = std::min(L, (int)seq.size() - 1), lac = std::min(L + 1, (int)seq.size() - 1);
                if (lac > laf) {
                    m |= 1 << a;
                    k++;
                }
            }
            (void)f;
            (void)c;
            P.lv[L].cmask = m;
            P.lv[L].ncoars = k;
        }
        const size_t nb = (size_t)block_cells(P.d);
        std::vector<size_t> &of = offs[l];
        of.push_back(bytes);   // phi
        bytes += up256(nb * 8);
        of.push_back(bytes);   // rho
        bytes += up256(nb * 8);
        of.push_back(bytes);   // f0
        bytes += up256(nb * 8);
        of.push_back(bytes);   // scal
        bytes += 256;
        for (int L = 0; L < depthL; L++) {
            const size_t c = P.lv[L].cells;
            if (!mixed(b)) {
                if (L > 0) {
                    of.push_back(bytes);
                    bytes += up256(c * 8);
                    of.push_back(bytes);
                    bytes += up256(c * 8);
                }
            } else {   // colour-split: two arrays of `half` cells, and the word past the last row
                const size_t cs = 2 * (size_t)P.lv[L].g.half + 16;
                of.push_back(bytes);
                bytes += up256(cs * 4);
                of.push_back(bytes);
                bytes += up256(cs * 4);
            }
        }
        long long om = 1;
        for (int a = 0; a < dim; a++)
            om *= P.n[a];
        stage = std::max(stage, std::max((size_t)nb * 3, (size_t)om * (dim + 1)));
    }
    const size_t stage_off = bytes;
    bytes += up256(stage * 8);
    if (!e)
        e = cudaMalloc(&b->arena, bytes);
    if (e) {
        cudaGetLastError();
        destroy_box(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA, "device memory (%zu bytes): %s",
                     bytes, cudaGetErrorString(e));
    }
    b->part = (double *)b->arena;
    b->stage = (double *)(b->arena + stage_off);
    b->stage_doubles = stage;
    for (int l = 0; l < desc->num_patches; l++) {
        BoxPatch &P = b->p[l];
        const std::vector<size_t> &of = offs[l];
        size_t q = 0;
        P.phi = (double *)(b->arena + of[q++]);
        P.rho = (double *)(b->arena + of[q++]);
        P.f0 = (double *)(b->arena + of[q++]);
        P.scal = (double *)(b->arena + of[q++]);
        for (int L = 0; L < (int)P.lv.size(); L++) {
            BoxLevel &v = P.lv[L];
            if (L == 0) {
                v.phi64 = P.phi;
                v.f64 = P.f0;
            }
            if (!mixed(b)) {
                if (L > 0) {
                    v.phi64 = (double *)(b->arena + of[q++]);
                    v.f64 = (double *)(b->arena + of[q++]);
                }
            } else {
                v.phi32 = (float *)(b->arena + of[q++]);
                v.f32 = (float *)(b->arena + of[q++]);
            }
        }
    }
    if (!e)
        e = cudaMemsetAsync(b->arena, 0, bytes, b->stream);
    if (!e)
        e = cudaMallocHost(&b->hscal, 2 * sizeof(double) * desc->num_patches);
    if (!e)
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (!e)
        e = cudaEventCreate(&b->ev0);
    if (!e)
        e = cudaEventCreate(&b->ev1);
    if (!e)
        e = cudaStreamSynchronize(b->stream);
    if (e) {
        cudaGetLastError();
        destroy_box(b);
        return bfail(nullptr, MG_ECUDA, "setup: %s", cudaGetErrorString(e));
    }
    *out = b;
    return MG_OK;
}

mg_status mg_box_set_density(mg_box *b, int patch, const double *rho, const double *bc_rho, const double *bc_phi)
{
    if (!b)
        return MG_EINVAL;
    if (b->poisoned)
        return bfail(b, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (patch < 0 || patch >= (int)b->p.size())
        return bfail(b, MG_EINVAL, "patch %d out of range", patch);
    if (!rho)
        return bfail(b, MG_EINVAL, "rho is NULL");
    if (patch == 0 && (!bc_rho || !bc_phi))
        return bfail(b, MG_EINVAL, "patch 0 needs bc_rho and bc_phi");
    if (patch > 0 && (bc_rho || bc_phi))
        return bfail(b, MG_EINVAL, "bc_rho/bc_phi must be NULL above patch 0 (the interface fills them)");
    BoxPatch &P = b->p[patch];
    const int dim = b->dim;
    const size_t nb = (size_t)block_cells(P.d);
    size_t nr = 1, ng = 1;
    for (int a = 0; a < dim; a++) {
        nr *= (size_t)P.n[a];
        ng *= (size_t)P.n[a] + 2;
    }
    const double *d_rho = rho, *d_bcr = bc_rho, *d_bcp = bc_phi;
    bool host_in = false;
    auto take = [&](const double *src, const double *&dst, double *st, size_t count) -> cudaError_t {
        if (device_ptr(src))
            return cudaSuccess;
        host_in = true;
        dst = st;
        return cudaMemcpyAsync(st, src, count * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    };
    BCK(b, take(rho, d_rho, b->stage, nr));
    if (patch == 0) {
        BCK(b, take(bc_rho, d_bcr, b->stage + nb, ng));
        BCK(b, take(bc_phi, d_bcp, b->stage + 2 * nb, nb));
    }
    BCK(b, launch_block(kx_place, P.d, b->stream, P.d, dim, d_rho, d_bcr, d_bcp, P.rho, P.phi));
    if (host_in)
        BCK(b, cudaStreamSynchronize(b->stream));
    P.density_set = true;
    b->solved = false;
    return MG_OK;
}

mg_status mg_box_solve(mg_box *b, mg_level_stats *stats)
{
    if (!b)
        return MG_EINVAL;
    if (b->poisoned)
        return bfail(b, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    for (size_t l = 0; l < b->p.size(); l++)
        if (!b->p[l].density_set)
            return bfail(b, MG_ESTATE, "patch %zu has no density", l);
    const mg_options &o = b->opt;
    const bool adapt = mixed(b) && o.inner_max > 0;
    mg_status worst = MG_OK;
    for (int pi = 0; pi < (int)b->p.size(); pi++) {
        BCK(b, prelude(b, pi, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        const double *hs = b->hscal + 2 * pi;
        const double bn = std::sqrt(hs[0]);
        double rel = bn > 0.0 ? std::sqrt(hs[1]) / bn : 0.0;
        int status = std::isfinite(bn) && std::isfinite(rel) ? 0 : 1;
        int cycles = 0, outer = 0, inner = o.inner_cycles;
        while (bn > 0.0 && !status && cycles < o.max_cycles && !(rel < o.rel_tol)) {
            const int ncyc = !mixed(b) ? 1 : adapt ? std::min(inner, o.max_cycles - cycles) : o.inner_cycles;
            cudaGraphExec_t x;
            BCK(b, iteration_graph(b, pi, ncyc, &x));
            BCK(b, cudaGraphLaunch(x, b->stream));
            BCK(b, cudaStreamSynchronize(b->stream));
            const double before = rel;
            cycles += ncyc;
            outer++;
            rel = std::sqrt(hs[1]) / bn;
            if (!std::isfinite(rel))
                status = 1;
            if (adapt)
                inner = mg_next_inner(before, rel, ncyc, o.rel_tol, o.inner_max);
        }
        int s = status ? MG_EDIVERGED : MG_OK;
        if (s == MG_OK && bn > 0.0 && o.rel_tol > 0.0 && !(rel < o.rel_tol))
            s = MG_ENOCONV;
        if (stats) {
            stats[pi].cycles = cycles;
            stats[pi].outer_steps = outer;
            stats[pi].rel_res = rel;
            stats[pi].b_norm = bn;
            stats[pi].status = s;
        }
        if (s == MG_EDIVERGED)
            worst = MG_EDIVERGED;
        else if (s == MG_ENOCONV && worst == MG_OK)
            worst = MG_ENOCONV;
    }
    b->solved = true;
    return worst;
}

mg_status mg_box_forces(mg_box *b, int patch, double *phi_out, double *F_out)
{
    if (!b)
        return MG_EINVAL;
    if (b->poisoned)
        return bfail(b, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (patch < 0 || patch >= (int)b->p.size())
        return bfail(b, MG_EINVAL, "patch %d out of range", patch);
    if (!b->solved)
        return bfail(b, MG_ESTATE, "mg_box_forces before mg_box_solve");
    const BoxPatch &P = b->p[patch];
    const int dim = b->dim;
    size_t nr = 1;
    for (int a = 0; a < dim; a++)
        nr *= (size_t)P.n[a];
    const bool F_dev = F_out && device_ptr(F_out), P_dev = phi_out && device_ptr(phi_out);
    double *dF = F_out ? (F_dev ? F_out : b->stage) : nullptr;
    double *dP = phi_out ? (P_dev ? phi_out : b->stage + (size_t)dim * nr) : nullptr;
    BCK(b, launch3(kx_forces, P.n[0], P.n[1], P.n[2], b->stream, P.d, dim, 1.0 / (2.0 * P.h), 1.0 / (4.0 * P.h),
                   (const double *)P.phi, dF, dP, b->opt.force_stencil));
    bool sync = false;
    if (F_out && !F_dev) {
        BCK(b, cudaMemcpyAsync(F_out, dF, (size_t)dim * nr * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        sync = true;
    }
    if (phi_out && !P_dev) {
        BCK(b, cudaMemcpyAsync(phi_out, dP, nr * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        sync = true;
    }
    if (sync)
        BCK(b, cudaStreamSynchronize(b->stream));
    return MG_OK;
}

int mg_box_level_sizes(const mg_box *b, int patch, int *N, int cap)
{
    if (!b || patch < 0 || patch >= (int)b->p.size() || cap < 0 || (cap > 0 && !N))
        return -1;
    const BoxPatch &P = b->p[patch];
    const int k = (int)P.lv.size();
    for (int L = 0; L < std::min(k, cap); L++)
        for (int a = 0; a < 3; a++)
            N[3 * L + a] = P.lv[L].g.N[a];
    return k;
}

mg_status mg_box_time_smoothing(mg_box *b, int patch, int L, int launches, double *us_per_launch,
                                double *bytes_per_launch)
{
    if (!b)
        return MG_EINVAL;
    if (b->poisoned)
        return bfail(b, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (patch < 0 || patch >= (int)b->p.size() || launches < 1)
        return bfail(b, MG_EINVAL, "patch %d / launches %d out of range", patch, launches);
    const BoxPatch &P = b->p[patch];
    if (L < 0 || L >= (int)P.lv.size())
        return bfail(b, MG_EINVAL, "multigrid level %d out of range", L);
    const BoxLevel &v = P.lv[L];
    auto pass = [&](int c) -> cudaError_t {
        if (mixed(b))
            return colour_pass(b->dim, v.phi32, (const float *)v.f32, v.g, c, b->stream);
        return colour_pass(b->dim, v.phi64, (const double *)v.f64, v.g, c, b->stream);
    };
    for (int w = 0; w < 3; w++)
        BCK(b, pass(w & 1));
    BCK(b, cudaEventRecord(b->ev0, b->stream));
    for (int r = 0; r < launches; r++)
        BCK(b, pass(r & 1));
    BCK(b, cudaEventRecord(b->ev1, b->stream));
    BCK(b, cudaEventSynchronize(b->ev1));
    float ms = 0.0f;
    BCK(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    const double cells = (double)v.g.N[0] * v.g.N[1] * v.g.N[2];
    if (us_per_launch)
        *us_per_launch = 1e3 * ms / launches;
    if (bytes_per_launch)
        *bytes_per_launch = 1.5 * cells * (mixed(b) ? 4.0 : 8.0);
    b->solved = false;
    return MG_OK;
}

const char *mg_box_error_message(const mg_box *b) { return b ? b->msg.c_str() : g_create_msg.c_str(); }

mg_status mg_box_destroy(mg_box *b)
{
    if (b)
        cudaSetDevice(b->device);
    destroy_box(b);
    return MG_OK;
}

}  // extern "C"
