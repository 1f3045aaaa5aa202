// mg_api.cu -- C ABI (include/mg.h) and host driver of the nested-grid
// multigrid Poisson solver.  Each refinement level is solved by V-cycles
// (Sec. 2.3) after the one-way interface has filled its buffer rings from the
// parent (Sec. 2.1); all arithmetic runs in the kernels of mg_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "../../include/unet.h"
#include "mg_internal.h"

namespace {

struct LevelData {
    int n = 0, M = 0, nmg = 0;
    int parent = -1;               // parent patch (-1 for the base)
    int off[3] = {0, 0, 0};
    double h = 0.0;
    MgGeom g[MG_MAX_MG];
    double *phi[MG_MAX_MG] = {};   // multigrid level arrays, (N^L+2)^d
    double *f[MG_MAX_MG] = {};
    double *blk = nullptr;         // the (n+4)^d level block of potential ...
    double *fblk = nullptr;        // ... and of 4 pi G rho; phi[0] / f[0] themselves
                                   // except on frozen-interface levels
    bool frozen = false;           // MG_IFACE_FROZEN level: multigrid on Omega only
    double *prev = nullptr;        // MG_STOP_FORCE: the (n+4)^d block before the iteration
    float *phi32[MG_MAX_MG] = {};  // mixed precision correction, all multigrid levels
    float *phi32b[MG_MAX_MG] = {}; // second FP32 buffer of the temporally blocked levels
    int tile[MG_MAX_MG] = {};      // FP32 temporal-blocking tile per level (0: one kernel per phase)
    int nsplit = 0;                // FP32 levels 0..nsplit-1 stored colour-split (MgGeom::sH > 0), tile 0
    float *f32[MG_MAX_MG] = {};
    double *rho = nullptr;         // (n+4)^d density (Omega and inner ring)
    double *guess = nullptr;       // (n+2)^d optional initial potential
    bool density_set = false, guess_set = false;
    double *tab64[MG_MAX_MG] = {}; // boundary diagonal tables of the coarse levels (device)
    float *tab32[MG_MAX_MG] = {};
    int Ls[2] = {0, 0};            // first level handled by the one-block kernel [fp64, fp32]
    int Lc[2] = {-1, -1};          // first level handled by the cluster kernel (-1: none)
    int Llim[2] = {0, 0};          // the level-size limit that chose it
    MgBottom bt[2];
    // device image of the one-block kernel's plan for the precision the
    // V-cycles run in, sized for the largest bottom the level admits
    void *bplan = nullptr;
    size_t bplan_bytes = 0;
    // outputs mg_solve writes once the level has converged (mg_set_outputs):
    // device pointers or device views of page-locked host arrays
    double *out_F = nullptr, *out_phi = nullptr;
};

// Largest multigrid level (cells per edge) given to the one-block bottom
// kernel.  Measured on the 4x64^3 workload: 8 beats 17 in both precisions
// (one SM runs FP64 at two FMA per clock; even in FP32 a 17^3 level is
// faster spread over the GPU).  MG_BOTTOM_N64 / MG_BOTTOM_N32 override
// (0 leaves only the one-cell level to the kernel).
int bottom_limit(bool fp32)
{
    const char *v = std::getenv(fp32 ? "MG_BOTTOM_N32" : "MG_BOTTOM_N64");
    if (v && *v)
        return std::atoi(v);
    return 8;
}

// Launch plan of an FP32 multigrid level above the bottom kernel, one int per
// level (LevelData::tile): 0 = one kernel per colour and phase; t > 0 = the
// temporally blocked legs with tile t; t < 0 = the plane-marching sweeps
// (mg_wave.cu: every smoothing stint one launch, phi32 -> phi32b before the
// restriction, phi32b + prolongation -> phi32 after it), encoded as
// -(variant * 256 + z-chunks).
int wave_code(int variant, int zchunks) { return -(variant * 256 + zchunks); }
int wave_variant(int code) { return (-code) >> 8; }
int wave_zchunks(int code) { return (-code) & 255; }

bool wave_ok(int dim, int nu_pre, int nu_post, int N)
{
    return mg_wave_applies(dim, nu_pre, N) && mg_wave_applies(dim, nu_post, N);
}

// The default plane-marching plan of a level of N cells per edge: 56 x 10
// tiles from 100 cells up, 56 x 6 below (two blocks per SM either way);
// z-chunks so that the blocks fill the SMs once.
int wave_default(int N)
{
    const int variant = N >= 100 ? 0 : 1;
    const int ty = variant == 0 ? 10 : 6;
    const int xy = (N / 56 + 1) * (N / ty + 1);
    int zc = std::max(1, 152 * 2 / xy);
    zc = std::min(zc, std::max(1, N / 8));
    return wave_code(variant, std::min(zc, 255));
}

// FP32 launch plan of each level above the bottom kernel.  Without tuning:
// one kernel per phase (measured fastest on every level but the largest,
// where the plane-marching sweeps are about even); MG_WAVE=1 selects the
// plane-marching sweeps wherever they apply (3D, 1-2 sweeps per stint),
// MG_WAVE_PLAN="variant,zchunks" fixes their tile shape and z split (for
// measurement); MG_TB_TILE forces one blocked-leg tile for every level (even,
// fitting the shared-memory limit).  mg_autotune times all the candidates.
void plan_tiles(LevelData &ld, int dim, int nu_pre, int nu_post)
{
    const char *v = std::getenv("MG_TB_TILE");
    const int forced = (v && *v) ? std::atoi(v) : -1;
    const char *wv = std::getenv("MG_WAVE");
    const bool wave = wv && wv[0] == '1';
    int wvar = -1, wzc = -1;
    if (const char *wp = std::getenv("MG_WAVE_PLAN"))
        if (std::sscanf(wp, "%d,%d", &wvar, &wzc) != 2 || wvar < 0 || wvar > 1 || wzc < 1 || wzc > 255)
            wvar = wzc = -1;
    for (int L = 0; L < ld.nmg; L++) {
        int t = forced >= 0 ? forced : 0;
        t &= ~1;
        while (t > 0 && (mg_tb_smem(dim, true, t, 2 * nu_pre + 1) > MG_TB_SMEM_MAX ||
                         mg_tb_smem(dim, true, t, 2 * nu_post) > MG_TB_SMEM_MAX))
            t -= 2;
        if (forced < 0 && wave && wave_ok(dim, nu_pre, nu_post, ld.g[L].N))
            t = wvar >= 0 ? wave_code(wvar, std::min(wzc, ld.g[L].N)) : wave_default(ld.g[L].N);
        ld.tile[L] = t;
    }
}

// Colour-split FP32 levels: the first S multigrid levels above the one-block
// bottom (none with the cluster kernel) keep each colour in its own array and
// run the box-patch kernels (mg_box.cu), whose colour pass moves exactly its
// algorithmic bytes; levels below stay plain for the bottom, plane-marching
// and blocked kernels.  MG_SPLIT=S fixes S; without it (and without tuning)
// the levels of 192 cells per edge or more are split (measured on 4 nested
// 256^3 levels: the 258^3 level gains 33.4 -> 28.6 ms, splitting the 129^3
// level as well costs 0.9 ms, and at 66^3 the tuner keeps plain), unless MG_WAVE,
// MG_WAVE_PLAN or MG_TB_TILE ask for the plain-layout plans.  mg_autotune
// times the choices; the batched kernels (MG_BATCHED=1) run plain levels
// only.  Changing the layout clears the level's FP32 arrays (their ghost
// layer must read zero in either layout).
constexpr int kTileSplit = 1 << 16;   // mg_tuning / tuning-cache code of a split level
constexpr int kSplitMinN = 192;

int split_default(const LevelData &ld)
{
    if (ld.Lc[1] >= 0 || ld.frozen)   // the cluster kernel runs plain levels
        return 0;
    const int Ls = ld.Ls[1];
    if (const char *v = std::getenv("MG_SPLIT"))
        if (*v)
            return std::max(0, std::min(std::atoi(v), Ls));
    for (const char *name : {"MG_WAVE", "MG_WAVE_PLAN", "MG_TB_TILE"})
        if (const char *v = std::getenv(name))
            if (*v)
                return 0;
    int S = 0;
    while (S < Ls && ld.g[S].N >= kSplitMinN)
        S++;
    return S;
}

cudaError_t plan_split(LevelData &ld, int dim, int S, cudaStream_t s)
{
    S = std::max(0, std::min(S, ld.Ls[1]));
    if (ld.Lc[1] >= 0)
        S = 0;
    const bool changed = S != ld.nsplit;
    for (int L = 0; L < ld.nmg; L++) {
        MgGeom &g = ld.g[L];
        if (L < S) {
            g.sH = mg_split_H(g.E);
            g.shalf = (long long)g.sH * g.E * (dim == 3 ? g.E : 1);
            ld.tile[L] = 0;
        } else {
            g.sH = 0;
            g.shalf = 0;
        }
    }
    ld.nsplit = S;
    if (!changed || !ld.phi32[0])
        return cudaSuccess;
    for (int L = 0; L < ld.nmg; L++)
        for (float *a : {ld.phi32[L], ld.phi32b[L], ld.f32[L]})
            if (cudaError_t e = cudaMemsetAsync(a, 0, mg_fp32_cells(ld.g[L].E, dim) * sizeof(float), s))
                return e;
    return cudaSuccess;
}

void plan_bottom(LevelData &ld, int dim, int lim32 = -1)
{
    for (int w = 0; w < 2; w++) {
        const bool fp32 = w == 1;
        const int lim = (fp32 && lim32 >= 0) ? lim32 : bottom_limit(fp32);
        int Ls = ld.nmg - 1;
        for (int L = 0; L < ld.nmg; L++) {
            if (ld.g[L].N > lim || ld.nmg - L > MG_BOTTOM_MAX)
                continue;
            MgBottom bt;
            bt.nlev = ld.nmg - L;
            for (int q = 0; q < bt.nlev; q++)
                bt.g[q] = ld.g[L + q];
            if (mg_bottom_smem(dim, fp32, bt) <= MG_BOTTOM_SMEM_MAX) {
                Ls = L;
                break;
            }
        }
        ld.Ls[w] = Ls;
        ld.bt[w].nlev = ld.nmg - Ls;
        for (int q = 0; q < ld.bt[w].nlev; q++)
            ld.bt[w].g[q] = ld.g[Ls + q];
        ld.bt[w].plan = nullptr;   // until refresh_bottom_plan writes the image for these levels
    }
}

// Bytes of the largest plan image a one-block kernel of this level can use
// (the first level from which the kernel's shared memory fits).
size_t max_bottom_plan_bytes(const LevelData &ld, int dim, bool fp32)
{
    for (int L = 0; L < ld.nmg; L++) {
        if (ld.nmg - L > MG_BOTTOM_MAX)
            continue;
        MgBottom bt;
        bt.nlev = ld.nmg - L;
        for (int q = 0; q < bt.nlev; q++)
            bt.g[q] = ld.g[L + q];
        if (mg_bottom_smem(dim, fp32, bt) <= MG_BOTTOM_SMEM_MAX)
            return mg_bottom_plan_bytes(dim, fp32, bt);
    }
    return 0;
}

long cells(int e, int dim) { return dim == 3 ? (long)e * e * e : (long)e * e; }

// Largest multigrid level (cells per edge) handed to the cluster kernel, per
// precision; 0 disables it.  MG_CLUSTER_N64 / MG_CLUSTER_N32 override.
int cluster_limit(bool fp32)
{
    const char *v = std::getenv(fp32 ? "MG_CLUSTER_N32" : "MG_CLUSTER_N64");
    if (v && *v)
        return std::atoi(v);
    return 0;
}

// Largest multigrid level (cells per edge) the cluster kernel leaves to its
// CTA 0 and the one-block path.  MG_CLUSTER_BOTTOM overrides.
int cluster_bottom_limit()
{
    const char *v = std::getenv("MG_CLUSTER_BOTTOM");
    if (v && *v)
        return std::atoi(v);
    return 8;
}

// The cluster kernel's plan for levels from Lc on (3D): Lc the first level of
// at most `lim` cells per edge, Lcb the first after it of at most the cluster
// bottom limit; false when it does not apply or does not fit.
bool cluster_plan(const LevelData &ld, int dim, int csize, bool fp32, int lim, const mg_options &o, MgClusterPlan &p,
                  size_t *smem, int *Lc_out)
{
    if (dim != 3 || csize <= 0 || lim <= 0 || ld.nmg < 3)
        return false;
    int Lc = -1, Lcb = ld.nmg - 1;
    for (int L = 0; L < ld.nmg - 1; L++)
        if (ld.g[L].N <= lim) {
            Lc = L;
            break;
        }
    if (Lc < 0)
        return false;
    const int cb = cluster_bottom_limit();
    for (int L = Lc + 1; L < ld.nmg; L++)
        if (ld.g[L].N <= cb) {
            Lcb = L;
            break;
        }
    if (Lcb <= Lc)
        return false;
    p = MgClusterPlan{};
    p.nlev = ld.nmg - Lc;
    p.nclu = Lcb - Lc;
    p.cycles = 1;
    p.nu_pre = o.nu_pre;
    p.nu_post = o.nu_post;
    for (int q = 0; q < p.nlev; q++)
        p.g[q] = ld.g[Lc + q];
    p.bt.nlev = ld.nmg - Lcb;
    if (p.bt.nlev > MG_BOTTOM_MAX)
        return false;
    for (int q = 0; q < p.bt.nlev; q++)
        p.bt.g[q] = ld.g[Lcb + q];
    if (!mg_cluster_layout(fp32, csize, p, smem))
        return false;
    *Lc_out = Lc;
    return true;
}

void plan_cluster(LevelData &ld, int dim, int csize, const mg_options &o, int lim64 = -1, int lim32 = -1)
{
    for (int w = 0; w < 2; w++) {
        const int lim = w ? (lim32 >= 0 ? lim32 : cluster_limit(true)) : (lim64 >= 0 ? lim64 : cluster_limit(false));
        MgClusterPlan p;
        size_t smem = 0;
        int Lc = -1;
        ld.Lc[w] = cluster_plan(ld, dim, csize, w == 1, lim, o, p, &smem, &Lc) ? Lc : -1;
        ld.Llim[w] = lim;
    }
}

// Sec. 2.2: N^L = round(M / 2^L), halves rounded up, until N^L = 1.
int level_sizes(int M, int *N, int cap)
{
    int L = 0;
    N[0] = M;
    while (N[L] > 1 && L + 1 < cap) {
        L++;
        // floor(M / 2^L + 1/2) in integers
        N[L] = (int)(((long)M + (1L << (L - 1))) >> L);
    }
    return L + 1;
}

void build_geometry(LevelData &ld, int dim)
{
    int N[MG_MAX_MG];
    ld.M = ld.frozen ? ld.n : ld.n + 2;
    ld.nmg = level_sizes(ld.M, N, MG_MAX_MG);
    (void)dim;
    for (int L = 0; L < ld.nmg; L++) {
        MgGeom &g = ld.g[L];
        g.tab64 = nullptr;
        g.tab32 = nullptr;
        g.N = N[L];
        g.E = N[L] + 2;
        g.L = L;
        // x_N = (N - 1/2) 2^L / M; tie <=> (2N - 1) 2^L == 2M
        const long num = 2L * ld.M - (2L * N[L] + 1) * (1L << L);   // 2M (1 - x_N - h^L)
        const long den = 2L * ld.M - (2L * N[L] - 1) * (1L << L);   // 2M (1 - x_N)
        g.tie = (den == 0);
        g.cR = g.tie ? 0.0 : (double)num / (double)den;
        const double hL = ld.h * (double)(1L << L);
        g.h2 = hL * hL;
        g.inv_h2 = 1.0 / g.h2;
        g.cRf = (float)g.cR;
        g.h2f = (float)g.h2;
        g.inv_h2f = (float)g.inv_h2;
        g.sH = 0;
        g.shalf = 0;
    }
    ld.nsplit = 0;
}

#define MG_BRANCHES 8   // parallel branches of the solve graph (hierarchies of a batch)

enum KernelKind { KK_SMOOTH, KK_RESTRICT, KK_PROLONG, KK_NORM, KK_DEFECT, KK_ACCUM, KK_IFACE, KK_FORCES,
                  KK_SETDENS, KK_BOTTOM, KK_TB_PRE, KK_TB_POST, KK_CLUSTER, KK_SMOOTH0, KK_WAVE, KK_WAVE0, KK_COUNT };
const char *const kKindName[KK_COUNT] = {"smooth_colour", "resid_restrict", "prolong_correct", "resid_norm",
                                         "defect",        "accumulate",     "interface",       "forces",
                                         "set_density",   "bottom",         "tb_pre",          "tb_post",
                                         "cluster_vcycle", "smooth_colour_finest", "smooth_wave",
                                         "smooth_wave_finest"};

// Per-launch CUDA-event timing on the hierarchy's stream (mg_profile).
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec { int kind; size_t e0; double bytes; };
    std::vector<Rec> recs;
    long launches[KK_COUNT] = {};
    double ms[KK_COUNT] = {};
    double bytes[KK_COUNT] = {};
};

}  // namespace

struct mg_hierarchy {
    int batch = 0, dim = 0;
    std::vector<mg_hierarchy_desc> desc;
    std::vector<std::vector<LevelData>> lev;   // [b][l]
    mg_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    double *stage = nullptr;        // device staging for host-pointer I/O
    size_t stage_elems = 0;
    double *partials = nullptr;     // MG_BRANCHES * 2 * MG_NORM_BLOCKS_MAX reduction scratch
    unsigned *counters = nullptr;   // MG_BRANCHES block counters of the norm kernel
    unsigned long long *fmax = nullptr; // MG_BRANCHES maxima of the force-change test
    double *scal = nullptr;         // device scalars: [b][l][2] = ||b||^2, ||r||^2
    double *hscal = nullptr;        // pinned mirror
    MgSolveCtl *ctl = nullptr;      // device loop state per (b, l)
    double *frho = nullptr;         // device 4 pi G h_l^2 per (b, l) (input scaling of the learned guess)
    mg_unet *unet = nullptr;        // learned initial guess (MG_GUESS_LEARNED)
    MgSolveCtl *hctl = nullptr;     // pinned mirror
    int *werr = nullptr;            // device word: MG_ETIMEOUT once a plane-marching load wait gave up
    int wfault = 0;                 // MG_FAULT_WAVE_WAIT=1: those waits are made to run out (test of that path)
    bool poisoned = false, solved = false;
    std::string err;
    Profiler prof;
    // solve graph
    bool use_graph = true;          // MG_SOLVE_GRAPH=0: host-driven loop (for kernel profilers)
    int csize = 0;                  // CTAs per cluster of the cluster kernel (0: unavailable)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<char> graph_sig;
    cudaStream_t cap[MG_BRANCHES] = {};
    // batched mixed-precision plan (one launch per phase over all hierarchies)
    struct BatchLevel {
        int nparts = 0, maxLs = 0;
        MgBPart *parts = nullptr;
        int *active = nullptr;
        std::vector<int> ntasks;              // per depth: blocked-leg tile tasks
        std::vector<MgBTask *> tasks;
        // per depth, one-kernel-per-phase chunk tasks of the parts without a tile
        std::vector<int> n_sm, n_rr, n_pr;
        std::vector<MgBCell *> t_sm, t_rr, t_pr;
        MgBCell *cells_act = nullptr, *cells_blk = nullptr;
        int ncells_act = 0, ncells_blk = 0;
        std::vector<size_t> smem_pre, smem_post;
        size_t smem_bottom = 0;
    };
    std::vector<BatchLevel> bl;
    char *batch_mem = nullptr;
    bool batched = false;
    // persistent batched plan (one launch: a block per hierarchy at a time)
    bool persist = false;
    std::vector<char> in_persist;  // per hierarchy: solved by the persistent launch
    cudaStream_t cap_p = nullptr;  // capture stream of the persistent launch's branch
    cudaEvent_t ev_pjoin = nullptr;
    char *persist_mem = nullptr;
    MgBPart *pparts = nullptr;
    MgPTask *ptasks = nullptr;
    unsigned *pnext = nullptr;
    int nptasks = 0, pgrid = 0;
    size_t psmem = 0;
    cudaStream_t body_stream = nullptr;
    cudaStream_t inner_stream = nullptr;   // captures the nested loop of an adaptive step
    cudaEvent_t ev_fork = nullptr, ev_join[MG_BRANCHES] = {};
};

namespace {

std::string g_create_error;

mg_status fail(mg_hierarchy *h, mg_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_error = buf;
    return s;
}

mg_status fail_cuda(mg_hierarchy *h, cudaError_t e, const char *what)
{
    if (h)
        h->poisoned = true;
    return fail(h, MG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess)                        \
            return fail_cuda((h), e_, #call);         \
    } while (0)

// Launch through `fn`, bracketed by events when profiling is on.
template <class Fn>
cudaError_t timed(mg_hierarchy *h, int kind, double bytes, Fn &&fn)
{
    Profiler &P = h->prof;
    if (!P.on)
        return fn();
    while (P.used + 2 > P.pool.size()) {
        cudaEvent_t e;
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess)
            return ce;
        P.pool.push_back(e);
    }
    const size_t e0 = P.used;
    P.used += 2;
    cudaError_t ce = cudaEventRecord(P.pool[e0], h->stream);
    if (ce == cudaSuccess)
        ce = fn();
    if (ce == cudaSuccess)
        ce = cudaEventRecord(P.pool[e0 + 1], h->stream);
    P.recs.push_back({kind, e0, bytes});
    return ce;
}

cudaError_t profile_flush(mg_hierarchy *h)
{
    Profiler &P = h->prof;
    if (P.recs.empty())
        return cudaSuccess;
    cudaError_t ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess)
        return ce;
    for (const auto &r : P.recs) {
        float ms = 0.f;
        ce = cudaEventElapsedTime(&ms, P.pool[r.e0], P.pool[r.e0 + 1]);
        if (ce != cudaSuccess)
            return ce;
        P.launches[r.kind]++;
        P.ms[r.kind] += ms;
        P.bytes[r.kind] += r.bytes;
    }
    P.recs.clear();
    P.used = 0;
    return cudaSuccess;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked host memory that CUDA maps into the device address space: the
// device address through which kernels read or write it directly over the
// host link (no staging copy); nullptr for any other memory.
template <typename P>
P *mapped_host_view(P *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<P *>(a.devicePointer) : nullptr;
}

mg_status check_options(const mg_options &o)
{
    if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre + o.nu_post < 1 || o.max_cycles < 0 || !(o.rel_tol >= 0.0) ||
        (o.precision != MG_FP64 && o.precision != MG_MIXED) || o.inner_cycles < 1 || o.inner_max < 0 ||
        o.inner_max > MG_INNER_MAX ||
        o.guess < MG_GUESS_INTERP || o.guess > MG_GUESS_LEARNED ||
        (o.force_stencil != MG_FORCE_EQ2 && o.force_stencil != MG_FORCE_CD2) ||
        (o.interface != MG_IFACE_BUFFER && o.interface != MG_IFACE_FROZEN) ||
        (o.stop != MG_STOP_RESIDUAL && o.stop != MG_STOP_FORCE) ||
        (o.stop == MG_STOP_FORCE && o.interface != MG_IFACE_BUFFER))
        return MG_EINVAL;
    return MG_OK;
}

// parent patch of patch l > 0, and the refinement depth of a patch
int desc_parent(const mg_hierarchy_desc &d, int l) { return d.tree ? d.parent[l] : l - 1; }
int desc_depth(const mg_hierarchy_desc &d, int l)
{
    int k = 0;
    while (l > 0 && k <= MG_MAX_LEVELS) {
        l = desc_parent(d, l);
        k++;
    }
    return k;
}

mg_status check_desc(const mg_hierarchy_desc &d, int b, int dim0)
{
    if (d.dim != 2 && d.dim != 3)
        return fail(nullptr, MG_EINVAL, "hierarchy %d: dim must be 2 or 3", b);
    if (d.dim != dim0)
        return fail(nullptr, MG_EINVAL, "hierarchy %d: all hierarchies of a batch share one dim", b);
    if (d.num_levels < 1 || d.num_levels > MG_MAX_LEVELS)
        return fail(nullptr, MG_EINVAL, "hierarchy %d: num_levels %d out of range", b, d.num_levels);
    if (!(d.h0 > 0.0) || !std::isfinite(d.h0) || !std::isfinite(d.G))
        return fail(nullptr, MG_EINVAL, "hierarchy %d: h0 must be positive and G finite", b);
    if (d.tree != 0 && d.tree != 1)
        return fail(nullptr, MG_EINVAL, "hierarchy %d: tree must be 0 or 1", b);
    for (int l = 1; l < d.num_levels; l++)
        if (d.tree && (d.parent[l] < 0 || d.parent[l] >= l))
            return fail(nullptr, MG_EINVAL, "hierarchy %d patch %d: parent %d not in [0, %d)", b, l, d.parent[l], l);
    for (int l = 0; l < d.num_levels; l++) {
        const int n = d.n[l];
        if (n < 2 || n + 2 > (1 << (MG_MAX_MG - 1)) || (l > 0 && (n & 1)))
            return fail(nullptr, MG_EINVAL, "hierarchy %d level %d: n=%d (need >= 2, even above level 0)", b, l, n);
        if (d.dim == 3 && n > 1286)   // (n+4)^3 cells indexed in 32 bits
            return fail(nullptr, MG_EINVAL, "hierarchy %d level %d: n=%d exceeds 1286 in 3D", b, l, n);
        if (l == 0)
            continue;
        const int pl = desc_parent(d, l);
        const double hp = d.h0 / (double)(1L << desc_depth(d, pl));
        for (int a = 0; a < d.dim; a++) {
            const double o = (d.lo[l][a] - d.lo[pl][a]) / hp;
            const double r = std::floor(o + 0.5);
            if (std::fabs(o - r) > 1e-6)
                return fail(nullptr, MG_EINVAL, "hierarchy %d level %d axis %d: patch not on parent cell faces", b, l, a);
            if (r < 1.0 || r > (double)(d.n[pl] - n / 2 - 1))
                return fail(nullptr, MG_EINVAL,
                            "hierarchy %d level %d axis %d: offset %g outside [1, %d] parent cells", b, l, a, r,
                            d.n[pl] - n / 2 - 1);
        }
    }
    return MG_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// After device work that ran plane-marching sweeps: MG_ETIMEOUT (and the
// handle poisoned) when one of their bounded load waits gave up.
mg_status wave_status(mg_hierarchy *h)
{
    int w = 0;
    cudaError_t e = cudaMemcpyAsync(&w, h->werr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
        return fail_cuda(h, e, "reading the device error word");
    if (w) {
        h->poisoned = true;
        return fail(h, MG_ETIMEOUT, "a plane-marching sweep's load wait ran out of its clock budget");
    }
    return MG_OK;
}

// --------------------------------------------------------------------------
// the V-cycle of Sec. 2.3 on the arrays of one refinement level
// --------------------------------------------------------------------------
double cells_d(int N, int dim) { return dim == 3 ? (double)N * N * N : (double)N * N; }

// sweeps red-black sweeps on level L; ctl != NULL: the last launch also
// counts one V-cycle of an adaptive step's nested loop (condition hi)
cudaError_t smooth(mg_hierarchy *h, const LevelData &ld, int L, bool fp32, int sweeps, cudaStream_t s,
                   MgSolveCtl *ctl = nullptr, cudaGraphConditionalHandle hi = 0, bool red_done = false)
{
    const int dim = h->dim;
    const MgGeom &g = ld.g[L];
    void *phi = fp32 ? (void *)ld.phi32[L] : (void *)ld.phi[L];
    const void *f = fp32 ? (const void *)ld.f32[L] : (const void *)ld.f[L];
    const bool split = fp32 && L < ld.nsplit;
    const double bytes = (split ? 1.5 : 2.0) * (fp32 ? 4 : 8) * cells_d(g.N, dim);   // read Phi, read/write one colour
    for (int sw = 0; sw < sweeps; sw++)
        for (int c = 0; c < 2; c++) {
            if (red_done && sw == 0 && c == 0)
                continue;   // the restriction into this level did the first red half-sweep
            // the finest multigrid level is profiled apart from the coarser ones
            const bool last = sw == sweeps - 1 && c == 1;
            cudaError_t e = timed(h, L == 0 ? KK_SMOOTH0 : KK_SMOOTH, bytes, [&] {
                if (split)
                    return mg_split_colour(dim, (float *)phi, (const float *)f, g, c, s);
                return mg_launch_smooth(dim, fp32, phi, f, g, c, s, last ? ctl : nullptr, hi);
            });
            if (e)
                return e;
            if (split && last && ctl && (e = mg_launch_inner_step(ctl, hi, s)))
                return e;
        }
    return cudaSuccess;
}

// Writes the one-block kernel's plan image for the levels plan_bottom chose
// (precision of the V-cycles) and hands it to the kernel; until then the
// kernel builds the plan itself.  Synchronous: runs at creation and tuning.
cudaError_t refresh_bottom_plan(mg_hierarchy *h, LevelData &ld)
{
    const bool fp32 = h->opt.precision == MG_MIXED;
    MgBottom &bt = ld.bt[fp32 ? 1 : 0];
    bt.plan = nullptr;
    if (!ld.bplan || mg_bottom_plan_bytes(h->dim, fp32, bt) > ld.bplan_bytes)
        return cudaSuccess;
    cudaError_t e = mg_launch_bottom_plan(h->dim, fp32, bt, ld.bplan, h->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess)
        bt.plan = ld.bplan;
    return e;
}

// the V-cycle of Sec. 2.3 (steps 2-13) on the arrays of one refinement level,
// `ncyc` times; the levels from Lc down run in the cluster kernel (when
// Lc < Ls), those from Ls down in the one-block kernel
// ctl != NULL (one V-cycle of an adaptive step's nested loop): when the
// cycle ends with a smoothing launch of level 0, that launch also counts the
// cycle and sets the loop condition hi, and *counted is set.
cudaError_t vcycle(mg_hierarchy *h, const LevelData &ld, bool fp32, cudaStream_t s, int ncyc = 1,
                   MgSolveCtl *ctl = nullptr, cudaGraphConditionalHandle hi = 0, bool *counted = nullptr)
{
    const int dim = h->dim;
    const mg_options &o = h->opt;
    const int w = fp32 ? 4 : 8;
    auto P = [&](int L) -> void * { return fp32 ? (void *)ld.phi32[L] : (void *)ld.phi[L]; };
    auto F = [&](int L) -> void * { return fp32 ? (void *)ld.f32[L] : (void *)ld.f[L]; };
    const int Ls = ld.Ls[fp32 ? 1 : 0];
    const MgBottom &bt = ld.bt[fp32 ? 1 : 0];
    const int Lc = ld.Lc[fp32 ? 1 : 0];
    const bool clu = Lc >= 0 && h->csize > 0;
    const int Lstop = clu ? Lc : Ls;
    auto bottom = [&]() {
        return timed(h, KK_BOTTOM, 3.0 * w * cells_d(ld.g[Ls].E, dim),
                     [&] { return mg_launch_bottom(dim, fp32, P(Ls), F(Ls), bt, o.nu_pre, o.nu_post, s); });
    };
    auto cluster = [&](int cycles) {
        MgClusterPlan p;
        size_t smem = 0;
        int L0 = -1;
        if (!cluster_plan(ld, dim, h->csize, fp32, ld.Llim[fp32 ? 1 : 0], o, p, &smem, &L0) ||
            L0 != Lc)
            return cudaErrorInvalidValue;
        p.cycles = cycles;
        p.phi0 = P(Lc);
        p.f0 = F(Lc);
        double by = 3.0 * w * cells_d(ld.g[Lc].E, dim);
        for (int q = 0; q < p.nclu; q++)   // smoothing sweeps, residual + restriction, prolongation (on chip)
            by += w * cells_d(ld.g[Lc + q].N, dim) * (4.0 * (o.nu_pre + o.nu_post) + 5.0);
        return timed(h, KK_CLUSTER, by * cycles, [&] { return mg_launch_cluster(fp32, p, h->csize, smem, s); });
    };
    cudaError_t e;
    if (Lstop == 0) {                                                                     // whole cycle
        if (clu)
            return cluster(ncyc);
        for (int c = 0; c < ncyc; c++)
            if ((e = bottom()))
                return e;
        return cudaSuccess;
    }
    for (int cyc = 0; cyc < ncyc; cyc++) {
    // descent: at each level above Lstop, nu_pre sweeps then residual and
    // restriction (steps 2/6, 4, 5) -- one temporally blocked kernel per
    // level in FP32 when the level has a tile, else one kernel per phase.
    // A plain restriction into a level smoothed next by one kernel per phase
    // also does that level's first red half-sweep (red_done).
    bool red_done = false;
    for (int L = 0; L < Lstop; L++) {
        const double nf = cells_d(ld.g[L].N, dim), nc = cells_d(ld.g[L + 1].N, dim);
        if (fp32 && ld.tile[L] < 0) {
            const int code = ld.tile[L];
            e = timed(h, L == 0 ? KK_WAVE0 : KK_WAVE, 3.0 * w * nf, [&] {
                return mg_launch_wave(ld.phi32[L], ld.phi32b[L], ld.f32[L], ld.g[L], o.nu_pre, wave_variant(code),
                                      wave_zchunks(code), s, nullptr, 0, h->werr, h->wfault);
            });
            if (e)
                return e;
            e = timed(h, KK_RESTRICT, w * (2.0 * nf + 2.0 * nc), [&] {
                return mg_launch_resid_restrict(dim, true, ld.phi32b[L], ld.f32[L], ld.g[L], ld.phi32[L + 1],
                                                ld.f32[L + 1], ld.g[L + 1], s);
            });
            if (e)
                return e;
            continue;
        }
        if (fp32 && ld.tile[L] > 0) {
            e = timed(h, KK_TB_PRE, w * (3.0 * nf + 2.0 * nc), [&] {
                return mg_launch_tb_pre(dim, ld.phi32[L], ld.phi32b[L], ld.f32[L], ld.g[L], ld.phi32[L + 1],
                                        ld.f32[L + 1], ld.g[L + 1], ld.tile[L], o.nu_pre, s);
            });
            if (e)
                return e;
            continue;
        }
        if ((e = smooth(h, ld, L, fp32, o.nu_pre, s, nullptr, 0, red_done)))
            return e;
        const bool split_here = fp32 && L < ld.nsplit;
        const bool fuse = !split_here && o.nu_pre >= 1 && L + 1 < Lstop && !(fp32 && ld.tile[L + 1] != 0) &&
                          !(fp32 && L + 1 < ld.nsplit);
        e = timed(h, KK_RESTRICT, 2.0 * w * (nf + nc), [&] {
            if (split_here)
                return mg_split_resid_restrict(dim, ld.phi32[L], ld.f32[L], ld.g[L], ld.phi32[L + 1], ld.f32[L + 1],
                                               ld.g[L + 1], s);
            return mg_launch_resid_restrict(dim, fp32, P(L), F(L), ld.g[L], P(L + 1), F(L + 1), ld.g[L + 1], s,
                                            fuse);
        });
        if (e)
            return e;
        red_done = fuse;
    }
    if ((e = clu ? cluster(1) : bottom()))                                                // steps 6-11, L >= Lstop
        return e;
    // ascent: prolongation + correction, then nu_post sweeps (steps 10-11)
    for (int L = Lstop; L > 0; L--) {
        const double nf = cells_d(ld.g[L - 1].N, dim), nc = cells_d(ld.g[L].N, dim);
        if (fp32 && ld.tile[L - 1] < 0) {
            const int code = ld.tile[L - 1];
            e = timed(h, KK_PROLONG, w * (nc + 2.0 * nf), [&] {
                return mg_launch_prolong(dim, true, ld.phi32[L], ld.g[L], ld.phi32b[L - 1], ld.g[L - 1], s);
            });
            if (e)
                return e;
            const bool fold = ctl && ncyc == 1 && L == 1;
            e = timed(h, L == 1 ? KK_WAVE0 : KK_WAVE, 3.0 * w * nf, [&] {
                return mg_launch_wave(ld.phi32b[L - 1], ld.phi32[L - 1], ld.f32[L - 1], ld.g[L - 1], o.nu_post,
                                      wave_variant(code), wave_zchunks(code), s, fold ? ctl : nullptr, hi, h->werr,
                                      h->wfault);
            });
            if (e)
                return e;
            if (fold && counted)
                *counted = true;
            continue;
        }
        if (fp32 && ld.tile[L - 1] > 0) {
            e = timed(h, KK_TB_POST, w * (3.0 * nf + nc), [&] {
                return mg_launch_tb_post(dim, ld.phi32b[L - 1], ld.phi32[L - 1], ld.f32[L - 1], ld.g[L - 1],
                                         ld.phi32[L], ld.g[L], ld.tile[L - 1], o.nu_post, s);
            });
            if (e)
                return e;
            continue;
        }
        e = timed(h, KK_PROLONG, w * (nc + 2.0 * nf), [&] {
            if (fp32 && L - 1 < ld.nsplit)
                return mg_split_prolong(dim, ld.phi32[L], ld.g[L], ld.phi32[L - 1], ld.g[L - 1], s);
            return mg_launch_prolong(dim, fp32, P(L), ld.g[L], P(L - 1), ld.g[L - 1], s);
        });
        if (e)
            return e;
        const bool fold = ctl && ncyc == 1 && L == 1 && o.nu_post > 0;
        if ((e = smooth(h, ld, L - 1, fp32, o.nu_post, s, fold ? ctl : nullptr, hi)))
            return e;
        if (fold && counted)
            *counted = true;
    }
    }
    return cudaSuccess;
}

// True when the residual norm also writes the next defect-correction step's
// FP32 right-hand side (mixed precision under the residual stopping rule):
// the residual is then computed once per step instead of twice.
bool fused_defect(const mg_hierarchy *h) { return h->opt.precision == MG_MIXED && h->opt.stop == MG_STOP_RESIDUAL; }

// ||b||^2 (which & 1) and ||r||^2 (which & 2) of a level into scal[0..1];
// `branch` selects the reduction scratch of a parallel graph branch.
cudaError_t norms(mg_hierarchy *h, const LevelData &ld, int which, double *scal, cudaStream_t s, int branch)
{
    const bool fd = (which & 2) && fused_defect(h);
    return timed(h, KK_NORM, (fd ? 24.0 : 16.0) * cells_d(ld.g[0].N, h->dim), [&] {
        return mg_launch_norms2(h->dim, ld.phi[0], ld.f[0], ld.g[0], which,
                                h->partials + (size_t)branch * 2 * MG_NORM_BLOCKS_MAX, h->counters + branch, scal, s,
                                fd ? ld.f32[0] : nullptr, fd ? ld.phi32[0] : nullptr);
    });
}

double *level_scal(mg_hierarchy *h, int b, int l) { return h->scal + 2 * ((size_t)b * MG_MAX_LEVELS + l); }
MgSolveCtl *level_ctl(mg_hierarchy *h, int b, int l) { return h->ctl + (size_t)b * MG_MAX_LEVELS + l; }

// Before the iterations of one level: the one-way interface from the parent
// (Sec. 2.1) with the initial potential (Sec. 2.4), then ||b||^2 and ||r||^2.
cudaError_t level_prelude(mg_hierarchy *h, int b, int l, cudaStream_t s, int branch)
{
    LevelData &ld = h->lev[b][l];
    const int dim = h->dim;
    const mg_options &o = h->opt;
    const double fourpiG = 4.0 * M_PI * h->desc[b].G;
    double *ds = level_scal(h, b, l);
    cudaError_t e;
    if (l > 0) {
        const LevelData &pd = h->lev[b][ld.parent];
        const int gmode = o.guess == MG_GUESS_USER ? (ld.guess_set ? 2 : 0) : (o.guess == MG_GUESS_ZERO ? 1 : 0);
        const double by = 8.0 * cells_d(ld.n + 4, dim) + 16.0 * (cells_d(ld.n + 2, dim) - cells_d(ld.n, dim));
        e = timed(h, KK_IFACE, by, [&] {
            return mg_launch_interface(dim, pd.n, pd.blk, pd.rho, ld.n, ld.off[0], ld.off[1], ld.off[2], ld.blk,
                                       ld.rho, ld.fblk, fourpiG, gmode, ld.guess, ld.frozen, s);
        });
        if (e)
            return e;
        if (o.guess == MG_GUESS_LEARNED && h->unet && dim == 3 && (ld.n & (ld.n - 1)) == 0) {
            // network correction of the interpolated potential on Omega
            const int r = mg_unet_predict_dev(h->unet, 1, ld.n, 1, ld.rho, ld.blk, nullptr,
                                              h->frho + (size_t)b * MG_MAX_LEVELS + l, 1, s);
            if (r == 3)
                return cudaErrorLaunchFailure;
        }
        if (ld.frozen) {
            // the (n+2)^d box of Omega and the inner ring into the multigrid arrays
            if ((e = mg_launch_copy_box(dim, ld.n + 2, ld.blk, ld.n + 4, 1, ld.phi[0], ld.n + 2, 0, s)) ||
                (e = mg_launch_copy_box(dim, ld.n + 2, ld.fblk, ld.n + 4, 1, ld.f[0], ld.n + 2, 0, s)))
                return e;
        }
    } else if (ld.guess_set) {
        if ((e = mg_launch_copy_guess(dim, ld.n, ld.guess, ld.blk, s)))
            return e;
    }
    if ((e = norms(h, ld, 3, ds, s, branch)))
        return e;
    if (o.stop == MG_STOP_FORCE)
        e = mg_launch_force_stop(0, dim, ld.n, ld.h, nullptr, nullptr, 0, nullptr, ds, s);
    return e;
}

// After the iterations of a frozen-interface level: Omega back into the level block.
cudaError_t level_epilogue(mg_hierarchy *h, int b, int l, cudaStream_t s)
{
    const LevelData &ld = h->lev[b][l];
    if (!ld.frozen)
        return cudaSuccess;
    return mg_launch_copy_box(h->dim, ld.n, ld.phi[0], ld.n + 2, 1, ld.blk, ld.n + 4, 2, s);
}

// One iteration of a level's loop (Sec. 2.3 step 14): an FP64 V-cycle, or in
// mixed precision an FP64 defect (already written by the previous residual
// norm under the residual stopping rule), inner_cycles FP32 V-cycles on the
// correction and its FP64 accumulation; then ||r||^2.
// True when each mixed-precision step chooses its FP32 V-cycles (options
// inner_max > 0, residual stopping rule).
bool adaptive_inner(const mg_hierarchy *h)
{
    return h->opt.precision == MG_MIXED && h->opt.stop == MG_STOP_RESIDUAL && h->opt.inner_max > 0;
}

// The FP32 V-cycles of an adaptive step while s captures a graph: a nested
// WHILE node whose body is one V-cycle, counted down in ctl.left by its last
// launch (the counted smoothing variant, else a separate kernel after it);
// the condition *hi starts at 1 and ctl_step re-arms it for the next step.
cudaError_t capture_inner_loop(mg_hierarchy *h, const LevelData &ld, MgSolveCtl *ctl, cudaStream_t s,
                               cudaGraphConditionalHandle *hi)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
    if (e)
        return e;
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    if ((e = cudaGraphConditionalHandleCreate(hi, g, 1, cudaGraphCondAssignDefault)))
        return e;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = *hi;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, dv.data(), nullptr, dv.size(), &p)))
        return e;
    cudaGraph_t body = p.conditional.phGraph_out[0];
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)))
        return e;
    if (!h->inner_stream && (e = cudaStreamCreateWithFlags(&h->inner_stream, cudaStreamNonBlocking)))
        return e;
    if ((e = cudaStreamBeginCaptureToGraph(h->inner_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
        return e;
    bool counted = false;
    cudaError_t eb = vcycle(h, ld, true, h->inner_stream, 1, ctl, *hi, &counted);
    if (!eb && !counted)
        eb = mg_launch_inner_step(ctl, *hi, h->inner_stream);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(h->inner_stream, &out);
    return eb ? eb : e;
}

// One step of level l: ncyc V-cycles (FP32 in mixed mode, where hi != NULL
// captures an adaptive step's nested loop instead), then the norms that
// decide the next.
cudaError_t level_iteration(mg_hierarchy *h, int b, int l, cudaStream_t s, int branch, int ncyc = -1,
                            cudaGraphConditionalHandle *hi = nullptr)
{
    const LevelData &ld = h->lev[b][l];
    const int dim = h->dim;
    const mg_options &o = h->opt;
    cudaError_t e;
    unsigned long long *cmax = h->fmax + branch;
    if (o.stop == MG_STOP_FORCE &&
        (e = mg_launch_force_stop(1, dim, ld.n, ld.h, ld.blk, ld.prev, 0, cmax, nullptr, s)))
        return e;
    if (o.precision != MG_MIXED) {
        if ((e = vcycle(h, ld, false, s)))
            return e;
    } else {
        const double nd = cells_d(ld.g[0].N, dim);
        if (!fused_defect(h)) {   // else the previous residual norm wrote it
            e = timed(h, KK_DEFECT, 24.0 * nd, [&] {
                return mg_launch_defect(dim, ld.phi[0], ld.f[0], ld.g[0], ld.f32[0], ld.phi32[0], s);
            });
            if (e)
                return e;
        }
        if (hi)
            e = capture_inner_loop(h, ld, level_ctl(h, b, l), s, hi);
        else
            e = vcycle(h, ld, true, s, ncyc > 0 ? ncyc : o.inner_cycles);
        if (e)
            return e;
        e = timed(h, KK_ACCUM, 20.0 * nd, [&] { return mg_launch_accumulate(dim, ld.phi[0], ld.phi32[0], ld.g[0], s); });
        if (e)
            return e;
    }
    if (o.stop == MG_STOP_FORCE)
        return mg_launch_force_stop(2, dim, ld.n, ld.h, ld.blk, ld.prev, o.force_stencil, cmax, level_scal(h, b, l), s);
    return norms(h, ld, 2, level_scal(h, b, l), s, branch);
}

int cycles_per_iteration(const mg_hierarchy *h) { return h->opt.precision == MG_MIXED ? h->opt.inner_cycles : 1; }

void fill_stats(const mg_hierarchy *h, const MgSolveCtl &c, mg_level_stats *st)
{
    int status = c.status ? MG_EDIVERGED : MG_OK;
    if (status == MG_OK && c.bnorm > 0.0 && h->opt.rel_tol > 0.0 && !(c.rel < h->opt.rel_tol))
        status = MG_ENOCONV;
    st->cycles = c.cycles;
    st->outer_steps = c.outer;
    st->rel_res = c.rel;
    st->b_norm = c.bnorm;
    st->status = status;
}

// Potential and forces (Eq. 2) of a converged level into its registered
// outputs, on stream s.
cudaError_t launch_outputs(mg_hierarchy *h, const LevelData &ld, cudaStream_t s)
{
    if (!ld.out_F)
        return cudaSuccess;
    const int dim = h->dim;
    const double nr = cells_d(ld.n, dim);
    return timed(h, KK_FORCES, 8.0 * (cells_d(ld.n + 4, dim) + (dim + 1) * nr), [&] {
        return mg_launch_forces(dim, ld.n, ld.h, ld.blk, ld.out_F, ld.out_phi, h->opt.force_stencil, s);
    });
}

// Host-driven loop (used while per-kernel profiling is on): the same
// launches as the graph, with the loop decision taken on the host.
mg_status solve_level_host(mg_hierarchy *h, int b, int l, mg_level_stats *st)
{
    const mg_options &o = h->opt;
    cudaStream_t s = h->stream;
    double *hs = h->hscal + 2 * ((size_t)b * MG_MAX_LEVELS + l);
    double *ds = level_scal(h, b, l);
    CK(h, level_prelude(h, b, l, s, 0));
    CK(h, cudaMemcpyAsync(hs, ds, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    MgSolveCtl c{};
    c.bnorm = std::sqrt(hs[0]);
    c.rel = c.bnorm > 0.0 ? std::sqrt(hs[1]) / c.bnorm : 0.0;
    if (!std::isfinite(c.bnorm))
        c.status = 1;
    const bool adapt = adaptive_inner(h);
    int inner = o.inner_cycles;   // adaptive: FP32 V-cycles of the next step, as the graph's ctl kernels choose
    while (c.bnorm > 0.0 && c.status == 0 && c.cycles < o.max_cycles && !(c.rel < o.rel_tol)) {
        const int ncyc = adapt ? std::min(inner, o.max_cycles - c.cycles) : cycles_per_iteration(h);
        CK(h, level_iteration(h, b, l, s, 0, ncyc));
        CK(h, cudaMemcpyAsync(hs, ds, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(h, cudaStreamSynchronize(s));
        const double before = c.rel;
        c.cycles += ncyc;
        c.outer++;
        c.rel = std::sqrt(hs[1]) / c.bnorm;
        if (!std::isfinite(c.rel))
            c.status = 1;
        if (adapt)
            inner = mg_next_inner(before, c.rel, ncyc, o.rel_tol, o.inner_max);
    }
    CK(h, level_epilogue(h, b, l, s));
    CK(h, launch_outputs(h, h->lev[b][l], s));
    fill_stats(h, c, st);
    return (mg_status)st->status;
}

// --------------------------------------------------------------------------
// The whole solve as one CUDA graph: per (hierarchy, level) the prelude and a
// conditional WHILE node whose body is one iteration plus a control kernel
// that counts cycles and decides, on the device, whether to go on.
// Hierarchies of a batch are independent and run as parallel branches.
// --------------------------------------------------------------------------
void destroy_graph(mg_hierarchy *h)
{
    if (h->gexec)
        cudaGraphExecDestroy(h->gexec);
    if (h->graph)
        cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
}

std::vector<char> graph_signature(const mg_hierarchy *h)
{
    std::vector<char> sig;
    sig.push_back(h->unet ? 1 : 0);
    for (const auto &hl : h->lev)
        for (const auto &ld : hl) {
            sig.push_back(ld.guess_set ? 1 : 0);
            for (const double *p : {ld.out_F, ld.out_phi}) {
                const uintptr_t v = (uintptr_t)p;
                for (size_t k = 0; k < sizeof v; k++)
                    sig.push_back((char)(v >> (8 * k)));
            }
        }
    return sig;
}

cudaError_t capture_level(mg_hierarchy *h, int b, int l, cudaStream_t s, int branch)
{
    const mg_options &o = h->opt;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (e)
        return e;
    cudaGraphConditionalHandle hc;
    if ((e = cudaGraphConditionalHandleCreate(&hc, g, 0, cudaGraphCondAssignDefault)))
        return e;
    if ((e = level_prelude(h, b, l, s, branch)))
        return e;
    if ((e = mg_launch_ctl_init(level_ctl(h, b, l), level_scal(h, b, l), o.rel_tol, o.max_cycles, o.inner_cycles,
                                hc, s)))
        return e;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd)))
        return e;
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hc;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, dv.data(), nullptr, dv.size(), &p)))
        return e;
    cudaGraph_t body = p.conditional.phGraph_out[0];
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)))
        return e;
    if ((e = cudaStreamBeginCaptureToGraph(h->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
        return e;
    const bool adapt = adaptive_inner(h);
    cudaGraphConditionalHandle hi = 0;
    cudaError_t eb = level_iteration(h, b, l, h->body_stream, branch, -1, adapt ? &hi : nullptr);
    if (!eb)
        eb = mg_launch_ctl_step(level_ctl(h, b, l), level_scal(h, b, l), adapt ? 0 : cycles_per_iteration(h),
                                o.rel_tol, o.max_cycles, adapt ? o.inner_max : 0, hc, hi, h->body_stream);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(h->body_stream, &out);
    if (eb || e)
        return eb ? eb : e;
    return level_epilogue(h, b, l, s);
}

// Plan of the batched mixed-precision solve: per refinement level the parts
// (hierarchies that have the level), their tile tasks per multigrid depth and
// their cell-chunk tasks.  Returns false (no batched plan) when some part has
// a level above its one-block kernel without an FP32 tile.
bool plan_batched(mg_hierarchy *h, mg_status &err)
{
    err = MG_OK;
    const int dim = h->dim;
    const mg_options &o = h->opt;
    int maxL = 0;
    for (int b = 0; b < h->batch; b++)
        maxL = std::max(maxL, h->desc[b].num_levels);
    struct HostLevel {
        std::vector<MgBPart> parts;
        std::vector<std::vector<MgBTask>> tasks;
        std::vector<std::vector<MgBCell>> sm, rr, pr;
        std::vector<MgBCell> act, blk;
    };
    std::vector<HostLevel> HL(maxL);
    size_t npart_total = 0;
    for (int l = 0; l < maxL; l++) {
        HostLevel &H = HL[l];
        for (int b = 0; b < h->batch; b++) {
            if (l >= h->desc[b].num_levels)
                continue;
            LevelData &ld = h->lev[b][l];
            MgBPart P;
            std::memset(&P, 0, sizeof P);
            P.b = b;
            P.l = l;
            P.nmg = ld.nmg;
            P.Ls = ld.Ls[1];
            for (int L = 0; L < ld.nmg; L++) {
                P.g[L] = ld.g[L];
                P.tile[L] = ld.tile[L] > 0 ? ld.tile[L] : 0;   // batched kernels: blocked legs or one kernel per phase
                P.phi32[L] = ld.phi32[L];
                P.phi32b[L] = ld.phi32b[L];
                P.f32[L] = ld.f32[L];
            }
            P.phi = ld.phi[0];
            P.f = ld.f[0];
            P.rho = ld.rho;
            P.scal = level_scal(h, b, l);
            P.ctl = level_ctl(h, b, l);
            const long act = (long)std::pow((double)ld.g[0].N, dim), blk = cells(ld.n + 4, dim);
            P.nblk_act = (int)std::max<long>(1, std::min<long>((act + 1023) / 1024, MG_NORM_BLOCKS_MAX));
            P.nblk_blk = (int)std::min<long>((blk + 255) / 256, 4096);
            P.bt = ld.bt[1];
            P.n = ld.n;
            P.fourpiG = 4.0 * M_PI * h->desc[b].G;
            P.guess = ld.guess;
            if (l == 0) {
                P.gmode = ld.guess_set ? 2 : -1;
            } else {
                const LevelData &pd = h->lev[b][ld.parent];
                P.np = pd.n;
                P.phi_p = pd.phi[0];
                P.rho_p = pd.rho;
                for (int a = 0; a < 3; a++)
                    P.off[a] = ld.off[a];
                P.gmode = o.guess == MG_GUESS_USER ? (ld.guess_set ? 2 : 0) : (o.guess == MG_GUESS_ZERO ? 1 : 0);
            }
            const int p = (int)H.parts.size();
            if ((int)H.tasks.size() < P.Ls) {
                H.tasks.resize(P.Ls);
                H.sm.resize(P.Ls);
                H.rr.resize(P.Ls);
                H.pr.resize(P.Ls);
            }
            for (int L = 0; L < P.Ls; L++) {
                if (ld.tile[L] > 0) {
                    const int nb = (ld.g[L].N + ld.tile[L] - 1) / ld.tile[L];
                    for (int z = 0; z < (dim == 3 ? nb : 1); z++)
                        for (int y = 0; y < nb; y++)
                            for (int x = 0; x < nb; x++)
                                H.tasks[L].push_back({p, x, y, z});
                    continue;
                }
                // one chunk of 256 threads per 256 cells of the level (same
                // count for the colour, coarse and fine passes: grid-stride)
                const long cl = (long)std::pow((double)ld.g[L].N, dim);
                P.nblk_lvl[L] = (int)std::max<long>(1, std::min<long>((cl + 255) / 256, 152 * 16));
                for (int c = 0; c < P.nblk_lvl[L]; c++) {
                    H.sm[L].push_back({p, c});
                    H.rr[L].push_back({p, c});
                    H.pr[L].push_back({p, c});
                }
            }
            for (int c = 0; c < P.nblk_act; c++)
                H.act.push_back({p, c});
            for (int c = 0; c < P.nblk_blk; c++)
                H.blk.push_back({p, c});
            H.parts.push_back(P);
        }
        npart_total += H.parts.size();
    }
    // one allocation for the metadata and the per-part reduction scratch
    size_t bytes = 0;
    auto add = [&](size_t b) { const size_t at = bytes; bytes += align256(b); return at; };
    std::vector<size_t> off_parts(maxL), off_active(maxL), off_act(maxL), off_blk(maxL);
    std::vector<std::vector<size_t>> off_tasks(maxL);
    for (int l = 0; l < maxL; l++) {
        off_parts[l] = add(HL[l].parts.size() * sizeof(MgBPart));
        off_active[l] = add(HL[l].parts.size() * sizeof(int));
        off_act[l] = add(HL[l].act.size() * sizeof(MgBCell));
        off_blk[l] = add(HL[l].blk.size() * sizeof(MgBCell));
        for (auto &t : HL[l].tasks)
            off_tasks[l].push_back(add(t.size() * sizeof(MgBTask)));
        for (auto *v : {&HL[l].sm, &HL[l].rr, &HL[l].pr})
            for (auto &t : *v)
                off_tasks[l].push_back(add(t.size() * sizeof(MgBCell)));
    }
    const size_t off_partials = add(npart_total * 2 * MG_NORM_BLOCKS_MAX * sizeof(double));
    const size_t off_counters = add(npart_total * sizeof(unsigned));
    if (h->batch_mem)
        cudaFree(h->batch_mem);
    h->batch_mem = nullptr;
    cudaError_t e = cudaMalloc((void **)&h->batch_mem, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = fail(h, MG_ENOMEM, "cudaMalloc of %zu bytes for the batched plan failed", bytes);
        return false;
    }
    char *base = h->batch_mem;
    e = cudaMemsetAsync(base, 0, bytes, h->stream);
    size_t pidx = 0;
    h->bl.assign(maxL, mg_hierarchy::BatchLevel());
    for (int l = 0; l < maxL && !e; l++) {
        HostLevel &H = HL[l];
        auto &B = h->bl[l];
        for (auto &P : H.parts) {
            P.partials = (double *)(base + off_partials) + pidx * 2 * MG_NORM_BLOCKS_MAX;
            P.counter = (unsigned *)(base + off_counters) + pidx;
            pidx++;
            B.maxLs = std::max(B.maxLs, P.Ls);
            B.smem_bottom = std::max(B.smem_bottom, mg_bottom_smem(dim, true, P.bt));
        }
        B.nparts = (int)H.parts.size();
        B.parts = (MgBPart *)(base + off_parts[l]);
        B.active = (int *)(base + off_active[l]);
        B.cells_act = (MgBCell *)(base + off_act[l]);
        B.cells_blk = (MgBCell *)(base + off_blk[l]);
        B.ncells_act = (int)H.act.size();
        B.ncells_blk = (int)H.blk.size();
        B.smem_pre.assign(B.maxLs, 0);
        B.smem_post.assign(B.maxLs, 0);
        for (auto &P : H.parts)
            for (int L = 0; L < P.Ls; L++) {
                B.smem_pre[L] = std::max(B.smem_pre[L], mg_tb_smem(dim, true, P.tile[L], 2 * o.nu_pre + 1));
                B.smem_post[L] = std::max(B.smem_post[L], mg_tb_smem(dim, true, P.tile[L], 2 * o.nu_post));
            }
        B.tasks.resize(H.tasks.size());
        B.ntasks.resize(H.tasks.size());
        const size_t nd = H.tasks.size();
        B.n_sm.assign(nd, 0);
        B.n_rr.assign(nd, 0);
        B.n_pr.assign(nd, 0);
        B.t_sm.assign(nd, nullptr);
        B.t_rr.assign(nd, nullptr);
        B.t_pr.assign(nd, nullptr);
        e = cudaMemcpyAsync(B.parts, H.parts.data(), H.parts.size() * sizeof(MgBPart), cudaMemcpyHostToDevice, h->stream);
        if (!e)
            e = cudaMemcpyAsync(B.cells_act, H.act.data(), H.act.size() * sizeof(MgBCell), cudaMemcpyHostToDevice, h->stream);
        if (!e)
            e = cudaMemcpyAsync(B.cells_blk, H.blk.data(), H.blk.size() * sizeof(MgBCell), cudaMemcpyHostToDevice, h->stream);
        size_t oi = 0;
        for (size_t d = 0; d < nd && !e; d++, oi++) {
            B.tasks[d] = (MgBTask *)(base + off_tasks[l][oi]);
            B.ntasks[d] = (int)H.tasks[d].size();
            if (!H.tasks[d].empty())
                e = cudaMemcpyAsync(B.tasks[d], H.tasks[d].data(), H.tasks[d].size() * sizeof(MgBTask),
                                    cudaMemcpyHostToDevice, h->stream);
        }
        std::vector<MgBCell *> *dst[3] = {&B.t_sm, &B.t_rr, &B.t_pr};
        std::vector<int> *cnt[3] = {&B.n_sm, &B.n_rr, &B.n_pr};
        std::vector<std::vector<MgBCell>> *src[3] = {&H.sm, &H.rr, &H.pr};
        for (int w = 0; w < 3 && !e; w++)
            for (size_t d = 0; d < nd && !e; d++, oi++) {
                (*dst[w])[d] = (MgBCell *)(base + off_tasks[l][oi]);
                (*cnt[w])[d] = (int)(*src[w])[d].size();
                if (!(*src[w])[d].empty())
                    e = cudaMemcpyAsync((*dst[w])[d], (*src[w])[d].data(), (*src[w])[d].size() * sizeof(MgBCell),
                                        cudaMemcpyHostToDevice, h->stream);
            }
    }
    if (!e)
        e = cudaStreamSynchronize(h->stream);
    if (e) {
        err = fail_cuda(h, e, "batched plan upload");
        return false;
    }
    return true;
}

// One iteration of the batched loop of level l: FP64 defect, inner_cycles
// FP32 V-cycles over all parts (pre legs by depth, the one-block kernels,
// post legs), FP64 accumulation, norms and the loop control.
// The persistent plan: every (hierarchy, level) as a part in level order,
// the hierarchies ordered by decreasing active cells (the largest start
// first, so the last block to finish holds a small one), FP32 levels plain.
// Eligible: mixed precision, buffer interface, residual stopping rule, no
// learned guess and no cluster levels.
bool persist_eligible(const mg_hierarchy *h)
{
    const mg_options &o = h->opt;
    if (o.precision != MG_MIXED || h->batch < 2 || o.interface != MG_IFACE_BUFFER || o.stop != MG_STOP_RESIDUAL ||
        o.guess == MG_GUESS_LEARNED)
        return false;
    for (const auto &hl : h->lev)
        for (const auto &ld : hl)
            if (ld.Lc[1] >= 0 || ld.frozen)
                return false;
    return true;
}

// Which hierarchies of an eligible batch the persistent launch takes.  Cost
// model, calibrated on GB300 batches of 512 hierarchies of 16-32 and 32-48
// cells per edge and of 64 and 512 hierarchies of 32-128: a graph branch
// costs about 2.3 us per kernel node (Ls (2 nu_pre + 1) + 1 + Ls (2 nu_post
// + 1) nodes per V-cycle, 12 V-cycles per level assumed, 8 branches at once)
// plus its cells at 1.5e9 per second; the persistent launch solves 6e6 cells
// per second per block, 2 blocks per SM, largest hierarchy first.  The whole
// batch goes to the persistent launch when that estimate is the shorter:
// run beside graph branches it takes SMs and bandwidth from them (measured:
// a split of the 512-hierarchy batch of 32-128 took 707 ms against 642 ms
// with graph branches only).  MG_PERSIST=1 / 0 forces all / none (the
// batched kernels, MG_BATCHED=1, exclude it); MG_PERSIST_COUNT=k gives the k
// smallest hierarchies to it and the rest to graph branches in the same
// graph.
void choose_persistent(mg_hierarchy *h)
{
    const int nb = h->batch;
    h->in_persist.assign(nb, 0);
    const char *v = std::getenv("MG_PERSIST");
    const char *vb = std::getenv("MG_BATCHED");
    if (!persist_eligible(h) || (v && v[0] == '0') || (vb && vb[0] == '1'))
        return;
    if (v && v[0] == '1') {
        h->in_persist.assign(nb, 1);
        return;
    }
    const mg_options &o = h->opt;
    std::vector<double> cells(nb, 0.0), lat(nb, 0.0);
    for (int b = 0; b < nb; b++)
        for (const auto &ld : h->lev[b]) {
            cells[b] += cells_d(ld.n, h->dim);
            const int Ls = ld.Ls[1];
            lat[b] += 12.0 * (Ls * (2.0 * o.nu_pre + 1) + 1 + Ls * (2.0 * o.nu_post + 1)) * 2.3e-6;
        }
    if (const char *kv = std::getenv("MG_PERSIST_COUNT")) {
        std::vector<int> order(nb);
        for (int b = 0; b < nb; b++)
            order[b] = b;
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cells[a] < cells[c]; });
        const int k = std::max(0, std::min(std::atoi(kv), nb));
        for (int i = 0; i < k; i++)
            h->in_persist[order[i]] = 1;
        return;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    double g_lat = 0.0, all = 0.0, big = 0.0;
    for (int b = 0; b < nb; b++) {
        g_lat += lat[b];
        all += cells[b];
        big = std::max(big, cells[b]);
    }
    const double tg = g_lat / 8.0 + all / 1.5e9;
    const double tp = std::max(big / 6e6, all / (std::min((double)nb, 2.0 * nsm) * 6e6));
    if (tp < tg)
        h->in_persist.assign(nb, 1);
}

bool plan_persistent(mg_hierarchy *h, mg_status &err)
{
    err = MG_OK;
    const int dim = h->dim;
    const mg_options &o = h->opt;
    std::vector<MgBPart> parts;
    std::vector<MgPTask> tasks;
    std::vector<double> work;
    size_t smem = 0;
    for (int b = 0; b < h->batch; b++) {
        if (!h->in_persist[b])
            continue;
        MgPTask T{(int)parts.size(), h->desc[b].num_levels};
        double cellsum = 0.0;
        for (int l = 0; l < h->desc[b].num_levels; l++) {
            LevelData &ld = h->lev[b][l];
            if (cudaError_t e = plan_split(ld, dim, 0, h->stream)) {
                err = fail_cuda(h, e, "persistent plan");
                return false;
            }
            MgBPart P;
            std::memset(&P, 0, sizeof P);
            P.b = b;
            P.l = l;
            P.nmg = ld.nmg;
            P.Ls = ld.Ls[1];
            for (int L = 0; L < ld.nmg; L++) {
                P.g[L] = ld.g[L];
                P.phi32[L] = ld.phi32[L];
                P.phi32b[L] = ld.phi32b[L];
                P.f32[L] = ld.f32[L];
            }
            P.phi = ld.phi[0];
            P.f = ld.f[0];
            P.rho = ld.rho;
            P.scal = level_scal(h, b, l);
            P.ctl = level_ctl(h, b, l);
            P.bt = ld.bt[1];
            P.n = ld.n;
            P.h = ld.h;
            P.fourpiG = 4.0 * M_PI * h->desc[b].G;
            P.guess = ld.guess;
            P.out_F = ld.out_F;
            P.out_phi = ld.out_phi;
            if (l == 0) {
                P.gmode = ld.guess_set ? 2 : -1;
            } else {
                const LevelData &pd = h->lev[b][ld.parent];
                P.np = pd.n;
                P.phi_p = pd.phi[0];
                P.rho_p = pd.rho;
                for (int a = 0; a < 3; a++)
                    P.off[a] = ld.off[a];
                P.gmode = o.guess == MG_GUESS_USER ? (ld.guess_set ? 2 : 0) : (o.guess == MG_GUESS_ZERO ? 1 : 0);
            }
            smem = std::max(smem, mg_bottom_smem(dim, true, P.bt));
            cellsum += cells_d(ld.g[0].N, dim);
            parts.push_back(P);
        }
        tasks.push_back(T);
        work.push_back(cellsum);
    }
    std::vector<int> order(tasks.size());
    for (size_t i = 0; i < order.size(); i++)
        order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<MgPTask> sorted;
    for (int i : order)
        sorted.push_back(tasks[i]);
    int per_sm = 0;
    cudaError_t e = mg_persist_prepare(dim, smem, &per_sm);
    if (e || per_sm < 1) {
        err = fail_cuda(h, e ? e : cudaErrorInvalidConfiguration, "persistent kernel occupancy");
        return false;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t bytes = align256(parts.size() * sizeof(MgBPart)) + align256(sorted.size() * sizeof(MgPTask)) + 256;
    if (h->persist_mem)
        cudaFree(h->persist_mem);
    h->persist_mem = nullptr;
    if ((e = cudaMalloc((void **)&h->persist_mem, bytes))) {
        cudaGetLastError();
        err = fail(h, MG_ENOMEM, "cudaMalloc of %zu bytes for the persistent plan failed", bytes);
        return false;
    }
    h->pparts = (MgBPart *)h->persist_mem;
    h->ptasks = (MgPTask *)(h->persist_mem + align256(parts.size() * sizeof(MgBPart)));
    h->pnext = (unsigned *)(h->persist_mem + align256(parts.size() * sizeof(MgBPart)) +
                            align256(sorted.size() * sizeof(MgPTask)));
    h->nptasks = (int)sorted.size();
    h->psmem = smem;
    h->pgrid = std::min(h->nptasks, per_sm * nsm);
    e = cudaMemcpyAsync(h->pparts, parts.data(), parts.size() * sizeof(MgBPart), cudaMemcpyHostToDevice, h->stream);
    if (!e)
        e = cudaMemcpyAsync(h->ptasks, sorted.data(), sorted.size() * sizeof(MgPTask), cudaMemcpyHostToDevice,
                            h->stream);
    if (!e)
        e = cudaStreamSynchronize(h->stream);
    if (e) {
        err = fail_cuda(h, e, "persistent plan upload");
        return false;
    }
    return true;
}

cudaError_t capture_batched_level(mg_hierarchy *h, int l, cudaStream_t s, cudaStream_t body)
{
    const int dim = h->dim;
    const mg_options &o = h->opt;
    auto &B = h->bl[l];
    if (B.nparts == 0)
        return cudaSuccess;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (e)
        return e;
    cudaGraphConditionalHandle hc;
    if ((e = cudaGraphConditionalHandleCreate(&hc, g, 0, cudaGraphCondAssignDefault)))
        return e;
    if ((e = mg_launch_b_interface(dim, B.parts, B.cells_blk, B.ncells_blk, s)))
        return e;
    if ((e = cudaMemsetAsync(B.active, 0x01, B.nparts * sizeof(int), s)))
        return e;
    if ((e = mg_launch_b_norms2(dim, B.parts, B.cells_act, B.ncells_act, B.active, 3, s)))
        return e;
    if ((e = mg_launch_b_ctl(B.parts, B.nparts, B.active, 1, 0, o.rel_tol, o.max_cycles, hc, s)))
        return e;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd)))
        return e;
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hc;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, dv.data(), nullptr, dv.size(), &p)))
        return e;
    cudaGraph_t bodyg = p.conditional.phGraph_out[0];
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)))
        return e;
    if ((e = cudaStreamBeginCaptureToGraph(body, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
        return e;
    cudaError_t eb = mg_launch_b_defect(dim, B.parts, B.cells_act, B.ncells_act, B.active, body);
    for (int c = 0; c < o.inner_cycles && !eb; c++) {
        for (int d = 0; d < B.maxLs && !eb; d++) {
            // parts without a tile at this depth: sweeps, then residual + restriction
            for (int sw = 0; sw < o.nu_pre && !eb; sw++)
                for (int col = 0; col < 2 && !eb; col++)
                    eb = mg_launch_b_smooth(dim, B.parts, B.t_sm[d], B.n_sm[d], B.active, d, col, body);
            if (!eb)
                eb = mg_launch_b_restrict(dim, B.parts, B.t_rr[d], B.n_rr[d], B.active, d, body);
            // parts with a tile: the blocked leg
            if (!eb)
                eb = mg_launch_b_tb_pre(dim, B.parts, B.tasks[d], B.ntasks[d], B.active, d, o.nu_pre, B.smem_pre[d],
                                        body);
        }
        if (!eb)
            eb = mg_launch_b_bottom(dim, B.parts, B.nparts, B.active, o.nu_pre, o.nu_post, B.smem_bottom, body);
        for (int d = B.maxLs - 1; d >= 0 && !eb; d--) {
            if (!eb)
                eb = mg_launch_b_prolong(dim, B.parts, B.t_pr[d], B.n_pr[d], B.active, d, body);
            for (int sw = 0; sw < o.nu_post && !eb; sw++)
                for (int col = 0; col < 2 && !eb; col++)
                    eb = mg_launch_b_smooth(dim, B.parts, B.t_sm[d], B.n_sm[d], B.active, d, col, body);
            if (!eb)
                eb = mg_launch_b_tb_post(dim, B.parts, B.tasks[d], B.ntasks[d], B.active, d, o.nu_post,
                                         B.smem_post[d], body);
        }
    }
    if (!eb)
        eb = mg_launch_b_accumulate(dim, B.parts, B.cells_act, B.ncells_act, B.active, body);
    if (!eb)
        eb = mg_launch_b_norms2(dim, B.parts, B.cells_act, B.ncells_act, B.active, 2, body);
    if (!eb)
        eb = mg_launch_b_ctl(B.parts, B.nparts, B.active, 0, o.inner_cycles, o.rel_tol, o.max_cycles, hc, body);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(body, &out);
    return eb ? eb : e;
}

mg_status build_graph(mg_hierarchy *h)
{
    destroy_graph(h);
    const int nbr = std::min(h->batch, MG_BRANCHES);
    for (int i = 0; i < nbr; i++)
        if (!h->cap[i])
            CK(h, cudaStreamCreateWithFlags(&h->cap[i], cudaStreamNonBlocking));
    if (!h->body_stream)
        CK(h, cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
    if (!h->ev_fork) {
        CK(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        for (int i = 0; i < MG_BRANCHES; i++)
            CK(h, cudaEventCreateWithFlags(&h->ev_join[i], cudaEventDisableTiming));
    }
    h->batched = false;
    h->persist = false;
    choose_persistent(h);
    for (char c : h->in_persist)
        h->persist |= c != 0;
    if (h->persist) {
        mg_status perr;
        if (!plan_persistent(h, perr))
            return perr ? perr : MG_ECUDA;
        if (!h->cap_p)
            CK(h, cudaStreamCreateWithFlags(&h->cap_p, cudaStreamNonBlocking));
        if (!h->ev_pjoin)
            CK(h, cudaEventCreateWithFlags(&h->ev_pjoin, cudaEventDisableTiming));
    }
    if (h->opt.precision == MG_MIXED && h->batch > 1 && h->opt.interface == MG_IFACE_BUFFER &&
        h->opt.stop == MG_STOP_RESIDUAL && h->opt.inner_max == 0) {   // the batched kernels run fixed steps
        // measured on 64 uneven hierarchies: graph branches 105 ms, batched
        // launches 143 ms (each batched block first loads its part's
        // descriptor); MG_BATCHED=1 selects the batched launches
        const char *v = std::getenv("MG_BATCHED");
        if (v && v[0] == '1') {
            for (auto &hl : h->lev)
                for (auto &ld : hl)
                    CK(h, plan_split(ld, h->dim, 0, h->stream));
            mg_status perr;
            h->batched = plan_batched(h, perr);
            if (perr)
                return perr;
        }
    }
    if (h->batched) {
        CK(h, cudaStreamBeginCapture(h->cap[0], cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int l = 0; l < (int)h->bl.size() && !e; l++)
            e = capture_batched_level(h, l, h->cap[0], h->body_stream);
        for (int b = 0; b < h->batch && !e; b++)       // registered outputs, after the batched solve
            for (int l = 0; l < h->desc[b].num_levels && !e; l++)
                e = launch_outputs(h, h->lev[b][l], h->cap[0]);
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(h->cap[0], &g);
        if (e || ee) {
            if (g)
                cudaGraphDestroy(g);
            return fail_cuda(h, e ? e : ee, "capture of the batched solve graph");
        }
        h->graph = g;
        CK(h, cudaGraphInstantiate(&h->gexec, g, 0));
        h->graph_sig = graph_signature(h);
        return MG_OK;
    }
    CK(h, cudaStreamBeginCapture(h->cap[0], cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(h->ev_fork, h->cap[0]);
    for (int i = 1; i < nbr && !e; i++)
        e = cudaStreamWaitEvent(h->cap[i], h->ev_fork, 0);
    if (h->persist && !e) {   // its own branch: the hierarchies the persistent launch takes
        const mg_options &o = h->opt;
        e = cudaStreamWaitEvent(h->cap_p, h->ev_fork, 0);
        if (!e)
            e = cudaMemsetAsync(h->pnext, 0, sizeof(unsigned), h->cap_p);
        if (!e)
            e = mg_launch_persist(h->dim, h->pparts, h->ptasks, h->nptasks, h->pnext, h->pgrid, h->psmem, o.nu_pre,
                                  o.nu_post, o.rel_tol, o.max_cycles, o.inner_cycles,
                                  adaptive_inner(h) ? o.inner_max : 0, o.force_stencil, h->cap_p);
        if (!e)
            e = cudaEventRecord(h->ev_pjoin, h->cap_p);
    }
    int q = 0;   // graph branches, round robin over the other hierarchies
    for (int b = 0; b < h->batch && !e; b++) {
        if (h->persist && h->in_persist[b])
            continue;
        for (int l = 0; l < h->desc[b].num_levels && !e; l++)
            e = capture_level(h, b, l, h->cap[q % nbr], q % nbr);
        q++;
    }
    for (int i = 1; i < nbr && !e; i++) {
        e = cudaEventRecord(h->ev_join[i], h->cap[i]);
        if (!e)
            e = cudaStreamWaitEvent(h->cap[0], h->ev_join[i], 0);
    }
    if (h->persist && !e)
        e = cudaStreamWaitEvent(h->cap[0], h->ev_pjoin, 0);
    // registered outputs after every solve (beside the solves of other
    // levels or branches they slowed those down: batch of 64, 90 vs 84 ms);
    // the persistent launch writes its own
    for (int b = 0; b < h->batch && !e; b++)
        for (int l = 0; l < h->desc[b].num_levels && !e; l++)
            if (!(h->persist && h->in_persist[b]))
                e = launch_outputs(h, h->lev[b][l], h->cap[0]);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(h->cap[0], &g);
    if (e || ee) {
        if (g)
            cudaGraphDestroy(g);
        return fail_cuda(h, e ? e : ee, "capture of the solve graph");
    }
    h->graph = g;
    CK(h, cudaGraphInstantiate(&h->gexec, g, 0));
    h->graph_sig = graph_signature(h);
    return MG_OK;
}

mg_status solve_graph(mg_hierarchy *h, mg_level_stats *stats)
{
    if (!h->gexec || h->graph_sig != graph_signature(h)) {
        mg_status s = build_graph(h);
        if (s)
            return s;
    }
    const size_t nctl = (size_t)h->batch * MG_MAX_LEVELS;
    CK(h, cudaGraphLaunch(h->gexec, h->stream));
    CK(h, cudaMemcpyAsync(h->hctl, h->ctl, nctl * sizeof(MgSolveCtl), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    mg_status worst = MG_OK;
    for (int b = 0; b < h->batch; b++)
        for (int l = 0; l < h->desc[b].num_levels; l++) {
            mg_level_stats st{};
            fill_stats(h, h->hctl[(size_t)b * MG_MAX_LEVELS + l], &st);
            if (stats)
                stats[(size_t)b * MG_MAX_LEVELS + l] = st;
            if (st.status == MG_EDIVERGED || (st.status == MG_ENOCONV && worst == MG_OK))
                worst = (mg_status)st.status;
        }
    return worst;
}

// --------------------------------------------------------------------------
// Autotuner of the FP32 V-cycle: per distinct level size, the temporal-
// blocking tile of every multigrid level above the one-block kernel and the
// one-block kernel's size limit.  Timing runs on the level's own FP32
// correction arrays (scratch: rewritten by the next defect), so tuning does
// not disturb a solve.
// --------------------------------------------------------------------------
struct TuneEntry {
    int dim, n, nu_pre, nu_post, bottom_n;
    int tile[MG_MAX_MG];
};

// Mean time of one replay of the launches of fn, captured into a CUDA graph
// (the solve runs as a graph: timing plain launches would favour plans with
// fewer launches for the wrong reason).  With the solve graph off
// (MG_SOLVE_GRAPH=0) the launches are timed as plain launches, as the solve
// then runs them.
float time_ms(mg_hierarchy *h, int reps, const std::function<cudaError_t(cudaStream_t)> &fn, cudaError_t &err)
{
    err = cudaSuccess;
    if (!h->use_graph) {
        cudaEvent_t a = nullptr, b = nullptr;
        err = fn(h->stream);                                // warm-up
        if (!err)
            err = cudaEventCreate(&a);
        if (!err)
            err = cudaEventCreate(&b);
        if (!err)
            err = cudaEventRecord(a, h->stream);
        for (int r = 0; r < reps && !err; r++)
            err = fn(h->stream);
        if (!err)
            err = cudaEventRecord(b, h->stream);
        if (!err)
            err = cudaEventSynchronize(b);
        float ms = 0.f;
        if (!err)
            err = cudaEventElapsedTime(&ms, a, b);
        if (a)
            cudaEventDestroy(a);
        if (b)
            cudaEventDestroy(b);
        return ms / reps;
    }
    if (!h->cap[0] && (err = cudaStreamCreateWithFlags(&h->cap[0], cudaStreamNonBlocking)))
        return 0.f;
    cudaStream_t cs = h->cap[0];
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if ((err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)))
        return 0.f;
    cudaError_t ef = fn(cs);
    err = cudaStreamEndCapture(cs, &g);
    if (ef)
        err = ef;
    if (!err)
        err = cudaGraphInstantiate(&ge, g, 0);
    cudaEvent_t a = nullptr, b = nullptr;
    if (!err)
        err = cudaEventCreate(&a);
    if (!err)
        err = cudaEventCreate(&b);
    if (!err)
        err = cudaGraphLaunch(ge, h->stream);              // warm-up
    if (!err)
        err = cudaEventRecord(a, h->stream);
    for (int r = 0; r < reps && !err; r++)
        err = cudaGraphLaunch(ge, h->stream);
    if (!err)
        err = cudaEventRecord(b, h->stream);
    if (!err)
        err = cudaEventSynchronize(b);
    float ms = 0.f;
    if (!err)
        err = cudaEventElapsedTime(&ms, a, b);
    if (a)
        cudaEventDestroy(a);
    if (b)
        cudaEventDestroy(b);
    if (ge)
        cudaGraphExecDestroy(ge);
    if (g)
        cudaGraphDestroy(g);
    return ms / reps;
}

bool tune_level(mg_hierarchy *h, LevelData &ld, TuneEntry &te, cudaError_t &err)
{
    const int dim = h->dim;
    const mg_options &o = h->opt;
    te.dim = dim;
    te.n = ld.n;
    te.nu_pre = o.nu_pre;
    te.nu_post = o.nu_post;
    // 1. the bottom limit, with the default tiles
    const int nbs[3] = {4, 8, 17};
    float best = 1e30f;
    int bestnb = 8;
    for (int nb : nbs) {
        plan_bottom(ld, dim, nb);
        if ((err = refresh_bottom_plan(h, ld)))
            return false;
        plan_tiles(ld, dim, o.nu_pre, o.nu_post);
        plan_cluster(ld, h->dim, h->csize, h->opt);
        if ((err = plan_split(ld, dim, 0, h->stream)))
            return false;
        const float ms = time_ms(h, 10, [&](cudaStream_t cs) { return vcycle(h, ld, true, cs); }, err);
        if (err)
            return false;
        if (ms < best) {
            best = ms;
            bestnb = nb;
        }
    }
    plan_bottom(ld, dim, bestnb);
    if ((err = refresh_bottom_plan(h, ld)))
        return false;
    plan_cluster(ld, h->dim, h->csize, h->opt);
    if ((err = plan_split(ld, dim, 0, h->stream)))
        return false;
    te.bottom_n = bestnb;
    // 2. per level above the bottom: the tile of its pre/post pair
    const int Ls = ld.Ls[1];
    for (int L = 0; L < MG_MAX_MG; L++)
        te.tile[L] = 0;
    for (int L = 0; L < Ls; L++) {
        float bl = 1e30f;
        int bt = 0;
        std::vector<int> cands = {0, 8, 12, 16};
        if (wave_ok(dim, o.nu_pre, o.nu_post, ld.g[L].N)) {
            // plane-marching sweeps: both tiles, z-chunks around the default
            const int N = ld.g[L].N;
            const int zd = wave_zchunks(wave_default(N));
            for (int v = 0; v < 2; v++)
                for (int zc : {std::max(1, zd / 2), zd, std::min(2 * zd, std::max(1, N / 4))})
                    if (std::find(cands.begin(), cands.end(), wave_code(v, zc)) == cands.end())
                        cands.push_back(wave_code(v, zc));
        }
        for (int t : cands) {
            if (t > 0 && (mg_tb_smem(dim, true, t, 2 * o.nu_pre + 1) > MG_TB_SMEM_MAX ||
                          mg_tb_smem(dim, true, t, 2 * o.nu_post) > MG_TB_SMEM_MAX))
                continue;
            ld.tile[L] = t;
            const float ms = time_ms(h, 10, [&](cudaStream_t s) {
                cudaError_t e;
                if (t < 0) {
                    e = mg_launch_wave(ld.phi32[L], ld.phi32b[L], ld.f32[L], ld.g[L], o.nu_pre, wave_variant(t),
                                       wave_zchunks(t), s, nullptr, 0, h->werr, h->wfault);
                    if (!e)
                        e = mg_launch_resid_restrict(dim, true, ld.phi32b[L], ld.f32[L], ld.g[L], ld.phi32[L + 1],
                                                     ld.f32[L + 1], ld.g[L + 1], s);
                    if (!e)
                        e = mg_launch_prolong(dim, true, ld.phi32[L + 1], ld.g[L + 1], ld.phi32b[L], ld.g[L], s);
                    if (!e)
                        e = mg_launch_wave(ld.phi32b[L], ld.phi32[L], ld.f32[L], ld.g[L], o.nu_post, wave_variant(t),
                                           wave_zchunks(t), s, nullptr, 0, h->werr, h->wfault);
                    return e;
                }
                if (t) {
                    e = mg_launch_tb_pre(dim, ld.phi32[L], ld.phi32b[L], ld.f32[L], ld.g[L], ld.phi32[L + 1],
                                         ld.f32[L + 1], ld.g[L + 1], t, o.nu_pre, s);
                    if (!e)
                        e = mg_launch_tb_post(dim, ld.phi32b[L], ld.phi32[L], ld.f32[L], ld.g[L], ld.phi32[L + 1],
                                              ld.g[L + 1], t, o.nu_post, s);
                    return e;
                }
                for (int sw = 0; sw < o.nu_pre; sw++)
                    for (int c = 0; c < 2; c++)
                        if ((e = mg_launch_smooth(dim, true, ld.phi32[L], ld.f32[L], ld.g[L], c, s)))
                            return e;
                if ((e = mg_launch_resid_restrict(dim, true, ld.phi32[L], ld.f32[L], ld.g[L], ld.phi32[L + 1],
                                                  ld.f32[L + 1], ld.g[L + 1], s)))
                    return e;
                if ((e = mg_launch_prolong(dim, true, ld.phi32[L + 1], ld.g[L + 1], ld.phi32[L], ld.g[L], s)))
                    return e;
                for (int sw = 0; sw < o.nu_post; sw++)
                    for (int c = 0; c < 2; c++)
                        if ((e = mg_launch_smooth(dim, true, ld.phi32[L], ld.f32[L], ld.g[L], c, s)))
                            return e;
                return cudaSuccess;
            }, err);
            if (err)
                return false;
            if (ms < bl) {
                bl = ms;
                bt = t;
            }
        }
        ld.tile[L] = bt;
        te.tile[L] = bt;
    }
    for (int L = Ls; L < ld.nmg; L++)
        ld.tile[L] = 0;
    // 3. how many leading levels run colour-split (their tiles give way)
    if (ld.Lc[1] < 0 && !ld.frozen) {
        int tiles[MG_MAX_MG];
        std::copy(ld.tile, ld.tile + MG_MAX_MG, tiles);
        float bs = 1e30f;
        int bestS = 0;
        for (int S = 0; S <= Ls; S++) {
            std::copy(tiles, tiles + MG_MAX_MG, ld.tile);
            if ((err = plan_split(ld, dim, S, h->stream)))
                return false;
            const float ms = time_ms(h, 10, [&](cudaStream_t cs) { return vcycle(h, ld, true, cs); }, err);
            if (err)
                return false;
            if (ms < bs) {
                bs = ms;
                bestS = S;
            }
        }
        std::copy(tiles, tiles + MG_MAX_MG, ld.tile);
        if ((err = plan_split(ld, dim, bestS, h->stream)))
            return false;
        for (int L = 0; L < bestS; L++)
            te.tile[L] = kTileSplit;
    }
    return true;
}

cudaError_t apply_entry(mg_hierarchy *h, LevelData &ld, const TuneEntry &te)
{
    plan_bottom(ld, h->dim, te.bottom_n);
    cudaError_t e = refresh_bottom_plan(h, ld);
    int S = 0;
    while (S < ld.Ls[1] && te.tile[S] == kTileSplit)
        S++;
    for (int L = 0; L < ld.nmg; L++)
        ld.tile[L] = L < ld.Ls[1] && te.tile[L] != kTileSplit ? te.tile[L] : 0;
    plan_cluster(ld, h->dim, h->csize, h->opt);
    if (!e)
        e = plan_split(ld, h->dim, S, h->stream);
    return e;
}

std::vector<TuneEntry> read_cache(const char *path)
{
    std::vector<TuneEntry> v;
    if (!path)
        return v;
    FILE *fp = std::fopen(path, "r");
    if (!fp)
        return v;
    char line[512];
    while (std::fgets(line, sizeof line, fp)) {
        TuneEntry te{};
        int pos = 0;
        if (line[0] == '#' || std::sscanf(line, "%d %d %d %d %d%n", &te.dim, &te.n, &te.nu_pre, &te.nu_post,
                                          &te.bottom_n, &pos) != 5)
            continue;
        for (int L = 0; L < MG_MAX_MG; L++) {
            int used = 0;
            if (std::sscanf(line + pos, "%d%n", &te.tile[L], &used) != 1)
                break;
            pos += used;
        }
        v.push_back(te);
    }
    std::fclose(fp);
    return v;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

mg_status mg_default_options(mg_options *opt)
{
    if (!opt)
        return MG_EINVAL;
    opt->nu_pre = 2;
    opt->nu_post = 1;
    opt->max_cycles = 50;
    opt->rel_tol = 1e-10;
    opt->precision = MG_FP64;
    opt->inner_cycles = 3;
    opt->inner_max = 0;
    opt->guess = MG_GUESS_INTERP;
    opt->force_stencil = MG_FORCE_EQ2;
    opt->interface = MG_IFACE_BUFFER;
    opt->stop = MG_STOP_RESIDUAL;
    opt->stream = nullptr;
    return MG_OK;
}

int mg_level_sizes(int M, int *N, int cap)
{
    if (M < 1 || !N || cap < 1)
        return 0;
    return level_sizes(M, N, cap);
}

const char *mg_status_str(mg_status s)
{
    switch (s) {
    case MG_OK: return "MG_OK";
    case MG_EINVAL: return "MG_EINVAL: invalid argument";
    case MG_ENOMEM: return "MG_ENOMEM: out of memory";
    case MG_ECUDA: return "MG_ECUDA: CUDA error";
    case MG_ESTATE: return "MG_ESTATE: call out of order or handle poisoned";
    case MG_ENOCONV: return "MG_ENOCONV: not converged within max_cycles";
    case MG_EDIVERGED: return "MG_EDIVERGED: residual not finite";
    case MG_ETIMEOUT: return "MG_ETIMEOUT: device wait timed out";
    }
    return "unknown mg_status";
}

const char *mg_error_message(const mg_hierarchy *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

mg_status mg_create_hierarchy(const mg_hierarchy_desc *descs, int batch, const mg_options *opt, mg_hierarchy **out)
{
    g_create_error.clear();
    if (!out)
        return fail(nullptr, MG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!descs || batch < 1)
        return fail(nullptr, MG_EINVAL, "descs is NULL or batch < 1");
    mg_options o;
    mg_default_options(&o);
    if (opt)
        o = *opt;
    if (check_options(o))
        return fail(nullptr, MG_EINVAL, "invalid options");
    for (int b = 0; b < batch; b++) {
        mg_status s = check_desc(descs[b], b, descs[0].dim);
        if (s)
            return s;
    }
    mg_hierarchy *h = new (std::nothrow) mg_hierarchy();
    if (!h)
        return fail(nullptr, MG_ENOMEM, "host allocation failed");
    h->batch = batch;
    h->dim = descs[0].dim;
    h->desc.assign(descs, descs + batch);
    h->opt = o;
    h->stream = (cudaStream_t)o.stream;
    const int dim = h->dim;
    if (h->stream) {
        // run on the device the caller's stream belongs to
        int sd = -1;
        if (cudaStreamGetDevice(h->stream, &sd) == cudaSuccess && sd >= 0)
            cudaSetDevice(sd);
        cudaGetLastError();
    }
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, MG_ECUDA, "no CUDA device");
    }

    // geometry and arena layout
    h->lev.resize(batch);
    size_t bytes = 0, stage = 0;
    struct Slot { void **dst; size_t bytes; };
    std::vector<Slot> slots;
    for (int b = 0; b < batch; b++) {
        const mg_hierarchy_desc &d = descs[b];
        h->lev[b].resize(d.num_levels);
        for (int l = 0; l < d.num_levels; l++) {
            LevelData &ld = h->lev[b][l];
            ld.n = d.n[l];
            ld.h = d.h0 / (double)(1L << desc_depth(d, l));
            ld.frozen = l > 0 && o.interface == MG_IFACE_FROZEN;
            if (l > 0) {
                ld.parent = desc_parent(d, l);
                const double hp = d.h0 / (double)(1L << desc_depth(d, ld.parent));
                for (int a = 0; a < dim; a++)
                    ld.off[a] = (int)std::floor((d.lo[l][a] - d.lo[ld.parent][a]) / hp + 0.5);
            }
            build_geometry(ld, dim);
            for (int L = 0; L < ld.nmg; L++) {
                const size_t c = (size_t)cells(ld.g[L].E, dim);
                slots.push_back({(void **)&ld.phi[L], align256(c * sizeof(double))});
                slots.push_back({(void **)&ld.f[L], align256(c * sizeof(double))});
                if (o.precision == MG_MIXED) {   // room for the plain and the colour-split layout
                    const size_t c32 = mg_fp32_cells(ld.g[L].E, dim);
                    slots.push_back({(void **)&ld.phi32[L], align256(c32 * sizeof(float))});
                    slots.push_back({(void **)&ld.phi32b[L], align256(c32 * sizeof(float))});
                    slots.push_back({(void **)&ld.f32[L], align256(c32 * sizeof(float))});
                }
            }
            for (int L = 1; L < ld.nmg; L++) {
                slots.push_back({(void **)&ld.tab64[L], align256(128 * sizeof(double))});
                slots.push_back({(void **)&ld.tab32[L], align256(128 * sizeof(float))});
            }
            ld.bplan_bytes = max_bottom_plan_bytes(ld, dim, o.precision == MG_MIXED);
            if (ld.bplan_bytes)
                slots.push_back({(void **)&ld.bplan, align256(ld.bplan_bytes)});
            if (o.stop == MG_STOP_FORCE)
                slots.push_back({(void **)&ld.prev, align256((size_t)cells(ld.n + 4, dim) * sizeof(double))});
            if (ld.frozen) {
                slots.push_back({(void **)&ld.blk, align256((size_t)cells(ld.n + 4, dim) * sizeof(double))});
                slots.push_back({(void **)&ld.fblk, align256((size_t)cells(ld.n + 4, dim) * sizeof(double))});
            }
            slots.push_back({(void **)&ld.rho, align256((size_t)cells(ld.n + 4, dim) * sizeof(double))});
            slots.push_back({(void **)&ld.guess, align256((size_t)cells(ld.n + 2, dim) * sizeof(double))});
            const size_t st = std::max((size_t)cells(ld.n + 4, dim) * 3, (size_t)cells(ld.n, dim) * (dim + 1));
            stage = std::max(stage, st);
        }
    }
    h->stage_elems = stage;
    slots.push_back({(void **)&h->stage, align256(stage * sizeof(double))});
    slots.push_back({(void **)&h->partials, align256((size_t)MG_BRANCHES * 2 * MG_NORM_BLOCKS_MAX * sizeof(double))});
    slots.push_back({(void **)&h->counters, align256((size_t)MG_BRANCHES * sizeof(unsigned))});
    slots.push_back({(void **)&h->fmax, align256((size_t)MG_BRANCHES * sizeof(unsigned long long))});
    slots.push_back({(void **)&h->ctl, align256((size_t)batch * MG_MAX_LEVELS * sizeof(MgSolveCtl))});
    slots.push_back({(void **)&h->frho, align256((size_t)batch * MG_MAX_LEVELS * sizeof(double))});
    slots.push_back({(void **)&h->scal, align256((size_t)batch * MG_MAX_LEVELS * 2 * sizeof(double))});
    slots.push_back({(void **)&h->werr, align256(sizeof(int))});
    for (auto &sl : slots)
        bytes += sl.bytes;
    cudaError_t e = cudaMalloc((void **)&h->arena, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, MG_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    h->arena_bytes = bytes;
    size_t pos = 0;
    for (auto &sl : slots) {
        *sl.dst = h->arena + pos;
        pos += sl.bytes;
    }
    for (auto &hl : h->lev)
        for (auto &ld : hl)
            if (!ld.frozen) {
                ld.blk = ld.phi[0];
                ld.fblk = ld.f[0];
            }
    e = cudaMallocHost((void **)&h->hscal, (size_t)batch * MG_MAX_LEVELS * 2 * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&h->hctl, (size_t)batch * MG_MAX_LEVELS * sizeof(MgSolveCtl));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->hscal)
            cudaFreeHost(h->hscal);
        cudaFree(h->arena);
        delete h;
        return fail(nullptr, MG_ENOMEM, "pinned host allocation failed");
    }
    {
        const char *v = std::getenv("MG_SOLVE_GRAPH");
        h->use_graph = !(v && v[0] == '0');
        const char *fw = std::getenv("MG_FAULT_WAVE_WAIT");
        h->wfault = fw && fw[0] == '1';
    }
    // ghost layers and rings start at zero
    e = mg_bottom_prepare();
    if (e == cudaSuccess)
        e = mg_tb_prepare();
    if (e == cudaSuccess)
        e = mg_wave_prepare();
    if (e == cudaSuccess)
        e = mg_batch_prepare();
    if (e == cudaSuccess)
        h->csize = mg_cluster_prepare();
    if (e == cudaSuccess)
        e = mg_launch_zero(h->arena, bytes, h->stream);
    if (e == cudaSuccess)   // the table copies below do not run on the caller's stream
        e = cudaStreamSynchronize(h->stream);
    // boundary-diagonal tables of the coarse multigrid levels, then the plan
    // of the one-block kernel (which copies the level descriptions) and its
    // image
    for (int b = 0; b < batch && e == cudaSuccess; b++)
        for (auto &ld : h->lev[b]) {
            for (int L = 1; L < ld.nmg && e == cudaSuccess; L++) {
                double t64[128];
                float t32[128];
                mg_fill_diag_table(ld.g[L], dim, t64);
                for (int c = 0; c < 128; c++)
                    t32[c] = (float)t64[c];
                e = cudaMemcpy(ld.tab64[L], t64, sizeof t64, cudaMemcpyHostToDevice);
                if (e == cudaSuccess)
                    e = cudaMemcpy(ld.tab32[L], t32, sizeof t32, cudaMemcpyHostToDevice);
                ld.g[L].tab64 = ld.tab64[L];
                ld.g[L].tab32 = ld.tab32[L];
            }
            plan_bottom(ld, dim);
            if (e == cudaSuccess)
                e = refresh_bottom_plan(h, ld);
            plan_tiles(ld, dim, o.nu_pre, o.nu_post);
            plan_cluster(ld, h->dim, h->csize, h->opt);
            if (e == cudaSuccess && o.precision == MG_MIXED)
                e = plan_split(ld, dim, split_default(ld), h->stream);
        }
    if (e == cudaSuccess) {
        std::vector<double> fr((size_t)batch * MG_MAX_LEVELS, 0.0);
        for (int b = 0; b < batch; b++)
            for (int l = 0; l < descs[b].num_levels; l++) {
                const double hl = h->lev[b][l].h;
                fr[(size_t)b * MG_MAX_LEVELS + l] = 4.0 * M_PI * descs[b].G * hl * hl;
            }
        e = cudaMemcpy(h->frho, fr.data(), fr.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(h->hscal);
        cudaFreeHost(h->hctl);
        cudaFree(h->arena);
        delete h;
        return fail(nullptr, MG_ECUDA, "arena initialisation failed: %s", cudaGetErrorString(e));
    }
    *out = h;
    return MG_OK;
}

mg_status mg_set_density(mg_hierarchy *h, int b, int level, const double *rho, const double *bc_rho,
                         const double *bc_phi)
{
    if (!h)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (b < 0 || b >= h->batch || level < 0 || level >= h->desc[b].num_levels)
        return fail(h, MG_EINVAL, "hierarchy %d level %d out of range", b, level);
    if (!rho)
        return fail(h, MG_EINVAL, "rho is NULL");
    if (level == 0 && (!bc_rho || !bc_phi))
        return fail(h, MG_EINVAL, "level 0 needs bc_rho and bc_phi");
    if (level > 0 && (bc_rho || bc_phi))
        return fail(h, MG_EINVAL, "bc_rho/bc_phi must be NULL above level 0 (the interface fills them)");
    LevelData &ld = h->lev[b][level];
    const int dim = h->dim;
    const size_t nr = (size_t)cells(ld.n, dim), nb = (size_t)cells(ld.n + 2, dim), np = (size_t)cells(ld.n + 4, dim);
    const double *d_rho = rho, *d_bcr = bc_rho, *d_bcp = bc_phi;
    double *stage = h->stage;
    bool host_in = false;
    // host arrays: read in place by the kernel when mapped (page-locked),
    // else copied to the staging area first
    auto take = [&](const double *src, const double *&dst, double *st, size_t count) -> cudaError_t {
        if (is_device_ptr(src))
            return cudaSuccess;
        host_in = true;
        if (const double *m = mapped_host_view(src)) {
            dst = m;
            return cudaSuccess;
        }
        dst = st;
        return cudaMemcpyAsync(st, src, count * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    };
    CK(h, take(rho, d_rho, stage, nr));
    if (level == 0) {
        CK(h, take(bc_rho, d_bcr, stage + np, nb));
        CK(h, take(bc_phi, d_bcp, stage + 2 * np, np));
    }
    const double fourpiG = 4.0 * M_PI * h->desc[b].G;
    CK(h, timed(h, KK_SETDENS, 24.0 * (double)nr, [&] {
           return mg_launch_set_density(dim, ld.n, d_rho, d_bcr, d_bcp, ld.rho, ld.fblk, ld.blk, fourpiG,
                                        h->stream);
       }));
    if (host_in)   // the caller may reuse its host arrays (and the staging area is reused) on return
        CK(h, cudaStreamSynchronize(h->stream));
    ld.density_set = true;
    ld.guess_set = false;
    h->solved = false;
    return MG_OK;
}

mg_status mg_set_guess(mg_hierarchy *h, int b, int level, const double *phi0)
{
    if (!h)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (b < 0 || b >= h->batch || level < 0 || level >= h->desc[b].num_levels || !phi0)
        return fail(h, MG_EINVAL, "bad hierarchy/level or NULL phi0");
    LevelData &ld = h->lev[b][level];
    if (!ld.density_set)
        return fail(h, MG_ESTATE, "mg_set_guess before mg_set_density");
    const size_t nb = (size_t)cells(ld.n + 2, h->dim);
    CK(h, cudaMemcpyAsync(ld.guess, phi0, nb * sizeof(double), cudaMemcpyDefault, h->stream));
    if (!is_device_ptr(phi0))
        CK(h, cudaStreamSynchronize(h->stream));
    ld.guess_set = true;
    return MG_OK;
}

mg_status mg_solve(mg_hierarchy *h, mg_level_stats *stats)
{
    if (!h)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    for (int b = 0; b < h->batch; b++)
        for (int l = 0; l < h->desc[b].num_levels; l++)
            if (!h->lev[b][l].density_set)
                return fail(h, MG_ESTATE, "density of hierarchy %d level %d not set", b, l);
    mg_status worst = MG_OK;
    if (!h->prof.on && h->use_graph) {
        worst = solve_graph(h, stats);
        if (worst == MG_ECUDA || worst == MG_ETIMEOUT)
            return worst;
    } else {
        for (int b = 0; b < h->batch; b++)
            for (int l = 0; l < h->desc[b].num_levels; l++) {
                mg_level_stats st{};
                mg_status s = solve_level_host(h, b, l, &st);
                if (s == MG_ECUDA || s == MG_ETIMEOUT)
                    return s;
                if (stats)
                    stats[(size_t)b * MG_MAX_LEVELS + l] = st;
                if (s == MG_EDIVERGED || (s == MG_ENOCONV && worst == MG_OK))
                    worst = s;
            }
        CK(h, cudaStreamSynchronize(h->stream));   // registered outputs complete on return
    }
    if (mg_status ws = wave_status(h))
        return ws;
    h->solved = true;
    return worst;
}

mg_status mg_set_outputs(mg_hierarchy *h, int b, int level, double *phi_out, double *F_out)
{
    if (!h)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (b < 0 || b >= h->batch || level < 0 || level >= h->desc[b].num_levels)
        return fail(h, MG_EINVAL, "hierarchy %d level %d out of range", b, level);
    if (!F_out && phi_out)
        return fail(h, MG_EINVAL, "a potential output needs a force output");
    auto usable = [](double *p) -> double * {
        if (!p)
            return nullptr;
        if (is_device_ptr(p))
            return p;
        return mapped_host_view(p);   // page-locked host memory, else NULL
    };
    double *F = usable(F_out), *P = usable(phi_out);
    if ((F_out && !F) || (phi_out && !P))
        return fail(h, MG_EINVAL, "outputs must be device memory or page-locked host memory");
    LevelData &ld = h->lev[b][level];
    ld.out_F = F;
    ld.out_phi = P;
    return MG_OK;
}

mg_status mg_forces(mg_hierarchy *h, int b, int level, double *phi_out, double *F_out)
{
    if (!h)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (b < 0 || b >= h->batch || level < 0 || level >= h->desc[b].num_levels)
        return fail(h, MG_EINVAL, "hierarchy %d level %d out of range", b, level);
    if (!h->solved)
        return fail(h, MG_ESTATE, "mg_forces before mg_solve");
    const LevelData &ld = h->lev[b][level];
    const int dim = h->dim;
    const size_t nr = (size_t)cells(ld.n, dim);
    // device arrays and mapped page-locked host arrays are written by the
    // kernel itself; other host arrays get a copy from the staging area
    double *mF = F_out && !is_device_ptr(F_out) ? mapped_host_view(F_out) : nullptr;
    double *mP = phi_out && !is_device_ptr(phi_out) ? mapped_host_view(phi_out) : nullptr;
    const bool phi_dev = phi_out && (mP || is_device_ptr(phi_out));
    const bool F_dev = F_out && (mF || is_device_ptr(F_out));
    double *dF = F_out ? (F_dev ? (mF ? mF : F_out) : h->stage) : nullptr;
    double *dP = phi_out ? (phi_dev ? (mP ? mP : phi_out) : h->stage + (size_t)dim * nr) : nullptr;
    if (!dF) {
        // potential only: the kernel still needs somewhere to write forces
        dF = h->stage;
        if (phi_out && !phi_dev)
            dP = h->stage + (size_t)dim * nr;
    }
    CK(h, timed(h, KK_FORCES, 8.0 * (cells_d(ld.n + 4, dim) + (dim + 1) * (double)nr), [&] {
           return mg_launch_forces(dim, ld.n, ld.h, ld.blk, dF, dP, h->opt.force_stencil, h->stream);
       }));
    bool sync = false;
    if (F_out && !F_dev) {
        CK(h, cudaMemcpyAsync(F_out, dF, (size_t)dim * nr * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        sync = true;
    }
    if (phi_out && !phi_dev) {
        CK(h, cudaMemcpyAsync(phi_out, dP, nr * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        sync = true;
    }
    if (mF || mP)
        sync = true;   // host memory written by the kernel: complete before returning
    if (sync)
        CK(h, cudaStreamSynchronize(h->stream));
    return MG_OK;
}

mg_status mg_profile(mg_hierarchy *h, int enable)
{
    if (!h)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    CK(h, profile_flush(h));
    Profiler &P = h->prof;
    P.on = enable != 0;
    for (int k = 0; k < KK_COUNT; k++) {
        P.launches[k] = 0;
        P.ms[k] = 0.0;
        P.bytes[k] = 0.0;
    }
    return MG_OK;
}

int mg_profile_read(mg_hierarchy *h, mg_kernel_stat *out, int cap)
{
    if (!h || h->poisoned || profile_flush(h) != cudaSuccess)
        return -1;
    int k = 0;
    for (int i = 0; i < KK_COUNT && k < cap; i++) {
        if (!h->prof.launches[i])
            continue;
        if (out) {
            std::snprintf(out[k].name, sizeof out[k].name, "%s", kKindName[i]);
            out[k].launches = h->prof.launches[i];
            out[k].ms = h->prof.ms[i];
            out[k].bytes = h->prof.bytes[i];
        }
        k++;
    }
    return k;
}

mg_status mg_set_unet(mg_hierarchy *h, struct mg_unet *net)
{
    if (!h)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (net && mg_unet_pack(net) != 0)
        return fail(h, MG_ECUDA, "packing the network weights failed");
    h->unet = net;
    destroy_graph(h);
    return MG_OK;
}

mg_status mg_interp_guess(mg_hierarchy *h, int b, int level, double *out, double *resid_out)
{
    if (!h || !out)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (b < 0 || b >= h->batch || level < 1 || level >= h->desc[b].num_levels)
        return fail(h, MG_EINVAL, "hierarchy %d level %d: need 1 <= level < num_levels", b, level);
    if (!h->solved)
        return fail(h, MG_ESTATE, "mg_interp_guess before mg_solve");
    LevelData &ld = h->lev[b][level];
    const LevelData &pd = h->lev[b][ld.parent];
    const int dim = h->dim;
    const size_t nr = (size_t)cells(ld.n, dim), nb = (size_t)cells(ld.n + 4, dim);
    double *blk = h->stage, *dense = h->stage + nb, *dres = h->stage + nb + nr;
    // the interface rewrites the inner-ring density and f with the values it
    // already holds; the potential goes to the staging block
    const double fourpiG = 4.0 * M_PI * h->desc[b].G;
    CK(h, mg_launch_interface(dim, pd.n, pd.blk, pd.rho, ld.n, ld.off[0], ld.off[1], ld.off[2], blk, ld.rho,
                              ld.fblk, fourpiG, 0, nullptr, ld.frozen, h->stream));
    const bool dev = is_device_ptr(out);
    CK(h, mg_launch_extract(dim, ld.n, blk, dev ? out : dense, h->stream));
    if (!dev)
        CK(h, cudaMemcpyAsync(out, dense, nr * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (resid_out) {
        const bool rdev = is_device_ptr(resid_out);
        CK(h, mg_launch_resid_h2(dim, ld.n, blk, ld.rho, fourpiG * ld.h * ld.h, rdev ? resid_out : dres, h->stream));
        if (!rdev)
            CK(h, cudaMemcpyAsync(resid_out, dres, nr * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return MG_OK;
}

mg_status mg_autotune(mg_hierarchy *h, const char *cache_path)
{
    if (!h)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (h->opt.precision != MG_MIXED)
        return MG_OK;                 // the FP64 path has nothing to tune
    std::vector<TuneEntry> cache = read_cache(cache_path);
    std::vector<TuneEntry> fresh;
    for (int b = 0; b < h->batch; b++)
        for (auto &ld : h->lev[b]) {
            if (ld.frozen)
                continue;             // the ablation keeps the default plan
            const TuneEntry *hit = nullptr;
            for (auto *v : {&cache, &fresh})
                for (auto &te : *v)
                    if (te.dim == h->dim && te.n == ld.n && te.nu_pre == h->opt.nu_pre &&
                        te.nu_post == h->opt.nu_post)
                        hit = &te;
            if (hit) {
                if (cudaError_t e = apply_entry(h, ld, *hit))
                    return fail_cuda(h, e, "bottom plan");
                continue;
            }
            TuneEntry te{};
            cudaError_t e = cudaSuccess;
            if (!tune_level(h, ld, te, e))
                return fail_cuda(h, e, "autotune timing");
            fresh.push_back(te);
        }
    if (cache_path && !fresh.empty()) {
        FILE *fp = std::fopen(cache_path, "a");
        if (fp) {
            for (auto &te : fresh) {
                std::fprintf(fp, "%d %d %d %d %d", te.dim, te.n, te.nu_pre, te.nu_post, te.bottom_n);
                for (int L = 0; L < MG_MAX_MG; L++)
                    std::fprintf(fp, " %d", te.tile[L]);
                std::fprintf(fp, "\n");
            }
            std::fclose(fp);
        }
    }
    destroy_graph(h);                 // the solve graph is rebuilt with the new plan
    return wave_status(h);
}

mg_status mg_time_smoothing(mg_hierarchy *h, int b, int level, int L, int launches, double *us_per_launch,
                            double *bytes_per_launch)
{
    if (!h || !us_per_launch || !bytes_per_launch)
        return MG_EINVAL;
    if (h->poisoned)
        return fail(h, MG_ESTATE, "handle poisoned by an earlier CUDA error");
    if (h->opt.precision != MG_MIXED)
        return fail(h, MG_EINVAL, "mg_time_smoothing times the FP32 plan of MG_MIXED");
    if (b < 0 || b >= h->batch || level < 0 || level >= h->desc[b].num_levels)
        return fail(h, MG_EINVAL, "hierarchy %d level %d out of range", b, level);
    LevelData &ld = h->lev[b][level];
    if (L < 0 || L >= ld.Ls[1] || ld.Lc[1] >= 0 || launches < 1 || launches > 4096)
        return fail(h, MG_EINVAL, "multigrid level %d is not run by per-level launches, or launches %d out of 1..4096",
                    L, launches);
    const int dim = h->dim, code = ld.tile[L];
    if (code > 0)
        return fail(h, MG_EINVAL, "multigrid level %d runs the temporally blocked legs", L);
    const mg_options &o = h->opt;
    cudaError_t err = cudaSuccess;
    const float ms = time_ms(h, 5, [&](cudaStream_t s) {
        cudaError_t e = cudaSuccess;
        for (int r = 0; r < launches && !e; r++) {
            if (code < 0) {
                const bool fwd = (r & 1) == 0;
                e = mg_launch_wave(fwd ? ld.phi32[L] : ld.phi32b[L], fwd ? ld.phi32b[L] : ld.phi32[L], ld.f32[L],
                                   ld.g[L], o.nu_pre, wave_variant(code), wave_zchunks(code), s, nullptr, 0,
                                   h->werr, h->wfault);
            } else if (L < ld.nsplit) {
                e = mg_split_colour(dim, ld.phi32[L], ld.f32[L], ld.g[L], r & 1, s);
            } else {
                e = mg_launch_smooth(dim, true, ld.phi32[L], ld.f32[L], ld.g[L], r & 1, s);
            }
        }
        return e;
    }, err);
    if (err)
        return fail_cuda(h, err, "smoothing timing");
    if (mg_status ws = wave_status(h))
        return ws;
    const double nc = cells_d(ld.g[L].N, dim);
    *us_per_launch = 1e3 * (double)ms / launches;
    *bytes_per_launch = (code < 0 ? 3.0 : 1.5) * sizeof(float) * nc;
    return MG_OK;
}

int mg_persistent_count(const mg_hierarchy *h)
{
    if (!h || !h->gexec)
        return -1;
    int k = 0;
    if (h->persist)
        for (char c : h->in_persist)
            k += c != 0;
    return k;
}

int mg_tuning(const mg_hierarchy *h, int b, int level, int *tiles, int cap)
{
    if (!h || b < 0 || b >= h->batch || level < 0 || level >= h->desc[b].num_levels || !tiles)
        return -1;
    const LevelData &ld = h->lev[b][level];
    for (int L = 0; L < cap && L < ld.nmg; L++)
        tiles[L] = L < ld.nsplit ? kTileSplit : ld.tile[L];
    return ld.g[ld.Ls[1]].N;
}

mg_status mg_destroy(mg_hierarchy *h)
{
    if (!h)
        return MG_OK;
    if (h->arena) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->arena);
    }
    for (cudaEvent_t e : h->prof.pool)
        cudaEventDestroy(e);
    destroy_graph(h);
    if (h->persist_mem)
        cudaFree(h->persist_mem);
    if (h->cap_p)
        cudaStreamDestroy(h->cap_p);
    if (h->ev_pjoin)
        cudaEventDestroy(h->ev_pjoin);
    if (h->batch_mem)
        cudaFree(h->batch_mem);
    for (int i = 0; i < MG_BRANCHES; i++) {
        if (h->cap[i])
            cudaStreamDestroy(h->cap[i]);
        if (h->ev_join[i])
            cudaEventDestroy(h->ev_join[i]);
    }
    if (h->body_stream)
        cudaStreamDestroy(h->body_stream);
    if (h->inner_stream)
        cudaStreamDestroy(h->inner_stream);

    if (h->ev_fork)
        cudaEventDestroy(h->ev_fork);
    if (h->hscal)
        cudaFreeHost(h->hscal);
    if (h->hctl)
        cudaFreeHost(h->hctl);
    cudaGetLastError();
    delete h;
    return MG_OK;
}

}  // extern "C"
