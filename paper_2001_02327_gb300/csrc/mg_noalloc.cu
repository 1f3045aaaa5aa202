// mg_noalloc.cu -- mg_solve_level_noalloc: a single-level FP64 solve that
// allocates no memory.  For callers that cannot call cudaMalloc: code that
// hands all of the device's memory to its own pool, or runs the Poisson solve
// inside a time step where an allocation (and the device-wide
// synchronisation cudaMalloc/cudaFree imply) is not allowed.  Its working
// arrays live in one file-scope device array (kNoAllocScratchBytes); the
// caller passes the density and the potential.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 4u << 20;   // 4 MiB: 3D n <= 69, 2D n <= 554 (the byte count below decides)

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
size_t ncells(int e, int dim) { return dim == 3 ? (size_t)e * e * e : (size_t)e * e; }

}  // namespace

// The working memory: the right-hand side of the finest multigrid level, the
// potential and right-hand side of every coarser multigrid level, and the
// norm reduction scratch.  Every GPU that loads this library holds it until
// the process exits.  Host code must not use this name as an address: the
// device address comes from cudaGetSymbolAddress (scratch_address below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_scratch_mtx;
std::vector<std::pair<int, unsigned char *>> g_scratch_addr;   // (device, address)

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (with that device current) and then cached.
cudaError_t scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lk(g_scratch_mtx);
    for (auto &p : g_scratch_addr)
        if (p.first == dev) {
            *out = p.second;
            return cudaSuccess;
        }
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
        return e;
    g_scratch_addr.push_back({dev, (unsigned char *)ptr});
    *out = (unsigned char *)ptr;
    return cudaSuccess;
}

// f = 4 pi G rho on the solved region Gamma of an (n+4)^d block, zero elsewhere.
template <int DIM>
__global__ void k_rhs_from_block(int n, const double *__restrict__ rho, double *__restrict__ f, double fourpiG)
{
    const int E = n + 4;
    const long total = (long)E * E * (DIM == 3 ? E : 1);
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t % E), j = (int)((t / E) % E), k = DIM == 3 ? (int)(t / ((long)E * E)) : 1;
        const bool gamma = i >= 1 && i <= n + 2 && j >= 1 && j <= n + 2 && k >= 1 && k <= n + 2;
        f[t] = gamma ? fourpiG * rho[t] : 0.0;
    }
}

// Sec. 2.2 level sizes and the Sec. 2.4 ghost factor for a solved region of M cells.
int geometry(int M, double h, MgGeom *g)
{
    int N[MG_MAX_MG];
    int L = 0;
    N[0] = M;
    while (N[L] > 1 && L + 1 < MG_MAX_MG) {
        L++;
        N[L] = (int)(((long)M + (1L << (L - 1))) >> L);
    }
    const int nmg = L + 1;
    for (int q = 0; q < nmg; q++) {
        g[q].tab64 = nullptr;   // boundary diagonals computed in place
        g[q].tab32 = nullptr;
        g[q].N = N[q];
        g[q].E = N[q] + 2;
        g[q].L = q;
        const long num = 2L * M - (2L * N[q] + 1) * (1L << q);
        const long den = 2L * M - (2L * N[q] - 1) * (1L << q);
        g[q].tie = den == 0;
        g[q].cR = g[q].tie ? 0.0 : (double)num / (double)den;
        const double hq = h * (double)(1L << q);
        g[q].h2 = hq * hq;
        g[q].inv_h2 = 1.0 / g[q].h2;
        g[q].cRf = (float)g[q].cR;
        g[q].h2f = (float)g[q].h2;
        g[q].inv_h2f = (float)g[q].inv_h2;
    }
    return nmg;
}

cudaError_t smooth(int dim, double *phi, const double *f, const MgGeom &g, int sweeps, cudaStream_t s)
{
    for (int sw = 0; sw < sweeps; sw++)
        for (int c = 0; c < 2; c++) {
            cudaError_t e = mg_launch_smooth(dim, false, phi, f, g, c, s);
            if (e)
                return e;
        }
    return cudaSuccess;
}

// Sec. 2.3 steps 2-13, FP64, same launch sequence as the allocating path.
cudaError_t vcycle(int dim, int nmg, const MgGeom *g, double **phi, double **f, int nu_pre, int nu_post,
                   cudaStream_t s)
{
    cudaError_t e;
    if (nmg == 1)
        return smooth(dim, phi[0], f[0], g[0], nu_pre + nu_post, s);
    if ((e = smooth(dim, phi[0], f[0], g[0], nu_pre, s)))
        return e;
    int L = 0;
    do {
        if ((e = mg_launch_resid_restrict(dim, false, phi[L], f[L], g[L], phi[L + 1], f[L + 1], g[L + 1], s)))
            return e;
        const int sweeps = g[L + 1].N == 1 ? (nu_pre > 0 ? 1 : 0) : nu_pre;
        if ((e = smooth(dim, phi[L + 1], f[L + 1], g[L + 1], sweeps, s)))
            return e;
        L++;
    } while (g[L].N > 1 && L + 1 < nmg);
    do {
        if ((e = mg_launch_prolong(dim, false, phi[L], g[L], phi[L - 1], g[L - 1], s)))
            return e;
        if ((e = smooth(dim, phi[L - 1], f[L - 1], g[L - 1], nu_post, s)))
            return e;
        L--;
    } while (L > 0);
    return cudaSuccess;
}

thread_local char g_msg[256];

mg_status reject(mg_status s, const char *msg)
{
    std::snprintf(g_msg, sizeof g_msg, "mg_solve_level_noalloc: %s", msg);
    std::fprintf(stderr, "%s\n", g_msg);
    return s;
}

}  // namespace

extern "C" mg_status mg_solve_level_noalloc(int dim, int n, double h, double G, const double *rho, double *phi,
                                            const mg_options *opt, mg_level_stats *stats)
{
    mg_options o;
    mg_default_options(&o);
    if (opt)
        o = *opt;
    if ((dim != 2 && dim != 3) || n < 2 || !(h > 0.0) || !std::isfinite(G) || !rho || !phi)
        return reject(MG_EINVAL, "bad dim, n, h, G or NULL array");
    if (o.precision != MG_FP64 || o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre + o.nu_post < 1 || o.max_cycles < 0 ||
        !(o.rel_tol >= 0.0) || o.stop != MG_STOP_RESIDUAL)
        return reject(MG_EINVAL, "options: FP64 only, nu_pre + nu_post >= 1, max_cycles >= 0, rel_tol >= 0, "
                                 "residual stopping rule");
    if (n + 2 > (1 << (MG_MAX_MG - 1)))
        return reject(MG_EINVAL, "n too large");

    // layout of the scratch array, checked against its size before any GPU work
    const int M = n + 2;
    MgGeom g[MG_MAX_MG] = {};
    const int nmg = geometry(M, h, g);
    size_t need = up256(ncells(n + 4, dim) * sizeof(double));                       // f on the finest level
    for (int L = 1; L < nmg; L++)
        need += 2 * up256(ncells(g[L].E, dim) * sizeof(double));                    // phi, f
    const size_t part_off = need;
    need += up256(MG_NORM_BLOCKS * sizeof(double)) + up256(2 * sizeof(double));
    if (need > kNoAllocScratchBytes) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "n=%d in %dD needs %zu bytes of scratch, the limit is %zu (3D n <= 69, 2D n <= 554)",
                      n, dim, need, kNoAllocScratchBytes);
        return reject(MG_EINVAL, buf);
    }
    cudaStream_t s = (cudaStream_t)o.stream;
    {
        // the call waits for its own norms on the host: a capturing stream
        // would have its capture invalidated, so it is refused up front
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
            cudaGetLastError();
            return reject(MG_EINVAL, "opt->stream is not a valid stream");
        }
        if (cs != cudaStreamCaptureStatusNone)
            return reject(MG_EINVAL, "opt->stream is capturing a graph; this call synchronises and cannot be captured");
    }
    for (const void *p : {(const void *)rho, (const void *)phi}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return reject(MG_EINVAL, "rho and phi must be device memory");
        }
    }

    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess)
        return reject(MG_ECUDA, cudaGetErrorString(e));
    double *phis[MG_MAX_MG], *fs[MG_MAX_MG];
    size_t pos = 0;
    phis[0] = phi;
    fs[0] = (double *)(base + pos);
    pos += up256(ncells(n + 4, dim) * sizeof(double));
    for (int L = 1; L < nmg; L++) {
        phis[L] = (double *)(base + pos);
        pos += up256(ncells(g[L].E, dim) * sizeof(double));
        fs[L] = (double *)(base + pos);
        pos += up256(ncells(g[L].E, dim) * sizeof(double));
    }
    double *partials = (double *)(base + part_off);
    double *scal = partials + up256(MG_NORM_BLOCKS * sizeof(double)) / sizeof(double);

    // once work is queued, a failing call waits for the stream before it
    // returns, so that no kernel of it still writes the shared array when the
    // caller's next call starts
    auto fail_queued = [&](cudaError_t err) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return reject(MG_ECUDA, cudaGetErrorString(err));
    };
    // the array keeps the previous call's contents: ghost layers of the
    // coarse levels must read as zero, so clear the part this call uses
    if ((e = mg_launch_zero(base, need, s)))
        return fail_queued(e);
    const double fourpiG = 4.0 * M_PI * G;
    const int E = n + 4;
    const long tot = (long)ncells(E, dim);
    const int grid = (int)std::min<long>((tot + 255) / 256, 152 * 16);
    if (dim == 3)
        k_rhs_from_block<3><<<grid, 256, 0, s>>>(n, rho, fs[0], fourpiG);
    else
        k_rhs_from_block<2><<<grid, 256, 0, s>>>(n, rho, fs[0], fourpiG);
    if ((e = cudaGetLastError()))
        return fail_queued(e);

    // loop of Sec. 2.3 with the stopping rule of mg_options (host-side test;
    // the two norms come back through a pageable host copy, no allocation)
    double hs[2];
    if ((e = mg_launch_resid_norm2(dim, phi, fs[0], g[0], true, partials, scal, s)) ||
        (e = mg_launch_resid_norm2(dim, phi, fs[0], g[0], false, partials, scal + 1, s)) ||
        (e = cudaMemcpyAsync(hs, scal, sizeof hs, cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s)))
        return fail_queued(e);
    const double bn = std::sqrt(hs[0]);
    double rel = bn > 0.0 ? std::sqrt(hs[1]) / bn : 0.0;
    int cycles = 0, status = std::isfinite(bn) ? MG_OK : MG_EDIVERGED;
    while (status == MG_OK && bn > 0.0 && cycles < o.max_cycles && !(rel < o.rel_tol)) {
        if ((e = vcycle(dim, nmg, g, phis, fs, o.nu_pre, o.nu_post, s)) ||
            (e = mg_launch_resid_norm2(dim, phi, fs[0], g[0], false, partials, scal + 1, s)) ||
            (e = cudaMemcpyAsync(hs + 1, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s)))
            return fail_queued(e);
        cycles++;
        rel = std::sqrt(hs[1]) / bn;
        if (!std::isfinite(rel)) {
            status = MG_EDIVERGED;
            break;
        }
    }
    if (status == MG_OK && bn > 0.0 && o.rel_tol > 0.0 && !(rel < o.rel_tol))
        status = MG_ENOCONV;
    if (stats) {
        stats->cycles = cycles;
        stats->outer_steps = cycles;
        stats->rel_res = rel;
        stats->b_norm = bn;
        stats->status = status;
    }
    return (mg_status)status;
}
