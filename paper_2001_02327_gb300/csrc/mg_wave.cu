// mg_wave.cu -- plane-marching red-black Gauss-Seidel sweeps of the FP32
// multigrid levels (3D), several colour passes per launch.
//
// One launch runs nsw complete red-black sweeps (Sec. 2.3 steps 2, 6 and 11;
// its 7-point Laplacian; the ghost rule of Sec. 2.4 folded into the boundary
// cells of the coarse multigrid levels) out of place, phi_in -> phi_out, so
// that a block reads only the input and never waits for another block.
//
// Dataflow.  A block owns a 56 x TY column of storage cells (tiles start at
// storage index 0; tile cells outside 1..N are ghosts and keep their values)
// over a range of z-planes [z0, z1] and marches through it.  The S = 2 nsw
// colour stages (red, black, red, black) are skewed by one plane: at march
// step t, stage s updates plane t - s.  Each plane lives in one shared-memory
// slot that the stages update in place, so stage s reads its neighbours in
// the state stage s - 1 left them (a red cell's six neighbours are black and
// vice versa, and the stages of a step run in order behind barriers).  Stage
// s is valid on a ring of S - 1 - s cells around the tile, which is all the
// next stage reads, so the last stage has every neighbour it needs.  The
// rows of a stage cover that ring; its columns cover the whole 64-wide slot
// (cells beyond the ring get values nothing reads; cells outside 1..N are
// never written).  Per launch the level's arrays are read once and written
// once, 3 words per cell for nsw sweeps, apart from the halo planes of the
// z-chunks.
//
// Block organisation.  Eight consumer warps run the stages; one producer warp
// keeps the planes coming: it waits for each plane's TMA load
// (cp.async.bulk.tensor, 64 x (TY + 8) boxes, zero fill outside the array;
// mbarrier waits with a clock budget, after which the kernel records
// MG_ETIMEOUT and returns), repacks the potential into a slot split by colour
// and issues the next loads, one step ahead of the consumers.  In the split
// slot a lane updates two cells of one colour (x, x + 2) with 64-bit shared
// loads and packed FP32x2 arithmetic, a warp's two rows of 16 lanes touch all
// 32 banks, and a lane keeps the same cells of a stage from plane to plane,
// so that two of its six neighbours come from registers: the plane below is
// what it read as its in-row neighbours one step earlier, and its in-row
// neighbours are what it read as the plane above.  The last stage writes the
// tile's cells, both colours, straight to phi_out, a lane's four consecutive
// cells as one 16-byte store.  Levels whose rows are not a multiple of 16
// bytes (E % 4 != 0: the odd coarse levels) are loaded by the producer with
// 4-byte cp.async and stored cell by cell.
//
// The arithmetic per cell, and its order, are those of the one-colour kernel
// (op_smooth_colour): the results are bit-identical.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "mg_internal.h"

namespace {

constexpr int kWX = 64;     // slot width: the tile's 56 columns and 4 halo columns on each side
constexpr int kTX = 56;
constexpr int kHalo = 4;
constexpr int kTimeout = 7; // MG_ETIMEOUT

template <int S, int TY>
struct WaveCfg {
    static constexpr int WY = TY + 2 * kHalo;      // slot height
    static constexpr int RP = kWX / 2;             // words per row of one colour half
    static constexpr int HALF = RP * WY + 16;      // one colour half (+16: the halves sit 16 banks apart)
    static constexpr int SPL = 2 * HALF;           // split potential slot
    static constexpr int NAT = kWX * WY;           // natural-layout slot (TMA destination)
    static constexpr int NS = 3;                   // potential staging buffers = load groups in flight
    static constexpr int RS = S + 3;               // split slots: planes t-S .. t+1, and t+2 being repacked
    static constexpr int RF = S + NS + 2;          // density slots (natural layout, loaded in place)
    static constexpr size_t off_f = (size_t)NS * NAT * 4;
    static constexpr size_t off_split = off_f + (size_t)RF * NAT * 4;
    static constexpr size_t off_bar = off_split + (size_t)RS * SPL * 4;
    static constexpr size_t smem = off_bar + NS * 8 + 16 + 128;   // mbarriers, a flag; base aligned up to 128
    static_assert((NAT * 4) % 128 == 0 && (SPL * 4) % 128 == 0, "TMA destinations 128-byte aligned");
    static_assert(TY % 2 == 0 && TY / 2 + S - 1 <= 8, "row pairs: at most one per consumer warp and stage");
};

constexpr int kConsumers = 256;               // eight consumer warps
constexpr int kWaveThreads = kConsumers + 32; // and the producer warp

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier, giving up after `budget` SM clocks.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long budget)
{
    if (mbar_try(bar, parity))
        return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > budget)
            return false;
    return true;
}

__device__ __forceinline__ void tma_load3(unsigned dst, const CUtensorMap *map, int x, int y, int z, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}


__device__ __forceinline__ void cp_async4(unsigned dst, const float *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

__device__ __forceinline__ void cp_async_arrive(unsigned bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// packed FP32x2 arithmetic: the sm_100 builtins, each lane of the pair
// rounded to nearest as the scalar operation
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

// ---------------------------------------------------------------------------
// one cell by the general rule of the coarse levels (Sec. 2.4 ghost rule
// folded in): the arithmetic of neighbour_sum_ptr / op_smooth_colour
// ---------------------------------------------------------------------------
__device__ __forceinline__ float cell_general(int i, int j, int k, float xl, float xr, float yd, float yu, float zd,
                                              float zu, float fv, const MgGeom &g)
{
    const int N = g.N;
    const bool tieN = g.tie && N >= 2;
    int cls = 0;
    auto axis = [&](int a, float lv, float rv, int shift) -> float {
        const bool lo = a == 1, hi = a == N;
        cls |= ((lo ? 1 : 0) | (hi ? 2 : 0)) << shift;
        const float l = (!lo && !(hi && tieN)) ? lv : 0.f;
        const float r = !hi ? rv : 0.f;
        return l + r;
    };
    float s = axis(i, xl, xr, 0) + axis(j, yd, yu, 2);
    s += axis(k, zd, zu, 4);
    float nid;
    if (cls == 0) {
        nid = float(1.0 / 6);
    } else if (g.tab32) {
        nid = g.tab32[64 + cls];
    } else {
        double d = mg_axis_diag(cls & 3, g) + mg_axis_diag((cls >> 2) & 3, g);
        d += mg_axis_diag((cls >> 4) & 3, g);
        nid = 1.f / (-float(d));
    }
    return __fmaf_rn(-g.h2f, fv, s) * nid;
}

struct WaveGeo {
    int gx0, gy0;   // storage indices of slot column 0 and slot row 0 (gx0 is even)
    int z0, z1;     // output planes of the block
    int base;       // plane of load group 0 (the first march step's plane - 1)
};

// What a consumer lane needs of the geometry, fixed for the whole launch.
// Lane a of a warp's two rows takes the compact pair (2a, 2a + 1) of its
// row's colour-c half: the cells x = 4a + q and x + 2, q the column parity of
// colour c in that row; per q in {0, 1}: the first cell's storage index and
// whether each cell lies inside 1..N (and away from the ghost rule).
struct WaveLane {
    int a, hr;                 // column pair, row within the warp's pair
    int ib;                    // storage index of the first cell at q = 0 (i0 = ib + q)
    unsigned in0, in1, inner;  // bit q: 1 <= i <= N for the first / second cell; both away from 1 and N
};

// What a consumer lane needs of one stage (ring w), fixed across steps: the
// warp's row pair (at most one per warp), the lane's row offset in a colour
// half and in the density slot, and the row's storage index.
struct WaveRow {
    bool act;                  // the warp has a row pair in this stage
    int ro, fo, j;
    bool jin, jint;            // 1 <= j <= N; 1 < j < N
};

template <int S, int TY, int W>
__device__ __forceinline__ WaveRow wave_row(const WaveGeo &wg, const WaveLane &ln, int N)
{
    using C = WaveCfg<S, TY>;
    constexpr int R0 = kHalo - W, NPAIRS = (TY + 2 * W) / 2;
    const int warp = threadIdx.x >> 5;
    WaveRow wr;
    wr.act = warp < NPAIRS;
    const int r = R0 + 2 * warp + ln.hr;
    wr.ro = r * C::RP + 2 * ln.a;
    wr.fo = r * kWX + 4 * ln.a;
    wr.j = wg.gy0 + r;
    wr.jin = (unsigned)(wr.j - 1) < (unsigned)N;
    wr.jint = wr.j > 1 && wr.j < N;
    return wr;
}

// One colour-c stage (ring W) of the lane on plane p: the potential slots of
// planes p - 1, p, p + 1 (P0 split slot, Pm / Pp their other-colour halves),
// the density slot F0, q the column parity of colour c on the lane's row.
// zr / orr carry the other colour at the lane's cells from the previous plane
// of this stage (FRESH: the stage's first plane, read them instead).  FINAL
// (W = 0): the lane's four cells 4a .. 4a+3 of the tile go to out (the
// storage row of plane p, at the span's first cell).
template <int S, int TY, bool FINAL, bool ALIGNED, bool COARSE, bool FRESH>
__device__ __forceinline__ void wave_cells(float *P0, const float *Pm, const float *Pp, const float *F0, int c, int q,
                                          int p, const WaveLane &ln, const WaveRow &wr, float2 &zr, float2 &orr,
                                          float *__restrict__ out, const MgGeom &g)
{
    using C = WaveCfg<S, TY>;
    const int N = g.N;
    const float *oth = P0 + (c ^ 1) * C::HALF + wr.ro;   // other colour, this row
    const float2 ot = FRESH ? lds2(oth) : orr;
    const float2 zd = FRESH ? lds2(Pm + wr.ro) : zr;
    const float2 zu = lds2(Pp + wr.ro);
    const float ow = q ? oth[2] : oth[-1];
    const float2 L = q ? ot : make_float2(ow, ot.x);
    const float2 R = q ? make_float2(ot.y, ow) : ot;
    const float2 yd = lds2(oth - C::RP), yu = lds2(oth + C::RP);
    const float *fr = F0 + wr.fo + q;
    const float2 fv = make_float2(fr[0], fr[2]);
    orr = zu;   // the next plane's in-row neighbours of the cells this lane takes there
    zr = ot;    // and the plane below them
    const bool in0 = wr.jin && ((ln.in0 >> q) & 1), in1 = wr.jin && ((ln.in1 >> q) & 1);
    const int i0 = ln.ib + q;
    float2 nv;
    if (!COARSE || (p > 1 && p < N && wr.jint && ((ln.inner >> q) & 1))) {
        float2 s2 = add2(add2(L, R), add2(yd, yu));
        s2 = add2(s2, add2(zd, zu));
        nv = mul2(fma2(make_float2(-g.h2f, -g.h2f), fv, s2), make_float2(float(1.0 / 6), float(1.0 / 6)));
    } else {
        nv.x = in0 ? cell_general(i0, wr.j, p, L.x, R.x, yd.x, yu.x, zd.x, zu.x, fv.x, g) : 0.f;
        nv.y = in1 ? cell_general(i0 + 2, wr.j, p, L.y, R.y, yd.y, yu.y, zd.y, zu.y, fv.y, g) : 0.f;
    }
    float *own = P0 + c * C::HALF + wr.ro;
    if (!FINAL) {
        if (in0 && in1) {
            *reinterpret_cast<float2 *>(own) = nv;
        } else {
            if (in0)
                own[0] = nv.x;
            if (in1)
                own[1] = nv.y;
        }
    } else if (ln.a >= 1 && ln.a <= kTX / 4 && (unsigned)wr.j < (unsigned)g.E) {
        const float2 old = lds2(own);
        const float b0 = in0 ? nv.x : old.x, b1 = in1 ? nv.y : old.y;
        const float4 v4 = q ? make_float4(ot.x, b0, ot.y, b1) : make_float4(b0, ot.x, b1, ot.y);
        const int ib = ln.ib;      // storage index of the span's first cell
        if (ALIGNED) {
            if (ib < g.E)           // E % 4 == 0: a span lies inside the row or beyond it
                *reinterpret_cast<float4 *>(out) = v4;
        } else {
            const float w4[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (ib + e < g.E)
                    out[e] = w4[e];
        }
    }
}

__device__ __forceinline__ void consumer_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory"); }

template <int S, int TY, bool TMA, bool COARSE>
__global__ void __launch_bounds__(kWaveThreads, 2)
    k_wave(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_f,
           const float *__restrict__ phi_in, float *__restrict__ phi_out, const float *__restrict__ f, MgGeom g,
           int TZ, MgSolveCtl *ctl, cudaGraphConditionalHandle hi, int *err, long long budget, int skip)
{
    using C = WaveCfg<S, TY>;
    extern __shared__ __align__(16) unsigned char wave_raw[];
    unsigned char *sm = wave_raw + ((128 - (smem_u32(wave_raw) & 127)) & 127);
    float *sStage = reinterpret_cast<float *>(sm);
    float *sF = reinterpret_cast<float *>(sm + C::off_f);
    float *sSplit = reinterpret_cast<float *>(sm + C::off_split);
    const unsigned bar0 = smem_u32(sm + C::off_bar);
    const int tid = threadIdx.x;
    const bool producer = tid >= kConsumers;
    const int plane_lane = tid - kConsumers;   // producer lanes 0..31
    pdl_begin();
    if (ctl && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0)
        inner_step_count(ctl, hi);
    const int N = g.N, E = g.E;
    WaveGeo wg;
    wg.gx0 = kTX * (int)blockIdx.x - kHalo;
    wg.gy0 = TY * (int)blockIdx.y - kHalo;
    wg.z0 = 1 + TZ * (int)blockIdx.z;
    wg.z1 = min(N, wg.z0 + TZ - 1);
    const int tf = wg.z0 - (S - 1), tl = wg.z1 + (S - 1);
    wg.base = tf - 1;
    const int nsteps = tl - tf + 1;
    const int ngroups = nsteps + 2;   // planes base .. tl + 1

    if (tid == kConsumers)
        for (int b = 0; b < C::NS; b++)
            mbar_init(bar0 + 8 * b, TMA ? 1 : 32);
    __syncthreads();

    // Producer: load group v = potential of plane base + v into staging slot
    // v % NS and its density into density slot v % RF, completing on
    // mbarrier v % NS.
    auto issue = [&](int v) {
        if (v >= ngroups || v == skip)
            return;
        const int pl = wg.base + v;
        const unsigned bar = bar0 + 8 * (v % C::NS);
        float *dst = sStage + (v % C::NS) * C::NAT;
        float *dstf = sF + (v % C::RF) * C::NAT;
        if (TMA) {
            if (plane_lane == 0) {
                mbar_expect_tx(bar, 2u * C::NAT * 4u);
                tma_load3(smem_u32(dst), &tm_in, wg.gx0, wg.gy0, pl, bar);
                tma_load3(smem_u32(dstf), &tm_f, wg.gx0, wg.gy0, pl, bar);
            }
        } else {
            const bool pin = (unsigned)pl < (unsigned)E;
            const long pb = (long)pl * E * E;
            for (int it = plane_lane; it < C::NAT; it += 32) {
                const int r = it / kWX, x = it - r * kWX;
                const int i = wg.gx0 + x, j = wg.gy0 + r;
                const bool ok = pin && (unsigned)i < (unsigned)E && (unsigned)j < (unsigned)E;
                const long gq = ok ? pb + (long)j * E + i : 0;
                cp_async4(smem_u32(dst + it), phi_in + gq, ok);
                cp_async4(smem_u32(dstf + it), f + gq, ok);
            }
            cp_async_arrive(bar);
        }
    };
    // Producer: wait for group v, repack its potential by colour into split
    // slot v % RS, then load group v + NS into the staging slot it frees.
    // False when the wait ran out of budget.
    auto produce = [&](int v) -> bool {
        if (v >= ngroups)
            return true;
        if (!mbar_wait(bar0 + 8 * (v % C::NS), (unsigned)((v / C::NS) & 1), budget))
            return false;
        __syncwarp();
        const int pl = wg.base + v;
        const float *src = sStage + (v % C::NS) * C::NAT;
        float *dst = sSplit + (v % C::RS) * C::SPL;
        // lane: columns 4 (lane & 15) .. +3 of rows 2k + (lane >> 4); all loads first
        constexpr int NIT = C::NAT / 4 / 32;
        static_assert(C::NAT % 128 == 0, "whole float4 per lane");
        const int x4 = 4 * (plane_lane & 15), rh = plane_lane >> 4;
        float4 w[NIT];
#pragma unroll
        for (int k = 0; k < NIT; k++)
            w[k] = *reinterpret_cast<const float4 *>(src + (2 * k + rh) * kWX + x4);
        const int c0 = (wg.gy0 + rh + pl) & 1;   // colour of the even columns of row rh (gx0 even)
#pragma unroll
        for (int k = 0; k < NIT; k++) {
            const int r = 2 * k + rh;
            *reinterpret_cast<float2 *>(dst + c0 * C::HALF + r * C::RP + x4 / 2) = make_float2(w[k].x, w[k].z);
            *reinterpret_cast<float2 *>(dst + (c0 ^ 1) * C::HALF + r * C::RP + x4 / 2) = make_float2(w[k].y, w[k].w);
        }
        __syncwarp();   // every lane's reads of the staging slot before its refill
        issue(v + C::NS);
        return true;
    };

    // prologue: groups 0 .. 2 ready (the first step reads planes t-1 .. t+1)
    bool ok = true;
    if (producer) {
        for (int v = 0; v < C::NS; v++)
            issue(v);
        for (int v = 0; v < 3 && ok; v++)
            ok = produce(v);
    }
    int failed_at = 0;
    bool fail = __syncthreads_or(!ok) != 0;

    // consumer constants
    WaveLane ln;
    ln.a = threadIdx.x & 15;
    ln.hr = (threadIdx.x >> 4) & 1;
    ln.ib = wg.gx0 + 4 * ln.a;
    ln.in0 = ln.in1 = ln.inner = 0;
    for (int qq = 0; qq < 2; qq++) {
        const int i0 = ln.ib + qq;
        ln.in0 |= ((unsigned)(i0 - 1) < (unsigned)N ? 1u : 0u) << qq;
        ln.in1 |= ((unsigned)(i0 + 1) < (unsigned)N ? 1u : 0u) << qq;
        ln.inner |= (i0 > 1 && i0 + 2 < N ? 1u : 0u) << qq;
    }
    WaveRow rows[S];
    int zlo[S], zhi[S];   // planes each stage updates
    rows[S - 1] = wave_row<S, TY, 0>(wg, ln, N);
    rows[S - 2] = wave_row<S, TY, 1>(wg, ln, N);
    if constexpr (S == 4) {
        rows[1] = wave_row<S, TY, 2>(wg, ln, N);
        rows[0] = wave_row<S, TY, 3>(wg, ln, N);
    }
    for (int sidx = 0; sidx < S; sidx++) {
        zlo[sidx] = max(1, wg.z0 - (S - 1 - sidx));
        zhi[sidx] = min(N, wg.z1 + (S - 1 - sidx));
    }
    float2 zr[S], orr[S];
    // the last stage's store target: storage row rows[S-1].j of plane z0 at the span's first cell
    float *out = phi_out + ((long)wg.z0 * E + rows[S - 1].j) * E + ln.ib;
    const long plane_stride = (long)E * E;
    int slot0 = 1 % C::RS;    // split slot of plane t (group t - base), t = base + 1 at step 0
    int fslot0 = 1 % C::RF;   // density slot of plane t
    int tpar = (wg.base + 1 + wg.gy0 + ln.hr) & 1;

    for (int st = 0; !fail && st < nsteps; st++) {
        const int t = wg.base + 1 + st;
        if (producer) {
            // group st + 3 for the next step while the consumers run this one
            ok = produce(st + 3);
            if (!ok)
                failed_at = st + 3;
        } else {
            auto stage = [&](auto sconst) {
                constexpr int sidx = decltype(sconst)::value, w = S - 1 - sidx, c = sidx & 1;
                constexpr bool final_stage = sidx == S - 1;
                const int p = t - sidx;
                if (rows[sidx].act && p >= zlo[sidx] && p <= zhi[sidx]) {
                    const int sl = slot0 >= sidx ? slot0 - sidx : slot0 - sidx + C::RS;
                    float *P0 = sSplit + sl * C::SPL;
                    const float *Pm = sSplit + (sl == 0 ? C::RS - 1 : sl - 1) * C::SPL + (c ^ 1) * C::HALF;
                    const float *Pp = sSplit + (sl == C::RS - 1 ? 0 : sl + 1) * C::SPL + (c ^ 1) * C::HALF;
                    const float *F0 = sF + (fslot0 >= sidx ? fslot0 - sidx : fslot0 - sidx + C::RF) * C::NAT;
                    const int q = tpar ^ ((c + (kHalo - w) - sidx) & 1);
                    if (p > zlo[sidx])
                        wave_cells<S, TY, final_stage, TMA, COARSE, false>(P0, Pm, Pp, F0, c, q, p, ln, rows[sidx],
                                                                          zr[sidx], orr[sidx], out, g);
                    else
                        wave_cells<S, TY, final_stage, TMA, COARSE, true>(P0, Pm, Pp, F0, c, q, p, ln, rows[sidx],
                                                                         zr[sidx], orr[sidx], out, g);
                }
                if (!final_stage)
                    consumer_barrier();
            };
            stage(std::integral_constant<int, 0>{});
            stage(std::integral_constant<int, 1>{});
            if constexpr (S == 4) {
                stage(std::integral_constant<int, 2>{});
                stage(std::integral_constant<int, 3>{});
            }
            if (t - (S - 1) >= wg.z0)
                out += plane_stride;
        }
        slot0 = slot0 + 1 == C::RS ? 0 : slot0 + 1;
        fslot0 = fslot0 + 1 == C::RF ? 0 : fslot0 + 1;
        tpar ^= 1;
        fail = __syncthreads_or(!ok) != 0;   // end of step: the repacked plane is visible to everyone
    }
    if (!fail)
        return;
    // a wait ran out: record it, let the copies this block started land, return
    if (producer) {
        if (plane_lane == 0 && err)
            atomicExch(err, kTimeout);
        if (TMA) {
            if (plane_lane == 0)
                for (int u = failed_at; u < min(failed_at + C::NS, ngroups); u++)
                    if (u != skip)
                        mbar_wait(bar0 + 8 * (u % C::NS), (unsigned)((u / C::NS) & 1), budget);
        } else {
            cp_async_wait_all();
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// A 3D tensor map over an E^3 FP32 array with a bx x by x 1 box.
bool encode3(CUtensorMap *m, const float *base, int E, int bx, int by)
{
    const PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
    if (!fn)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)E, (cuuint64_t)E, (cuuint64_t)E};
    const cuuint64_t strides[2] = {(cuuint64_t)E * 4, (cuuint64_t)E * E * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S, int TY, bool TMA, bool COARSE>
cudaError_t wave_attr()
{
    return cudaFuncSetAttribute(k_wave<S, TY, TMA, COARSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)WaveCfg<S, TY>::smem);
}

template <int S, int TY>
cudaError_t wave_attrs()
{
    cudaError_t e = wave_attr<S, TY, true, false>();
    for (cudaError_t r : {wave_attr<S, TY, true, true>(), wave_attr<S, TY, false, false>(),
                          wave_attr<S, TY, false, true>()})
        if (r && !e)
            e = r;
    return e;
}

template <int S, int TY>
cudaError_t wave_launch(const float *in, float *out, const float *f, const MgGeom &g, int zchunks, cudaStream_t s,
                        MgSolveCtl *ctl, cudaGraphConditionalHandle hi, int *err, long long budget, int skip)
{
    const int TZ = (g.N + zchunks - 1) / zchunks;
    const dim3 grid(g.N / kTX + 1, g.N / TY + 1, (g.N + TZ - 1) / TZ);
    CUtensorMap m_in{}, m_f{};
    const bool tma = g.E % 4 == 0 && encode3(&m_in, in, g.E, kWX, WaveCfg<S, TY>::WY) &&
                     encode3(&m_f, f, g.E, kWX, WaveCfg<S, TY>::WY);
    const size_t sm = WaveCfg<S, TY>::smem;
    auto go = [&](auto kernel) {
        mg_launch_kernel(kernel, grid, kWaveThreads, sm, s, m_in, m_f, in, out, f, g, TZ, ctl, hi, err, budget, skip);
    };
    if (tma)
        g.L > 0 ? go(k_wave<S, TY, true, true>) : go(k_wave<S, TY, true, false>);
    else
        g.L > 0 ? go(k_wave<S, TY, false, true>) : go(k_wave<S, TY, false, false>);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mg_wave_prepare()
{
    cudaError_t e = wave_attrs<4, 10>();
    for (cudaError_t r : {wave_attrs<4, 6>(), wave_attrs<2, 10>(), wave_attrs<2, 6>()})
        if (r && !e)
            e = r;
    return e;
}

bool mg_wave_applies(int dim, int nsw, int N) { return dim == 3 && (nsw == 1 || nsw == 2) && N >= 4; }

cudaError_t mg_launch_wave(const float *phi_in, float *phi_out, const float *f, const MgGeom &g, int nsw,
                           int variant, int zchunks, cudaStream_t s, MgSolveCtl *ctl, cudaGraphConditionalHandle hi,
                           int *err, int fault)
{
    if (!mg_wave_applies(3, nsw, g.N) || phi_in == phi_out || zchunks < 1)
        return cudaErrorInvalidValue;
    // about two seconds at the part's clock: no correct wait comes near it;
    // a fault-injection run (a load group never issued) gives up after ~1 ms
    const long long budget = fault ? (2LL << 20) : (4LL << 30);
    const int skip = fault ? 0 : -1;
    if (nsw == 2)
        return variant == 0 ? wave_launch<4, 10>(phi_in, phi_out, f, g, zchunks, s, ctl, hi, err, budget, skip)
                            : wave_launch<4, 6>(phi_in, phi_out, f, g, zchunks, s, ctl, hi, err, budget, skip);
    return variant == 0 ? wave_launch<2, 10>(phi_in, phi_out, f, g, zchunks, s, ctl, hi, err, budget, skip)
                        : wave_launch<2, 6>(phi_in, phi_out, f, g, zchunks, s, ctl, hi, err, budget, skip);
}
