// unet.cu -- the learned initial guess: a small 3D U-Net that predicts the
// correction of a refinement level's interpolated initial potential, with
// hand-written BF16 tensor-core convolutions (FP32 accumulate), its backward
// pass, AdamW training and the hook into the solver.
//
// Network (channels-last BF16 activations, n = 2^k spatial edge, 4 scales):
//   x0 = [4 pi G rho h^2 / s, Phi_interp / s, h^2 r / s_r]   on Omega, with
//        r = 4 pi G rho - lap(Phi_interp) the residual of the interpolated
//        potential, s = max |Phi_interp|, s_r = max |h^2 r|
//   a0 = relu(c3(x0; 3->16))      s0 = relu(c3(a0; 16->16))          n
//   a1 = relu(c3(pool s0; 16->32)) s1 = relu(c3(a1; 32->32))         n/2
//   s2 = relu(c3(pool s1; 32->64))                                   n/4
//   a3 = relu(c3(pool s2; 64->64))                                   n/8
//   d2 = relu(c3([up a3, s2]; 128->32))                              n/4
//   d1 = relu(c3([up d2, s1]; 64->16))                               n/2
//   d0 = relu(c3([up d1, s0]; 32->16))                               n
//   y  = c1(d0; 16->1);   Phi_guess = Phi_interp + (s_r n^2 / 16) y  on Omega
// (the inverse 7-point Laplacian amplifies smooth residuals by ~n^2: the
// factor keeps y of order one across level sizes).
// c3: 3x3x3 convolution, zero padding, bias; pool: 2x2x2 mean; up: nearest.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/unet.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kT = 256;

inline int blocks_for(long n, int cap = 152 * 32)
{
    long b = (n + kT - 1) / kT;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t ld2(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
__device__ __forceinline__ uint32_t ld2(const float *p)
{
    const float2 f = *reinterpret_cast<const float2 *>(p);
    return pack2(f.x, f.y);
}

// D += A (16x16, row) * B (16x8, col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float *d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 3x3x3 convolution as an implicit GEMM on the tensor cores.
//   out[v][nn] = sum_{tap, c} in[v +/- off(tap)][c] * W[tap][nn][c]  (+ bias, relu)
// in: [V][CK] (CK a multiple of 16), W: [27][NT*8][CK] BF16, V = batch * n^3
// with n = 2^lg.  FLIP = true gathers at v - off (the transpose convolution of
// the backward data pass).  A block of 4 warps covers 64 voxels; a warp owns
// 16 voxels and all NT*8 output channels.
template <int NT, bool FLIP, typename TIn>
__global__ void __launch_bounds__(128) k_conv3(const TIn *__restrict__ in, int CK, const bf16 *__restrict__ W,
                                               const float *__restrict__ bias, void *__restrict__ out, int out_bf16,
                                               int relu, int lg, int V)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int n = 1 << lg, msk = n - 1;
    const int r0 = blockIdx.x * 64 + warp * 16 + g, r1 = r0 + 8;
    const bool ok0 = r0 < V, ok1 = r1 < V;
    const int x0 = r0 & msk, y0 = (r0 >> lg) & msk, z0 = (r0 >> (2 * lg)) & msk, b0 = r0 >> (3 * lg);
    const int x1 = r1 & msk, y1 = (r1 >> lg) & msk, z1 = (r1 >> (2 * lg)) & msk, b1 = r1 >> (3 * lg);
    float acc[NT][4];
#pragma unroll
    for (int q = 0; q < NT; q++)
        acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    constexpr int N = NT * 8;
    for (int tap = 0; tap < 27; tap++) {
        int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        if (FLIP) {
            dz = -dz;
            dy = -dy;
            dx = -dx;
        }
        int q0 = -1, q1 = -1;
        {
            const int zz = z0 + dz, yy = y0 + dy, xx = x0 + dx;
            if (ok0 && (unsigned)zz < (unsigned)n && (unsigned)yy < (unsigned)n && (unsigned)xx < (unsigned)n)
                q0 = (((b0 << lg | zz) << lg | yy) << lg) | xx;
        }
        {
            const int zz = z1 + dz, yy = y1 + dy, xx = x1 + dx;
            if (ok1 && (unsigned)zz < (unsigned)n && (unsigned)yy < (unsigned)n && (unsigned)xx < (unsigned)n)
                q1 = (((b1 << lg | zz) << lg | yy) << lg) | xx;
        }
        const bf16 *Wt = W + (size_t)tap * N * CK;
        for (int c0 = 0; c0 < CK; c0 += 16) {
            const uint32_t a0 = q0 >= 0 ? ld2(in + (size_t)q0 * CK + c0 + 2 * t) : 0u;
            const uint32_t a1 = q1 >= 0 ? ld2(in + (size_t)q1 * CK + c0 + 2 * t) : 0u;
            const uint32_t a2 = q0 >= 0 ? ld2(in + (size_t)q0 * CK + c0 + 2 * t + 8) : 0u;
            const uint32_t a3 = q1 >= 0 ? ld2(in + (size_t)q1 * CK + c0 + 2 * t + 8) : 0u;
#pragma unroll
            for (int q = 0; q < NT; q++) {
                const bf16 *wp = Wt + (size_t)(q * 8 + g) * CK + c0 + 2 * t;
                mma16816(acc[q], a0, a1, a2, a3, ld2(wp), ld2(wp + 8));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NT; q++) {
        const int c = q * 8 + 2 * t;
        float v[4] = {acc[q][0], acc[q][1], acc[q][2], acc[q][3]};
        if (bias) {
            v[0] += bias[c];
            v[1] += bias[c + 1];
            v[2] += bias[c];
            v[3] += bias[c + 1];
        }
        if (relu)
            for (int e = 0; e < 4; e++)
                v[e] = fmaxf(v[e], 0.f);
        if (out_bf16) {
            bf16 *o = reinterpret_cast<bf16 *>(out);
            if (ok0)
                *reinterpret_cast<uint32_t *>(o + (size_t)r0 * N + c) = pack2(v[0], v[1]);
            if (ok1)
                *reinterpret_cast<uint32_t *>(o + (size_t)r1 * N + c) = pack2(v[2], v[3]);
        } else {
            float *o = reinterpret_cast<float *>(out);
            if (ok0)
                *reinterpret_cast<float2 *>(o + (size_t)r0 * N + c) = make_float2(v[0], v[1]);
            if (ok1)
                *reinterpret_cast<float2 *>(o + (size_t)r1 * N + c) = make_float2(v[2], v[3]);
        }
    }
}

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): the same implicit GEMM with the
// accumulator in tensor memory.  Inline PTX after the PTX ISA's tcgen05
// section: TMEM allocation by one warp, tcgen05.mma issued by one thread
// from shared-memory matrix descriptors, completion through tcgen05.commit
// on an mbarrier, tcgen05.ld for the epilogue.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy stores to shared memory made visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A * B^T, kind::f16 (BF16 operands, FP32 accumulate)
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
                 : "memory");
}
// arrive once on the mbarrier when every tcgen05.mma this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++)
        v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init1(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok)
                 : "r"(mbar), "r"(parity)
                 : "memory");
    return ok != 0;
}
// wait for completion `parity` of the mbarrier; false when the clock budget ran out first
__device__ __forceinline__ bool mbar_wait_for(uint32_t mbar, uint32_t parity, long long budget)
{
    const long long t0 = clock64();
    while (!mbar_test(mbar, parity))
        if (clock64() - t0 > budget)
            return false;
    return true;
}

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension
// byte offset (between core matrices adjacent along K), stride-dimension byte
// offset (between 8-row groups along M or N), the fixed 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Operand tiles in shared memory, K-major without swizzle: K in slabs of 16
// (one MMA each); within a slab, core matrices of 8 rows x 8 BF16 (128
// contiguous bytes, rows 16 B apart), the two core matrices of a row group
// 128 B apart (LBO), row groups 256 B apart (SBO).  Byte offset of the
// 16-byte chunk holding elements k8*8..k8*8+7 of row m in a tile of `rows`
// rows:
__device__ __forceinline__ uint32_t tc_chunk(int rows, int m, int k8)
{
    return (uint32_t)((k8 >> 1) * rows * 32 + (m >> 3) * 256 + (k8 & 1) * 128 + (m & 7) * 16);
}

// 16-byte asynchronous copy global -> shared through L1, zero-filled when
// `valid` is false (a padding voxel); groups committed and waited on per tap
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

constexpr long long kTcBudget = 1ll << 31;   // clock cycles an mbarrier wait may take (about 1 s)
constexpr int kTcStages = 4;                  // taps in flight

// 3x3x3 convolution on tcgen05: a block of 128 threads computes 128 voxels
// (thread m gathers voxel m's rows and owns its outputs) x N output channels.
// Taps run through kTcStages shared-memory stages: the 128 gathered input
// rows (CK channels, zero rows at the padding) and the tap's N x CK weights
// arrive by cp.async kTcStages - 2 taps ahead; once a tap's copies have
// landed, thread 0 issues CK/16 MMAs into the TMEM accumulator and commits
// them to the stage's mbarrier, which the stage's next fill (two taps later)
// waits on.
// Epilogue: each warp reads its 32 TMEM lanes, adds the bias, applies relu,
// stores.  FLIP and the operand layouts as in k_conv3 (BF16 input).  A wait
// that outlasts kTcBudget sets *err and stops issuing; the block still waits
// (bounded) for what it issued and frees its TMEM.
template <int N, bool FLIP>
__global__ void __launch_bounds__(128) k_conv3_tc(const bf16 *__restrict__ in, int CK, const bf16 *__restrict__ W,
                                                  const float *__restrict__ bias, void *__restrict__ out,
                                                  int out_bf16, int relu, int lg, int V, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[kTcStages];
    __shared__ uint32_t tslot;
    constexpr int NCOL = N < 32 ? 32 : N;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, N);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int abytes = 128 * CK * 2, bbytes = N * CK * 2, sbytes = abytes + bbytes;
    const uint32_t sm0 = smem_u32(smem), mb0 = smem_u32(&mbar[0]);   // stage s: tiles at sm0 + s sbytes, mbarrier mb0 + 8 s
    if (warp == 0) {
        tc_alloc(smem_u32(&tslot), NCOL);
        tc_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < kTcStages; q++)
            mbar_init1(mb0 + 8 * q);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int n = 1 << lg, msk = n - 1;
    const int r = blockIdx.x * 128 + tid;
    const bool ok = r < V;
    const int x = r & msk, y = (r >> lg) & msk, z = (r >> (2 * lg)) & msk, b = r >> (3 * lg);
    const int nk8 = CK >> 3;
    // the copies of one tap into stage s
    auto fill = [&](int tap, int s) {
        int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        if (FLIP) {
            dz = -dz;
            dy = -dy;
            dx = -dx;
        }
        const int zz = z + dz, yy = y + dy, xx = x + dx;
        const bool inside = ok && (unsigned)zz < (unsigned)n && (unsigned)yy < (unsigned)n && (unsigned)xx < (unsigned)n;
        const bf16 *src = inside ? in + (size_t)((((b << lg | zz) << lg | yy) << lg) | xx) * CK : in;
        const uint32_t As = sm0 + s * sbytes, Bs = As + abytes;
        for (int k8 = 0; k8 < nk8; k8++)
            cp16(As + tc_chunk(128, tid, k8), src + k8 * 8, inside);
        const bf16 *Wt = W + (size_t)tap * N * CK;
        for (int e = tid; e < N * nk8; e += 128) {
            const int row = e / nk8, k8 = e - row * nk8;
            cp16(Bs + tc_chunk(N, row, k8), Wt + (size_t)row * CK + k8 * 8, true);
        }
    };
    for (int t = 0; t < kTcStages - 2; t++) {
        fill(t, t);
        cp_commit();
    }
    uint32_t phases = 0u;    // bit s: parity of stage s's next completion
    int issued = 0;          // taps whose MMAs were issued (uniform)
    bool bad = false;
    for (int tap = 0; tap < 27; tap++) {
        const int s = tap % kTcStages;
        // refill the stage of tap - 2 with tap + kTcStages - 2, once tap - 2's MMAs are done with it
        // (a tap's MMAs get one tap of slack; the copies of two taps stay in flight)
        const int tn = tap + kTcStages - 2;
        if (tn < 27) {
            const int sn = tn % kTcStages;
            if (tap >= 2) {
                const bool done = mbar_wait_for(mb0 + 8 * sn, (phases >> sn) & 1u, kTcBudget);
                if (__syncthreads_or(!done)) {   // the final wait covers tap - 2 and what followed it
                    bad = true;
                    break;
                }
                phases ^= 1u << sn;
            }
            fill(tn, sn);
        }
        cp_commit();                 // (an empty group past the last tap keeps the count)
        cp_wait<kTcStages - 2>();    // this thread's copies of `tap` have landed
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint32_t a0 = sm0 + s * sbytes, b0 = a0 + abytes;
            for (int k = 0; k < CK / 16; k++)
                tc_mma(tmem, tc_sdesc(a0 + k * 128 * 32, 128, 256), tc_sdesc(b0 + k * N * 32, 128, 256), IDESC,
                       (tap > 0 || k > 0) ? 1u : 0u);
            tc_commit(mb0 + 8 * s);
        }
        issued = tap + 1;
    }
    cp_wait<0>();
    // the last commit covers every MMA issued before it
    bool done = true;
    if (issued > 0) {
        const int s = (issued - 1) % kTcStages;
        done = mbar_wait_for(mb0 + 8 * s, (phases >> s) & 1u, kTcBudget);
    }
    done = !__syncthreads_or(!done);
    tc_fence_after();
    if (done && !bad) {
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc_ld16(lane_base + c0, v);
            if (bias)
#pragma unroll
                for (int i = 0; i < 16; i++)
                    v[i] += bias[c0 + i];
            if (relu)
#pragma unroll
                for (int i = 0; i < 16; i++)
                    v[i] = fmaxf(v[i], 0.f);
            if (!ok)
                continue;
            if (out_bf16) {
                uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<bf16 *>(out) + (size_t)r * N + c0);
                o[0] = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
                o[1] = make_uint4(pack2(v[8], v[9]), pack2(v[10], v[11]), pack2(v[12], v[13]), pack2(v[14], v[15]));
            } else {
                float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(out) + (size_t)r * N + c0);
#pragma unroll
                for (int i = 0; i < 4; i++)
                    o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tc_dealloc(tmem, NCOL);
    if ((bad || !done) && tid == 0)
        atomicExch(err, 1);
}

// Weight gradients of a 3x3x3 convolution on tcgen05 (bias gradient apart):
//   dW[tap][ci][co] += sum_v in[v + off(tap)][ci] * bf16(d[v][co])
// as D = A B^T with the voxels as K: a block takes TG = 128 / CK taps (rows
// m = tap_local * CK + ci; rows of taps past 26 stay zero) and a run of
// `vchunk` voxels, gathers 64 voxels per stage -- A[m][k] from the voxels'
// shifted input rows, B[co][k] from their output gradients rounded to BF16,
// both transposed into the K-major tiles of k_conv3_tc -- issues 4 MMAs per
// stage into its TMEM accumulator (two stages, a stage refilled once its
// MMAs of two stages back have completed), and adds its 128 x N partial sums
// into dW (FP32 atomics, real channels only).  Waits bounded as in
// k_conv3_tc.
template <int CK, int N>
__global__ void __launch_bounds__(128) k_wgrad_tc(const bf16 *__restrict__ in, int Cin, const float *__restrict__ d,
                                                  float *__restrict__ dW, int lg, int V, int vchunk,
                                                  int *__restrict__ err)
{
    constexpr int TG = 128 / CK, KB = 64, NS = 2;
    constexpr int NCOL = N < 32 ? 32 : N;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, N);
    constexpr int ABYTES = 128 * KB * 2, BBYTES = N * KB * 2, SBYTES = ABYTES + BBYTES;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[NS];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sm0 = smem_u32(smem), mb0 = smem_u32(&mbar[0]);
    if (warp == 0) {
        tc_alloc(smem_u32(&tslot), NCOL);
        tc_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < NS; q++)
            mbar_init1(mb0 + 8 * q);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int n = 1 << lg, msk = n - 1;
    const int tap0 = blockIdx.y * TG;
    const int v0 = blockIdx.x * vchunk, v1 = min(v0 + vchunk, V);
    const int nst = (v1 - v0 + KB - 1) / KB;
    // rows of the tap `tap` shifted from voxel v, or NULL (padding, past the run, or no such tap)
    auto row_of = [&](int v, int tap) -> const bf16 * {
        if (v >= v1 || tap >= 27)
            return nullptr;
        const int x = v & msk, y = (v >> lg) & msk, z = (v >> (2 * lg)) & msk, b = v >> (3 * lg);
        const int zz = z + tap / 9 - 1, yy = y + (tap / 3) % 3 - 1, xx = x + tap % 3 - 1;
        if ((unsigned)zz >= (unsigned)n || (unsigned)yy >= (unsigned)n || (unsigned)xx >= (unsigned)n)
            return nullptr;
        return in + (size_t)((((b << lg | zz) << lg | yy) << lg) | xx) * CK;
    };
    auto fill = [&](int j, int s) {
        unsigned char *As = smem + s * SBYTES, *Bs = As + ABYTES;
        const int vb = v0 + j * KB;
        // A: (voxel pair p, tap_local) items; a pair of voxels k = 2p, 2p + 1 makes one 32-bit word per row
        for (int it = tid; it < (KB / 2) * TG; it += 128) {
            const int p = it % (KB / 2), tl = it / (KB / 2), k = 2 * p;
            const bf16 *ra = row_of(vb + k, tap0 + tl), *rb = row_of(vb + k + 1, tap0 + tl);
#pragma unroll 2
            for (int k8 = 0; k8 < CK / 8; k8++) {
                const uint4 qa = ra ? *reinterpret_cast<const uint4 *>(ra + 8 * k8) : make_uint4(0u, 0u, 0u, 0u);
                const uint4 qb = rb ? *reinterpret_cast<const uint4 *>(rb + 8 * k8) : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t wa[4] = {qa.x, qa.y, qa.z, qa.w}, wb[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const uint32_t lo = (wa[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                    const uint32_t hi = (wb[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                    const int m = tl * CK + 8 * k8 + e;
                    *reinterpret_cast<uint32_t *>(As + tc_chunk(128, m, k >> 3) + (k & 7) * 2) = lo | (hi << 16);
                }
            }
        }
        // B: (voxel pair p, 4 output channels) items from the FP32 gradient rows
        for (int it = tid; it < (KB / 2) * (N / 4); it += 128) {
            const int p = it % (KB / 2), c4 = it / (KB / 2), k = 2 * p;
            const int va = vb + k, vbb = vb + k + 1;
            const float4 ga = va < v1 ? *reinterpret_cast<const float4 *>(d + (size_t)va * N + 4 * c4)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 gb = vbb < v1 ? *reinterpret_cast<const float4 *>(d + (size_t)vbb * N + 4 * c4)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
            const float fa[4] = {ga.x, ga.y, ga.z, ga.w}, fb[4] = {gb.x, gb.y, gb.z, gb.w};
#pragma unroll
            for (int e = 0; e < 4; e++)
                *reinterpret_cast<uint32_t *>(Bs + tc_chunk(N, 4 * c4 + e, k >> 3) + (k & 7) * 2) = pack2(fa[e], fb[e]);
        }
    };
    uint32_t phases = 0u;
    int issued = 0;
    bool bad = false;
    for (int j = 0; j < nst; j++) {
        const int s = j % NS;
        if (j >= NS) {       // the stage's MMAs of stage j - 2 have finished reading it
            const bool done = mbar_wait_for(mb0 + 8 * s, (phases >> s) & 1u, kTcBudget);
            if (__syncthreads_or(!done)) {
                bad = true;
                break;
            }
            phases ^= 1u << s;
        }
        fill(j, s);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint32_t a0 = sm0 + s * SBYTES, b0 = a0 + ABYTES;
            for (int k = 0; k < KB / 16; k++)
                tc_mma(tmem, tc_sdesc(a0 + k * 128 * 32, 128, 256), tc_sdesc(b0 + k * N * 32, 128, 256), IDESC,
                       (j > 0 || k > 0) ? 1u : 0u);
            tc_commit(mb0 + 8 * s);
        }
        issued = j + 1;
    }
    bool done = true;
    if (issued > 0) {
        const int s = (issued - 1) % NS;
        done = mbar_wait_for(mb0 + 8 * s, (phases >> s) & 1u, kTcBudget);
    }
    done = !__syncthreads_or(!done);
    tc_fence_after();
    if (done && !bad && issued > 0) {
        const int tl = tid / CK, ci = tid - tl * CK, tap = tap0 + tl;
        const bool mine = tap < 27 && ci < Cin;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc_ld16(lane_base + c0, v);
            if (mine)
#pragma unroll
                for (int i = 0; i < 16; i++)
                    atomicAdd(&dW[((size_t)tap * Cin + ci) * N + c0 + i], v[i]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tc_dealloc(tmem, NCOL);
    if ((bad || !done) && tid == 0)
        atomicExch(err, 1);
}

// db[co] += sum_v d[v][co]: a block of 256 threads takes a run of voxels,
// thread t the channel t % N of voxels v0 + t / N, v0 + t / N + 256 / N, ...
// (coalesced rows), then sums per channel in shared memory and adds once
__global__ void __launch_bounds__(256) k_bias_grad(const float *__restrict__ d, int N, int V, int vchunk,
                                                   float *__restrict__ db)
{
    __shared__ float part[256];
    const int v0 = blockIdx.x * vchunk, v1 = min(v0 + vchunk, V);
    const int c = threadIdx.x % N, step = 256 / N;
    float s = 0.f;
    for (int v = v0 + threadIdx.x / N; v < v1; v += step)
        s += d[(size_t)v * N + c];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < N) {
        float t = 0.f;
        for (int q = threadIdx.x; q < 256; q += N)
            t += part[q];
        atomicAdd(&db[threadIdx.x], t);
    }
}

// ---------------------------------------------------------------------------
// The same convolution from a TMA-loaded halo: a tile of 8 (x) x 16 (y) x 1
// (z) voxels of one sample; one TMA box per 8 input channels brings the
// 10 x 18 x 3 voxels around it (zero outside the grid) into shared memory as
// 16-byte rows, x fastest.  Tap (dz, dy, dx) is then the 128 x CK operand
// whose row (x, y) is halo row ((dz+1) 18 + y + dy + 1) 10 + x + dx + 1: a
// descriptor at that start with 8-row groups one halo row (160 B) apart
// (SBO) and the channel chunks kHaloChunk apart (LBO) -- no copy per tap.
// All 27 taps' weights (N x CK each) come in by cp.async from every thread,
// N rows of 16 B per chunk.  One thread issues the TMA and every MMA; the
// block waits once for the accumulator.
// ---------------------------------------------------------------------------
constexpr int kHaloRows = 10 * 18 * 3;                 // 540 rows of one channel chunk
constexpr int kHaloChunk = (kHaloRows * 16 + 127) / 128 * 128;   // 8704 B, 128-byte aligned chunks

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load5(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                          uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                 "%3, %4, %5, %6}], [%7];" ::"r"(dst),
                 "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mbar)
                 : "memory");
}
template <int N, bool FLIP>
__global__ void __launch_bounds__(128) k_conv3_halo(const __grid_constant__ CUtensorMap tm_in,
                                                    const bf16 *__restrict__ in, int halo_by_tma,
                                                    const bf16 *__restrict__ W, int CK,
                                                    const float *__restrict__ bias, void *__restrict__ out,
                                                    int out_bf16, int relu, int lg, int B, int fault,
                                                    int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];   // 0: halo and weights arrived; 1: accumulator complete
    __shared__ uint32_t tslot;
    constexpr int NCOL = N < 32 ? 32 : N;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, N);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nk8 = CK >> 3;
    const uint32_t halo = smem_u32(smem), wts = halo + nk8 * kHaloChunk;
    const uint32_t mb_in = smem_u32(&mbar[0]), mb_acc = smem_u32(&mbar[1]);
    const int n = 1 << lg;
    const int tx = n >> 3, ty = (n + 15) >> 4;          // tiles per row and per column of a plane
    int t = blockIdx.x;
    const int x0 = (t % tx) * 8;
    t /= tx;
    const int y0 = (t % ty) * 16;
    t /= ty;
    const int z0 = t % n, b = t / n;
    if (warp == 0) {
        tc_alloc(smem_u32(&tslot), NCOL);
        tc_relinquish();
    }
    if (tid == 0) {
        mbar_init1(mb_in);
        mbar_init1(mb_acc);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    if (halo_by_tma) {
        if (tid == 0) {
            mbar_expect_tx(mb_in, (uint32_t)(nk8 * kHaloRows * 16));
            for (int k8 = 0; k8 < nk8; k8++)
                tma_load5(halo + k8 * kHaloChunk, &tm_in, 8 * k8, x0 - 1, y0 - 1, z0 - 1, b, mb_in);
        }
    } else {
        // the halo rows by every thread, zero outside the grid
        for (int e = tid; e < nk8 * kHaloRows; e += 128) {
            const int k8 = e / kHaloRows, row = e - k8 * kHaloRows;
            const int hx = row % 10, hy = (row / 10) % 18, hz = row / 180;
            const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
            const bool inside = (unsigned)gx < (unsigned)n && (unsigned)gy < (unsigned)n && (unsigned)gz < (unsigned)n;
            const bf16 *src = inside ? in + ((((size_t)b * n + gz) * n + gy) * n + gx) * CK + 8 * k8 : in;
            cp16(halo + k8 * kHaloChunk + row * 16, src, inside);
        }
    }
    // the weights by every thread (16-byte copies), N rows of 16 B per (tap, chunk)
    for (int e = tid; e < 27 * N * nk8; e += 128) {
        const int k8 = e % nk8, row = e / nk8;   // row = tap * N + output channel
        const int tap = row / N, nn = row - tap * N;
        cp16(wts + ((tap * nk8 + k8) * N + nn) * 16, W + (size_t)row * CK + 8 * k8, true);
    }
    cp_commit();
    cp_wait<0>();
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        if (halo_by_tma) {
            ok = mbar_wait_for(mb_in, 0, kTcBudget);
            if (!ok)
                mbar_wait_for(mb_in, 0, kTcBudget);   // the copies still in flight land before the block leaves
        }
        if (ok && !fault) {   // fault (test of the timeout path): nothing is issued, the accumulator wait runs out
            tc_fence_after();
            for (int tap = 0; tap < 27; tap++) {
                int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                if (FLIP) {
                    dz = -dz;
                    dy = -dy;
                    dx = -dx;
                }
                const uint32_t a0 = halo + (uint32_t)((((dz + 1) * 18 + dy + 1) * 10 + dx + 1) * 16);
                for (int k = 0; k < CK / 16; k++)
                    tc_mma(tmem, tc_sdesc(a0 + 2 * k * kHaloChunk, kHaloChunk, 160),
                           tc_sdesc(wts + (tap * nk8 + 2 * k) * N * 16, N * 16, 128), IDESC,
                           (tap > 0 || k > 0) ? 1u : 0u);
            }
            tc_commit(mb_acc);
        }
    }
    ok = !__syncthreads_or(!ok);
    bool done = ok && mbar_wait_for(mb_acc, 0, fault ? (1ll << 21) : kTcBudget);
    done = !__syncthreads_or(!done);
    tc_fence_after();
    if (done) {
        const int x = x0 + (tid & 7), y = y0 + (tid >> 3);
        const bool mine = y < n;
        const size_t r = ((((size_t)b * n + z0) * n + y) * n + x);
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc_ld16(lane_base + c0, v);
            if (bias)
#pragma unroll
                for (int i = 0; i < 16; i++)
                    v[i] += bias[c0 + i];
            if (relu)
#pragma unroll
                for (int i = 0; i < 16; i++)
                    v[i] = fmaxf(v[i], 0.f);
            if (!mine)
                continue;
            if (out_bf16) {
                uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<bf16 *>(out) + r * N + c0);
                o[0] = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
                o[1] = make_uint4(pack2(v[8], v[9]), pack2(v[10], v[11]), pack2(v[12], v[13]), pack2(v[14], v[15]));
            } else {
                float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(out) + r * N + c0);
#pragma unroll
                for (int i = 0; i < 4; i++)
                    o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tc_dealloc(tmem, NCOL);
    if (!done && tid == 0)
        atomicExch(err, 1);
}

// The halo convolution as a persistent kernel: each block loads all 27 taps'
// weights once and then walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// with two halo buffers and two TMEM accumulators, so that the TMA of tile
// i + 2 and the MMAs of tile i + 1 run while the block stores tile i.  Thread
// 0 issues every copy and product; the mbarriers of buffer s (halo arrived,
// accumulator complete) complete once per tile on that buffer, the k-th time
// with parity k & 1, and a phase is always waited for before the next copy or
// product on that buffer is issued.  Every wait is bounded; on a timeout the
// block stops issuing, waits (bounded) for what it has in flight, frees its
// TMEM and raises *err.
template <int N, bool FLIP>
__global__ void __launch_bounds__(128) k_conv3_halo_p(const __grid_constant__ CUtensorMap tm_in,
                                                      const bf16 *__restrict__ W, int CK,
                                                      const float *__restrict__ bias, void *__restrict__ out,
                                                      int out_bf16, int relu, int lg, int ntiles, int fault,
                                                      int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[4];   // 0, 1: halo of buffer s arrived; 2, 3: accumulator s complete
    __shared__ uint32_t tslot;
    constexpr int NCOL = N < 32 ? 32 : N;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, N);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nk8 = CK >> 3;
    const uint32_t hbytes = (uint32_t)(nk8 * kHaloChunk);
    const uint32_t halo0 = smem_u32(smem), wts = halo0 + 2 * hbytes;
    const int n = 1 << lg;
    const int tx = n >> 3, ty = (n + 15) >> 4;
    if (warp == 0) {
        tc_alloc(smem_u32(&tslot), 2 * NCOL);
        tc_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < 4; q++)
            mbar_init1(smem_u32(&mbar[q]));
        fence_mbar_init();
    }
    for (int e = tid; e < 27 * N * nk8; e += 128) {
        const int k8 = e % nk8, row = e / nk8;   // row = tap * N + output channel
        const int tap = row / N, nn = row - tap * N;
        cp16(wts + ((tap * nk8 + k8) * N + nn) * 16, W + (size_t)row * CK + 8 * k8, true);
    }
    cp_commit();
    cp_wait<0>();
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int first = blockIdx.x, stride = gridDim.x;
    const int nt = first < ntiles ? (ntiles - 1 - first) / stride + 1 : 0;
    auto coords = [&](int i, int &x0, int &y0, int &z0, int &b) {
        int t = first + i * stride;
        x0 = (t % tx) * 8;
        t /= tx;
        y0 = (t % ty) * 16;
        t /= ty;
        z0 = t % n;
        b = t / n;
    };
    auto load = [&](int i) {   // thread 0: the halo of tile i into buffer i & 1
        int x0, y0, z0, b;
        coords(i, x0, y0, z0, b);
        const uint32_t mb = smem_u32(&mbar[i & 1]), dst = halo0 + (uint32_t)(i & 1) * hbytes;
        mbar_expect_tx(mb, (uint32_t)(nk8 * kHaloRows * 16));
        for (int k8 = 0; k8 < nk8; k8++)
            tma_load5(dst + k8 * kHaloChunk, &tm_in, 8 * k8, x0 - 1, y0 - 1, z0 - 1, b, mb);
    };
    auto issue = [&](int i) {   // thread 0: the 27 taps' products of tile i into accumulator i & 1
        const uint32_t hb = halo0 + (uint32_t)(i & 1) * hbytes, d = tmem + (uint32_t)((i & 1) * NCOL);
        tc_fence_after();
        for (int tap = 0; tap < 27; tap++) {
            int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            if (FLIP) {
                dz = -dz;
                dy = -dy;
                dx = -dx;
            }
            const uint32_t a0 = hb + (uint32_t)((((dz + 1) * 18 + dy + 1) * 10 + dx + 1) * 16);
            for (int k = 0; k < CK / 16; k++)
                tc_mma(d, tc_sdesc(a0 + 2 * k * kHaloChunk, kHaloChunk, 160),
                       tc_sdesc(wts + (tap * nk8 + 2 * k) * N * 16, N * 16, 128), IDESC,
                       (tap > 0 || k > 0) ? 1u : 0u);
        }
        tc_commit(smem_u32(&mbar[2 + (i & 1)]));
    };
    // thread 0's count of tiles whose copies were issued / waited for and
    // whose products were issued (for the exit after a timeout)
    int tma_issued = 0, tma_waited = 0, mma_issued = 0;
    bool ok = true;
    if (tid == 0 && nt > 0) {
        load(0);
        tma_issued = 1;
        if (nt > 1) {
            load(1);
            tma_issued = 2;
        }
        ok = mbar_wait_for(smem_u32(&mbar[0]), 0, kTcBudget);
        if (ok) {
            tma_waited = 1;
            if (!fault) {   // fault (test of the timeout path): nothing is issued, the accumulator wait runs out
                issue(0);
                mma_issued = 1;
            }
        }
    }
    ok = !__syncthreads_or(!ok);
    int i = 0;
    for (; ok && i < nt; i++) {
        const int s = i & 1;
        bool good = true;
        if (tid == 0 && i + 1 < nt) {
            good = mbar_wait_for(smem_u32(&mbar[(i + 1) & 1]), ((i + 1) >> 1) & 1, kTcBudget);
            if (good) {
                tma_waited = i + 2;
                if (!fault) {
                    issue(i + 1);
                    mma_issued = i + 2;
                }
            }
        }
        good = good && mbar_wait_for(smem_u32(&mbar[2 + s]), (i >> 1) & 1, fault ? (1ll << 21) : kTcBudget);
        if (__syncthreads_or(!good)) {
            ok = false;
            break;
        }
        if (tid == 0 && i + 2 < nt) {   // buffer s is free: the products of tile i have completed
            load(i + 2);
            tma_issued = i + 3;
        }
        tc_fence_after();
        int x0, y0, z0, b;
        coords(i, x0, y0, z0, b);
        const int x = x0 + (tid & 7), y = y0 + (tid >> 3);
        const bool mine = y < n;
        const size_t r = ((((size_t)b * n + z0) * n + y) * n + x);
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * NCOL);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc_ld16(lane_base + c0, v);
            if (bias)
#pragma unroll
                for (int q = 0; q < 16; q++)
                    v[q] += bias[c0 + q];
            if (relu)
#pragma unroll
                for (int q = 0; q < 16; q++)
                    v[q] = fmaxf(v[q], 0.f);
            if (!mine)
                continue;
            if (out_bf16) {
                uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<bf16 *>(out) + r * N + c0);
                o[0] = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
                o[1] = make_uint4(pack2(v[8], v[9]), pack2(v[10], v[11]), pack2(v[12], v[13]), pack2(v[14], v[15]));
            } else {
                float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(out) + r * N + c0);
#pragma unroll
                for (int q = 0; q < 4; q++)
                    o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
        tc_fence_before();
        __syncthreads();   // accumulator s read by every thread before tile i + 2's products
    }
    if (!ok && tid == 0) {   // what is still in flight lands before the block leaves
        for (int j = tma_waited; j < tma_issued; j++)
            mbar_wait_for(smem_u32(&mbar[j & 1]), (j >> 1) & 1, kTcBudget);
        for (int j = i; j < mma_issued; j++)
            mbar_wait_for(smem_u32(&mbar[2 + (j & 1)]), (j >> 1) & 1, kTcBudget);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tc_dealloc(tmem, 2 * NCOL);
    if (!ok && tid == 0)
        atomicExch(err, 1);
}

// FP32 -> BF16 (round to nearest even), 8 values per thread
__global__ void k_to_bf16(const float *__restrict__ src, bf16 *__restrict__ dst, long n8)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n8; e += (long)gridDim.x * blockDim.x) {
        const float4 a = reinterpret_cast<const float4 *>(src)[2 * e], c = reinterpret_cast<const float4 *>(src)[2 * e + 1];
        reinterpret_cast<uint4 *>(dst)[e] =
            make_uint4(pack2(a.x, a.y), pack2(a.z, a.w), pack2(c.x, c.y), pack2(c.z, c.w));
    }
}

// Weight and bias gradients of a 3x3x3 convolution (FP32 on the CUDA cores):
//   dW[tap][ci][co] += sum_v in[v + off(tap)][ci] * d[v][co],  db[co] += sum_v d[v][co]
// Each block takes one tap and a run of voxels, stages 32 voxels at a time
// in shared memory and accumulates 4x4 (ci, co) tiles per thread.
__global__ void __launch_bounds__(kT) k_wgrad(const bf16 *__restrict__ in, int CKin, int Cin, const float *__restrict__ d,
                                              int N, float *__restrict__ dW, float *__restrict__ db, int lg, int V,
                                              int vox_per_block)
{
    constexpr int VS = 32;
    __shared__ float sIn[VS][128 + 1];
    __shared__ float sD[VS][64 + 1];
    const int tap = blockIdx.y;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int n = 1 << lg, msk = n - 1;
    const int ntc = Cin / 4 > 0 ? (Cin + 3) / 4 : 1, nto = N / 4;
    const int ntiles = ntc * nto;
    float acc[2][16];
    for (int u = 0; u < 2; u++)
        for (int e = 0; e < 16; e++)
            acc[u][e] = 0.f;
    float bacc = 0.f;
    const int vbeg = blockIdx.x * vox_per_block, vend = min(vbeg + vox_per_block, V);
    for (int v0 = vbeg; v0 < vend; v0 += VS) {
        __syncthreads();
        for (int e = threadIdx.x; e < VS * Cin; e += kT) {
            const int vv = e / Cin, ci = e - vv * Cin;
            const int v = v0 + vv;
            float val = 0.f;
            if (v < vend) {
                const int x = v & msk, y = (v >> lg) & msk, z = (v >> (2 * lg)) & msk, b = v >> (3 * lg);
                const int zz = z + dz, yy = y + dy, xx = x + dx;
                if ((unsigned)zz < (unsigned)n && (unsigned)yy < (unsigned)n && (unsigned)xx < (unsigned)n)
                    val = __bfloat162float(in[(size_t)((((b << lg | zz) << lg | yy) << lg) | xx) * CKin + ci]);
            }
            sIn[vv][ci] = val;
        }
        for (int e = threadIdx.x; e < VS * N; e += kT) {
            const int vv = e / N, co = e - vv * N;
            const int v = v0 + vv;
            sD[vv][co] = v < vend ? d[(size_t)v * N + co] : 0.f;
        }
        __syncthreads();
        for (int u = 0; u < 2; u++) {
            const int tile = threadIdx.x + u * kT;
            if (tile >= ntiles)
                break;
            const int tc = tile / nto, to = tile - tc * nto;
            for (int vv = 0; vv < VS; vv++) {
                float a[4], bb[4];
                for (int e = 0; e < 4; e++) {
                    const int ci = tc * 4 + e;
                    a[e] = ci < Cin ? sIn[vv][ci] : 0.f;
                    bb[e] = sD[vv][to * 4 + e];
                }
                for (int i = 0; i < 4; i++)
                    for (int j = 0; j < 4; j++)
                        acc[u][i * 4 + j] = fmaf(a[i], bb[j], acc[u][i * 4 + j]);
            }
        }
        if (tap == 13 && threadIdx.x < N)
            for (int vv = 0; vv < VS; vv++)
                bacc += sD[vv][threadIdx.x];
    }
    for (int u = 0; u < 2; u++) {
        const int tile = threadIdx.x + u * kT;
        if (tile >= ntiles)
            break;
        const int tc = tile / nto, to = tile - tc * nto;
        for (int i = 0; i < 4; i++) {
            const int ci = tc * 4 + i;
            if (ci >= Cin)
                continue;
            for (int j = 0; j < 4; j++)
                atomicAdd(&dW[((size_t)tap * Cin + ci) * N + to * 4 + j], acc[u][i * 4 + j]);
        }
    }
    if (tap == 13 && threadIdx.x < N && db)
        atomicAdd(&db[threadIdx.x], bacc);
}

// master FP32 weights [27][Cin][Cout] -> forward layout [27][Cout][CKin] and
// backward-data layout [27][Cin_p16][Cout] (BF16, zero padded)
__global__ void k_pack_weights(const float *__restrict__ w, int Cin, int CKin, int Cout, bf16 *__restrict__ wf,
                               bf16 *__restrict__ wd)
{
    const int total = 27 * CKin * Cout;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int co = e % Cout, ci = (e / Cout) % CKin, tap = e / (Cout * CKin);
        const float v = ci < Cin ? w[((size_t)tap * Cin + ci) * Cout + co] : 0.f;
        wf[((size_t)tap * Cout + co) * CKin + ci] = __float2bfloat16_rn(v);
        if (wd)
            wd[((size_t)tap * CKin + ci) * Cout + co] = __float2bfloat16_rn(v);
    }
}

// 2x2x2 mean pool (BF16, C channels): fine n = 2^lg -> coarse
__global__ void k_pool(const bf16 *__restrict__ in, bf16 *__restrict__ out, int C, int lgc, int Vc)
{
    const int nc = 1 << lgc, m = nc - 1, lgf = lgc + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Vc * C; e += gridDim.x * blockDim.x) {
        const int c = e % C, v = e / C;
        const int x = v & m, y = (v >> lgc) & m, z = (v >> (2 * lgc)) & m, b = v >> (3 * lgc);
        float s = 0.f;
        for (int k = 0; k < 8; k++) {
            const int fz = 2 * z + (k >> 2), fy = 2 * y + ((k >> 1) & 1), fx = 2 * x + (k & 1);
            s += __bfloat162float(in[(size_t)((((b << lgf | fz) << lgf | fy) << lgf) | fx) * C + c]);
        }
        out[e] = __float2bfloat16_rn(0.125f * s);
    }
}

// pool backward, added: dIn[fine] += dOut[coarse] / 8
__global__ void k_pool_bwd_add(const float *__restrict__ dout, float *__restrict__ din, int C, int lgf, int Vf)
{
    const int nf = 1 << lgf, m = nf - 1, lgc = lgf - 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Vf * C; e += gridDim.x * blockDim.x) {
        const int c = e % C, v = e / C;
        const int x = v & m, y = (v >> lgf) & m, z = (v >> (2 * lgf)) & m, b = v >> (3 * lgf);
        din[e] += 0.125f * dout[(size_t)((((b << lgc | (z >> 1)) << lgc | (y >> 1)) << lgc) | (x >> 1)) * C + c];
    }
}

// [up(low), skip] at the fine level: channels 0..Cu-1 from the parent, Cu..Cu+Cs-1 from skip
__global__ void k_upcat(const bf16 *__restrict__ low, int Cu, const bf16 *__restrict__ skip, int Cs,
                        bf16 *__restrict__ out, int lgf, int Vf)
{
    const int nf = 1 << lgf, m = nf - 1, lgc = lgf - 1, C = Cu + Cs;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Vf * C; e += gridDim.x * blockDim.x) {
        const int c = e % C, v = e / C;
        if (c < Cu) {
            const int x = v & m, y = (v >> lgf) & m, z = (v >> (2 * lgf)) & m, b = v >> (3 * lgf);
            out[e] = low[(size_t)((((b << lgc | (z >> 1)) << lgc | (y >> 1)) << lgc) | (x >> 1)) * Cu + c];
        } else {
            out[e] = skip[(size_t)v * Cs + c - Cu];
        }
    }
}

// backward of k_upcat: dLow[coarse] = sum of the 8 children's channels 0..Cu-1; dSkip = channels Cu.. (written)
__global__ void k_upcat_bwd(const float *__restrict__ dout, int Cu, int Cs, float *__restrict__ dlow,
                            float *__restrict__ dskip, int lgc, int Vc)
{
    const int nc = 1 << lgc, m = nc - 1, lgf = lgc + 1, C = Cu + Cs;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Vc * Cu; e += gridDim.x * blockDim.x) {
        const int c = e % Cu, v = e / Cu;
        const int x = v & m, y = (v >> lgc) & m, z = (v >> (2 * lgc)) & m, b = v >> (3 * lgc);
        float s = 0.f;
        for (int k = 0; k < 8; k++) {
            const int fz = 2 * z + (k >> 2), fy = 2 * y + ((k >> 1) & 1), fx = 2 * x + (k & 1);
            s += dout[(size_t)((((b << lgf | fz) << lgf | fy) << lgf) | fx) * C + c];
        }
        dlow[e] = s;
    }
    const int Vf = Vc * 8;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Vf * Cs; e += gridDim.x * blockDim.x) {
        const int c = e % Cs, v = e / Cs;
        dskip[e] = dout[(size_t)v * C + Cu + c];
    }
}

// d *= (act > 0)
__global__ void k_relu_mask(float *__restrict__ d, const bf16 *__restrict__ act, long n)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(act[e]) > 0.f))
            d[e] = 0.f;
}

// y[v] = sum_c d0[v][c] w[c] + b
__global__ void k_out1(const bf16 *__restrict__ d0, const float *__restrict__ w, const float *__restrict__ b,
                       float *__restrict__ y, int V)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        float s = b[0];
        for (int c = 0; c < 16; c++)
            s += __bfloat162float(d0[(size_t)v * 16 + c]) * w[c];
        y[v] = s;
    }
}

// loss = mean (y - t)^2 per element; dy = 2 (y - t) / V; dd0 = dy w; dw, db of the 1x1 layer
__global__ void k_out1_bwd(const float *__restrict__ y, const float *__restrict__ tgt, const bf16 *__restrict__ d0,
                           const float *__restrict__ w, float *__restrict__ dd0, float *__restrict__ dw,
                           float *__restrict__ db, float *__restrict__ loss, int V)
{
    float accw[16], accb = 0.f, accl = 0.f;
    for (int c = 0; c < 16; c++)
        accw[c] = 0.f;
    const float inv = 1.f / (float)V;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        const float r = y[v] - tgt[v];
        const float dy = 2.f * r * inv;
        accl += r * r * inv;
        accb += dy;
        for (int c = 0; c < 16; c++) {
            accw[c] += dy * __bfloat162float(d0[(size_t)v * 16 + c]);
            dd0[(size_t)v * 16 + c] = dy * w[c];
        }
    }
    // block reductions of the 16 weight gradients, the bias gradient and the loss
    float vals[18];
    for (int c = 0; c < 16; c++)
        vals[c] = accw[c];
    vals[16] = accb;
    vals[17] = accl;
    for (int q = 0; q < 18; q++) {
        float v = vals[q];
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, o);
        vals[q] = v;
    }
    __shared__ float red2[18][kT / 32];
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 18; q++)
            red2[q][threadIdx.x >> 5] = vals[q];
    __syncthreads();
    if (threadIdx.x < 18) {
        float s = 0.f;
        for (int wv = 0; wv < kT / 32; wv++)
            s += red2[threadIdx.x][wv];
        if (threadIdx.x < 16)
            atomicAdd(&dw[threadIdx.x], s);
        else if (threadIdx.x == 16)
            atomicAdd(db, s);
        else
            atomicAdd(loss, s);
    }
}

// AdamW on FP32 master weights
__global__ void k_adamw(float *__restrict__ p, const float *__restrict__ gr, float *__restrict__ m, float *__restrict__ v,
                        long n, float lr, float b1, float b2, float eps, float wd, float c1, float c2)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const float gg = gr[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * ((mm / c1) / (sqrtf(vv / c2) + eps) + wd * p[e]);
    }
}

// h^2 r = 4 pi G rho h^2 - (sum of the 6 neighbours - 6 Phi) on Omega, from
// (n+4)^3 level blocks (blk = 1) or copied from a dense array (blk = 0).
__global__ void k_resid_in(const double *__restrict__ rho, const double *__restrict__ phi,
                           const double *__restrict__ resid, int n, int blk, int lg, int B,
                           const double *__restrict__ frho, double *__restrict__ rh2)
{
    const int V = 1 << (3 * lg), m = (1 << lg) - 1, E = n + 4;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * V; e += gridDim.x * blockDim.x) {
        if (!blk) {
            rh2[e] = resid[e];
            continue;
        }
        const int b = e / V, v = e - b * V;
        const int x = v & m, y = (v >> lg) & m, z = v >> (2 * lg);
        const size_t q = (size_t)b * E * E * E + ((size_t)(z + 2) * E + y + 2) * E + x + 2;
        const size_t s1 = 1, s2 = E, s3 = (size_t)E * E;
        const double nb = phi[q - s1] + phi[q + s1] + phi[q - s2] + phi[q + s2] + phi[q - s3] + phi[q + s3];
        rh2[e] = frho[b] * rho[q] - (nb - 6.0 * phi[q]);
    }
}

// per sample b (blockIdx.y): the maxima of |Phi| on Omega and of |h^2 r| over
// this block's share of the cells, folded into bits[2b], bits[2b+1] by an
// atomic max on the float bit patterns (non-negative floats order as their
// bits: the result is the exact maximum, whatever the order)
__global__ void k_scales(const double *__restrict__ phi, const double *__restrict__ rh2, int n, int blk, int lg,
                         unsigned *__restrict__ bits)
{
    __shared__ float red[2][kT / 32];
    const int b = blockIdx.y;
    const int V = 1 << (3 * lg), m = (1 << lg) - 1, E = n + 4;
    float mx = 0.f, mr = 0.f;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        const int x = v & m, y = (v >> lg) & m, z = v >> (2 * lg);
        const size_t q = blk ? (size_t)b * E * E * E + ((size_t)(z + 2) * E + y + 2) * E + x + 2 : (size_t)b * V + v;
        mx = fmaxf(mx, fabsf((float)phi[q]));
        mr = fmaxf(mr, fabsf((float)rh2[(size_t)b * V + v]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        mr = fmaxf(mr, __shfl_down_sync(0xffffffffu, mr, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = mx;
        red[1][threadIdx.x >> 5] = mr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f, sr = 0.f;
        for (int w = 0; w < kT / 32; w++) {
            s = fmaxf(s, red[0][w]);
            sr = fmaxf(sr, red[1][w]);
        }
        atomicMax(&bits[2 * b], __float_as_uint(s));
        atomicMax(&bits[2 * b + 1], __float_as_uint(sr));
    }
}

// scale[2b] = max |Phi|, scale[2b+1] = max |h^2 r| (1 where the maximum is zero)
__global__ void k_scales_fin(const unsigned *__restrict__ bits, int B, float *__restrict__ scale)
{
    for (int e = threadIdx.x; e < 2 * B; e += blockDim.x) {
        const float v = __uint_as_float(bits[e]);
        scale[e] = v > 0.f ? v : 1.f;
    }
}

__global__ void k_make_input(const double *__restrict__ rho, const double *__restrict__ phi,
                             const double *__restrict__ rh2, int n, int blk, int lg, int B,
                             const double *__restrict__ frho, const float *__restrict__ scale, bf16 *__restrict__ x0)
{
    const int V = 1 << (3 * lg), m = (1 << lg) - 1, E = n + 4;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * V; e += gridDim.x * blockDim.x) {
        const int b = e / V, v = e - b * V;
        const int x = v & m, y = (v >> lg) & m, z = v >> (2 * lg);
        const size_t q = blk ? (size_t)b * E * E * E + ((size_t)(z + 2) * E + y + 2) * E + x + 2 : (size_t)e;
        const float s = scale[2 * b], sr = scale[2 * b + 1];
        bf16 *o = x0 + (size_t)e * 16;
        o[0] = __float2bfloat16_rn((float)(frho[b] * rho[q]) / s);
        o[1] = __float2bfloat16_rn((float)phi[q] / s);
        o[2] = __float2bfloat16_rn((float)rh2[e] / sr);
        for (int c = 3; c < 16; c++)
            o[c] = __float2bfloat16_rn(0.f);
    }
}

// output scale of sample b: s_r n^2 / 16
__device__ __forceinline__ double out_scale(const float *scale, int b, int n)
{
    return (double)scale[2 * b + 1] * (double)n * (double)n / 16.0;
}

// training target: (phi_true - phi_interp) / out_scale
__global__ void k_make_target(const double *__restrict__ phi_t, const double *__restrict__ phi_i,
                              const float *__restrict__ scale, int n, int V, int B, float *__restrict__ tgt)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * V; e += gridDim.x * blockDim.x)
        tgt[e] = (float)((phi_t[e] - phi_i[e]) / out_scale(scale, e / V, n));
}

// Phi += out_scale * y on Omega (block or dense layout)
__global__ void k_apply(double *__restrict__ phi, int n, int blk, int lg, int B, const float *__restrict__ scale,
                        const float *__restrict__ y)
{
    const int V = 1 << (3 * lg), m = (1 << lg) - 1, E = n + 4;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * V; e += gridDim.x * blockDim.x) {
        const int b = e / V, v = e - b * V;
        const int x = v & m, yy = (v >> lg) & m, z = v >> (2 * lg);
        const size_t q = blk ? (size_t)b * E * E * E + ((size_t)(z + 2) * E + yy + 2) * E + x + 2 : (size_t)e;
        phi[q] += out_scale(scale, b, n) * (double)y[e];
    }
}

__global__ void k_fill(float *p, long n, float v)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        p[e] = v;
}

// ---------------------------------------------------------------------------
// layers
// ---------------------------------------------------------------------------
struct Conv {
    int cin, ckin, cout;     // real input channels, padded K channels, outputs
    long woff, boff;         // offsets into the parameter vector
};

// the nine 3x3x3 convolutions, then the 1x1 output (16 weights + bias)
const int kConvDims[9][2] = {{3, 16}, {16, 16}, {16, 32}, {32, 32}, {32, 64}, {64, 64}, {128, 32}, {64, 16}, {32, 16}};

int pad16(int c) { return (c + 15) / 16 * 16; }

}  // namespace

struct mg_unet {
    int nmax = 0, bmax = 0;
    Conv conv[9];
    long nparam = 0;
    float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // FP32 master parameters and AdamW state
    bf16 *wf[9] = {}, *wd[9] = {};                                     // packed BF16 weights
    // activations (BF16) and gradients (FP32), sized for bmax * nmax^3
    bf16 *x0 = nullptr, *a0 = nullptr, *s0 = nullptr, *p0 = nullptr, *a1 = nullptr, *s1 = nullptr, *p1 = nullptr,
         *s2 = nullptr, *p2 = nullptr, *a3 = nullptr, *u2 = nullptr, *d2 = nullptr, *u1 = nullptr, *d1 = nullptr,
         *u0 = nullptr, *d0 = nullptr;
    float *y = nullptr, *tgt = nullptr, *scale = nullptr, *loss = nullptr, *gA = nullptr, *gB = nullptr, *gC = nullptr;
    double *frho = nullptr, *rh2 = nullptr;
    int *tcerr = nullptr;          // set when a tensor-core completion wait ran out
    bf16 *gbf = nullptr;           // BF16 copy of a data-gradient pass's input gradient
    unsigned *scale_bits = nullptr; // per-sample maxima as float bit patterns
    char *mem = nullptr;
    long step = 0;
    cudaStream_t stream = nullptr;
    bool packed = false;
};

namespace {

// The convolutions run on tcgen05 (k_conv3_tc); UNET_MMA_SYNC=1 selects the
// warp-level mma.sync kernel instead (for comparison).
bool use_mma_sync()
{
    static const bool on = [] {
        const char *v = std::getenv("UNET_MMA_SYNC");
        return v && v[0] == '1';
    }();
    return on;
}

constexpr int kTcSmemMax = 200 * 1024;  // kTcStages stages of 128 x CK and N x CK BF16 tiles

template <int N, bool FLIP>
cudaError_t conv_launch_tc(const bf16 *in, int CK, const bf16 *W, const float *bias, void *out, int out_bf16,
                           int relu, int lg, int V, int *err, cudaStream_t s)
{
    static cudaError_t attr = cudaFuncSetAttribute(k_conv3_tc<N, FLIP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   kTcSmemMax);
    if (attr)
        return attr;
    const size_t smem = (size_t)kTcStages * ((size_t)128 * CK * 2 + (size_t)N * CK * 2);
    if (smem > (size_t)kTcSmemMax || CK % 16 || CK > 128)
        return cudaErrorInvalidValue;
    k_conv3_tc<N, FLIP><<<(V + 127) / 128, 128, smem, s>>>(in, CK, W, bias, out, out_bf16, relu, lg, V, err);
    return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
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

// the persistent halo kernel with UNET_HALO_P=1 (measured as fast as the
// one-tile-per-block kernel at 4 x 64^3: 0.996 vs 0.989 ms a forward pass)
bool use_persistent_halo()
{
    static const bool on = [] {
        const char *v = std::getenv("UNET_HALO_P");
        return v && v[0] == '1';
    }();
    return on;
}

// the halo kernel applies when all 27 taps' weights fit beside the halo and
// the grid has at least 8 cells per edge
bool halo_applies(int CK, int N, int lg) { return 27 * N * CK * 2 <= 64 * 1024 && lg >= 3 && CK <= 64; }

template <int N, bool FLIP>
cudaError_t conv_launch_halo(const bf16 *in, int CK, const bf16 *W, const float *bias, void *out, int out_bf16,
                             int relu, int lg, int V, int *err, cudaStream_t s)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc)
        return cudaErrorNotSupported;
    const int n = 1 << lg, B = V >> (3 * lg);
    CUtensorMap mi{};
    const cuuint64_t di[5] = {(cuuint64_t)CK, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)B};
    const cuuint64_t si[4] = {(cuuint64_t)CK * 2, (cuuint64_t)n * CK * 2, (cuuint64_t)n * n * CK * 2,
                              (cuuint64_t)n * n * n * CK * 2};
    const cuuint32_t bi[5] = {8, 10, 18, 3, 1}, e5[5] = {1, 1, 1, 1, 1};
    if (enc(&mi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(in), di, si, bi, e5,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)(CK / 8) * kHaloChunk + (size_t)27 * (CK / 8) * N * 16;
    static cudaError_t attr = cudaFuncSetAttribute(k_conv3_halo<N, FLIP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   200 * 1024);
    if (attr)
        return attr;
    const int tiles = B * n * ((n + 15) / 16) * (n / 8);
    static const bool by_tma = [] {   // the halo by one TMA box per chunk; UNET_HALO_TMA=0: cp.async rows
        const char *v = std::getenv("UNET_HALO_TMA");
        return !(v && v[0] == '0');
    }();
    static const int fault = [] {   // UNET_FAULT_WAIT=1: the accumulator waits run out (test of that path)
        const char *v = std::getenv("UNET_FAULT_WAIT");
        return v && v[0] == '1' ? 1 : 0;
    }();
    if (by_tma && use_persistent_halo()) {
        // persistent form: as many blocks as fit on the SMs at once, but never
        // more per SM than TMEM holds (each block keeps two accumulators of
        // NCOL columns allocated for its whole life; a block that could not
        // allocate would wait for one that never leaves)
        constexpr int NCOL = N < 32 ? 32 : N;
        constexpr int tmem_blocks = 512 / (2 * NCOL);
        size_t psmem = 2 * (size_t)(CK / 8) * kHaloChunk + (size_t)27 * (CK / 8) * N * 16;
        const size_t floor_smem = 233472 / (tmem_blocks + 1);   // more than 1/(t+1) of an SM's shared memory
        if (psmem < floor_smem)
            psmem = floor_smem;
        static cudaError_t pattr = [] {   // all of the SM's shared memory for several blocks
            cudaError_t e = cudaFuncSetAttribute(k_conv3_halo_p<N, FLIP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 200 * 1024);
            if (!e)
                e = cudaFuncSetAttribute(k_conv3_halo_p<N, FLIP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
            return e;
        }();
        if (pattr)
            return pattr;
        int per_sm = 0, dev = 0, nsm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3_halo_p<N, FLIP>, 128, psmem);
        if (!e)
            e = cudaGetDevice(&dev);
        if (!e)
            e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e)
            return e;
        // with one block per SM a block's tiles run one after another with
        // little to overlap: the one-tile-per-block kernel is faster there
        if (psmem <= 200 * 1024 && per_sm >= 2 && per_sm <= tmem_blocks) {
            const int grid = std::min(tiles, per_sm * nsm);
            k_conv3_halo_p<N, FLIP><<<grid, 128, psmem, s>>>(mi, W, CK, bias, out, out_bf16, relu, lg, tiles, fault,
                                                             err);
            return cudaGetLastError();
        }
    }
    k_conv3_halo<N, FLIP><<<tiles, 128, smem, s>>>(mi, in, by_tma ? 1 : 0, W, CK, bias, out, out_bf16, relu, lg, B,
                                                   fault, err);
    return cudaGetLastError();
}

// the halo kernel unless UNET_HALO=0
bool use_halo()
{
    static const bool on = [] {
        const char *v = std::getenv("UNET_HALO");
        return !(v && v[0] == '0');
    }();
    return on;
}

// tcgen05 path: FP32 input (the data-gradient pass) is rounded to BF16 first
// (into scratch), as the mma.sync kernel rounds it when it loads it
template <int NT, bool FLIP, typename TIn>
cudaError_t conv_launch(const TIn *in, int CK, const bf16 *W, const float *bias, void *out, int out_bf16, int relu,
                        int lg, int V, int *err, bf16 *scratch, cudaStream_t s)
{
    if (!use_mma_sync()) {
        const bf16 *src;
        if constexpr (sizeof(TIn) == 4) {
            const long n8 = (long)V * CK / 8;
            k_to_bf16<<<blocks_for(n8), kT, 0, s>>>(in, scratch, n8);
            src = scratch;
        } else {
            src = in;
        }
        if (use_halo() && halo_applies(CK, NT * 8, lg))
            return conv_launch_halo<NT * 8, FLIP>(src, CK, W, bias, out, out_bf16, relu, lg, V, err, s);
        return conv_launch_tc<NT * 8, FLIP>(src, CK, W, bias, out, out_bf16, relu, lg, V, err, s);
    }
    k_conv3<NT, FLIP, TIn><<<(V + 63) / 64, 128, 0, s>>>(in, CK, W, bias, out, out_bf16, relu, lg, V);
    return cudaGetLastError();
}

template <bool FLIP, typename TIn>
cudaError_t conv_any(const TIn *in, int CK, const bf16 *W, const float *bias, int N, void *out, int out_bf16, int relu,
                     int lg, int V, int *err, bf16 *scratch, cudaStream_t s)
{
    switch (N) {
    case 16: return conv_launch<2, FLIP, TIn>(in, CK, W, bias, out, out_bf16, relu, lg, V, err, scratch, s);
    case 32: return conv_launch<4, FLIP, TIn>(in, CK, W, bias, out, out_bf16, relu, lg, V, err, scratch, s);
    case 64: return conv_launch<8, FLIP, TIn>(in, CK, W, bias, out, out_bf16, relu, lg, V, err, scratch, s);
    case 128: return conv_launch<16, FLIP, TIn>(in, CK, W, bias, out, out_bf16, relu, lg, V, err, scratch, s);
    }
    return cudaErrorInvalidValue;
}

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n)
        l++;
    return l;
}

cudaError_t pack_all(mg_unet *u)
{
    for (int i = 0; i < 9; i++) {
        const Conv &c = u->conv[i];
        k_pack_weights<<<blocks_for(27L * c.ckin * c.cout), kT, 0, u->stream>>>(u->p + c.woff, c.cin, c.ckin, c.cout,
                                                                              u->wf[i], u->wd[i]);
    }
    u->packed = true;
    return cudaGetLastError();
}

// forward through the network for B samples of edge n = 2^lg (x0 ready)
cudaError_t forward(mg_unet *u, int B, int lg)
{
    cudaStream_t s = u->stream;
    const int V0 = B << (3 * lg), V1 = V0 >> 3, V2 = V1 >> 3, V3 = V2 >> 3;
    cudaError_t e;
    auto C = [&](int i) -> const Conv & { return u->conv[i]; };
    float *P = u->p;
#define FWD(i, in, out, lgv, V)                                                                                   \
    if ((e = conv_any<false, bf16>(in, C(i).ckin, u->wf[i], P + C(i).boff, C(i).cout, out, 1, 1, lgv, V, u->tcerr, \
                                   nullptr, s)))                                                                \
        return e;
    FWD(0, u->x0, u->a0, lg, V0);
    FWD(1, u->a0, u->s0, lg, V0);
    k_pool<<<blocks_for((long)V1 * 16), kT, 0, s>>>(u->s0, u->p0, 16, lg - 1, V1);
    FWD(2, u->p0, u->a1, lg - 1, V1);
    FWD(3, u->a1, u->s1, lg - 1, V1);
    k_pool<<<blocks_for((long)V2 * 32), kT, 0, s>>>(u->s1, u->p1, 32, lg - 2, V2);
    FWD(4, u->p1, u->s2, lg - 2, V2);
    k_pool<<<blocks_for((long)V3 * 64), kT, 0, s>>>(u->s2, u->p2, 64, lg - 3, V3);
    FWD(5, u->p2, u->a3, lg - 3, V3);
    k_upcat<<<blocks_for((long)V2 * 128), kT, 0, s>>>(u->a3, 64, u->s2, 64, u->u2, lg - 2, V2);
    FWD(6, u->u2, u->d2, lg - 2, V2);
    k_upcat<<<blocks_for((long)V1 * 64), kT, 0, s>>>(u->d2, 32, u->s1, 32, u->u1, lg - 1, V1);
    FWD(7, u->u1, u->d1, lg - 1, V1);
    k_upcat<<<blocks_for((long)V0 * 32), kT, 0, s>>>(u->d1, 16, u->s0, 16, u->u0, lg, V0);
    FWD(8, u->u0, u->d0, lg, V0);
#undef FWD
    k_out1<<<blocks_for(V0), kT, 0, s>>>(u->d0, P + u->nparam - 17, P + u->nparam - 1, u->y, V0);
    return cudaGetLastError();
}

template <int CK, int N>
cudaError_t wgrad_tc(const bf16 *in, int Cin, const float *g, float *dW, int lg, int V, int *err, cudaStream_t s)
{
    constexpr size_t smem = 2 * ((size_t)128 * 64 * 2 + (size_t)N * 64 * 2);
    static cudaError_t attr = cudaFuncSetAttribute(k_wgrad_tc<CK, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
    if (attr)
        return attr;
    const int vchunk = 4096;
    dim3 grid((V + vchunk - 1) / vchunk, (27 + 128 / CK - 1) / (128 / CK));
    k_wgrad_tc<CK, N><<<grid, 128, smem, s>>>(in, Cin, g, dW, lg, V, vchunk, err);
    return cudaGetLastError();
}

cudaError_t wgrad_tc_any(int CK, int N, const bf16 *in, int Cin, const float *g, float *dW, int lg, int V, int *err,
                         cudaStream_t s)
{
#define WG(ck, nn)                   \
    if (CK == ck && N == nn)         \
        return wgrad_tc<ck, nn>(in, Cin, g, dW, lg, V, err, s);
    WG(16, 16) WG(16, 32) WG(32, 32) WG(32, 64) WG(64, 64) WG(128, 32) WG(64, 16) WG(32, 16)
#undef WG
    return cudaErrorInvalidValue;
}

// weight gradients of conv i from its input activation and output gradient g (FP32, N channels)
cudaError_t wgrad(mg_unet *u, int i, const bf16 *in, const float *g, int lg, int V)
{
    const Conv &c = u->conv[i];
    if (use_mma_sync()) {
        const int vpb = 4096;
        dim3 grid((V + vpb - 1) / vpb, 27);
        k_wgrad<<<grid, kT, 0, u->stream>>>(in, c.ckin, c.cin, g, c.cout, u->grad + c.woff, u->grad + c.boff, lg, V,
                                            vpb);
        return cudaGetLastError();
    }
    cudaError_t e = wgrad_tc_any(c.ckin, c.cout, in, c.cin, g, u->grad + c.woff, lg, V, u->tcerr, u->stream);
    if (e)
        return e;
    const int vchunk = 4096;
    k_bias_grad<<<(V + vchunk - 1) / vchunk, 256, 0, u->stream>>>(g, c.cout, V, vchunk, u->grad + c.boff);
    return cudaGetLastError();
}

cudaError_t dgrad(mg_unet *u, int i, const float *g, float *out, int lg, int V)
{
    const Conv &c = u->conv[i];
    return conv_any<true, float>(g, c.cout, u->wd[i], nullptr, c.ckin, out, 0, 0, lg, V, u->tcerr, u->gbf,
                                 u->stream);
}

cudaError_t mask(mg_unet *u, float *g, const bf16 *act, long n)
{
    k_relu_mask<<<blocks_for(n), kT, 0, u->stream>>>(g, act, n);
    return cudaGetLastError();
}

// backward pass (loss gradient from y vs tgt), accumulating into u->grad
cudaError_t backward(mg_unet *u, int B, int lg)
{
    cudaStream_t s = u->stream;
    const int V0 = B << (3 * lg), V1 = V0 >> 3, V2 = V1 >> 3, V3 = V2 >> 3;
    float *gA = u->gA, *gB = u->gB, *gC = u->gC;
    cudaError_t e;
    k_out1_bwd<<<blocks_for(V0, 152 * 4), kT, 0, s>>>(u->y, u->tgt, u->d0, u->p + u->nparam - 17, gA,
                                                     u->grad + u->nparam - 17, u->grad + u->nparam - 1, u->loss, V0);
    // D0 (u0 -> d0), gA = dd0 [V0][16]
    if ((e = mask(u, gA, u->d0, (long)V0 * 16)) || (e = wgrad(u, 8, u->u0, gA, lg, V0)) ||
        (e = dgrad(u, 8, gA, gB, lg, V0)))
        return e;                                                        // gB = du0 [V0][32]
    // split du0 -> dd1 (coarse) and ds0 (gC)
    k_upcat_bwd<<<blocks_for((long)V0 * 16), kT, 0, s>>>(gB, 16, 16, gA, gC, lg - 1, V1);   // gA = dd1 [V1][16], gC = ds0 [V0][16]
    if ((e = mask(u, gA, u->d1, (long)V1 * 16)) || (e = wgrad(u, 7, u->u1, gA, lg - 1, V1)) ||
        (e = dgrad(u, 7, gA, gB, lg - 1, V1)))
        return e;                                                        // gB = du1 [V1][64]
    // ds1 lives behind ds0 in gC
    float *ds1 = gC + (size_t)V0 * 16;
    k_upcat_bwd<<<blocks_for((long)V1 * 32), kT, 0, s>>>(gB, 32, 32, gA, ds1, lg - 2, V2);  // gA = dd2 [V2][32]
    if ((e = mask(u, gA, u->d2, (long)V2 * 32)) || (e = wgrad(u, 6, u->u2, gA, lg - 2, V2)) ||
        (e = dgrad(u, 6, gA, gB, lg - 2, V2)))
        return e;                                                        // gB = du2 [V2][128]
    float *ds2 = ds1 + (size_t)V1 * 32;
    k_upcat_bwd<<<blocks_for((long)V2 * 64), kT, 0, s>>>(gB, 64, 64, gA, ds2, lg - 3, V3);  // gA = da3 [V3][64]
    if ((e = mask(u, gA, u->a3, (long)V3 * 64)) || (e = wgrad(u, 5, u->p2, gA, lg - 3, V3)) ||
        (e = dgrad(u, 5, gA, gB, lg - 3, V3)))
        return e;                                                        // gB = dp2 [V3][64]
    k_pool_bwd_add<<<blocks_for((long)V2 * 64), kT, 0, s>>>(gB, ds2, 64, lg - 2, V2);
    if ((e = mask(u, ds2, u->s2, (long)V2 * 64)) || (e = wgrad(u, 4, u->p1, ds2, lg - 2, V2)) ||
        (e = dgrad(u, 4, ds2, gB, lg - 2, V2)))
        return e;                                                        // gB = dp1 [V2][32]
    k_pool_bwd_add<<<blocks_for((long)V1 * 32), kT, 0, s>>>(gB, ds1, 32, lg - 1, V1);
    if ((e = mask(u, ds1, u->s1, (long)V1 * 32)) || (e = wgrad(u, 3, u->a1, ds1, lg - 1, V1)) ||
        (e = dgrad(u, 3, ds1, gB, lg - 1, V1)))
        return e;                                                        // gB = da1 [V1][32]
    if ((e = mask(u, gB, u->a1, (long)V1 * 32)) || (e = wgrad(u, 2, u->p0, gB, lg - 1, V1)) ||
        (e = dgrad(u, 2, gB, gA, lg - 1, V1)))
        return e;                                                        // gA = dp0 [V1][16]
    float *ds0 = gC;
    k_pool_bwd_add<<<blocks_for((long)V0 * 16), kT, 0, s>>>(gA, ds0, 16, lg, V0);
    if ((e = mask(u, ds0, u->s0, (long)V0 * 16)) || (e = wgrad(u, 1, u->a0, ds0, lg, V0)) ||
        (e = dgrad(u, 1, ds0, gB, lg, V0)))
        return e;                                                        // gB = da0 [V0][16]
    if ((e = mask(u, gB, u->a0, (long)V0 * 16)) || (e = wgrad(u, 0, u->x0, gB, lg, V0)))
        return e;
    return cudaGetLastError();
}

// He-style initialisation from a counter-based hash (deterministic per seed)
float hash_uniform(unsigned long long seed, unsigned long long i)
{
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)((z >> 11) * (1.0 / 9007199254740992.0));
}

}  // namespace

namespace {

// 4 once a tensor-core completion wait of a convolution ran out (the flag
// stays set), else 0; synchronises the stream
int tc_status(mg_unet *u)
{
    int f = 0;
    if (cudaMemcpyAsync(&f, u->tcerr, sizeof(int), cudaMemcpyDeviceToHost, u->stream) ||
        cudaStreamSynchronize(u->stream))
        return 3;
    return f ? 4 : 0;
}

}  // namespace

extern "C" {

long mg_unet_param_count(void)
{
    long n = 0;
    for (int i = 0; i < 9; i++)
        n += 27L * kConvDims[i][0] * kConvDims[i][1] + kConvDims[i][1];
    return n + 17;
}

int mg_unet_create(int nmax, int bmax, unsigned long long seed, void *stream, mg_unet **out)
{
    if (!out)
        return 1;
    *out = nullptr;
    if (nmax < 8 || (nmax & (nmax - 1)) || bmax < 1 || bmax > 1024)
        return 1;
    mg_unet *u = new (std::nothrow) mg_unet();
    if (!u)
        return 2;
    u->nmax = nmax;
    u->bmax = bmax;
    u->stream = (cudaStream_t)stream;
    long off = 0;
    for (int i = 0; i < 9; i++) {
        Conv &c = u->conv[i];
        c.cin = kConvDims[i][0];
        c.ckin = pad16(c.cin);
        c.cout = kConvDims[i][1];
        c.woff = off;
        off += 27L * c.cin * c.cout;
        c.boff = off;
        off += c.cout;
    }
    u->nparam = off + 17;
    const long V0 = (long)bmax * nmax * nmax * nmax;
    // arena
    std::vector<std::pair<void **, size_t>> sl;
    auto A = [&](void **p, size_t b) { sl.push_back({p, (b + 255) & ~(size_t)255}); };
    for (void **pp : {(void **)&u->p, (void **)&u->grad, (void **)&u->m, (void **)&u->v})
        A(pp, u->nparam * sizeof(float));
    for (int i = 0; i < 9; i++) {
        A((void **)&u->wf[i], 27L * u->conv[i].ckin * u->conv[i].cout * sizeof(bf16));
        A((void **)&u->wd[i], 27L * u->conv[i].ckin * u->conv[i].cout * sizeof(bf16));
    }
    const long V1 = V0 / 8, V2 = V1 / 8, V3 = V2 / 8;
    A((void **)&u->x0, V0 * 16 * sizeof(bf16));
    A((void **)&u->a0, V0 * 16 * sizeof(bf16));
    A((void **)&u->s0, V0 * 16 * sizeof(bf16));
    A((void **)&u->p0, V1 * 16 * sizeof(bf16));
    A((void **)&u->a1, V1 * 32 * sizeof(bf16));
    A((void **)&u->s1, V1 * 32 * sizeof(bf16));
    A((void **)&u->p1, V2 * 32 * sizeof(bf16));
    A((void **)&u->s2, V2 * 64 * sizeof(bf16));
    A((void **)&u->p2, V3 * 64 * sizeof(bf16));
    A((void **)&u->a3, V3 * 64 * sizeof(bf16));
    A((void **)&u->u2, V2 * 128 * sizeof(bf16));
    A((void **)&u->d2, V2 * 32 * sizeof(bf16));
    A((void **)&u->u1, V1 * 64 * sizeof(bf16));
    A((void **)&u->d1, V1 * 16 * sizeof(bf16));
    A((void **)&u->u0, V0 * 32 * sizeof(bf16));
    A((void **)&u->d0, V0 * 16 * sizeof(bf16));
    A((void **)&u->y, V0 * sizeof(float));
    A((void **)&u->tgt, V0 * sizeof(float));
    A((void **)&u->scale, 2048 * sizeof(float));
    A((void **)&u->scale_bits, 2048 * sizeof(unsigned));
    A((void **)&u->rh2, V0 * sizeof(double));
    A((void **)&u->loss, 256);
    A((void **)&u->tcerr, 256);
    A((void **)&u->gbf, V0 * 32 * sizeof(bf16));
    A((void **)&u->frho, bmax * sizeof(double));
    A((void **)&u->gA, V0 * 32 * sizeof(float));
    A((void **)&u->gB, V0 * 32 * sizeof(float));
    A((void **)&u->gC, (V0 * 16 + V1 * 32 + V2 * 64) * sizeof(float));
    size_t bytes = 0;
    for (auto &x : sl)
        bytes += x.second;
    if (cudaMalloc((void **)&u->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete u;
        return 2;
    }
    size_t pos = 0;
    for (auto &x : sl) {
        *x.first = u->mem + pos;
        pos += x.second;
    }
    cudaMemsetAsync(u->mem, 0, bytes, u->stream);
    // initial parameters: uniform(-a, a), a = sqrt(6 / fan_in); zero biases
    std::vector<float> h(u->nparam, 0.f);
    for (int i = 0; i < 9; i++) {
        const Conv &c = u->conv[i];
        const float a = std::sqrt(6.f / (27.f * c.cin));
        for (long k = 0; k < 27L * c.cin * c.cout; k++)
            h[c.woff + k] = a * (2.f * hash_uniform(seed, c.woff + k) - 1.f);
    }
    for (int c = 0; c < 16; c++)
        h[u->nparam - 17 + c] = 0.01f * (2.f * hash_uniform(seed, u->nparam + c) - 1.f);
    cudaMemcpyAsync(u->p, h.data(), u->nparam * sizeof(float), cudaMemcpyHostToDevice, u->stream);
    if (cudaStreamSynchronize(u->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(u->mem);
        delete u;
        return 3;
    }
    *out = u;
    return 0;
}

int mg_unet_destroy(mg_unet *u)
{
    if (!u)
        return 0;
    cudaStreamSynchronize(u->stream);
    cudaFree(u->mem);
    cudaGetLastError();
    delete u;
    return 0;
}

int mg_unet_get_params(mg_unet *u, float *out)
{
    if (!u || !out)
        return 1;
    if (cudaMemcpyAsync(out, u->p, u->nparam * sizeof(float), cudaMemcpyDeviceToHost, u->stream) ||
        cudaStreamSynchronize(u->stream))
        return 3;
    return 0;
}

int mg_unet_set_params(mg_unet *u, const float *in)
{
    if (!u || !in)
        return 1;
    if (cudaMemcpyAsync(u->p, in, u->nparam * sizeof(float), cudaMemcpyHostToDevice, u->stream) ||
        cudaStreamSynchronize(u->stream))
        return 3;
    u->packed = false;
    u->step = 0;
    return 0;
}

// Pack the BF16 weight copies now (before a solve graph captures inference).
int mg_unet_pack(mg_unet *u)
{
    if (!u)
        return 1;
    if (pack_all(u) || cudaStreamSynchronize(u->stream))
        return 3;
    return 0;
}

int mg_unet_get_grad(mg_unet *u, float *out)
{
    if (!u || !out)
        return 1;
    if (cudaMemcpyAsync(out, u->grad, u->nparam * sizeof(float), cudaMemcpyDeviceToHost, u->stream) ||
        cudaStreamSynchronize(u->stream))
        return 3;
    return 0;
}

// Internal entry used by the solver and by the public calls: from (n+4)^3
// blocks (blk = 1) or dense n^3 arrays (blk = 0) of B samples, predict y and
// (apply = 1) add scale * y to phi on Omega.
int mg_unet_predict_dev(mg_unet *u, int B, int n, int blk, const double *rho, double *phi, const double *resid,
                        const double *frho_dev, int apply, void *stream)
{
    if (!u || B < 1 || B > u->bmax || n < 8 || n > u->nmax || (n & (n - 1)) || (!blk && !resid))
        return 1;
    cudaStream_t s = stream ? (cudaStream_t)stream : u->stream;
    cudaStream_t keep = u->stream;
    u->stream = s;
    const int lg = ilog2(n);
    const int V0 = B << (3 * lg);
    if (!u->packed && pack_all(u)) {
        u->stream = keep;
        return 3;
    }
    k_resid_in<<<blocks_for(V0), kT, 0, s>>>(rho, phi, resid, n, blk, lg, B, frho_dev, u->rh2);
    cudaMemsetAsync(u->scale_bits, 0, 2 * B * sizeof(unsigned), s);
    k_scales<<<dim3(std::min(64, std::max(1, V0 / B / (kT * 16))), B), kT, 0, s>>>(phi, u->rh2, n, blk, lg,
                                                                                  u->scale_bits);
    k_scales_fin<<<1, 256, 0, s>>>(u->scale_bits, B, u->scale);
    k_make_input<<<blocks_for(V0), kT, 0, s>>>(rho, phi, u->rh2, n, blk, lg, B, frho_dev, u->scale, u->x0);
    cudaError_t e = forward(u, B, lg);
    if (!e && apply) {
        k_apply<<<blocks_for(V0), kT, 0, s>>>(phi, n, blk, lg, B, u->scale, u->y);
        e = cudaGetLastError();
    }
    u->stream = keep;
    return e ? 3 : 0;
}

int mg_unet_forward(mg_unet *u, int B, int n, const double *rho, const double *phi_interp, const double *resid,
                    const double *frho, float *y_out)
{
    if (!u || !frho || B > u->bmax)
        return 1;
    if (cudaMemcpyAsync(u->frho, frho, B * sizeof(double), cudaMemcpyHostToDevice, u->stream))
        return 3;
    int r = mg_unet_predict_dev(u, B, n, 0, rho, const_cast<double *>(phi_interp), resid, u->frho, 0, nullptr);
    if (r)
        return r;
    const long V0 = (long)B * n * n * n;
    if (y_out && (cudaMemcpyAsync(y_out, u->y, V0 * sizeof(float), cudaMemcpyDeviceToHost, u->stream) ||
                  cudaStreamSynchronize(u->stream)))
        return 3;
    return tc_status(u);
}

int mg_unet_train_step(mg_unet *u, int B, int n, const double *rho, const double *phi_interp,
                       const double *resid, const double *phi_true, const double *frho, float lr, float wd, int update,
                       float *loss_out)
{
    if (!u || !frho || B > u->bmax || n < 8 || n > u->nmax || (n & (n - 1)))
        return 1;
    cudaStream_t s = u->stream;
    const int lg = ilog2(n);
    const int V0 = B << (3 * lg);
    if (cudaMemcpyAsync(u->frho, frho, B * sizeof(double), cudaMemcpyHostToDevice, s))
        return 3;
    int r = mg_unet_predict_dev(u, B, n, 0, rho, const_cast<double *>(phi_interp), resid, u->frho, 0, nullptr);
    if (r)
        return r;
    k_make_target<<<blocks_for(V0), kT, 0, s>>>(phi_true, phi_interp, u->scale, n, 1 << (3 * lg), B, u->tgt);
    k_fill<<<blocks_for(u->nparam), kT, 0, s>>>(u->grad, u->nparam, 0.f);
    k_fill<<<1, 32, 0, s>>>(u->loss, 1, 0.f);
    if (backward(u, B, lg))
        return 3;
    if (update) {
        u->step++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)u->step), c2 = 1.f - std::pow(b2, (float)u->step);
        k_adamw<<<blocks_for(u->nparam), kT, 0, s>>>(u->p, u->grad, u->m, u->v, u->nparam, lr, b1, b2, 1e-8f, wd, c1, c2);
        u->packed = false;
    }
    float l = 0.f;
    if (cudaMemcpyAsync(&l, u->loss, sizeof(float), cudaMemcpyDeviceToHost, s) || cudaStreamSynchronize(s))
        return 3;
    if (loss_out)
        *loss_out = l;
    if (cudaGetLastError())
        return 3;
    return tc_status(u);
}

}  // extern "C"
