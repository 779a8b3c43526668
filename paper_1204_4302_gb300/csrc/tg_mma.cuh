// Dense block-CP contraction of the tensor-grid method (paper Sec. 3.2,
// Eq. "sumpot" with the factors already transformed) on the 5th-generation
// tensor cores:
//
//   Phi[g][i] = sum_K A[g][K] X[K][i],   A[g][K] = Z[K][k] Y[K][j],  g = k ny + j,
//
// a GEMM of M = nz ny rows, N = nx columns and K = 3 R r terms whose first
// operand is formed on the fly. FP32 accuracy from TF32 tensor operations by
// the three-term split (a = a_hi + a_lo, each rounded to TF32):
//   a b ~= a_hi b_hi + a_hi b_lo + a_lo b_hi
// (the dropped a_lo b_lo is below 2^-22 |a b|), accumulated in FP32 in tensor
// memory: the a_hi b_hi products in one accumulator, the two small cross
// terms in a second one, added in the epilogue. The tensor cores' FP32
// accumulation does not round to nearest (it leaves a bias of a fraction of
// an ulp of the accumulator per update), so keeping the small terms out of
// the large accumulator cuts its updates per 8 terms from three to one.
//
// One persistent CTA per SM loops over tiles of 128 rows by BN <= 256
// columns. Warp roles (320 threads):
//   warp 0, one lane: bulk-copies (TMA) the stage's B operand (X^T hi and lo,
//     pre-arranged in the swizzled shared-memory layout) on an mbarrier;
//   warp 1: allocates tensor memory; one lane issues tcgen05.mma (M 128,
//     N BN, K 8 per instruction; 6 per stage) and commits them to the
//     stage's "empty" barrier and, after a tile, to "tile full";
//   warps 2..9: form A = Z Y for 128 rows x 16 K per stage from the
//     transposed factors (two threads per row, 8 K each), split it into hi
//     and lo and store them in the 64-byte-swizzled K-major layout; after a
//     tile, read both accumulators back (tcgen05.ld; warp w reads TMEM lanes
//     32 (w mod 4) .., warps 2..5 and 6..9 alternate 32-column chunks), add
//     them and store Phi rows.
// Four stages of 16 K (A 16 KB + B 2 BN 64 B each). Every wait is bounded;
// a wait that runs out sets the error word and the CTA drains its copies
// and MMAs (bounded), frees its tensor memory and returns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace demag {
namespace tgm {

constexpr int kBM = 128;                       // rows per MMA (TMEM lanes)
constexpr int kBK = 16;                        // K per stage (64-byte rows)
constexpr int kStages = 4;
constexpr int kProd = 256;                     // producer / epilogue threads
constexpr int kThreads = 64 + kProd;
constexpr int kAMat = kBM * kBK * 4;           // one 128 x 16 FP32 matrix: 8 KB
constexpr int kAStage = 2 * kAMat;             // hi and lo: 16 KB
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s

__host__ __device__ constexpr int b_stage_bytes(int BN) { return BN * 2 * kBK * 4; }

__host__ inline size_t smem_bytes(int BN)
{
    return 1024 + (size_t)kStages * (kAStage + b_stage_bytes(BN)) + 256;
}

// Tensor-memory columns: two accumulators of BN columns (large terms, small
// cross terms), a power of two >= 32.
__host__ __device__ inline int tmem_cols(int BN)
{
    int c = 32;
    while (c < 2 * BN) c *= 2;
    return c;
}

// Offset (bytes) of the 16-byte chunk `c` (K elements 4c .. 4c + 3) of row
// `r` in a K-major tile of 64-byte rows with the 64-byte swizzle: rows at 64 B,
// the chunk index XORed with address bits 7..8 (row / 2 mod 4).
__host__ __device__ inline int sw64_off(int r, int c)
{
    return r * 64 + ((c ^ ((r >> 1) & 3)) << 4);
}

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t s_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(uint64_t *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(s_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(s_u32(b)) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(s_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t *b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(s_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity`; false when another role has
// aborted the CTA or the cycle budget ran out (then abort it and flag it).
__device__ __forceinline__ bool bar_wait(uint64_t *b, unsigned parity, volatile int *abort_flag, int *err)
{
    const long long t0 = clock64();
    while (!bar_try(b, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// Plain bounded wait (draining after an abort).
__device__ __forceinline__ void bar_drain(uint64_t *b, unsigned parity)
{
    const long long t0 = clock64();
    while (!bar_try(b, parity))
        if (clock64() - t0 > kWaitCycles) return;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *b)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            s_u32(dst)),
        "l"(src), "r"(bytes), "r"(s_u32(b))
        : "memory");
}

__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, int ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, int ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 B apart (stride byte offset), leading byte offset unused by swizzled
// K-major layouts (16 B), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// N >> 3 at bits 17..22, M >> 4 at bits 24..28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `b` once every tcgen05 operation this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(s_u32(b))
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes (one row per
// lane). The wait names the registers, so no use of them moves above it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;\n"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
          "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
          "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
          "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
        :
        : "memory");
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ------------------------------------------------------------ operand prep
// X[K][nx] -> B operand in stage order: for n tile nt and K chunk kc, the hi
// matrix (BN rows x 16 K) then the lo matrix, each in the swizzled layout.
// Rows past nx and K past the term count are zero.
__global__ void k_tg_prep_b(const float *__restrict__ X, int K, int nx, int BN, int ntn, int nkc,
                            float *__restrict__ Bsw)
{
    const int64_t total = (int64_t)ntn * nkc * BN * kBK;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(e % BN);
        const int64_t rest = e / BN;
        const int kk = (int)(rest % kBK);
        const int64_t blk = rest / kBK;  // nt * nkc + kc
        const int kc = (int)(blk % nkc), nt = (int)(blk / nkc);
        const int Kk = kc * kBK + kk, i = nt * BN + n;
        const float v = (Kk < K && i < nx) ? X[(int64_t)Kk * nx + i] : 0.0f;
        const float hi = to_tf32(v), lo = to_tf32(v - hi);
        float *base = Bsw + blk * 2 * BN * kBK;
        const int off = sw64_off(n, kk >> 2) / 4 + (kk & 3);
        base[off] = hi;
        base[(int64_t)BN * kBK + off] = lo;
    }
}

// F[K][n] -> Ft[n][Kp] (zero for K >= the term count).
__global__ void k_tg_transpose(const float *__restrict__ F, int K, int n, int Kp, float *__restrict__ Ft)
{
    const int64_t total = (int64_t)n * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int Kk = (int)(e % Kp), j = (int)(e / Kp);
        Ft[e] = Kk < K ? F[(int64_t)Kk * n + j] : 0.0f;
    }
}

// ------------------------------------------------------------ the contraction
__global__ void __launch_bounds__(kThreads, 1)
k_tg_mma(const float *__restrict__ Yt, const float *__restrict__ Zt, const float *__restrict__ Bsw, int Kp, int nx,
         int ny, int nz, int BN, int ntn, int ntiles, float *__restrict__ phi, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *sm = smraw + ((1024u - (s_u32(smraw) & 1023u)) & 1023u);
    unsigned char *sA = sm;
    const int BS = b_stage_bytes(BN);
    unsigned char *sB = sA + kStages * kAStage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + kStages * BS);
    uint64_t *fullA = bars, *fullB = bars + kStages, *empty = bars + 2 * kStages;
    uint64_t *tfull = bars + 3 * kStages, *tempty = tfull + 1, *done = tempty + 1;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *s_abort = reinterpret_cast<volatile int *>(s_tmem + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkc = Kp / kBK;
    const int M = nz * ny;
    const int ncols = tmem_cols(BN), half = ncols / 2;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(&fullA[s], kProd);
            bar_init(&fullB[s], 1);
            bar_init(&empty[s], 1);
        }
        bar_init(tfull, 1);
        bar_init(tempty, kProd);
        bar_init(done, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) tmem_alloc(s_tmem, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
                const int nt = t % ntn;
                for (int kc = 0; kc < nkc; ++kc, ++it) {
                    const int s = it % kStages;
                    if (!bar_wait(&empty[s], ((it / kStages) & 1) ^ 1, s_abort, err)) { ok = false; break; }
                    bar_expect_tx(&fullB[s], BS);
                    bulk_load(sB + s * BS, Bsw + ((int64_t)nt * nkc + kc) * 2 * BN * kBK, BS, &fullB[s]);
                }
            }
            if (!ok)  // copies in flight land before the CTA exits
                for (int i = it > kStages ? it - kStages : 0; i < it; ++i)
                    bar_drain(&fullB[i % kStages], (i / kStages) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kBM, BN);
            int it = 0, lt = 0;
            bool ok = true, issued = false;
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++lt) {
                if (!bar_wait(tempty, (lt & 1) ^ 1, s_abort, err)) { ok = false; break; }
                tc_fence_after();
                for (int kc = 0; kc < nkc; ++kc, ++it) {
                    const int s = it % kStages;
                    const unsigned ph = (it / kStages) & 1;
                    if (!bar_wait(&fullA[s], ph, s_abort, err) || !bar_wait(&fullB[s], ph, s_abort, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t aS = s_u32(sA + s * kAStage), bS = s_u32(sB + s * BS);
#pragma unroll
                    for (int ks = 0; ks < kBK / 8; ++ks) {
                        const uint64_t ahi = sdesc(aS + ks * 32), alo = sdesc(aS + kAMat + ks * 32);
                        const uint64_t bhi = sdesc(bS + ks * 32), blo = sdesc(bS + BN * kBK * 4 + ks * 32);
                        const uint32_t first = (kc > 0 || ks > 0) ? 1u : 0u;
                        mma_tf32(tbase, ahi, bhi, idesc, first);
                        mma_tf32(tbase + (uint32_t)half, ahi, blo, idesc, first);
                        mma_tf32(tbase + (uint32_t)half, alo, bhi, idesc, 1u);
                    }
                    issued = true;
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(tfull);
            }
            if (!ok && issued) {  // MMAs in flight complete before the memory is freed
                mma_commit(done);
                bar_drain(done, 0);
            }
        }
    } else {
        const int pt = threadIdx.x - 64, kh = pt >> 7, m = pt & 127;
        const int eg = (warp - 2) >> 2, q = warp & 3, erow = q * 32 + lane;
        const bool vec = (nx & 3) == 0;
        int it = 0, lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const int mt = t / ntn, nt = t % ntn;
            const int g = mt * kBM + m;
            const bool valid = g < M;
            const int k = valid ? g / ny : 0, j = valid ? g % ny : 0;
            const float4 *yrow = reinterpret_cast<const float4 *>(Yt + (int64_t)j * Kp) + 2 * kh;
            const float4 *zrow = reinterpret_cast<const float4 *>(Zt + (int64_t)k * Kp) + 2 * kh;
            bool ok = true;
            for (int kc = 0; kc < nkc; ++kc, ++it) {
                const int s = it % kStages;
                float4 y[2], z[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    y[c] = valid ? __ldg(yrow + kc * 4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                    z[c] = valid ? __ldg(zrow + kc * 4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                // exits stay warp-uniform: the epilogue's tcgen05.ld is a warp-wide instruction
                const bool w = bar_wait(&empty[s], ((it / kStages) & 1) ^ 1, s_abort, err);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                unsigned char *ahi = sA + s * kAStage;
                unsigned char *alo = ahi + kAMat;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float p0 = y[c].x * z[c].x, p1 = y[c].y * z[c].y, p2 = y[c].z * z[c].z,
                                p3 = y[c].w * z[c].w;
                    const float h0 = to_tf32(p0), h1 = to_tf32(p1), h2 = to_tf32(p2), h3 = to_tf32(p3);
                    const int off = sw64_off(m, 2 * kh + c);
                    *reinterpret_cast<float4 *>(ahi + off) = make_float4(h0, h1, h2, h3);
                    *reinterpret_cast<float4 *>(alo + off) =
                        make_float4(to_tf32(p0 - h0), to_tf32(p1 - h1), to_tf32(p2 - h2), to_tf32(p3 - h3));
                }
                fence_async_smem();
                bar_arrive(&fullA[s]);
            }
            if (!ok) break;
            // epilogue: this warp's 32 rows, every other 32-column chunk
            const bool w = bar_wait(tfull, lt & 1, s_abort, err);
            if (!__all_sync(0xffffffffu, w)) break;
            tc_fence_after();
            const int ge = mt * kBM + erow;
            const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16);
            for (int c0 = eg * 32; c0 < BN; c0 += 64) {
                float v[32], u[32];
                tmem_ld32(taddr + (uint32_t)c0, v);
                tmem_ld32(taddr + (uint32_t)(half + c0), u);
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] += u[e];
                const int i0 = nt * BN + c0;
                if (ge < M && i0 < nx) {
                    float *dst = phi + (int64_t)ge * nx + i0;
                    if (vec && i0 + 32 <= nx) {
#pragma unroll
                        for (int e = 0; e < 32; e += 4)
                            *reinterpret_cast<float4 *>(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (i0 + e < nx) dst[e] = v[e];
                    }
                }
            }
            tc_fence_before();
            bar_arrive(tempty);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_free(tbase, ncols);
    }
}

}  // namespace tgm
}  // namespace demag
