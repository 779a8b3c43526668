// Pipelined x passes: persistent CTAs stream their tiles of whole rows
// through shared memory with bulk asynchronous copies (TMA, cp.async.bulk)
// completing on mbarriers, two tiles in flight per CTA, so the loads of the
// next tiles overlap the transforms of the current one. Same arithmetic and
// results as k_x_fwd2 / k_x_inv2; used when the tile's rows are contiguous
// and 16-byte multiples (the field passes of plans with nx % 4 == 0 for the
// forward pass; always for the inverse pass, whose rows are Kxp complex).
#pragma once
#include <cuda.h>  // CUtensorMap (the map is built on the host, see passes_impl.cuh)

#include "fft2.cuh"

namespace demag {

// Set when a bounded wait for a bulk copy gave up (read and cleared by the
// host through Passes<T>::pipe_error_take). One per element type.
static __device__ int g_xpipe_error;

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arrive once and expect `bytes` of asynchronous transactions on the barrier.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the barrier's phase with the given parity, giving up after
// `budget` SM clock cycles. Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long budget)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

// Global -> shared bulk copy of `bytes` (16-byte aligned addresses, size a
// multiple of 16) completing as transactions on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy ones (a bulk copy into a buffer just read).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

constexpr long long kPipeWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// Shared-memory plan of a pipelined x pass: exchange rows [TR][RS] complex,
// two input buffers of `in_elems` elements of type E each, two barriers.
template <typename T, int L, typename E>
struct XPipeSmem {
    static constexpr int TR = XShape<T, L>::TR, RS = XShape<T, L>::RS;
    static size_t bytes(int in_elems)
    {
        const size_t ex = (size_t)TR * RS * sizeof(typename Cplx<T>::type);
        const size_t in = ((size_t)in_elems * sizeof(E) + 15) / 16 * 16;
        return ex + 2 * in + 2 * sizeof(uint64_t);
    }
};

// One buffer of the inverse pass: a tile of TR rows of in_rs complex, or the
// tile's exchange rows [TR][RS], whichever is larger (16-byte multiple).
template <typename T, int L>
__host__ __device__ inline size_t xinv_slot_bytes(int in_rs)
{
    using S = XShape<T, L>;
    const size_t a = (size_t)S::TR * in_rs * sizeof(typename Cplx<T>::type);
    const size_t b = (size_t)S::TR * S::RS * sizeof(typename Cplx<T>::type);
    return ((a > b ? a : b) + 15) / 16 * 16;
}

// Issue the bulk copy of tile t (rows [t TR, min((t+1) TR, nrows)) of
// rowlen elements, contiguous in global memory) into buffer b.
template <typename E>
__device__ __forceinline__ void xpipe_issue(const E *src, int rowlen, int nrows, int TR, int t, E *buf,
                                            uint64_t *bar)
{
    const int r0 = t * TR;
    const int rows = min(TR, nrows - r0);
    const unsigned bytes = (unsigned)((size_t)rows * rowlen * sizeof(E));
    mbar_expect_tx(bar, bytes);
    bulk_g2s(buf, src + (int64_t)r0 * rowlen, bytes, bar);
}

// Error exit at the wait of iteration first_i: the copies of tiles first_i
// and first_i + 1 may still be in flight; wait for them (bounded) so that no
// copy lands after the CTA exits, and flag the failure for the host.
__device__ __forceinline__ void xpipe_abort(uint64_t *bars, int first_i, int gridstep, int ntiles)
{
    if (threadIdx.x == 0) {
        for (int i = first_i; i < first_i + 2; ++i) {
            const int t = blockIdx.x + i * gridstep;
            if (t < ntiles) mbar_wait_bounded(&bars[i & 1], (unsigned)((i >> 1) & 1), kPipeWaitCycles);
        }
        atomicExch(&g_xpipe_error, 1);
    }
}

// Forward R2C rows (PIN: at most L reals per row, rows of nvalid reals stored
// back to back, nvalid % 4 == 0), persistent over tiles.
template <typename T, int L>
__global__ void __launch_bounds__(Tile2<T>::NT)
k_x_fwd_tma(const T *__restrict__ in, T wscalar, int nrows, int nvalid, typename Cplx<T>::type *__restrict__ out,
            int64_t out_rs, const typename Cplx<T>::type *__restrict__ twx, int ntiles)
{
    using C = typename Cplx<T>::type;
    using S = XShape<T, L>;
    constexpr int R1 = S::R1, R2 = S::R2, TR = S::TR, RS = S::RS;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const size_t inb = ((size_t)TR * nvalid * sizeof(T) + 15) / 16 * 16;
    T *buf[2] = {reinterpret_cast<T *>(smraw + (size_t)TR * RS * sizeof(C)),
                 reinterpret_cast<T *>(smraw + (size_t)TR * RS * sizeof(C) + inb)};
    uint64_t *bars = reinterpret_cast<uint64_t *>(smraw + (size_t)TR * RS * sizeof(C) + 2 * inb);
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int step = gridDim.x;
    if (threadIdx.x == 0)
        for (int i = 0; i < 2; ++i) {
            const int t = blockIdx.x + i * step;
            if (t < ntiles) xpipe_issue(in, nvalid, nrows, TR, t, buf[i], &bars[i]);
        }
    for (int i = 0;; ++i) {
        const int t = blockIdx.x + i * step;
        if (t >= ntiles) break;
        const int b = i & 1;
        // every thread waits for the tile itself; a wait that gives up is
        // acted on after stage 1's barrier (stage 1 then read a partly
        // filled buffer: shared memory only, and the tile is abandoned)
        if (!mbar_wait_bounded(&bars[b], (unsigned)((i >> 1) & 1), kPipeWaitCycles)) s_fail = 1;
        const int row0 = t * TR;
        // stage 1 from shared memory: thread (row, j1) reads z[j1 + r R2], r < R1/2
        if (threadIdx.x < TR * R2) {
            const int rr = threadIdx.x / R2, j1 = threadIdx.x % R2, row = row0 + rr;
            C u[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
            if (row < nrows) {
                const T *p = buf[b] + rr * nvalid;
#pragma unroll
                for (int r = 0; r < R1 / 2; ++r) {
                    const int x0 = 2 * (j1 + r * R2);
                    if (x0 < nvalid) {  // nvalid is even
                        const C q = *reinterpret_cast<const C *>(p + x0);
                        u[r] = cmk<C>(q.x * wscalar, q.y * wscalar);
                    }
                }
            }
            RegDFTHalfIn<R1, false, C>::run(u);
            C *s = sm + rr * RS;
#pragma unroll
            for (int r = 0; r < R1; ++r) s[xex<R1>(j1, r)] = u[r];
        }
        __syncthreads();  // buffer b consumed, exchange rows written
        if (s_fail) {
            xpipe_abort(bars, i, step, ntiles);
            return;
        }
        if (threadIdx.x == 0) {
            const int tn = blockIdx.x + (i + 2) * step;
            if (tn < ntiles) {
                fence_proxy_async_smem();
                xpipe_issue(in, nvalid, nrows, TR, tn, buf[b], &bars[b]);
            }
        }
        // stage 2 + split, as k_x_fwd2
        if (threadIdx.x < TR * R1) {
            const int rr = threadIdx.x / R1, j2 = threadIdx.x % R1, row = row0 + rr;
            const C *s = sm + rr * RS;
            C v[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = s[xex<R1>(r, j2)];
#pragma unroll
            for (int r = 1; r < R2; ++r) v[r] = cmul(v[r], __ldg(&twx[2 * r * j2]));
            RegDFT<R2, false, C>::run(v);
            const int lane = threadIdx.x & 31;
            const int partner = (lane & ~(R1 - 1)) | ((R1 - j2) & (R1 - 1));
            const T h = (T)0.5;
            C *o = out + (int64_t)row * out_rs;
            const bool live = row < nrows;
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                const C q = shfl_c(v[R2 - 1 - r], partner);
                const C pz = j2 == 0 ? v[(R2 - r) % R2] : q;
                const int k = j2 + r * R1;
                const C E = cmk<C>(h * (v[r].x + pz.x), h * (v[r].y - pz.y));
                const C O = cmk<C>(h * (v[r].y + pz.y), -h * (v[r].x - pz.x));
                if (live) o[k] = cadd(E, cmul(O, __ldg(&twx[k])));
            }
            if (live && j2 == 0) o[L] = cmk<C>(v[0].x - v[0].y, (T)0);
        }
        __syncthreads();  // exchange rows read before the next tile rewrites them
    }
}

// Inverse C2R rows with the XOut epilogue (energy partials per tile into
// partials[t]); input rows of in_rs complex (even) stored back to back.
// P1 as in k_x_inv2 (one output pair beyond the half length). Each of the two
// buffers first receives a tile by bulk copy and then, once stage 1 has read
// it into registers, serves as that tile's exchange rows, so a CTA needs two
// buffers in all and three CTAs fit on an SM; the buffer is refilled with the
// tile after next when stage 2 is done with it.
template <typename T, int L, bool P1>
__global__ void __launch_bounds__(Tile2<T>::NT)
k_x_inv_tma(const typename Cplx<T>::type *__restrict__ in, int in_rs, int nrows, int nvalid, XOut<T> o,
            const typename Cplx<T>::type *__restrict__ twx, int ntiles)
{
    using C = typename Cplx<T>::type;
    using S = XShape<T, L>;
    constexpr int R1 = S::R1, R2 = S::R2, NT = S::NT, TR = S::TR, RS = S::RS;
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t slot = xinv_slot_bytes<T, L>(in_rs);
    C *buf[2] = {reinterpret_cast<C *>(smraw), reinterpret_cast<C *>(smraw + slot)};
    uint64_t *bars = reinterpret_cast<uint64_t *>(smraw + 2 * slot);
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int step = gridDim.x;
    if (threadIdx.x == 0)
        for (int i = 0; i < 2; ++i) {
            const int t = blockIdx.x + i * step;
            if (t < ntiles) xpipe_issue(in, in_rs, nrows, TR, t, buf[i], &bars[i]);
        }
    const T g = o.gdev ? (T)(*o.gdev) : (T)1;
    const T oscale = o.oscale * g;
    for (int i = 0;; ++i) {
        const int t = blockIdx.x + i * step;
        if (t >= ntiles) break;
        const int b = i & 1;
        if (!mbar_wait_bounded(&bars[b], (unsigned)((i >> 1) & 1), kPipeWaitCycles)) s_fail = 1;
        __syncthreads();
        if (s_fail) {
            xpipe_abort(bars, i, step, ntiles);
            return;
        }
        const int row0 = t * TR;
        const bool act1 = threadIdx.x < TR * R2;
        const int rr1 = threadIdx.x / R2, j1 = threadIdx.x % R2;
        C u[R1];
        if (act1) {
#pragma unroll
            for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
            if (row0 + rr1 < nrows) {
                const C *p = buf[b] + rr1 * in_rs;
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    const int k = j1 + r * R2;
                    const C a = p[k];
                    const C bb = p[L - k];
                    const C E2 = cmk<C>(a.x + bb.x, a.y - bb.y);
                    const C D = cmk<C>(a.x - bb.x, a.y + bb.y);
                    const C O2 = cmulc(D, __ldg(&twx[k]));
                    u[r] = cmk<C>(E2.x - O2.y, E2.y + O2.x);
                }
            }
            RegDFT<R1, true, C>::run(u);
        }
        __syncthreads();  // the tile is in registers: the buffer becomes the exchange rows
        C *sm = buf[b];
        if (act1) {
            C *s = sm + rr1 * RS;
#pragma unroll
            for (int r = 0; r < R1; ++r) s[xex<R1>(j1, r)] = u[r];
        }
        __syncthreads();
        T acc = 0;
        if (threadIdx.x < TR * R1) {
            const int rr = threadIdx.x / R1, j2 = threadIdx.x % R1, row = row0 + rr;
            const C *s = sm + rr * RS;
            C v[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = s[xex<R1>(r, j2)];
#pragma unroll
            for (int r = 1; r < R2; ++r) v[r] = cmulc(v[r], __ldg(&twx[2 * r * j2]));
            if constexpr (P1) RegDFTHalfOutP1<R2, true, C>::run(v);
            else RegDFTHalfOut<R2, true, C>::run(v);
            if (row < nrows) {
#pragma unroll
                for (int r = 0; r < (P1 ? R2 / 2 + 1 : R2 / 2); ++r) {
                    const int n = j2 + r * R1;
                    x_out_pair<T>(o, row, 2 * n, v[r].x * o.scale, v[r].y * o.scale, oscale, nvalid, nullptr, acc);
                }
            }
        }
        if (o.partials) block_partial<NT>((double)acc, o.partials, t);  // has its own barrier
        __syncthreads();  // exchange rows read: the buffer can take the tile after next
        if (threadIdx.x == 0) {
            const int tn = blockIdx.x + (i + 2) * step;
            if (tn < ntiles) {
                fence_proxy_async_smem();
                xpipe_issue(in, in_rs, nrows, TR, tn, buf[b], &bars[b]);
            }
        }
    }
}

// ------------------------------------------------------------ y forward pass
// Tiled 3-D tensor copy (TMA) of box `coords` of the map into shared memory,
// completing as transactions on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Pruned forward column transform (the y pass: nin <= L/2 rows in, all L rows
// out) by persistent CTAs: each tile of TC columns of one slab arrives by
// TMA tensor copies (box: 2 TC reals wide, BR rows, one slab; nb boxes stacked
// in rows) into one of two buffers while the previous tile is transformed in
// the three-stage layout of k_col3; two tiles in flight per CTA. Columns past
// the slab's width and rows past nin arrive as zeros (out-of-bounds fill).
template <typename T, int L>
__global__ void __launch_bounds__(Col3Shape<T, L>::NT, L >= 1024 ? 2 : 3)
k_col_tma_fwd(const __grid_constant__ CUtensorMap map, typename Cplx<T>::type *__restrict__ out, int width, int nslabs,
              int nin, int BR, int nb, int64_t oss, int64_t ors, const typename Cplx<T>::type *__restrict__ tw,
              int twstride)
{
    using C = typename Cplx<T>::type;
    using S = Col3Shape<T, L>;
    constexpr int R1 = S::R1, R2 = S::R2, R3 = S::R3, NT = S::NT, TC = S::TC;
    extern __shared__ __align__(16) unsigned char smraw[];
    // tensor-copy destinations 128-byte aligned (the launch adds 128 bytes of slack)
    unsigned char *base = smraw + ((128 - (smem_u32(smraw) & 127)) & 127);
    C *sm = reinterpret_cast<C *>(base);
    const size_t ex = ((size_t)swsize(L * TC) * sizeof(C) + 127) / 128 * 128;
    const unsigned tile_bytes = (unsigned)((size_t)nb * BR * TC * sizeof(C));  // whole boxes, fill included
    const size_t inb = ((size_t)tile_bytes + 127) / 128 * 128;
    C *buf[2] = {reinterpret_cast<C *>(base + ex), reinterpret_cast<C *>(base + ex + inb)};
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + ex + 2 * inb);
    __shared__ int s_fail;
    const int tps = (width + TC - 1) / TC;
    const int ntiles = tps * nslabs;
    auto issue = [&](int t, int bsel) {
        const int slab = t / tps, x = 2 * (t - slab * tps) * TC;
        mbar_expect_tx(&bars[bsel], tile_bytes);
        for (int k = 0; k < nb; ++k)
            tma_load_3d(buf[bsel] + (size_t)k * BR * TC, &map, x, k * BR, slab, &bars[bsel]);
    };
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int step = gridDim.x;
    if (threadIdx.x == 0)
        for (int i = 0; i < 2; ++i)
            if (blockIdx.x + i * step < ntiles) issue(blockIdx.x + i * step, i);
    for (int i = 0;; ++i) {
        const int t = blockIdx.x + i * step;
        if (t >= ntiles) break;
        const int b = i & 1;
        if (!mbar_wait_bounded(&bars[b], (unsigned)((i >> 1) & 1), kPipeWaitCycles)) s_fail = 1;
        __syncthreads();
        if (s_fail) {
            xpipe_abort(bars, i, step, ntiles);
            return;
        }
        const int slab = t / tps, kx0 = (t - slab * tps) * TC;
        // stage 1: radix R1 over rows j1 + r L/R1 (r < R1/2 hold data) -> rows j1 R1 + r
#pragma unroll
        for (int q = 0; q < (TC * (L / R1) + NT - 1) / NT; ++q) {
            const int bq = threadIdx.x + q * NT;
            if (bq < TC * (L / R1)) {
                const int c = bq % TC, j1 = bq / TC;
                C u[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
#pragma unroll
                for (int r = 0; r < R1 / 2; ++r) {
                    const int row = j1 + r * (L / R1);
                    if (row < nin) u[r] = buf[b][row * TC + c];
                }
                RegDFTHalfIn<R1, false, C>::run(u);
                C *s = sm + sw(j1 * R1 * TC + c);
#pragma unroll
                for (int r = 0; r < R1; ++r) s[r * TC + (r * TC) / 32] = u[r];
            }
        }
        __syncthreads();  // buffer b consumed
        if (threadIdx.x == 0 && t + 2 * step < ntiles) {
            fence_proxy_async_smem();
            issue(t + 2 * step, b);
        }
        fft_stage<C, L, R2, R1, false, NT, TC>(sm, tw, twstride);
#pragma unroll
        for (int q = 0; q < (TC * (L / R3) + NT - 1) / NT; ++q) {
            const int bq = threadIdx.x + q * NT;
            if (bq < TC * (L / R3)) {
                const int c = bq % TC, j = bq / TC, kx = kx0 + c;
                C v[R3];
                const C *s = sm + sw(j * TC + c);
#pragma unroll
                for (int r = 0; r < R3; ++r) v[r] = s[r * ((L / R3) * TC + (L / R3) * TC / 32)];
                twiddle_row<R3, L, false>(v, j, tw, twstride);
                RegDFT<R3, false, C>::run(v);
                if (kx < width) {
                    C *col = out + (int64_t)slab * oss + kx;
#pragma unroll
                    for (int r = 0; r < R3; ++r) col[(int64_t)(j + r * (L / R3)) * ors] = v[r];
                }
            }
        }
        __syncthreads();  // exchange rows read before the next tile rewrites them
    }
}

// ------------------------------------------------------------ z pass (DM)
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// The tensor block of the columns kx0 .. kx0 + TC - 1 of spectral row ky (as
// tensor_block_prefetch, for row-aligned tiles).
template <typename T, int TC, int NT, int NC, int HZ>
__device__ __forceinline__ void tensor_block_prefetch_row(T *smT, const T *__restrict__ tab, int ky, int kx0, int Kx,
                                                          int Py, int64_t plane, int tid)
{
    constexpr int G = NT / TC, GQ = G / NC, GR = G % NC;
    const int c = tid % TC, g = tid / TC, kx = kx0 + c;
    if (kx >= Kx) return;
    const int kyf = ky > Py / 2 ? Py - ky : ky;
    const int64_t zs = (int64_t)(Py / 2 + 1) * Kx;
    const T *src = tab + (int64_t)kyf * Kx + kx;
    int comp = g % NC;
    int64_t off = comp * plane + (int64_t)(g / NC) * zs;
    const int64_t step = GQ * zs + GR * plane, wrap = zs - NC * plane;
    for (int idx = g; idx < HZ * NC; idx += G) {
        cp_async_elem(&smT[idx * TC + c], src + off);
        comp += GR;
        off += step;
        if (comp >= NC) {
            comp -= NC;
            off += wrap;
        }
    }
}

// Fused z pass by persistent CTAs with the input columns staged by TMA:
// tiles are TC consecutive kx of one spectral row ky (rows taken in fold-pair
// order); a tile's three components (nrows z-rows each) arrive in one 4-D
// tensor copy while the previous tile's forward stage 2, product and inverse
// run, and its tensor block is copied (cp.async) during the previous tile's
// inverse stage. Arithmetic as k_z_conv2.
// Thread layout of the TMA z pass: as k_z_conv2 variant 0, except at L = 512
// where the 256-thread layout (variant 2) leaves the persistent loop enough
// registers.
template <int L> struct ZTmaV { static constexpr int V = 0; };

template <typename T, int L>
__global__ void __launch_bounds__(ZShape<T, L, ZTmaV<L>::V>::NT, 1)
k_z_conv_tma(const __grid_constant__ CUtensorMap map, typename Cplx<T>::type *__restrict__ S, int Kx, int Py,
             int64_t ss, int64_t rs, int64_t cs, int nrows, const T *__restrict__ nhat,
             const typename Cplx<T>::type *__restrict__ tw, int ntr, int ntiles)
{
    using C = typename Cplx<T>::type;
    using Sh = ZShape<T, L, ZTmaV<L>::V>;
    constexpr int R1 = Sh::R1, R2 = Sh::R2, NT = Sh::NT, TC = Sh::TC;
    constexpr int TS = swsize(L * TC);
    constexpr int NB1 = TC * R2;
    constexpr int HZ = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((128 - (smem_u32(smraw) & 127)) & 127);
    const unsigned in_bytes = (unsigned)(3u * nrows * TC * sizeof(C));
    const size_t stg_bytes = ((size_t)in_bytes + 127) / 128 * 128;
    C *stg = reinterpret_cast<C *>(base);               // [3][nrows][TC]
    C *sm = reinterpret_cast<C *>(base + stg_bytes);    // exchange [3][TS]
    T *smT = reinterpret_cast<T *>(sm + 3 * TS);        // tensor block [HZ][6][TC]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smT + HZ * 6 * TC);
    __shared__ int s_fail;
    const int hy = Py / 2 + 1;
    const int64_t plane = (int64_t)HZ * hy * Kx;
    auto tile_ky = [&](int t) { return ky_pair_order(t / ntr, Py); };
    auto tile_kx0 = [&](int t) { return (t % ntr) * TC; };
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    int t = blockIdx.x;
    if (t < ntiles) {
        if (threadIdx.x == 0) {
            mbar_expect_tx(bar, in_bytes);
            tma_load_4d(stg, &map, 2 * tile_kx0(t), tile_ky(t), 0, 0, bar);
        }
        tensor_block_prefetch_row<T, TC, NT, 6, HZ>(smT, nhat, tile_ky(t), tile_kx0(t), Kx, Py, plane, threadIdx.x);
    }
    for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
        const int next = t + gridDim.x;
        const int ky = tile_ky(t), kx0 = tile_kx0(t);
        if (!mbar_wait_bounded(bar, (unsigned)(k & 1), kPipeWaitCycles)) s_fail = 1;
        cp_async_wait_all();
        __syncthreads();
        if (s_fail) {
            // only this tile's copy is in flight: give it one more bounded wait
            // so that it does not land after the CTA has exited, then flag
            if (threadIdx.x == 0) {
                mbar_wait_bounded(bar, (unsigned)(k & 1), kPipeWaitCycles);
                atomicExch(&g_xpipe_error, 1);
            }
            return;
        }
        // forward stage 1 from the staged rows: rows j1 + r R2 -> rows j1 R1 + r
#pragma unroll
        for (int q = 0; q < (3 * NB1 + NT - 1) / NT; ++q) {
            const int b = threadIdx.x + q * NT;
            if (b < 3 * NB1) {
                const int comp = b / NB1, bb = b - comp * NB1;
                const int c = bb % TC, j1 = bb / TC;
                C u[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
                const C *col = stg + ((size_t)comp * nrows + j1) * TC + c;
#pragma unroll
                for (int r = 0; r < R1 / 2; ++r)
                    if (j1 + r * R2 < nrows) u[r] = col[r * R2 * TC];
                RegDFTHalfIn<R1, false, C>::run(u);
                C *s = sm + comp * TS + sw(j1 * R1 * TC + c);
#pragma unroll
                for (int r = 0; r < R1; ++r) s[r * TC + (r * TC) / 32] = u[r];
            }
        }
        __syncthreads();  // staging buffer consumed
        if (threadIdx.x == 0 && next < ntiles) {
            fence_proxy_async_smem();
            mbar_expect_tx(bar, in_bytes);
            tma_load_4d(stg, &map, 2 * tile_kx0(next), tile_ky(next), 0, 0, bar);
        }
        const bool act2 = threadIdx.x < TC * R1;
        const int c2 = threadIdx.x % TC, j2 = threadIdx.x / TC;
        C v0[R2], v1[R2], v2[R2];
        if (act2) {
            const C *s = sm + sw(j2 * TC + c2);
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                constexpr int step = R1 * TC + (R1 * TC) / 32;
                v0[r] = s[r * step];
                v1[r] = s[TS + r * step];
                v2[r] = s[2 * TS + r * step];
            }
#pragma unroll
            for (int r = 1; r < R2; ++r) {
                const C w = __ldg(&tw[r * j2]);
                v0[r] = cmul(v0[r], w);
                v1[r] = cmul(v1[r], w);
                v2[r] = cmul(v2[r], w);
            }
            RegDFT<R2, false, C>::run(v0);
            RegDFT<R2, false, C>::run(v1);
            RegDFT<R2, false, C>::run(v2);
            const T sy = ky > Py / 2 ? (T)-1 : (T)1;
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                const int kz = j2 + r * R1;
                const bool up = kz > L / 2;
                const int kzf = up ? L - kz : kz;
                const T sz = up ? (T)-1 : (T)1;
                const T *tt = smT + kzf * 6 * TC + c2;
                const T nxx = tt[0], nyy = tt[TC], nzz = tt[2 * TC];
                const T nxy = sy * tt[3 * TC], nxz = sz * tt[4 * TC], nyz = sy * sz * tt[5 * TC];
                const C mx = v0[r], my = v1[r], mz = v2[r];
                v0[r] = cmk<C>(-(nxx * mx.x + nxy * my.x + nxz * mz.x), -(nxx * mx.y + nxy * my.y + nxz * mz.y));
                v1[r] = cmk<C>(-(nxy * mx.x + nyy * my.x + nyz * mz.x), -(nxy * mx.y + nyy * my.y + nyz * mz.y));
                v2[r] = cmk<C>(-(nxz * mx.x + nyz * my.x + nzz * mz.x), -(nxz * mx.y + nyz * my.y + nzz * mz.y));
            }
            RegDFT<R2, true, C>::run(v0);
            RegDFT<R2, true, C>::run(v1);
            RegDFT<R2, true, C>::run(v2);
        }
        __syncthreads();  // exchange and tensor block read
        if (next < ntiles)
            tensor_block_prefetch_row<T, TC, NT, 6, HZ>(smT, nhat, tile_ky(next), tile_kx0(next), Kx, Py, plane,
                                                        threadIdx.x);
        if (act2) {
            C *s = sm + sw(j2 * R2 * TC + c2);
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                const int o = r * TC + (r * TC) / 32;
                s[o] = v0[r];
                s[TS + o] = v1[r];
                s[2 * TS + o] = v2[r];
            }
        }
        __syncthreads();
        // inverse stage 2: radix R1 over rows j1 + r R2, rows < nrows stored
#pragma unroll
        for (int q = 0; q < (3 * NB1 + NT - 1) / NT; ++q) {
            const int b = threadIdx.x + q * NT;
            if (b < 3 * NB1) {
                const int comp = b / NB1, bb = b - comp * NB1;
                const int c = bb % TC, j1 = bb / TC, kx = kx0 + c;
                const C *s = sm + comp * TS + sw(j1 * TC + c);
                C u[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    constexpr int step = R2 * TC + (R2 * TC) / 32;
                    u[r] = s[r * step];
                }
#pragma unroll
                for (int r = 1; r < R1; ++r) u[r] = cmulc(u[r], __ldg(&tw[r * j1]));
                RegDFTHalfOut<R1, true, C>::run(u);
                if (kx < Kx) {
                    C *col = S + (int64_t)ky * ss + kx + comp * cs + j1 * rs;
#pragma unroll
                    for (int r = 0; r < R1 / 2; ++r)
                        if (j1 + r * R2 < nrows) col[(int64_t)r * R2 * rs] = u[r];
                }
            }
        }
        __syncthreads();  // exchange rows read before the next tile writes them
    }
}

// ------------------------------------------------------------ z pass (SP)
// Persistent SP z pass with TMA-staged input columns: as k_z_conv_tma for
// the three forward transforms; the product forms the potential spectrum
// (sp_product with the half-cell phase) and one inverse transform writes the
// nout = nz + 1 node planes over component 0 of the tile's own columns (the
// last plane lands in component 1's first plane, which only this tile reads,
// and it has been read). POUT: nout <= L/2.
template <typename T, int L, bool POUT>
__global__ void __launch_bounds__(ZShape<T, L, 0>::NT, 1)
k_sp_z_tma(const __grid_constant__ CUtensorMap map, typename Cplx<T>::type *__restrict__ S, int Kx, int Py,
           int64_t ss, int64_t rs, int64_t cs, int nrows, int nout, const T *__restrict__ that,
           const typename Cplx<T>::type *__restrict__ tw, const typename Cplx<T>::type *__restrict__ phx,
           const typename Cplx<T>::type *__restrict__ phy, const typename Cplx<T>::type *__restrict__ phz, int ntr,
           int ntiles)
{
    using C = typename Cplx<T>::type;
    using Sh = ZShape<T, L, 0>;
    constexpr int R1 = Sh::R1, R2 = Sh::R2, NT = Sh::NT, TC = Sh::TC;
    constexpr int TS = swsize(L * TC);
    constexpr int NB1 = TC * R2;
    constexpr int HZ = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((128 - (smem_u32(smraw) & 127)) & 127);
    const unsigned in_bytes = (unsigned)(3u * nrows * TC * sizeof(C));
    const size_t stg_bytes = ((size_t)in_bytes + 127) / 128 * 128;
    C *stg = reinterpret_cast<C *>(base);
    C *sm = reinterpret_cast<C *>(base + stg_bytes);
    T *smT = reinterpret_cast<T *>(sm + 3 * TS);  // [kzf][3][TC]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smT + ((HZ * 3 * TC + 1) / 2) * 2);
    __shared__ int s_fail;
    const int hy = Py / 2 + 1;
    const int64_t plane = (int64_t)HZ * hy * Kx;
    auto tile_ky = [&](int t) { return ky_pair_order(t / ntr, Py); };
    auto tile_kx0 = [&](int t) { return (t % ntr) * TC; };
    if (threadIdx.x == 0) {
        s_fail = 0;
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    int t = blockIdx.x;
    if (t < ntiles) {
        if (threadIdx.x == 0) {
            mbar_expect_tx(bar, in_bytes);
            tma_load_4d(stg, &map, 2 * tile_kx0(t), tile_ky(t), 0, 0, bar);
        }
        tensor_block_prefetch_row<T, TC, NT, 3, HZ>(smT, that, tile_ky(t), tile_kx0(t), Kx, Py, plane, threadIdx.x);
    }
    for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
        const int next = t + gridDim.x;
        const int ky = tile_ky(t), kx0 = tile_kx0(t);
        if (!mbar_wait_bounded(bar, (unsigned)(k & 1), kPipeWaitCycles)) s_fail = 1;
        cp_async_wait_all();
        __syncthreads();
        if (s_fail) {
            if (threadIdx.x == 0) {  // as in k_z_conv_tma
                mbar_wait_bounded(bar, (unsigned)(k & 1), kPipeWaitCycles);
                atomicExch(&g_xpipe_error, 1);
            }
            return;
        }
#pragma unroll
        for (int q = 0; q < (3 * NB1 + NT - 1) / NT; ++q) {
            const int b = threadIdx.x + q * NT;
            if (b < 3 * NB1) {
                const int comp = b / NB1, bb = b - comp * NB1;
                const int c = bb % TC, j1 = bb / TC;
                C u[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) u[r] = cmk<C>(0, 0);
                const C *col = stg + ((size_t)comp * nrows + j1) * TC + c;
#pragma unroll
                for (int r = 0; r < R1 / 2; ++r)
                    if (j1 + r * R2 < nrows) u[r] = col[r * R2 * TC];
                RegDFTHalfIn<R1, false, C>::run(u);
                C *s = sm + comp * TS + sw(j1 * R1 * TC + c);
#pragma unroll
                for (int r = 0; r < R1; ++r) s[r * TC + (r * TC) / 32] = u[r];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && next < ntiles) {
            fence_proxy_async_smem();
            mbar_expect_tx(bar, in_bytes);
            tma_load_4d(stg, &map, 2 * tile_kx0(next), tile_ky(next), 0, 0, bar);
        }
        const bool act2 = threadIdx.x < TC * R1;
        const int c2 = threadIdx.x % TC, j2 = threadIdx.x / TC;
        C p[R2];
        if (act2) {
            C v0[R2], v1[R2], v2[R2];
            const C *s = sm + sw(j2 * TC + c2);
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                constexpr int step = R1 * TC + (R1 * TC) / 32;
                v0[r] = s[r * step];
                v1[r] = s[TS + r * step];
                v2[r] = s[2 * TS + r * step];
            }
#pragma unroll
            for (int r = 1; r < R2; ++r) {
                const C w = __ldg(&tw[r * j2]);
                v0[r] = cmul(v0[r], w);
                v1[r] = cmul(v1[r], w);
                v2[r] = cmul(v2[r], w);
            }
            RegDFT<R2, false, C>::run(v0);
            RegDFT<R2, false, C>::run(v1);
            RegDFT<R2, false, C>::run(v2);
            const int kx = kx0 + c2;
            const T sy = ky > Py / 2 ? (T)-1 : (T)1;
            const C pxy = cmul(__ldg(&phx[kx < Kx ? kx : 0]), __ldg(&phy[ky]));
            const C cxy = cmk<C>(pxy.y, -pxy.x);
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                const int kz = j2 + r * R1;
                const bool up = kz > L / 2;
                const int kzf = up ? L - kz : kz;
                const T sz = up ? (T)-1 : (T)1;
                const T *tt = smT + kzf * 3 * TC + c2;
                p[r] = sp_product<T, C>(sy * sz * tt[0], sz * tt[TC], sy * tt[2 * TC], v0[r], v1[r], v2[r],
                                        cmul(cxy, __ldg(&phz[kz])));
            }
            RegDFT<R2, true, C>::run(p);
        }
        __syncthreads();
        if (next < ntiles)
            tensor_block_prefetch_row<T, TC, NT, 3, HZ>(smT, that, tile_ky(next), tile_kx0(next), Kx, Py, plane,
                                                        threadIdx.x);
        if (act2) {
            C *s = sm + sw(j2 * R2 * TC + c2);
#pragma unroll
            for (int r = 0; r < R2; ++r) s[r * TC + (r * TC) / 32] = p[r];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < (NB1 + NT - 1) / NT; ++q) {
            const int b = threadIdx.x + q * NT;
            if (b < NB1) {
                const int c = b % TC, j1 = b / TC, kx = kx0 + c;
                const C *s = sm + sw(j1 * TC + c);
                C u[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    constexpr int step = R2 * TC + (R2 * TC) / 32;
                    u[r] = s[r * step];
                }
#pragma unroll
                for (int r = 1; r < R1; ++r) u[r] = cmulc(u[r], __ldg(&tw[r * j1]));
                if constexpr (POUT) RegDFTHalfOut<R1, true, C>::run(u);
                else RegDFT<R1, true, C>::run(u);
                if (kx < Kx) {
                    C *col = S + (int64_t)ky * ss + kx + j1 * rs;
#pragma unroll
                    for (int r = 0; r < (POUT ? R1 / 2 : R1); ++r)
                        if (j1 + r * R2 < nout) col[(int64_t)r * R2 * rs] = u[r];
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace demag
