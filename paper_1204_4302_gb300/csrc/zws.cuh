// Fused z pass of the tensor method for FP32 plans (paper Sec. 3.1: forward
// z transform of the three components, the element-wise product with the
// real symmetric tensor spectrum H^ = -N^ M^, inverse z transform), as one
// persistent kernel per SM that streams column tiles through shared memory:
//
//  * the tile's input rows (three components, z < nz, TC columns kx at one
//    ky) arrive by one 4-D TMA tensor copy, and the tile's block of the
//    tensor spectrum by one bulk copy of a tile-ordered copy of the octant
//    table, both issued one tile ahead and completed on mbarriers (bounded
//    waits);
//  * a length-L transform (L = 512 = 2 x 16 x 16 with the zero padding) runs
//    as: stage 1, two 16-point DFTs per 32-point column segment (the even and
//    the odd outputs of a 32-point DFT whose upper half input is zero);
//    stage 2, the 16-point DFTs of the three components in registers, the
//    3x3 product, the inverse 16-point DFTs and the twiddles between the
//    inverse stages (the conjugates of the forward ones, held in registers),
//    in place; stage 3, the 32-point inverse DFT of which only the outputs
//    z < L/2 are formed, stored straight to global memory;
//  * the exchange tile is [component][row][TC] with one padding row every 32
//    rows: every warp access of stages 1-3 then touches consecutive 64-byte
//    rows alternating between the two halves of the banks (no conflicts);
//  * butterflies add and subtract both halves of a complex value with one
//    packed FP32x2 instruction (add.rn.f32x2 / sub.rn.f32x2).
#pragma once
#include <cuda.h>

#include <type_traits>

#include "fft2.cuh"
#include "xpipe.cuh"

namespace demag {
namespace zw {

// ------------------------------------------------------------ complex ops
__device__ __forceinline__ unsigned long long f2u(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 u2f(unsigned long long r)
{
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
// a - i b and a + i b
__device__ __forceinline__ float2 add_mi(float2 a, float2 b) { return make_float2(a.x + b.y, a.y - b.x); }
__device__ __forceinline__ float2 add_pi(float2 a, float2 b) { return make_float2(a.x - b.y, a.y + b.x); }
// a * w and a * conj(w)
__device__ __forceinline__ float2 mul(float2 a, float2 w)
{
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
__device__ __forceinline__ float2 mulc(float2 a, float2 w)
{
    return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}

// v * W_N^M (forward, W_N = exp(-2 pi i / N)) or v * W_N^-M (INV), N <= 32,
// M a compile-time constant: the angle 2 pi M / N in units of pi/16 is
// m = 32 M / N; multiples of pi/4 use adds and one scale.
template <int N, int M, bool INV>
__device__ __forceinline__ float2 tw(float2 v)
{
    constexpr int m = ((M % N) * (32 / N)) % 32;  // 0 <= m < 32, angle m pi / 16
    constexpr float r = 0.70710678118654752440f;
    if constexpr (m == 0) {
        return v;
    } else if constexpr (m == 16) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (m == 8) {  // -i (forward) / +i (inverse)
        return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else if constexpr (m == 24) {  // +i / -i
        return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    } else if constexpr (m == 4) {  // (1 - i)/sqrt2, inverse (1 + i)/sqrt2
        return INV ? make_float2((v.x - v.y) * r, (v.x + v.y) * r) : make_float2((v.x + v.y) * r, (v.y - v.x) * r);
    } else if constexpr (m == 12) {  // (-1 - i)/sqrt2, inverse (-1 + i)/sqrt2
        return INV ? make_float2(-(v.x + v.y) * r, (v.x - v.y) * r) : make_float2((v.y - v.x) * r, -(v.x + v.y) * r);
    } else {
        // cos and sin of m pi / 16 from the quarter-wave table of 2 pi k / 32
        constexpr double c = m <= 8 ? cos2pi32(m) : (m <= 16 ? -cos2pi32(16 - m) : (m <= 24 ? -cos2pi32(m - 16) : cos2pi32(32 - m)));
        constexpr double s = m <= 8 ? cos2pi32(8 - m) : (m <= 16 ? cos2pi32(m - 8) : (m <= 24 ? -cos2pi32(24 - m) : -cos2pi32(m - 24)));
        const float cf = (float)c, sf = (float)s;
        // forward: v (c - i s); inverse: v (c + i s)
        return INV ? make_float2(v.x * cf - v.y * sf, v.y * cf + v.x * sf)
                   : make_float2(v.x * cf + v.y * sf, v.y * cf - v.x * sf);
    }
}

// 4-point DFT in place (natural order).
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 s0 = add(a0, a2), d0 = sub(a0, a2), s1 = add(a1, a3), d1 = sub(a1, a3);
    a0 = add(s0, s1);
    a2 = sub(s0, s1);
    if (INV) {
        a1 = add_pi(d0, d1);
        a3 = add_mi(d0, d1);
    } else {
        a1 = add_mi(d0, d1);
        a3 = add_pi(d0, d1);
    }
}

// 16-point DFT, natural order in and out: n = 4 n1 + n2, k = k1 + 4 k2.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16])
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    // v[n2 + 4 k1] = a[n2][k1]; twiddle W16^(n2 k1)
    v[5] = tw<16, 1, INV>(v[5]);
    v[9] = tw<16, 2, INV>(v[9]);
    v[13] = tw<16, 3, INV>(v[13]);
    v[6] = tw<16, 2, INV>(v[6]);
    v[10] = tw<16, 4, INV>(v[10]);
    v[14] = tw<16, 6, INV>(v[14]);
    v[7] = tw<16, 3, INV>(v[7]);
    v[11] = tw<16, 6, INV>(v[11]);
    v[15] = tw<16, 9, INV>(v[15]);
    // DFT over n2 for each k1 (the values v[n2 + 4 k1], n2 = 0..3): output
    // X[k1 + 4 k2] lands in v[4 k1 + k2]; transpose to natural order
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    float2 t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

// 16-point forward DFT of v[0..7] (v[8..15] are zero padding): the first
// level's 4-point DFTs see two non-zero inputs each.
__device__ __forceinline__ void dft16_half_in(float2 (&v)[16])
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        const float2 a0 = v[n2], a1 = v[n2 + 4];
        v[n2] = add(a0, a1);
        v[n2 + 4] = add_mi(a0, a1);
        v[n2 + 8] = sub(a0, a1);
        v[n2 + 12] = add_pi(a0, a1);
    }
    v[5] = tw<16, 1, false>(v[5]);
    v[9] = tw<16, 2, false>(v[9]);
    v[13] = tw<16, 3, false>(v[13]);
    v[6] = tw<16, 2, false>(v[6]);
    v[10] = tw<16, 4, false>(v[10]);
    v[14] = tw<16, 6, false>(v[14]);
    v[7] = tw<16, 3, false>(v[7]);
    v[11] = tw<16, 6, false>(v[11]);
    v[15] = tw<16, 9, false>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<false>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    float2 t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

// 16-point inverse DFT of which only the outputs 0..7 are formed (into
// v[0..7]); v[8..15] are left undefined.
__device__ __forceinline__ void idft16_lo(float2 (&v)[16])
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<true>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    v[5] = tw<16, 1, true>(v[5]);
    v[9] = tw<16, 2, true>(v[9]);
    v[13] = tw<16, 3, true>(v[13]);
    v[6] = tw<16, 2, true>(v[6]);
    v[10] = tw<16, 4, true>(v[10]);
    v[14] = tw<16, 6, true>(v[14]);
    v[7] = tw<16, 3, true>(v[7]);
    v[11] = tw<16, 6, true>(v[11]);
    v[15] = tw<16, 9, true>(v[15]);
    float2 o[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        // outputs k2 = 0, 1 of the 4-point inverse DFT over v[4 k1 + n2]
        const float2 s0 = add(v[4 * k1], v[4 * k1 + 2]), d0 = sub(v[4 * k1], v[4 * k1 + 2]);
        const float2 s1 = add(v[4 * k1 + 1], v[4 * k1 + 3]), d1 = sub(v[4 * k1 + 1], v[4 * k1 + 3]);
        o[k1] = add(s0, s1);
        o[k1 + 4] = add_pi(d0, d1);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = o[i];
}

// 32-point inverse DFT of u[0..31] of which the outputs 0..15 are formed
// into y[0..15]: even outputs from u[k] + u[k+16], odd outputs from
// (u[k] - u[k+16]) W32^-k, each a 16-point inverse DFT keeping 8 outputs.
__device__ __forceinline__ void idft32_lo(const float2 (&u)[32], float2 (&y)[16])
{
    float2 a[16], b[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        a[k] = add(u[k], u[k + 16]);
        b[k] = sub(u[k], u[k + 16]);
    }
    b[1] = tw<32, 1, true>(b[1]);
    b[2] = tw<32, 2, true>(b[2]);
    b[3] = tw<32, 3, true>(b[3]);
    b[4] = tw<32, 4, true>(b[4]);
    b[5] = tw<32, 5, true>(b[5]);
    b[6] = tw<32, 6, true>(b[6]);
    b[7] = tw<32, 7, true>(b[7]);
    b[8] = tw<32, 8, true>(b[8]);
    b[9] = tw<32, 9, true>(b[9]);
    b[10] = tw<32, 10, true>(b[10]);
    b[11] = tw<32, 11, true>(b[11]);
    b[12] = tw<32, 12, true>(b[12]);
    b[13] = tw<32, 13, true>(b[13]);
    b[14] = tw<32, 14, true>(b[14]);
    b[15] = tw<32, 15, true>(b[15]);
    idft16_lo(a);
    idft16_lo(b);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        y[2 * m] = a[m];
        y[2 * m + 1] = b[m];
    }
}

// v[r] *= W32^r for r = 0..15 (the odd outputs of a 32-point DFT whose
// inputs 16..31 are zero are the 16-point DFT of x[r] W32^r).
__device__ __forceinline__ void tw32_half(float2 (&v)[16])
{
    v[1] = tw<32, 1, false>(v[1]);
    v[2] = tw<32, 2, false>(v[2]);
    v[3] = tw<32, 3, false>(v[3]);
    v[4] = tw<32, 4, false>(v[4]);
    v[5] = tw<32, 5, false>(v[5]);
    v[6] = tw<32, 6, false>(v[6]);
    v[7] = tw<32, 7, false>(v[7]);
    v[8] = tw<32, 8, false>(v[8]);
    v[9] = tw<32, 9, false>(v[9]);
    v[10] = tw<32, 10, false>(v[10]);
    v[11] = tw<32, 11, false>(v[11]);
    v[12] = tw<32, 12, false>(v[12]);
    v[13] = tw<32, 13, false>(v[13]);
    v[14] = tw<32, 14, false>(v[14]);
    v[15] = tw<32, 15, false>(v[15]);
}

// h = -N^ m at one frequency with the stored octant values t[0..5] = (xx, yy,
// zz, xy, xz, yz) and the fold signs sy (ky > Py/2: xy, yz flip) and sz
// (kz > L/2: xz, yz flip); SY is the tile's sign, sz a per-call value.
template <bool SYNEG>
__device__ __forceinline__ void product(float2 &mx, float2 &my, float2 &mz, float txx, float tyy, float tzz,
                                        float txy, float txz, float tyz)
{
    // each product term as one packed FP32x2 multiply-add with the negated
    // tensor value in both halves
    const float nxy = SYNEG ? txy : -txy, nyz = SYNEG ? tyz : -tyz;
    const float2 x = mx, y = my, z = mz;
    const float2 pxx = make_float2(-txx, -txx), pyy = make_float2(-tyy, -tyy), pzz = make_float2(-tzz, -tzz);
    const float2 pxy = make_float2(nxy, nxy), pxz = make_float2(-txz, -txz), pyz = make_float2(nyz, nyz);
    mx = __ffma2_rn(pxz, z, __ffma2_rn(pxy, y, __fmul2_rn(pxx, x)));
    my = __ffma2_rn(pyz, z, __ffma2_rn(pyy, y, __fmul2_rn(pxy, x)));
    mz = __ffma2_rn(pzz, z, __ffma2_rn(pyz, y, __fmul2_rn(pxz, x)));
}

}  // namespace zw

// Tile width TC (columns kx per tile, 4 or 8) and block size of the
// persistent z pass. The tensor block of a tile is TC/4 sub-blocks of 4
// columns ([6][HZ][4] floats each, TZB floats), laid TZS floats apart in
// shared memory (TZS = 16 mod 32 banks: the two sub-blocks of an 8-column
// tile fall in different bank halves).
// L = 512 runs as 2 x 16 x 16 (R1 = 32: a 32-point stage whose input half is
// padding, done as two 16-point DFTs), L = 256 as 16 x 16 (R1 = 16: a
// 16-point stage on 8 input rows). The exchange rows R1 j + k are padded by
// one row every R1 rows (EXR rows per component).
template <int L, int TC> struct ZwsShape {
    static_assert(L == 256 || L == 512, "the persistent z pass is built for L = 256 and 512");
    static_assert(TC == 4 || TC == 8, "tile width 4 or 8");
    static constexpr int R1 = L / 16;
    static constexpr int NT = R1 * TC, HZ = L / 2 + 1, EXR = L + 16;
    static constexpr int TZB = 6 * HZ * 4, TZS = TZB + 24, NSUB = TC / 4;  // HZ odd: TZS = 16 mod 32
    static constexpr int MIN_CTAS = (L == 512 && TC == 8) ? 1 : 2;
};

// Tile-ordered copy of the FP32 octant tensor spectrum for the persistent z
// pass: [Py/2+1][ntx4][6][Pz/2+1][4] (4-column sub-blocks, ntx4 = ceil(Kx/4)
// rounded up to even), zero for kx >= Kx; each sub-block is contiguous and
// fetched with one bulk copy.
template <typename T>
__global__ void k_tile_tensor(const T *__restrict__ nhat, T *__restrict__ out, int Kx, int hy, int HZ, int ntx4)
{
    const int64_t total = (int64_t)hy * ntx4 * 6 * HZ * 4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i;
        const int c = (int)(r & 3); r >>= 2;
        const int kzf = (int)(r % HZ); r /= HZ;
        const int comp = (int)(r % 6); r /= 6;
        const int kxt = (int)(r % ntx4);
        const int kyf = (int)(r / ntx4);
        const int kx = kxt * 4 + c;
        out[i] = kx < Kx ? nhat[(((int64_t)comp * HZ + kzf) * hy + kyf) * Kx + kx] : (T)0;
    }
}

// 4-column sub-blocks per ky row of the tile-ordered tensor copy.
__host__ __device__ inline int zws_ntx4(int Kx) { return ((Kx + 3) / 4 + 1) / 2 * 2; }

// Shared memory of the persistent z pass for nrows input rows.
template <int L, int TC>
__host__ __device__ inline size_t zws_smem_bytes(int nrows)
{
    using Sh = ZwsShape<L, TC>;
    const size_t stg = ((size_t)3 * nrows * TC * sizeof(float2) + 127) / 128 * 128;
    const size_t ex = (size_t)3 * Sh::EXR * TC * sizeof(float2);
    const size_t tz = (size_t)Sh::NSUB * Sh::TZS * sizeof(float);
    return 128 + stg + ex + tz + 2 * sizeof(uint64_t);
}

// The persistent fused z pass (L = 256 or 512, FP32). Tile t covers the columns
// kx = kxt TC .. kxt TC + TC - 1 (kxt = t % ntx) of the ky row
// ky_pair_order(t / ntx), so that the two ky rows sharing a folded tensor
// block are processed at about the same time. map: S2 [3][nz][Py][Kxp] as
// reals, box (2 TC, 1, nz, 3). ntile: the tile-ordered tensor copy. twg: the
// z axis twiddle table W_L^m, m < L.
//
// EONLY: the spectral (Parseval) energy instead of the field: after the
// forward transforms each thread sums w(kx) m^H N^ m over its frequencies,
// nothing is transformed back or written; partials[blockIdx.x] receives the
// CTA's sum over all its tiles (NaN if a wait gave up).
// FE: the field and the same energy sum, taken at the product as
// -Re(m^H h) with h = -N^ m (both in registers there).
template <int L, int TC, bool EONLY = false, bool FE = false>
__global__ void __launch_bounds__(ZwsShape<L, TC>::NT, ZwsShape<L, TC>::MIN_CTAS)
k_z_ws(const __grid_constant__ CUtensorMap map, float2 *__restrict__ S, int Kx, int Py, int64_t ss, int64_t rs,
       int64_t cs, int nrows, const float *__restrict__ ntile, const float2 *__restrict__ twg, int ntx, int ntiles,
       double *__restrict__ partials = nullptr)
{
    using Sh = ZwsShape<L, TC>;
    constexpr int NT = Sh::NT, HZ = Sh::HZ, EXR = Sh::EXR, TZB = Sh::TZB, TZS = Sh::TZS, NSUB = Sh::NSUB;
    constexpr int R1 = Sh::R1, RP = R1 + 1;  // stage-1 radix; padded row stride of the row groups
    constexpr unsigned TZ_BYTES = (unsigned)(NSUB * TZB * sizeof(float));
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((128 - (smem_u32(smraw) & 127)) & 127);
    const unsigned in_bytes = 3u * (unsigned)nrows * TC * (unsigned)sizeof(float2);
    const size_t stg_bytes = ((size_t)in_bytes + 127) / 128 * 128;
    float2 *stg = reinterpret_cast<float2 *>(base);                 // [3][nrows][TC]
    float2 *ex = reinterpret_cast<float2 *>(base + stg_bytes);      // [3][EXR][TC]
    float *tz = reinterpret_cast<float *>(ex + 3 * EXR * TC);       // [NSUB][TZS]: [6][HZ][4] each
    uint64_t *bar = reinterpret_cast<uint64_t *>(tz + NSUB * TZS);  // [0] input, [1] tensor
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    const int c = tid & (TC - 1);
    const int ntx4 = zws_ntx4(Kx);

    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // stage-2 twiddles W_L^(r j2), fixed per thread
    const int j2 = tid / TC;
    float2 w2[16];
#pragma unroll
    for (int r = 1; r < 16; ++r) w2[r] = twg[r * j2];

    auto tile_ky = [&](int t) { return ky_pair_order(t / ntx, Py); };
    auto issue_in = [&](int t) {
        mbar_expect_tx(&bar[0], in_bytes);
        tma_load_4d(stg, &map, 2 * (t % ntx) * TC, tile_ky(t), 0, 0, &bar[0]);
    };
    auto issue_tz = [&](int t) {
        const int ky = tile_ky(t);
        const int kyf = ky > Py / 2 ? Py - ky : ky;
        mbar_expect_tx(&bar[1], TZ_BYTES);
        const float *src = ntile + ((size_t)kyf * ntx4 + (t % ntx) * NSUB) * TZB;
#pragma unroll
        for (int h = 0; h < NSUB; ++h) bulk_g2s(tz + h * TZS, src + h * TZB, TZB * (unsigned)sizeof(float), &bar[1]);
    };

    static_assert(!(EONLY && FE), "one energy form at a time");
    double eacc = 0.0;  // EONLY / FE: this thread's sum over its tiles
    auto fail_exit_partial = [&]() {
        if constexpr (EONLY || FE) {
            if (tid == 0) partials[blockIdx.x] = __longlong_as_double(0x7ff8000000000000LL);
        }
    };
    int t = blockIdx.x;
    if (tid == 0 && t < ntiles) {
        issue_in(t);
        issue_tz(t);
    }
    for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
        const int next = t + gridDim.x;
        const unsigned par = (unsigned)(k & 1);
        const int ky = tile_ky(t), kx0 = (t % ntx) * TC;
        if (!mbar_wait_bounded(&bar[0], par, kPipeWaitCycles)) s_fail = 1;

        // ---- stage 1. L = 512: rows j1 + 16 r (r < 16; the upper half is
        // padding) -> 32-point DFT outputs 2m + p at rows 32 j1 + 2m + p
        // (p = 0 even, 1 odd). L = 256: rows j1 + 16 r (r < 8) -> 16-point
        // DFT outputs at rows 16 j1 + m.
        {
            const int j1 = (tid / TC) & 15, p = L == 512 ? tid / (16 * TC) : 0;
            // the three components' loads first, then their transforms
            float2 v[3][16];
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                const float2 *src = stg + ((size_t)comp * nrows + j1) * TC + c;
#pragma unroll
                for (int r = 0; r < 16; ++r)
                    v[comp][r] = (r < L / 32 && j1 + 16 * r < nrows) ? src[16 * r * TC] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                if constexpr (L == 512) {
                    if (p) zw::tw32_half(v[comp]);
                    zw::dft16<false>(v[comp]);
                    float2 *dst = ex + ((size_t)comp * EXR + RP * j1 + p) * TC + c;
#pragma unroll
                    for (int m = 0; m < 16; ++m) dst[2 * m * TC] = v[comp][m];
                } else {
                    zw::dft16_half_in(v[comp]);
                    float2 *dst = ex + ((size_t)comp * EXR + RP * j1) * TC + c;
#pragma unroll
                    for (int m = 0; m < 16; ++m) dst[m * TC] = v[comp][m];
                }
            }
        }
        __syncthreads();  // staging buffer consumed, exchange written
        if (s_fail) {
            // the input copy of this tile timed out; its tensor copy was issued
            if (tid == 0) {
                mbar_wait_bounded(&bar[0], par, kPipeWaitCycles);
                mbar_wait_bounded(&bar[1], par, kPipeWaitCycles);
                atomicExch(&g_xpipe_error, 1);
            }
            fail_exit_partial();
            return;
        }
        if (tid == 0 && next < ntiles) {
            fence_proxy_async_smem();
            issue_in(next);
        }

        // ---- stage 2: rows R1 r + j2 of the three components: twiddle,
        // 16-point DFTs (kz = j2 + R1 m), product, inverse DFTs, in place
        {
            float2 a[16], b[16], d[16];
            const float2 *s = ex + (size_t)j2 * TC + c;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                a[r] = s[RP * r * TC];
                b[r] = s[(EXR + RP * r) * TC];
                d[r] = s[(2 * EXR + RP * r) * TC];
            }
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                a[r] = zw::mul(a[r], w2[r]);
                b[r] = zw::mul(b[r], w2[r]);
                d[r] = zw::mul(d[r], w2[r]);
            }
            zw::dft16<false>(a);
            zw::dft16<false>(b);
            zw::dft16<false>(d);
            if (!mbar_wait_bounded(&bar[1], par, kPipeWaitCycles)) s_fail = 1;
            const float *tb = tz + (c >> 2) * TZS + (c & 3);
            const float szm = j2 == 0 ? 1.f : -1.f;  // kz = L/2 + j2: folded unless j2 = 0
            if constexpr (EONLY) {
                float e = 0.f;
                auto quad_all = [&](auto syneg) {
                    constexpr bool SN = decltype(syneg)::value;
#pragma unroll
                    for (int m = 0; m < 16; ++m) {
                        const int kzf = m < 8 ? j2 + R1 * m : (m == 8 ? L / 2 - j2 : L - j2 - R1 * m);
                        const float *q = tb + kzf * 4;
                        float txz = q[4 * HZ * 4], tyz = q[5 * HZ * 4];
                        if (m == 8) {
                            txz *= szm;
                            tyz *= szm;
                        } else if (m > 8) {
                            txz = -txz;
                            tyz = -tyz;
                        }
                        const float nxy = SN ? -q[3 * HZ * 4] : q[3 * HZ * 4], nyz = SN ? -tyz : tyz;
                        e += quad_form<float>(a[m], b[m], d[m], q[0], q[HZ * 4], q[2 * HZ * 4], nxy, txz, nyz);
                    }
                };
                if (ky > Py / 2) quad_all(std::true_type{});
                else quad_all(std::false_type{});
                eacc += (double)(e * kx_weight<float>(kx0 + c, Kx));
            } else {
            // FE: Re(m^H h) over this thread's frequencies, one packed
            // accumulator per component
            float2 ex2 = make_float2(0.f, 0.f), ey2 = ex2, ez2 = ex2;
            auto prod_all = [&](auto syneg) {
                constexpr bool SN = decltype(syneg)::value;
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    const int kzf = m < 8 ? j2 + R1 * m : (m == 8 ? L / 2 - j2 : L - j2 - R1 * m);
                    const float *q = tb + kzf * 4;
                    float txz = q[4 * HZ * 4], tyz = q[5 * HZ * 4];
                    if (m == 8) {
                        txz *= szm;
                        tyz *= szm;
                    } else if (m > 8) {
                        txz = -txz;
                        tyz = -tyz;
                    }
                    if constexpr (FE) {
                        const float2 mx = a[m], my = b[m], mz = d[m];
                        zw::product<SN>(a[m], b[m], d[m], q[0], q[HZ * 4], q[2 * HZ * 4], q[3 * HZ * 4], txz, tyz);
                        ex2 = __ffma2_rn(mx, a[m], ex2);
                        ey2 = __ffma2_rn(my, b[m], ey2);
                        ez2 = __ffma2_rn(mz, d[m], ez2);
                    } else {
                        zw::product<SN>(a[m], b[m], d[m], q[0], q[HZ * 4], q[2 * HZ * 4], q[3 * HZ * 4], txz, tyz);
                    }
                }
            };
            if (ky > Py / 2) prod_all(std::true_type{});
            else prod_all(std::false_type{});
            if constexpr (FE)
                eacc -= (double)(((ex2.x + ex2.y) + (ey2.x + ey2.y) + (ez2.x + ez2.y)) * kx_weight<float>(kx0 + c, Kx));
            zw::dft16<true>(a);
            zw::dft16<true>(b);
            zw::dft16<true>(d);
            // the stage-3 twiddles W_L^-(n1 k1) with k1 = j2: conj(w2[n1])
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                a[r] = zw::mulc(a[r], w2[r]);
                b[r] = zw::mulc(b[r], w2[r]);
                d[r] = zw::mulc(d[r], w2[r]);
            }
            float2 *o = ex + (size_t)j2 * TC + c;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                o[RP * r * TC] = a[r];
                o[(EXR + RP * r) * TC] = b[r];
                o[(2 * EXR + RP * r) * TC] = d[r];
            }
            }  // !EONLY
        }
        __syncthreads();  // tensor block consumed, exchange written
        if (s_fail) {
            // the tensor copy of this tile timed out; the next input copy may be in flight
            if (tid == 0) {
                if (next < ntiles) mbar_wait_bounded(&bar[0], par ^ 1u, kPipeWaitCycles);
                mbar_wait_bounded(&bar[1], par, kPipeWaitCycles);
                atomicExch(&g_xpipe_error, 1);
            }
            fail_exit_partial();
            return;
        }
        if (tid == 0 && next < ntiles) {
            fence_proxy_async_smem();
            issue_tz(next);
        }

        if constexpr (EONLY) continue;  // no inverse transforms

        // ---- stage 3: rows R1 n1 + k1 (k1 < R1, already twiddled by
        // W_L^-(n1 k1) in stage 2), R1-point inverse DFT of which the outputs
        // n2 < R1/2 are formed: z = n1 + 16 n2 < nz to global memory
        if constexpr (L == 512) {
#pragma unroll 1
            for (int b = tid; b < 3 * 16 * TC; b += NT) {
                const int comp = b / (16 * TC), n1 = (b / TC) & 15;
                float2 u[32];
                const float2 *s = ex + ((size_t)comp * EXR + RP * n1) * TC + c;
#pragma unroll
                for (int k1 = 0; k1 < 32; ++k1) u[k1] = s[k1 * TC];
                float2 y[16];
                zw::idft32_lo(u, y);
                if (kx0 + c < Kx) {
                    float2 *col = S + (int64_t)comp * cs + (int64_t)ky * ss + kx0 + c;
#pragma unroll
                    for (int n2 = 0; n2 < 16; ++n2) {
                        const int z = n1 + 16 * n2;
                        if (z < nrows) col[(int64_t)z * rs] = y[n2];
                    }
                }
            }
        } else {
            const int n1 = tid / TC;
#pragma unroll 1
            for (int comp = 0; comp < 3; ++comp) {
                float2 u[16];
                const float2 *s = ex + ((size_t)comp * EXR + RP * n1) * TC + c;
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) u[k1] = s[k1 * TC];
                zw::idft16_lo(u);
                if (kx0 + c < Kx) {
                    float2 *col = S + (int64_t)comp * cs + (int64_t)ky * ss + kx0 + c;
#pragma unroll
                    for (int n2 = 0; n2 < 8; ++n2) {
                        const int z = n1 + 16 * n2;
                        if (z < nrows) col[(int64_t)z * rs] = u[n2];
                    }
                }
            }
        }
        __syncthreads();  // exchange read before the next tile's stage 1 writes it
    }
    if constexpr (EONLY || FE) block_partial<NT>(eacc, partials, blockIdx.x);
}

}  // namespace demag
