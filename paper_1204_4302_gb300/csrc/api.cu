// C ABI of the FFT demagnetization-tensor library (declared in
// include/demag.h). Host-side plan management and the pass sequence:
//
//   x R2C (pruned to nx inputs) -> y FFT (ny of Py inputs) ->
//   z FFT . (H^ = -N^ M^) . z IFFT (nz outputs kept) ->
//   y IFFT (ny outputs kept) -> x C2R (nx outputs, scaled 1/(Px Py Pz),
//   optional per-block energy sums) [-> energy finalise]
//
// which is the zero-padded convolution H = -N * M of paper Sec. 3.1 (Eq.
// "demag" evaluated through Eq. "convolution").
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

using demag::Passes;

namespace {

// Allocation hook for tests of the error paths (demag_debug_fail_alloc):
// when armed with n, the n-th next device allocation of the plan code fails
// as if the device were out of memory.
std::atomic<long> g_fail_alloc{0};

// Debug allocations (DEMAG_DEBUG=1): guard zones of kGuardBytes before and
// after each buffer, filled with kGuardByte, registered by the buffer's
// address so dfree releases the whole block and demag_check_pipeline scans
// the zones.
constexpr size_t kGuardBytes = 4096;
constexpr unsigned char kGuardByte = 0xA5;
struct GuardBlock {
    void *base;
    size_t bytes;
    long serial;
};
std::mutex g_guard_mu;
std::map<void *, GuardBlock> g_guards;
long g_guard_serial = 0;

bool debug_allocations()
{
    const char *v = getenv("DEMAG_DEBUG");
    return v && v[0] && strcmp(v, "0") != 0;
}

template <typename P>
cudaError_t dmalloc(P **ptr, size_t bytes)
{
    long n = g_fail_alloc.load();
    while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    if (!debug_allocations()) return cudaMalloc(reinterpret_cast<void **>(ptr), bytes);
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes + 2 * kGuardBytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return e;
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    if ((e = cudaMemset(b, kGuardByte, kGuardBytes)) != cudaSuccess ||
        (e = cudaMemset(b + kGuardBytes + bytes, kGuardByte, kGuardBytes)) != cudaSuccess) {
        cudaFree(base);
        *ptr = nullptr;
        return e;
    }
    void *user = b + kGuardBytes;
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        g_guards[user] = GuardBlock{base, bytes, ++g_guard_serial};
    }
    *ptr = static_cast<P *>(user);
    return cudaSuccess;
}

// cudaFree for buffers from dmalloc (the guarded block when it has one).
void dfree(void *ptr)
{
    if (!ptr) return;
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        auto it = g_guards.find(ptr);
        if (it != g_guards.end()) {
            void *base = it->second.base;
            g_guards.erase(it);
            cudaFree(base);
            return;
        }
    }
    cudaFree(ptr);
}

__global__ void k_guard_scan(const unsigned char *__restrict__ z, int n, unsigned int *__restrict__ bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (z[i] != kGuardByte) atomicAdd(bad, 1u);
}

thread_local std::string g_err;
// The plan whose entry point the calling thread is in (its failures are also
// kept on the plan, for demag_last_error(plan)).
thread_local demag_plan *g_err_plan = nullptr;

struct PlanScope {
    demag_plan *prev;
    explicit PlanScope(demag_plan *p) : prev(g_err_plan) { g_err_plan = p; }
    ~PlanScope() { g_err_plan = prev; }
};

demag_status fail(demag_status s, const std::string &msg)
{
    g_err = msg;
    if (g_err_plan) snprintf(g_err_plan->last_err, sizeof g_err_plan->last_err, "%s", msg.c_str());
    return s;
}

#define DEMAG_CUDA(call)                                                                      \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? DEMAG_ERR_OOM : DEMAG_ERR_CUDA,     \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

constexpr int kMaxN = 512;
constexpr int kMaxP = 1024;
constexpr double kMu0 = 4e-7 * 3.14159265358979323846;

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int default_pad(int n)
{
    int p = 1;
    while (p < 2 * n - 1) p *= 2;
    return p;
}

// even, with no prime factor above 7 (the mixed-radix passes' lengths)
bool is_smooth_even(int v)
{
    if (v < 2 || v % 2) return false;
    for (int f : {2, 3, 5, 7})
        while (v % f == 0) v /= f;
    return v == 1;
}

int smooth_pad(int n)
{
    if (n == 1) return 1;
    int p = 2 * n - 1;
    while (!is_smooth_even(p)) ++p;
    return p;
}

// Padded lengths of a DM plan from its options (pad_mode powers of two or
// smooth, explicit lengths checked); DEMAG_PAD_TUNED is resolved by timing
// elsewhere and is UNSUPPORTED here.
demag_status pad_lengths(const int n[3], const demag_options *opt, int P[3])
{
    if (opt && opt->pad_mode != DEMAG_PAD_POW2 && opt->pad_mode != DEMAG_PAD_SMOOTH &&
        opt->pad_mode != DEMAG_PAD_TUNED)
        return fail(DEMAG_ERR_INVALID_ARG, "unknown pad_mode");
    if (opt && opt->pad_mode == DEMAG_PAD_TUNED)
        return fail(DEMAG_ERR_UNSUPPORTED, "tuned padded lengths come from demag_tune_padding");
    const bool smooth = opt && opt->pad_mode == DEMAG_PAD_SMOOTH;
    for (int a = 0; a < 3; ++a) P[a] = smooth ? smooth_pad(n[a]) : default_pad(n[a]);
    if (opt) {
        const int req[3] = {opt->px, opt->py, opt->pz};
        for (int a = 0; a < 3; ++a) {
            if (req[a] == 0) continue;
            if (!(is_pow2(req[a]) || is_smooth_even(req[a])) || req[a] < 2 * n[a] - 1)
                return fail(DEMAG_ERR_INVALID_ARG,
                            "padded lengths must be >= 2n - 1 and powers of two or even products of 2, 3, 5, 7");
            if (req[a] > kMaxP) return fail(DEMAG_ERR_UNSUPPORTED, "padded lengths above 1024 are not built");
            P[a] = req[a];
        }
    }
    return DEMAG_OK;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t elem_size(const demag_plan *p) { return p->prec == DEMAG_F32 ? sizeof(float) : sizeof(double); }

int64_t ncell(const demag_plan *p) { return (int64_t)p->nx * p->ny * p->nz; }

// The pointer must be device (or managed) memory of the plan's device, 16-byte
// aligned. Host pointers are rejected before any kernel could touch them.
demag_status check_dev_ptr(const demag_plan *p, const void *ptr, const char *name)
{
    if (!ptr) return fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is NULL");
    if (((uintptr_t)ptr & 15u) != 0) return fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not device memory");
    if (a.type == cudaMemoryTypeDevice && a.device != p->device)
        return fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " lives on another device");
    return DEMAG_OK;
}

bool overlap(const void *a, const void *b, size_t bytes)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

// [a, a + abytes) and [b, b + bbytes) intersect
bool overlap2(const void *a, size_t abytes, const void *b, size_t bbytes)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bbytes && y < x + abytes;
}

// Twiddle table W_P^m = exp(-2 pi i m / P), m < P, from long double sin/cos.
template <typename C>
std::vector<C> twiddles(int P)
{
    std::vector<C> t(P);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int m = 0; m < P; ++m) {
        const long double a = 2.0L * pi * (long double)m / (long double)P;
        t[m].x = (decltype(t[m].x))cosl(a);
        t[m].y = (decltype(t[m].y))(-sinl(a));
    }
    return t;
}

// --- per-kernel timing: a ring of call slots with one event per pass edge.
constexpr int kRing = 64;
constexpr int kEvPerCall = 8;

struct TimingRing {
    cudaEvent_t ev[kRing][kEvPerCall];
    int used[kRing];  // number of events recorded in the slot (0 = free)
    int next;
};

TimingRing *ring_of(demag_plan *p) { return static_cast<TimingRing *>(p->ring); }

void ring_collect_slot(demag_plan *p, TimingRing *R, int s)
{
    if (R->used[s] < 2) { R->used[s] = 0; return; }
    cudaEventSynchronize(R->ev[s][R->used[s] - 1]);
    for (int i = 0; i + 1 < R->used[s]; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, R->ev[s][i], R->ev[s][i + 1]) == cudaSuccess) {
            p->pass_ms[i] += ms;
            p->pass_n[i] += 1;
        }
    }
    R->used[s] = 0;
}

struct PassTimer {
    demag_plan *p;
    TimingRing *R = nullptr;
    int slot = -1, k = 0;
    cudaStream_t st;
    PassTimer(demag_plan *p_, cudaStream_t s) : p(p_), st(s)
    {
        if (!p->timing) return;
        R = ring_of(p);
        slot = R->next;
        R->next = (R->next + 1) % kRing;
        if (R->used[slot]) ring_collect_slot(p, R, slot);
        mark();
    }
    void mark()
    {
        if (R && k < kEvPerCall) { cudaEventRecord(R->ev[slot][k], st); ++k; R->used[slot] = k; }
    }
};

// What one pass through the pipeline reads and writes (see XIn / XOut).
struct FieldJob {
    const void *in;       // input field [3][nz][ny][nx]
    void *phi = nullptr;  // SP only: optional node potential [nz+1][ny+1][nx+1]
    const void *wcell;    // optional per-cell weight [nz][ny][nx]
    double wscalar;       // input = in * wscalar * wcell
    void *out;            // optional output = H * oscale * wcell * g
    double oscale;
    const double *gdev;   // optional device scalar g
    double *E_dev;        // optional energy -(mu0/2) V sum input . H
};

// Field calls with the energy take its spectral sum in the persistent z pass
// (FP32 plans of the tensor method whose z form is 6 or 7 at length 256 or
// 512, spectral route on); the last pass then does not read M.
bool energy_in_z(const demag_plan *p)
{
    return p->method == DEMAG_METHOD_DM && p->prec == DEMAG_F32 && p->spectral_energy && p->ntile &&
           (p->zvariant == 6 || p->zvariant == 7) && (p->Pz == 256 || p->Pz == 512);
}

template <typename T>
demag_status run_field(demag_plan *p, const FieldJob &job, cudaStream_t st)
{
    using C = typename demag::CplxOf<T>::type;
    C *S1 = static_cast<C *>(p->S1);
    C *S2 = static_cast<C *>(p->S2);
    const bool f32 = p->prec == DEMAG_F32;
    const C *twx = f32 ? (const C *)(const void *)p->tw32[0] : (const C *)(const void *)p->tw64[0];
    const C *twy = f32 ? (const C *)(const void *)p->tw32[1] : (const C *)(const void *)p->tw64[1];
    const C *twz = f32 ? (const C *)(const void *)p->tw32[2] : (const C *)(const void *)p->tw64[2];
    const T *nhat = f32 ? (const T *)(const void *)p->nhat32 : (const T *)(const void *)p->nhat64;
    const int nx = p->nx, ny = p->ny, nz = p->nz, Px = p->Px, Py = p->Py, Pz = p->Pz, Kx = p->Kx, Kxp = p->Kxp;
    const int rows = 3 * nz * ny;
    demag::XIn<T> xi;
    xi.in = static_cast<const T *>(job.in);
    xi.in_rs = nx;
    xi.wcell = static_cast<const T *>(job.wcell);
    xi.wscalar = (T)job.wscalar;
    xi.rows_per_comp = nz * ny;
    demag::XOut<T> xo;
    xo.out = static_cast<T *>(job.out);
    xo.out_rs = nx;
    xo.scale = (T)(1.0 / ((double)Px * Py * Pz));
    xo.oscale = (T)job.oscale;
    xo.wcell = static_cast<const T *>(job.wcell);
    xo.gdev = job.gdev;
    xo.Mref = job.E_dev ? static_cast<const T *>(job.in) : nullptr;
    xo.mscale = (T)job.wscalar;
    xo.partials = job.E_dev ? p->partials : nullptr;
    xo.rows_per_comp = nz * ny;
    PassTimer tm(p, st);
    cudaError_t e;
    // energy without a field: the spectral (Parseval) sum in the z pass,
    // E = (mu0/2) (V / (Px Py Pz)) sum_k w(kx) M^H N^ M, no inverse passes
    const bool spectral = !job.out && job.E_dev && p->spectral_energy &&
                          Passes<T>::zenergy_blocks(Pz, Py, Kx) > 0;
    // x forward
    if (Px == 1) e = Passes<T>::x1_fwd(xi, rows, S1, st);
    else e = Passes<T>::x_fwd(Px / 2, xi, rows, nx, S1, Kxp, twx, st, p->xvariant);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("x forward: ") + cudaGetErrorString(e));
    p->launches++;
    tm.mark();
    // y forward
    if (Py > 1) {
        e = Passes<T>::col(Py, false, S1, S2, 3 * nz * Kx, Kx, (int64_t)ny * Kxp, Kxp, ny,
                           (int64_t)Py * Kxp, Kxp, Py, twy, 1, st, p->yvariant);
        if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("y forward: ") + cudaGetErrorString(e));
        p->launches++;
    }
    tm.mark();
    if (spectral) {
        int nparts = p->npartials;
        e = cudaErrorNotSupported;
        if ((p->zvariant == 6 || p->zvariant == 7) && f32 && p->ntile)
            e = Passes<T>::zconv_ws_energy(Pz, S2, Kx, Py, Kxp, (int64_t)Py * Kxp, (int64_t)nz * Py * Kxp, nz,
                                           (const T *)(const void *)p->ntile, twz, p->partials, &nparts, st,
                                           p->zvariant == 7 ? 4 : 8);
        if (e == cudaErrorNotSupported)
            e = Passes<T>::zconv_energy(Pz, S2, Py * Kx, Kx, Kxp, (int64_t)Py * Kxp, (int64_t)nz * Py * Kxp, nz, nhat,
                                        Py, Kx, twz, 1, p->partials, &nparts, st);
        if (e != cudaSuccess)
            return fail(DEMAG_ERR_CUDA, std::string("z spectral energy: ") + cudaGetErrorString(e));
        p->launches++;
        tm.mark();
        tm.mark();  // no inverse y pass
        tm.mark();  // no inverse x pass
        const double V = p->dx * p->dy * p->dz;
        e = demag::energy_finalize(p->partials, nparts, 0.5 * kMu0 * V / ((double)Px * Py * Pz), job.E_dev,
                                   p->partials + p->npartials, st);
        if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("energy: ") + cudaGetErrorString(e));
        p->launches++;
        tm.mark();
        return DEMAG_OK;
    }
    // z forward . product . z inverse; with the energy and the persistent
    // form, the energy's spectral sum is taken there (so the x inverse pass
    // does not read M)
    e = cudaErrorNotSupported;
    int zparts = p->npartials;
    const bool zenergy = job.E_dev && energy_in_z(p);
    if ((p->zvariant == 6 || p->zvariant == 7) && f32 && p->ntile)  // persistent TMA forms, FP32 only
        e = Passes<T>::zconv_ws(Pz, S2, Kx, Py, Kxp, (int64_t)Py * Kxp, (int64_t)nz * Py * Kxp, nz,
                                (const T *)(const void *)p->ntile, twz, st, p->zvariant == 7 ? 4 : 8,
                                zenergy ? p->partials : nullptr, zenergy ? &zparts : nullptr);
    if (!(e == cudaSuccess && zenergy)) zparts = 0;
    if (zparts > 0) {
        xo.Mref = nullptr;
        xo.partials = nullptr;
    }
    if (e == cudaErrorNotSupported)
        e = Passes<T>::zconv(Pz, S2, Py * Kx, Kx, Kxp, (int64_t)Py * Kxp, (int64_t)nz * Py * Kxp, nz, nhat, Py, Kx,
                             twz, 1, st, (p->zvariant == 6 || p->zvariant == 7) ? 0 : p->zvariant);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("z convolution: ") + cudaGetErrorString(e));
    p->launches++;
    tm.mark();
    // y inverse
    if (Py > 1) {
        e = Passes<T>::col(Py, true, S2, S1, 3 * nz * Kx, Kx, (int64_t)Py * Kxp, Kxp, Py, (int64_t)ny * Kxp, Kxp,
                           ny, twy, 1, st, p->yvariant);
        if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("y inverse: ") + cudaGetErrorString(e));
        p->launches++;
    }
    tm.mark();
    // x inverse (+ epilogue)
    int nblocks;
    if (Px == 1) {
        nblocks = p->npartials;
        e = Passes<T>::x1_inv(S1, rows, xo, nblocks, st);
    } else {
        nblocks = Passes<T>::x_blocks(Px / 2, rows);
        e = Passes<T>::x_inv(Px / 2, S1, Kxp, rows, nx, xo, twx, st, p->xvariant);
    }
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("x inverse: ") + cudaGetErrorString(e));
    p->launches++;
    tm.mark();
    if (job.E_dev) {
        const double V = p->dx * p->dy * p->dz;
        if (zparts > 0)  // spectral sum of the z pass
            e = demag::energy_finalize(p->partials, zparts, 0.5 * kMu0 * V / ((double)Px * Py * Pz), job.E_dev,
                                       p->partials + p->npartials, st);
        else
            e = demag::energy_finalize(p->partials, nblocks, -0.5 * kMu0 * V, job.E_dev, p->partials + p->npartials,
                                       st);
        if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("energy: ") + cudaGetErrorString(e));
        p->launches++;
        tm.mark();
    }
    return DEMAG_OK;
}

// Scalar-potential method (paper Sec. 3.1): x and y forward passes as for
// the tensor method, the SP z pass to the potential spectrum (one component,
// nz + 1 node rows, written over component 0), inverse y and x passes of that
// one component to the node potential (nz+1)(ny+1)(nx+1), then the field by
// finite differences (and the energy partials).
template <typename T>
demag_status run_field_sp(demag_plan *p, const FieldJob &job, cudaStream_t st)
{
    using C = typename demag::CplxOf<T>::type;
    C *S1 = static_cast<C *>(p->S1);
    C *S2 = static_cast<C *>(p->S2);
    const bool f32 = p->prec == DEMAG_F32;
    auto pick = [&](float2 *a, double2 *b) { return f32 ? (const C *)(const void *)a : (const C *)(const void *)b; };
    const C *twx = pick(p->tw32[0], p->tw64[0]), *twy = pick(p->tw32[1], p->tw64[1]), *twz = pick(p->tw32[2], p->tw64[2]);
    const C *phx = pick(p->ph32[0], p->ph64[0]), *phy = pick(p->ph32[1], p->ph64[1]), *phz = pick(p->ph32[2], p->ph64[2]);
    const T *that = f32 ? (const T *)(const void *)p->nhat32 : (const T *)(const void *)p->nhat64;
    const int nx = p->nx, ny = p->ny, nz = p->nz, Px = p->Px, Py = p->Py, Pz = p->Pz, Kx = p->Kx, Kxp = p->Kxp;
    demag::XIn<T> xi;
    xi.in = static_cast<const T *>(job.in);
    xi.in_rs = nx;
    xi.wcell = nullptr;
    xi.wscalar = (T)1;
    xi.rows_per_comp = nz * ny;
    T *phi = job.phi ? static_cast<T *>(job.phi) : reinterpret_cast<T *>(S2);  // S2 is free after y inverse
    demag::XOut<T> xo;
    xo.out = phi;
    xo.out_rs = nx + 1;
    xo.scale = (T)(1.0 / ((double)Px * Py * Pz));
    xo.oscale = (T)1;
    xo.wcell = nullptr;
    xo.gdev = nullptr;
    xo.Mref = nullptr;
    xo.mscale = (T)1;
    xo.partials = nullptr;
    xo.rows_per_comp = (nz + 1) * (ny + 1);
    PassTimer tm(p, st);
    cudaError_t e = Passes<T>::x_fwd(Px / 2, xi, 3 * nz * ny, nx, S1, Kxp, twx, st, p->xvariant);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("x forward: ") + cudaGetErrorString(e));
    p->launches++;
    tm.mark();
    e = Passes<T>::col(Py, false, S1, S2, 3 * nz * Kx, Kx, (int64_t)ny * Kxp, Kxp, ny, (int64_t)Py * Kxp, Kxp, Py,
                       twy, 1, st, p->yvariant);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("y forward: ") + cudaGetErrorString(e));
    p->launches++;
    tm.mark();
    e = Passes<T>::sp_zconv(Pz, S2, Py * Kx, Kx, Kxp, (int64_t)Py * Kxp, (int64_t)nz * Py * Kxp, nz, nz + 1, that, Py,
                            Kx, twz, phx, phy, phz, st, p->zvariant);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("SP z pass: ") + cudaGetErrorString(e));
    p->launches++;
    tm.mark();
    e = Passes<T>::col(Py, true, S2, S1, (nz + 1) * Kx, Kx, (int64_t)Py * Kxp, Kxp, Py, (int64_t)(ny + 1) * Kxp, Kxp,
                       ny + 1, twy, 1, st, 0);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("y inverse: ") + cudaGetErrorString(e));
    p->launches++;
    tm.mark();
    e = Passes<T>::x_inv(Px / 2, S1, Kxp, (nz + 1) * (ny + 1), nx + 1, xo, twx, st, p->xvariant);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("x inverse: ") + cudaGetErrorString(e));
    p->launches++;
    tm.mark();
    if (job.out || job.E_dev) {
        e = Passes<T>::sp_grad(phi, nx, ny, nz, p->dx, p->dy, p->dz, static_cast<T *>(job.out),
                               job.E_dev ? static_cast<const T *>(job.in) : nullptr,
                               job.E_dev ? p->partials : nullptr, st);
        if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("SP field: ") + cudaGetErrorString(e));
        p->launches++;
        tm.mark();
    }
    if (job.E_dev) {
        const double V = p->dx * p->dy * p->dz;
        e = demag::energy_finalize(p->partials, Passes<T>::sp_grad_blocks(nx, ny, nz), -0.5 * kMu0 * V, job.E_dev,
                                   p->partials + p->npartials, st);
        if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("energy: ") + cudaGetErrorString(e));
        p->launches++;
        tm.mark();
    }
    return DEMAG_OK;
}

demag_status check_scalar_ptr(const void *ptr, const char *name)
{
    if (((uintptr_t)ptr & 7u) != 0) return fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not 8-byte aligned");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(DEMAG_ERR_INVALID_ARG, std::string(name) + " is not device memory");
    return DEMAG_OK;
}

// ----- CUDA-graph replay: each distinct call (pointers, scales, variants) is
// captured once on a private stream and replayed with one graph launch, so
// the host issues one launch per call instead of five or six (small grids
// are launch-bound).
struct GraphEntry {
    FieldJob job;
    int z, y, x;
    cudaGraphExec_t exec;
    long kernels;
    unsigned long long stamp;
};
struct GraphCache {
    std::vector<GraphEntry> entries;
    cudaStream_t cap = nullptr;
    unsigned long long clock = 0;
};
constexpr size_t kGraphSlots = 4;

bool same_job(const FieldJob &a, const FieldJob &b)
{
    return a.in == b.in && a.phi == b.phi && a.wcell == b.wcell && a.wscalar == b.wscalar && a.out == b.out &&
           a.oscale == b.oscale && a.gdev == b.gdev && a.E_dev == b.E_dev;
}

void graphs_free(demag_plan *p)
{
    GraphCache *G = static_cast<GraphCache *>(p->graphs);
    if (!G) return;
    for (auto &en : G->entries) cudaGraphExecDestroy(en.exec);
    if (G->cap) cudaStreamDestroy(G->cap);
    delete G;
    p->graphs = nullptr;
}

demag_status run_direct(demag_plan *p, const FieldJob &job, cudaStream_t st)
{
    if (p->method == DEMAG_METHOD_SP) {
        if (p->prec == DEMAG_F32) return run_field_sp<float>(p, job, st);
        return run_field_sp<double>(p, job, st);
    }
    if (p->prec == DEMAG_F32) return run_field<float>(p, job, st);
    return run_field<double>(p, job, st);
}

demag_status run_graph(demag_plan *p, const FieldJob &job, cudaStream_t st)
{
    GraphCache *G = static_cast<GraphCache *>(p->graphs);
    for (auto &en : G->entries)
        if (same_job(en.job, job) && en.z == p->zvariant && en.y == p->yvariant && en.x == p->xvariant) {
            en.stamp = ++G->clock;
            const cudaError_t e = cudaGraphLaunch(en.exec, st);
            if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
            p->launches += en.kernels;
            return DEMAG_OK;
        }
    cudaError_t e;
    if (!G->cap && (e = cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(DEMAG_ERR_CUDA, std::string("capture stream: ") + cudaGetErrorString(e));
    const long l0 = p->launches;
    if ((e = cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return fail(DEMAG_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    const demag_status s = run_direct(p, job, G->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(G->cap, &graph);
    const long kernels = p->launches - l0;
    p->launches = l0;  // the capture itself ran nothing
    if (s != DEMAG_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return s != DEMAG_OK ? s : fail(DEMAG_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    if (G->entries.size() >= kGraphSlots) {  // evict the least recently used call
        size_t old = 0;
        for (size_t i = 1; i < G->entries.size(); ++i)
            if (G->entries[i].stamp < G->entries[old].stamp) old = i;
        cudaGraphExecDestroy(G->entries[old].exec);
        G->entries.erase(G->entries.begin() + old);
    }
    G->entries.push_back(GraphEntry{job, p->zvariant, p->yvariant, p->xvariant, exec, kernels, ++G->clock});
    if ((e = cudaGraphLaunch(exec, st)) != cudaSuccess)
        return fail(DEMAG_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    p->launches += kernels;
    return DEMAG_OK;
}

demag_status run_job(demag_plan *p, const FieldJob &job, void *stream)
{
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (!p->setup_done) return fail(DEMAG_ERR_NOT_SETUP, "demag_tensor_setup() has not run on this plan");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    demag_status s;
    const size_t bytes = 3 * (size_t)ncell(p) * elem_size(p);
    if ((s = check_dev_ptr(p, job.in, "input field")) != DEMAG_OK) return s;
    if (job.out) {
        if ((s = check_dev_ptr(p, job.out, "output field")) != DEMAG_OK) return s;
        if (overlap(job.in, job.out, bytes))
            return fail(DEMAG_ERR_INVALID_ARG, "output overlaps input (in-place is not supported)");
    }
    if (job.wcell) {
        if ((s = check_dev_ptr(p, job.wcell, "cell weight")) != DEMAG_OK) return s;
        if (job.out && overlap2(job.wcell, bytes / 3, job.out, bytes))
            return fail(DEMAG_ERR_INVALID_ARG, "output overlaps the cell weight");
    }
    if (job.gdev && (s = check_scalar_ptr(job.gdev, "gradient scale")) != DEMAG_OK) return s;
    if (job.E_dev && (s = check_scalar_ptr(job.E_dev, "E_dev")) != DEMAG_OK) return s;
    if (p->method == DEMAG_METHOD_SP) {
        if (job.wcell || job.gdev || job.wscalar != 1.0 || job.oscale != 1.0)
            return fail(DEMAG_ERR_UNSUPPORTED, "scalar-potential plans take plain fields (no weights or scales)");
        if (job.phi) {
            if ((s = check_dev_ptr(p, job.phi, "phi")) != DEMAG_OK) return s;
            const size_t pb = (size_t)(p->nx + 1) * (p->ny + 1) * (p->nz + 1) * elem_size(p);
            if (overlap2(job.phi, pb, job.in, bytes) || (job.out && overlap2(job.phi, pb, job.out, bytes)))
                return fail(DEMAG_ERR_INVALID_ARG, "phi overlaps the input or the output");
        }
        if (!job.out && !job.E_dev && !job.phi)
            return fail(DEMAG_ERR_INVALID_ARG, "nothing to compute (no output, no energy)");
    } else if (!job.out && !job.E_dev) {
        return fail(DEMAG_ERR_INVALID_ARG, "nothing to compute (no output, no energy)");
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (p->use_graphs && p->graphs && !p->timing) return run_graph(p, job, st);
    return run_direct(p, job, st);
}

// ----- autotuner cache: one line per tuned geometry, "key zvariant yvariant ms"
std::string tune_path()
{
    if (const char *e = getenv("DEMAG_TUNE_CACHE")) return e;
    const char *home = getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/demag_tune.txt";
}

std::string tune_key(const demag_plan *p)
{
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) name = prop.name;
    for (auto &c : name)
        if (c == ' ') c = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "v2|%s|%s|%dx%dx%d|%dx%dx%d%s", name.c_str(), p->prec == DEMAG_F32 ? "f32" : "f64", p->Px,
             p->Py, p->Pz, p->nx, p->ny, p->nz, p->method == DEMAG_METHOD_SP ? "|sp" : "");
    return buf;
}

bool tune_lookup(const std::string &key, int &z, int &y, int &x, double &ms)
{
    FILE *f = fopen(tune_path().c_str(), "r");
    if (!f) return false;
    char line[768], k[512];
    int zz, yy, xx;
    double m;
    bool found = false;
    while (fgets(line, sizeof line, f))
        if (sscanf(line, "%511s %d %d %d %lf", k, &zz, &yy, &xx, &m) == 5 && key == k) {
            z = zz; y = yy; x = xx; ms = m; found = true;  // the last entry wins
        }
    fclose(f);
    return found;
}

void tune_store(const std::string &key, int z, int y, int x, double ms)
{
    const std::string path = tune_path();
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        const std::string dir = path.substr(0, slash);
        mkdir(dir.c_str(), 0755);  // one level is enough for the default location
    }
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;  // a cache that cannot be written is not an error
    fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), z, y, x, ms);
    fclose(f);
}

FieldJob plain_job(const void *M, void *H, double *E_dev)
{
    FieldJob j;
    j.in = M; j.wcell = nullptr; j.wscalar = 1.0;
    j.out = H; j.oscale = 1.0; j.gdev = nullptr;
    j.E_dev = E_dev;
    return j;
}

constexpr int kMaxSPZ = 256;  // the SP z pass is built for padded z lengths <= 512

// SP padding: node-minus-cell offsets take 2n values per axis.
int sp_pad(int n)
{
    int p = 2;
    while (p < 2 * n) p *= 2;
    return p;
}

// smallest even length >= 2n with prime factors 2, 3, 5, 7
int sp_smooth_pad(int n)
{
    int p = 2 * n;
    while (!is_smooth_even(p)) p += 2;
    return p;
}

// Allocates a plan with padded lengths P for the given method (no launches).
demag_status create_plan(int nx, int ny, int nz, double dx, double dy, double dz, demag_prec prec, const int P[3],
                         int method, demag_plan_t *out)
{
    demag_plan *p = new demag_plan;
    memset(p, 0, sizeof(*p));
    p->method = method;
    p->xvariant = 1;  // pipelined x passes where the rows allow them
    p->nx = nx; p->ny = ny; p->nz = nz;
    p->dx = dx; p->dy = dy; p->dz = dz;
    p->prec = prec;
    p->Px = P[0]; p->Py = P[1]; p->Pz = P[2];
    p->Kx = P[0] == 1 ? 1 : P[0] / 2 + 1;
    p->Kxp = P[0] == 1 ? 1 : (p->Kx + 1) / 2 * 2;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(DEMAG_ERR_CUDA, "no CUDA device");
    }
    const size_t cs = prec == DEMAG_F32 ? sizeof(float2) : sizeof(double2);
    const bool sp = method == DEMAG_METHOD_SP;
    // SP: the inverse y pass writes (nz+1)(ny+1) rows of one component into S1
    const size_t s1 = std::max((size_t)3 * nz * ny, sp ? (size_t)(nz + 1) * (ny + 1) : (size_t)0) * p->Kxp * cs;
    const int ntab = sp ? 3 : 6;
    const size_t s2 = (size_t)3 * nz * p->Py * p->Kxp * cs;
    const size_t plane = (size_t)(p->Pz / 2 + 1) * (p->Py / 2 + 1) * p->Kx;
    const int rows = 3 * nz * ny;
    p->npartials = p->Px == 1 ? std::max(1, std::min(4096, (rows + 255) / 256))
                              : (prec == DEMAG_F32 ? Passes<float>::x_blocks(p->Px / 2, rows)
                                                   : Passes<double>::x_blocks(p->Px / 2, rows));
    if (sp) p->npartials = Passes<float>::sp_grad_blocks(nx, ny, nz);
    if (!sp) {  // room for the spectral energy's per-CTA sums
        const int ze = prec == DEMAG_F32 ? Passes<float>::zenergy_blocks(p->Pz, p->Py, p->Kx)
                                         : Passes<double>::zenergy_blocks(p->Pz, p->Py, p->Kx);
        p->npartials = std::max(p->npartials, ze);
    }
    p->spectral_energy = true;
    auto cleanup_fail = [&](cudaError_t e, const char *what) {
        demag_plan_destroy(p);
        return fail(e == cudaErrorMemoryAllocation ? DEMAG_ERR_OOM : DEMAG_ERR_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = dmalloc(&p->S1, s1)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc S1");
    if (p->Py > 1) {
        if ((e = dmalloc(&p->S2, s2)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc S2");
    } else {
        p->S2 = p->S1;
    }
    if (prec == DEMAG_F32) {
        if ((e = dmalloc(&p->nhat32, ntab * plane * sizeof(float))) != cudaSuccess) return cleanup_fail(e, "cudaMalloc tensor");
    } else {
        if ((e = dmalloc(&p->nhat64, ntab * plane * sizeof(double))) != cudaSuccess) return cleanup_fail(e, "cudaMalloc tensor");
    }
    if ((e = dmalloc(&p->partials, sizeof(double) * (p->npartials + demag::kFinalizeScratch))) != cudaSuccess)
        return cleanup_fail(e, "cudaMalloc partials");
    if ((e = cudaMemset(p->partials, 0, sizeof(double) * (p->npartials + demag::kFinalizeScratch))) != cudaSuccess)
        return cleanup_fail(e, "clear partials");
    if ((e = dmalloc(&p->e_dev, sizeof(double))) != cudaSuccess) return cleanup_fail(e, "cudaMalloc energy");
    for (int a = 0; a < 3; ++a) {
        const auto t64 = twiddles<double2>(P[a]);
        if ((e = dmalloc(&p->tw64[a], sizeof(double2) * P[a])) != cudaSuccess) return cleanup_fail(e, "cudaMalloc twiddles");
        if ((e = cudaMemcpy(p->tw64[a], t64.data(), sizeof(double2) * P[a], cudaMemcpyHostToDevice)) != cudaSuccess)
            return cleanup_fail(e, "twiddle upload");
        if (prec == DEMAG_F32) {
            const auto t32 = twiddles<float2>(P[a]);
            if ((e = dmalloc(&p->tw32[a], sizeof(float2) * P[a])) != cudaSuccess) return cleanup_fail(e, "cudaMalloc twiddles");
            if ((e = cudaMemcpy(p->tw32[a], t32.data(), sizeof(float2) * P[a], cudaMemcpyHostToDevice)) != cudaSuccess)
                return cleanup_fail(e, "twiddle upload");
        }
        if (sp) {  // exp(-pi i k / P): the half-cell shift of the node offsets
            const auto h64 = twiddles<double2>(2 * P[a]);
            if ((e = dmalloc(&p->ph64[a], sizeof(double2) * P[a])) != cudaSuccess) return cleanup_fail(e, "cudaMalloc phases");
            if ((e = cudaMemcpy(p->ph64[a], h64.data(), sizeof(double2) * P[a], cudaMemcpyHostToDevice)) != cudaSuccess)
                return cleanup_fail(e, "phase upload");
            if (prec == DEMAG_F32) {
                const auto h32 = twiddles<float2>(2 * P[a]);
                if ((e = dmalloc(&p->ph32[a], sizeof(float2) * P[a])) != cudaSuccess) return cleanup_fail(e, "cudaMalloc phases");
                if ((e = cudaMemcpy(p->ph32[a], h32.data(), sizeof(float2) * P[a], cudaMemcpyHostToDevice)) != cudaSuccess)
                    return cleanup_fail(e, "phase upload");
            }
        }
    }
    if ((e = cudaMemset(p->S1, 0, s1)) != cudaSuccess) return cleanup_fail(e, "cudaMemset");
    if (p->S2 != p->S1 && (e = cudaMemset(p->S2, 0, s2)) != cudaSuccess) return cleanup_fail(e, "cudaMemset");
    p->device_bytes = s1 + (p->S2 != p->S1 ? s2 : 0) + ntab * plane * (prec == DEMAG_F32 ? 4 : 8) +
                      sizeof(double) * (p->npartials + demag::kFinalizeScratch) +
                      (size_t)(P[0] + P[1] + P[2]) * (sizeof(double2) + (prec == DEMAG_F32 ? sizeof(float2) : 0)) *
                          (sp ? 2 : 1);
    *out = p;
    g_err.clear();
    return DEMAG_OK;
}

// ----- tensor-spectrum files (demag_plan_save / demag_plan_load)
struct SpecHeader {
    char magic[8];  // "DMGSPEC" and a zero byte
    int32_t version;
    int32_t method, prec;
    int32_t nx, ny, nz, Px, Py, Pz;
    int32_t ntab;
    double dx, dy, dz;
    double imag_max;
    uint64_t count;     // table values that follow (float for FP32 plans, double for FP64)
    uint64_t checksum;  // FNV-1a 64 of the table bytes
};
constexpr int32_t kSpecVersion = 1;

uint64_t fnv1a64(const unsigned char *b, size_t n)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

size_t table_count(const demag_plan *p)
{
    const size_t plane = (size_t)(p->Pz / 2 + 1) * (p->Py / 2 + 1) * p->Kx;
    return (size_t)(p->method == DEMAG_METHOD_SP ? 3 : 6) * plane;
}

// The tile-ordered copy of the FP32 tensor spectrum read by the persistent
// TMA z pass (z variant 6), built from nhat32 on the plan's stream; plans whose
// z length that kernel does not support keep none.
cudaError_t build_ntile(demag_plan *p, cudaStream_t st)
{
    if (p->prec != DEMAG_F32 || p->method != DEMAG_METHOD_DM || !p->nhat32) return cudaSuccess;
    const size_t n = Passes<float>::tile_tensor_elems(p->Pz, p->Py, p->Kx);
    if (n == 0) return cudaSuccess;
    if (!p->ntile) {
        cudaError_t e = dmalloc(&p->ntile, n * sizeof(float));
        if (e != cudaSuccess) {
            p->ntile = nullptr;
            return e;
        }
        p->ntile_bytes = n * sizeof(float);
        p->device_bytes += p->ntile_bytes;
    }
    return Passes<float>::tile_tensor(p->Pz, p->nhat32, p->ntile, p->Py, p->Kx, st);
}

// A plan that is only timed (padding autotuner): its tensor spectrum is
// zeroed instead of set up. The field passes do the same work whatever the
// spectrum holds, so the timing is that of a set-up plan, without the FP64
// tensor evaluation. The plan is destroyed right after.
demag_status zero_spectrum_for_timing(demag_plan *p, cudaStream_t st)
{
    const size_t plane = (size_t)(p->Pz / 2 + 1) * (p->Py / 2 + 1) * p->Kx;
    cudaError_t e = p->nhat32 ? cudaMemsetAsync(p->nhat32, 0, 6 * plane * sizeof(float), st)
                              : cudaMemsetAsync(p->nhat64, 0, 6 * plane * sizeof(double), st);
    if (e == cudaSuccess) e = build_ntile(p, st);
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? DEMAG_ERR_OOM : DEMAG_ERR_CUDA,
                    std::string("timing plan: ") + cudaGetErrorString(e));
    p->setup_done = true;
    return DEMAG_OK;
}

}  // namespace

void demag::set_last_error(const std::string &msg) { g_err = msg; }

extern "C" {

const char *demag_last_error(demag_plan_t plan) { return plan ? plan->last_err : g_err.c_str(); }

const char *demag_status_string(demag_status s)
{
    switch (s) {
    case DEMAG_OK: return "DEMAG_OK";
    case DEMAG_ERR_INVALID_ARG: return "DEMAG_ERR_INVALID_ARG";
    case DEMAG_ERR_NOT_SETUP: return "DEMAG_ERR_NOT_SETUP";
    case DEMAG_ERR_OOM: return "DEMAG_ERR_OOM";
    case DEMAG_ERR_CUDA: return "DEMAG_ERR_CUDA";
    case DEMAG_ERR_TIMEOUT: return "DEMAG_ERR_TIMEOUT";
    case DEMAG_ERR_UNSUPPORTED: return "DEMAG_ERR_UNSUPPORTED";
    case DEMAG_ERR_GUARD: return "DEMAG_ERR_GUARD";
    }
    return "DEMAG_ERR_UNKNOWN";
}

void demag_plan_destroy(demag_plan_t p)
{
    if (!p) return;
    DeviceGuard g(p->device);
    graphs_free(p);
    if (p->S2 && p->S2 != p->S1) dfree(p->S2);
    dfree(p->S1);
    dfree(p->nhat32);
    dfree(p->nhat64);
    dfree(p->ntile);
    for (int a = 0; a < 3; ++a) {
        dfree(p->tw64[a]); dfree(p->tw32[a]);
        dfree(p->ph64[a]); dfree(p->ph32[a]);
    }
    dfree(p->partials);
    dfree(p->e_dev);
    dfree(p->dM);
    dfree(p->dH);
    if (p->async_ready) {
        cudaStreamSynchronize(p->s_in);
        cudaStreamSynchronize(p->s_out);
        for (int k = 0; k < demag_plan::kAsyncSlots; ++k) {
            dfree(p->aM[k]);
            dfree(p->aH[k]);
            dfree(p->aE[k]);
            cudaEventDestroy(p->ev_in[k]);
            cudaEventDestroy(p->ev_done[k]);
            cudaEventDestroy(p->ev_out[k]);
        }
        cudaStreamDestroy(p->s_in);
        cudaStreamDestroy(p->s_out);
    }
    if (p->ring) {
        TimingRing *R = ring_of(p);
        for (int s = 0; s < kRing; ++s)
            for (int i = 0; i < kEvPerCall; ++i) cudaEventDestroy(R->ev[s][i]);
        delete R;
    }
    delete p;
}

demag_status demag_padded_lengths(int nx, int ny, int nz, const demag_options *opt, int *P)
{
    if (!P) return fail(DEMAG_ERR_INVALID_ARG, "P is NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(DEMAG_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (nx > kMaxN || ny > kMaxN || nz > kMaxN)
        return fail(DEMAG_ERR_UNSUPPORTED, "grid sizes above 512 per axis are not built");
    const int n[3] = {nx, ny, nz};
    int Q[3];
    demag_status s = pad_lengths(n, opt, Q);
    if (s != DEMAG_OK) return s;
    for (int a = 0; a < 3; ++a) P[a] = Q[a];
    return DEMAG_OK;
}

demag_status demag_plan_create_ex(int nx, int ny, int nz, double dx, double dy, double dz, demag_prec prec,
                                  const demag_options *opt, demag_plan_t *out)
{
    if (!out) return fail(DEMAG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(DEMAG_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz))
        return fail(DEMAG_ERR_INVALID_ARG, "cell edges must be positive and finite");
    if (prec != DEMAG_F32 && prec != DEMAG_F64) return fail(DEMAG_ERR_INVALID_ARG, "unknown precision");
    if (nx > kMaxN || ny > kMaxN || nz > kMaxN)
        return fail(DEMAG_ERR_UNSUPPORTED, "grid sizes above 512 per axis are not built");
    const int n[3] = {nx, ny, nz};
    int P[3];
    if (opt && opt->pad_mode == DEMAG_PAD_TUNED) {
        if (opt->px || opt->py || opt->pz)
            return fail(DEMAG_ERR_INVALID_ARG, "DEMAG_PAD_TUNED takes no explicit padded lengths");
        demag_options t;
        memset(&t, 0, sizeof t);
        demag_status s = demag_tune_padding(nx, ny, nz, dx, dy, dz, prec, 1, &t, nullptr, nullptr, nullptr);
        if (s != DEMAG_OK) return s;
        P[0] = t.px; P[1] = t.py; P[2] = t.pz;
        return create_plan(nx, ny, nz, dx, dy, dz, prec, P, DEMAG_METHOD_DM, out);
    }
    demag_status s = pad_lengths(n, opt, P);
    if (s != DEMAG_OK) return s;
    return create_plan(nx, ny, nz, dx, dy, dz, prec, P, DEMAG_METHOD_DM, out);
}

demag_status demag_plan_create_sp(int nx, int ny, int nz, double dx, double dy, double dz, demag_prec prec,
                                  const demag_options *opt, demag_plan_t *out)
{
    if (!out) return fail(DEMAG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(DEMAG_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz))
        return fail(DEMAG_ERR_INVALID_ARG, "cell edges must be positive and finite");
    if (prec != DEMAG_F32 && prec != DEMAG_F64) return fail(DEMAG_ERR_INVALID_ARG, "unknown precision");
    if (nx > kMaxN || ny > kMaxN || nz > kMaxSPZ)
        return fail(DEMAG_ERR_UNSUPPORTED, "scalar-potential grids are built up to 512 x 512 x 256");
    const int n[3] = {nx, ny, nz};
    if (opt && opt->pad_mode == DEMAG_PAD_TUNED)
        return fail(DEMAG_ERR_UNSUPPORTED, "scalar-potential plans take power-of-two or smooth padding");
    if (opt && opt->pad_mode != DEMAG_PAD_POW2 && opt->pad_mode != DEMAG_PAD_SMOOTH)
        return fail(DEMAG_ERR_INVALID_ARG, "unknown pad_mode");
    const bool smooth = opt && opt->pad_mode == DEMAG_PAD_SMOOTH;
    int P[3];
    for (int a = 0; a < 3; ++a) P[a] = smooth ? sp_smooth_pad(n[a]) : sp_pad(n[a]);
    if (opt) {
        const int req[3] = {opt->px, opt->py, opt->pz};
        for (int a = 0; a < 3; ++a) {
            if (req[a] == 0) continue;
            if (!(is_pow2(req[a]) || is_smooth_even(req[a])) || req[a] < 2 * n[a])
                return fail(DEMAG_ERR_INVALID_ARG,
                            "scalar-potential padded lengths must be >= 2n and powers of two or even products of 2, 3, 5, 7");
            if (req[a] > (a == 2 ? 2 * kMaxSPZ : kMaxP))
                return fail(DEMAG_ERR_UNSUPPORTED, "padded length above what is built");
            P[a] = req[a];
        }
    }
    return create_plan(nx, ny, nz, dx, dy, dz, prec, P, DEMAG_METHOD_SP, out);
}

demag_status demag_plan_create(int nx, int ny, int nz, double dx, double dy, double dz, demag_prec prec,
                               demag_plan_t *out)
{
    return demag_plan_create_ex(nx, ny, nz, dx, dy, dz, prec, nullptr, out);
}

// Kernel setup of the scalar-potential method: the cell kernel S at the
// half-integer node offsets (FP64), per component wrapped onto the padded
// grid, transformed, and reduced to the real table T_j (phase removed).
demag_status sp_setup(demag_plan *p, cudaStream_t st)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz, Px = p->Px, Py = p->Py, Pz = p->Pz, Kx = p->Kx, Kxp = p->Kxp;
    const size_t plane = (size_t)(Pz / 2 + 1) * (Py / 2 + 1) * Kx;
    double *oct = nullptr, *W = nullptr, *t64 = p->nhat64;
    double2 *St = nullptr;
    unsigned long long *imag = nullptr;
    bool own64 = false;
    demag_status rs = DEMAG_OK;
    auto done = [&](demag_status s) {
        dfree(oct); dfree(W); dfree(St); dfree(imag);
        if (own64) dfree(t64);
        return s;
    };
#define SETUP_CUDA(call)                                                                       \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            rs = fail(e_ == cudaErrorMemoryAllocation ? DEMAG_ERR_OOM : DEMAG_ERR_CUDA,        \
                      std::string("SP kernel setup: ") + #call + ": " + cudaGetErrorString(e_)); \
            return done(rs);                                                                   \
        }                                                                                      \
    } while (0)
    SETUP_CUDA(dmalloc(&oct, sizeof(double) * 3 * (size_t)nx * ny * nz));
    SETUP_CUDA(dmalloc(&W, sizeof(double) * (size_t)Px * Py * Pz));
    SETUP_CUDA(dmalloc(&St, sizeof(double2) * (size_t)Pz * Py * Kxp));
    SETUP_CUDA(dmalloc(&imag, sizeof(unsigned long long)));
    SETUP_CUDA(cudaMemsetAsync(imag, 0, sizeof(unsigned long long), st));
    if (!t64) {
        SETUP_CUDA(dmalloc(&t64, sizeof(double) * 3 * plane));
        own64 = true;
    }
    SETUP_CUDA(demag::sp_octant(oct, nx, ny, nz, p->dx, p->dy, p->dz, st));
    demag::XIn<double> xin;
    xin.in = W;
    xin.in_rs = Px;
    xin.wcell = nullptr;
    xin.wscalar = 1.0;
    xin.rows_per_comp = Pz * Py;
    for (int c = 0; c < 3; ++c) {
        SETUP_CUDA(demag::sp_wrap(oct, c, nx, ny, nz, Px, Py, Pz, W, st));
        SETUP_CUDA(Passes<double>::x_fwd(Px / 2, xin, Pz * Py, Px, St, Kxp, p->tw64[0], st));
        SETUP_CUDA(Passes<double>::col(Py, false, St, St, Pz * Kx, Kx, (int64_t)Py * Kxp, Kxp, Py, (int64_t)Py * Kxp,
                                       Kxp, Py, p->tw64[1], 1, st));
        SETUP_CUDA(Passes<double>::col(Pz, false, St, St, Py * Kx, Kx, Kxp, (int64_t)Py * Kxp, Pz, Kxp,
                                       (int64_t)Py * Kxp, Pz, p->tw64[2], 1, st));
        SETUP_CUDA(demag::sp_extract(St, c, Px, Py, Pz, Kxp, t64, p->nhat32, imag, st));
    }
    unsigned long long bits = 0;
    SETUP_CUDA(cudaMemcpyAsync(&bits, imag, sizeof(bits), cudaMemcpyDeviceToHost, st));
    SETUP_CUDA(cudaStreamSynchronize(st));
    memcpy(&p->imag_max, &bits, sizeof(double));
    p->launches += 1 + 3 * 5;
    p->setup_done = true;
    g_err.clear();
    return done(DEMAG_OK);
#undef SETUP_CUDA
}

demag_status demag_tensor_setup(demag_plan_t p, void *stream)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (p->setup_done) return DEMAG_OK;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->method == DEMAG_METHOD_SP) return sp_setup(p, st);
    const int nx = p->nx, ny = p->ny, nz = p->nz, Px = p->Px, Py = p->Py, Pz = p->Pz, Kx = p->Kx, Kxp = p->Kxp;
    const size_t plane = (size_t)(Pz / 2 + 1) * (Py / 2 + 1) * Kx;
    double *oct = nullptr, *W = nullptr, *nh64 = p->nhat64;
    double2 *St = nullptr;
    unsigned long long *imag = nullptr;
    bool own64 = false;
    demag_status rs = DEMAG_OK;
    auto done = [&](demag_status s) {
        dfree(oct); dfree(W); dfree(St); dfree(imag);
        if (own64) dfree(nh64);
        return s;
    };
#define SETUP_CUDA(call)                                                                       \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            rs = fail(e_ == cudaErrorMemoryAllocation ? DEMAG_ERR_OOM : DEMAG_ERR_CUDA,        \
                      std::string("tensor setup: ") + #call + ": " + cudaGetErrorString(e_));  \
            return done(rs);                                                                   \
        }                                                                                      \
    } while (0)
    SETUP_CUDA(dmalloc(&oct, sizeof(double) * 6 * (size_t)nx * ny * nz));
    SETUP_CUDA(dmalloc(&W, sizeof(double) * (size_t)Px * Py * Pz));
    SETUP_CUDA(dmalloc(&St, sizeof(double2) * (size_t)Pz * Py * Kxp));
    SETUP_CUDA(dmalloc(&imag, sizeof(unsigned long long)));
    SETUP_CUDA(cudaMemsetAsync(imag, 0, sizeof(unsigned long long), st));
    if (!nh64) {
        SETUP_CUDA(dmalloc(&nh64, sizeof(double) * 6 * plane));
        own64 = true;
    }
    SETUP_CUDA(demag::tensor_octant(oct, nx, ny, nz, p->dx, p->dy, p->dz, st));
    demag::XIn<double> xin;
    xin.in = W;
    xin.in_rs = Px;
    xin.wcell = nullptr;
    xin.wscalar = 1.0;
    xin.rows_per_comp = Pz * Py;
    for (int c = 0; c < 6; ++c) {
        SETUP_CUDA(demag::tensor_wrap(oct, c, nx, ny, nz, Px, Py, Pz, W, st));
        if (Px == 1) SETUP_CUDA(Passes<double>::x1_fwd(xin, (int64_t)Pz * Py, St, st));
        else SETUP_CUDA(Passes<double>::x_fwd(Px / 2, xin, Pz * Py, Px, St, Kxp, p->tw64[0], st));
        if (Py > 1)
            SETUP_CUDA(Passes<double>::col(Py, false, St, St, Pz * Kx, Kx, (int64_t)Py * Kxp, Kxp, Py,
                                           (int64_t)Py * Kxp, Kxp, Py, p->tw64[1], 1, st));
        if (Pz > 1)
            SETUP_CUDA(Passes<double>::col(Pz, false, St, St, Py * Kx, Kx, Kxp, (int64_t)Py * Kxp, Pz, Kxp,
                                           (int64_t)Py * Kxp, Pz, p->tw64[2], 1, st));
        SETUP_CUDA(demag::tensor_extract(St, c, Px, Py, Pz, Kxp, nh64, p->nhat32, imag, st));
    }
    SETUP_CUDA(build_ntile(p, st));
    unsigned long long bits = 0;
    SETUP_CUDA(cudaMemcpyAsync(&bits, imag, sizeof(bits), cudaMemcpyDeviceToHost, st));
    SETUP_CUDA(cudaStreamSynchronize(st));
    memcpy(&p->imag_max, &bits, sizeof(double));
    p->launches += 1 + 6 * (2 + (Py > 1) + (Pz > 1));
    p->setup_done = true;
    g_err.clear();
    return done(DEMAG_OK);
#undef SETUP_CUDA
}

demag_status demag_sp_potential(demag_plan_t p, const void *M, void *phi, void *stream)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (p->method != DEMAG_METHOD_SP) return fail(DEMAG_ERR_INVALID_ARG, "not a scalar-potential plan");
    if (!phi) return fail(DEMAG_ERR_INVALID_ARG, "phi is NULL");
    FieldJob j = plain_job(M, nullptr, nullptr);
    j.phi = phi;
    return run_job(p, j, stream);
}

demag_status demag_field(demag_plan_t p, const void *M, void *H, void *stream)
{
    PlanScope scope_(p);
    if (!H) return fail(DEMAG_ERR_INVALID_ARG, "H is NULL");
    return run_job(p, plain_job(M, H, nullptr), stream);
}

demag_status demag_field_adjoint(demag_plan_t p, const void *G, void *out, void *stream)
{
    PlanScope scope_(p);
    // N_ij = N_ji and N(-r) = N(r): the operator equals its adjoint.
    if (!out) return fail(DEMAG_ERR_INVALID_ARG, "out is NULL");
    if (p && p->method == DEMAG_METHOD_SP)
        return fail(DEMAG_ERR_UNSUPPORTED, "the scalar-potential operator is not self-adjoint; its adjoint is not built");
    return run_job(p, plain_job(G, out, nullptr), stream);
}

demag_status demag_field_energy(demag_plan_t p, const void *M, void *H, double *E_dev, void *stream)
{
    PlanScope scope_(p);
    if (!E_dev) return fail(DEMAG_ERR_INVALID_ARG, "E_dev is NULL");
    if (!H) return fail(DEMAG_ERR_INVALID_ARG, "H is NULL");
    return run_job(p, plain_job(M, H, E_dev), stream);
}

demag_status demag_energy(demag_plan_t p, const void *M, double *E_out, void *stream)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (!E_out) return fail(DEMAG_ERR_INVALID_ARG, "E_out is NULL");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    demag_status s = run_job(p, plain_job(M, nullptr, p->e_dev), stream);
    if (s != DEMAG_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    DEMAG_CUDA(cudaMemcpyAsync(E_out, p->e_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    DEMAG_CUDA(cudaStreamSynchronize(st));
    return DEMAG_OK;
}

demag_status demag_field_host(demag_plan_t p, const void *M_host, void *H_host, void *stream)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (!M_host || !H_host) return fail(DEMAG_ERR_INVALID_ARG, "host buffers must not be NULL");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    const size_t bytes = 3 * (size_t)ncell(p) * elem_size(p);
    if (!p->dM) DEMAG_CUDA(dmalloc(&p->dM, bytes));
    if (!p->dH) DEMAG_CUDA(dmalloc(&p->dH, bytes));
    cudaStream_t st = (cudaStream_t)stream;
    DEMAG_CUDA(cudaMemcpyAsync(p->dM, M_host, bytes, cudaMemcpyHostToDevice, st));
    demag_status s = run_job(p, plain_job(p->dM, p->dH, nullptr), stream);
    if (s != DEMAG_OK) return s;
    DEMAG_CUDA(cudaMemcpyAsync(H_host, p->dH, bytes, cudaMemcpyDeviceToHost, st));
    DEMAG_CUDA(cudaStreamSynchronize(st));
    return DEMAG_OK;
}

demag_status demag_energy_grad(demag_plan_t p, const void *m, const void *w, double Ms, double *E_dev,
                               void *grad, const double *gscale_dev, void *stream)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (p->method == DEMAG_METHOD_SP)
        return fail(DEMAG_ERR_UNSUPPORTED, "energy gradients need the adjoint, which scalar-potential plans do not build");
    if (!isfinite(Ms)) return fail(DEMAG_ERR_INVALID_ARG, "Ms must be finite");
    FieldJob j;
    j.in = m; j.wcell = w; j.wscalar = Ms;
    j.out = grad;
    // dE/dm = Ms w dE/dM = -mu0 V Ms w H (the operator is self-adjoint)
    j.oscale = -kMu0 * p->dx * p->dy * p->dz * Ms;
    j.gdev = gscale_dev;
    j.E_dev = E_dev;
    return run_job(p, j, stream);
}

demag_status demag_field_host_async(demag_plan_t p, const void *M_host, void *H_host, void *stream)
{
    PlanScope scope_(p);
    return demag_field_energy_host_async(p, M_host, H_host, nullptr, stream);
}

demag_status demag_field_energy_host_async(demag_plan_t p, const void *M_host, void *H_host, double *E_host,
                                           void *stream)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (!M_host || !H_host) return fail(DEMAG_ERR_INVALID_ARG, "host buffers must not be NULL");
    if (!p->setup_done) return fail(DEMAG_ERR_NOT_SETUP, "demag_tensor_setup() has not run on this plan");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    const size_t bytes = 3 * (size_t)ncell(p) * elem_size(p);
    if (!p->async_ready) {
        for (int k = 0; k < demag_plan::kAsyncSlots; ++k) {
            DEMAG_CUDA(dmalloc(&p->aM[k], bytes));
            DEMAG_CUDA(dmalloc(&p->aH[k], bytes));
            DEMAG_CUDA(dmalloc(&p->aE[k], sizeof(double)));
            DEMAG_CUDA(cudaEventCreateWithFlags(&p->ev_in[k], cudaEventDisableTiming));
            DEMAG_CUDA(cudaEventCreateWithFlags(&p->ev_done[k], cudaEventDisableTiming));
            DEMAG_CUDA(cudaEventCreateWithFlags(&p->ev_out[k], cudaEventDisableTiming));
            p->out_recorded[k] = false;
        }
        DEMAG_CUDA(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
        DEMAG_CUDA(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
        p->slot = 0;
        p->async_ready = true;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int k = p->slot;
    p->slot = (p->slot + 1) % demag_plan::kAsyncSlots;
    // the slot's previous download must be done before its buffers are reused
    if (p->out_recorded[k]) DEMAG_CUDA(cudaStreamWaitEvent(p->s_in, p->ev_out[k], 0));
    DEMAG_CUDA(cudaMemcpyAsync(p->aM[k], M_host, bytes, cudaMemcpyHostToDevice, p->s_in));
    DEMAG_CUDA(cudaEventRecord(p->ev_in[k], p->s_in));
    DEMAG_CUDA(cudaStreamWaitEvent(st, p->ev_in[k], 0));
    demag_status s = run_job(p, plain_job(p->aM[k], p->aH[k], E_host ? p->aE[k] : nullptr), stream);
    if (s != DEMAG_OK) return s;
    DEMAG_CUDA(cudaEventRecord(p->ev_done[k], st));
    DEMAG_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_done[k], 0));
    DEMAG_CUDA(cudaMemcpyAsync(H_host, p->aH[k], bytes, cudaMemcpyDeviceToHost, p->s_out));
    if (E_host) DEMAG_CUDA(cudaMemcpyAsync(E_host, p->aE[k], sizeof(double), cudaMemcpyDeviceToHost, p->s_out));
    DEMAG_CUDA(cudaEventRecord(p->ev_out[k], p->s_out));
    p->out_recorded[k] = true;
    return DEMAG_OK;
}

demag_status demag_host_wait(demag_plan_t p)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (!p->async_ready) return DEMAG_OK;
    DeviceGuard g(p->device);
    DEMAG_CUDA(cudaStreamSynchronize(p->s_in));
    DEMAG_CUDA(cudaStreamSynchronize(p->s_out));
    return DEMAG_OK;
}

void demag_debug_fail_alloc(long n) { g_fail_alloc.store(n > 0 ? n : 0); }

demag_status demag_plan_save(demag_plan_t p, const char *path)
{
    PlanScope scope_(p);
    if (!p || !path) return fail(DEMAG_ERR_INVALID_ARG, "NULL argument");
    if (!p->setup_done) return fail(DEMAG_ERR_NOT_SETUP, "demag_tensor_setup() has not run on this plan");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    SpecHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "DMGSPEC", 8);
    h.version = kSpecVersion;
    h.method = p->method;
    h.prec = p->prec;
    h.nx = p->nx; h.ny = p->ny; h.nz = p->nz;
    h.Px = p->Px; h.Py = p->Py; h.Pz = p->Pz;
    h.ntab = p->method == DEMAG_METHOD_SP ? 3 : 6;
    h.dx = p->dx; h.dy = p->dy; h.dz = p->dz;
    h.imag_max = p->imag_max;
    h.count = table_count(p);
    const size_t bytes = h.count * (p->prec == DEMAG_F32 ? sizeof(float) : sizeof(double));
    std::vector<unsigned char> buf(bytes);
    const void *src = p->prec == DEMAG_F32 ? (const void *)p->nhat32 : (const void *)p->nhat64;
    cudaError_t e = cudaMemcpy(buf.data(), src, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("spectrum download: ") + cudaGetErrorString(e));
    h.checksum = fnv1a64(buf.data(), bytes);
    FILE *f = fopen(path, "wb");
    if (!f) return fail(DEMAG_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
    const bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(buf.data(), 1, bytes, f) == bytes;
    if (fclose(f) != 0 || !ok) return fail(DEMAG_ERR_INVALID_ARG, std::string("cannot write ") + path);
    return DEMAG_OK;
}

demag_status demag_plan_load(const char *path, demag_plan_t *out)
{
    if (!out || !path) return fail(DEMAG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(DEMAG_ERR_INVALID_ARG, std::string("cannot open ") + path);
    SpecHeader h;
    std::vector<unsigned char> buf;
    std::string why;
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, "DMGSPEC", 8) != 0) {
        why = "not a tensor-spectrum file";
    } else if (h.version != kSpecVersion) {
        why = "unknown file version";
    } else if ((h.method != DEMAG_METHOD_DM && h.method != DEMAG_METHOD_SP) || (h.prec != DEMAG_F32 && h.prec != DEMAG_F64) ||
               h.ntab != (h.method == DEMAG_METHOD_SP ? 3 : 6)) {
        why = "bad method, precision or table count";
    } else {
        const int n[3] = {h.nx, h.ny, h.nz}, P[3] = {h.Px, h.Py, h.Pz};
        const double d[3] = {h.dx, h.dy, h.dz};
        for (int a = 0; a < 3 && why.empty(); ++a) {
            const bool sp = h.method == DEMAG_METHOD_SP;
            const int nmax = sp && a == 2 ? kMaxSPZ : kMaxN;
            if (n[a] < 1 || n[a] > nmax || !(d[a] > 0) || !isfinite(d[a])) why = "bad grid sizes or cell edges";
            else if (n[a] == 1 && P[a] == 1) continue;
            else if (P[a] > (sp && a == 2 ? 2 * kMaxSPZ : kMaxP) || P[a] < (sp ? 2 * n[a] : 2 * n[a] - 1) ||
                     !(is_pow2(P[a]) || is_smooth_even(P[a])))
                why = "bad padded lengths";
        }
        if (why.empty()) {
            const int Kx = h.Px == 1 ? 1 : h.Px / 2 + 1;
            const uint64_t want = (uint64_t)h.ntab * (uint64_t)(h.Pz / 2 + 1) * (uint64_t)(h.Py / 2 + 1) * (uint64_t)Kx;
            const size_t bytes = (size_t)want * (h.prec == DEMAG_F32 ? sizeof(float) : sizeof(double));
            if (h.count != want) {
                why = "table size does not match the sizes";
            } else {
                buf.resize(bytes);
                if (fread(buf.data(), 1, bytes, f) != bytes || fgetc(f) != EOF) why = "truncated or oversized file";
                else if (fnv1a64(buf.data(), bytes) != h.checksum) why = "checksum mismatch";
            }
        }
    }
    fclose(f);
    if (!why.empty()) return fail(DEMAG_ERR_INVALID_ARG, std::string(path) + ": " + why);
    const int P[3] = {h.Px, h.Py, h.Pz};
    demag_plan_t p = nullptr;
    demag_status s = create_plan(h.nx, h.ny, h.nz, h.dx, h.dy, h.dz, (demag_prec)h.prec, P, h.method, &p);
    if (s != DEMAG_OK) return s;
    void *dst = h.prec == DEMAG_F32 ? (void *)p->nhat32 : (void *)p->nhat64;
    cudaError_t e = cudaMemcpy(dst, buf.data(), buf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        demag_plan_destroy(p);
        return fail(DEMAG_ERR_CUDA, std::string("spectrum upload: ") + cudaGetErrorString(e));
    }
    if ((e = build_ntile(p, nullptr)) == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        demag_plan_destroy(p);
        return fail(e == cudaErrorMemoryAllocation ? DEMAG_ERR_OOM : DEMAG_ERR_CUDA,
                    std::string("tile-ordered tensor: ") + cudaGetErrorString(e));
    }
    p->imag_max = h.imag_max;
    p->setup_done = true;
    *out = p;
    return DEMAG_OK;
}

demag_status demag_plan_info(demag_plan_t p, demag_info *info)
{
    PlanScope scope_(p);
    if (!p || !info) return fail(DEMAG_ERR_INVALID_ARG, "NULL argument");
    info->nx = p->nx; info->ny = p->ny; info->nz = p->nz;
    info->px = p->Px; info->py = p->Py; info->pz = p->Pz;
    info->kx = p->Kx;
    info->prec = p->prec;
    info->device_bytes = p->device_bytes;
    info->launches_per_field = p->method == DEMAG_METHOD_SP ? 6 : 3 + 2 * (p->Py > 1);
    info->tensor_imag_max = p->imag_max;
    info->method = p->method;
    info->dx = p->dx; info->dy = p->dy; info->dz = p->dz;
    info->energy_in_z = energy_in_z(p) ? 1 : 0;
    return DEMAG_OK;
}

demag_status demag_set_graphs(demag_plan_t p, int enable)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    DeviceGuard g(p->device);
    if (enable) {
        if (!p->graphs) p->graphs = new GraphCache;
    } else {
        graphs_free(p);
    }
    p->use_graphs = enable != 0;
    return DEMAG_OK;
}

demag_status demag_set_timing(demag_plan_t p, int enable)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    DeviceGuard g(p->device);
    if (enable && !p->ring) {
        TimingRing *R = new TimingRing;
        memset(R, 0, sizeof(*R));
        for (int s = 0; s < kRing; ++s)
            for (int i = 0; i < kEvPerCall; ++i) DEMAG_CUDA(cudaEventCreate(&R->ev[s][i]));
        p->ring = R;
    }
    p->timing = enable != 0;
    for (int i = 0; i < 8; ++i) { p->pass_ms[i] = 0; p->pass_n[i] = 0; }
    if (p->ring) {
        TimingRing *R = ring_of(p);
        for (int s = 0; s < kRing; ++s) R->used[s] = 0;
        R->next = 0;
    }
    return DEMAG_OK;
}

demag_status demag_get_timing(demag_plan_t p, double *ms, long *counts, int n)
{
    PlanScope scope_(p);
    if (!p || !ms || !counts || n < 0 || n > 8) return fail(DEMAG_ERR_INVALID_ARG, "bad arguments");
    DeviceGuard g(p->device);
    if (p->ring) {
        TimingRing *R = ring_of(p);
        for (int s = 0; s < kRing; ++s)
            if (R->used[s]) ring_collect_slot(p, R, s);
    }
    for (int i = 0; i < n; ++i) { ms[i] = p->pass_ms[i]; counts[i] = p->pass_n[i]; }
    return DEMAG_OK;
}

long demag_launch_count(demag_plan_t p) { return p ? p->launches : 0; }

demag_status demag_autotune(demag_plan_t p, int use_cache, double *best_ms, void *stream)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (!p->setup_done) return fail(DEMAG_ERR_NOT_SETUP, "demag_tensor_setup() has not run on this plan");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    const std::string key = tune_key(p);
    int zc = 0, yc = 0, xc = 1;
    double ms_cached = 0;
    if (use_cache && tune_lookup(key, zc, yc, xc, ms_cached)) {
        p->zvariant = zc;
        p->yvariant = yc;
        p->xvariant = xc;
        p->tuned = true;
        if (best_ms) *best_ms = ms_cached;
        return DEMAG_OK;
    }
    // candidates: z-pass tile width where the two-stage z kernel runs, y-pass
    // radix order where the two radices differ
    std::vector<int> zs = {0}, ys = {0}, xs = {0, 1, 2};
    const bool dm = p->method == DEMAG_METHOD_DM;  // the SP z pass has one form
    // (lengths that are not powers of two have the one mixed-radix form)
    const bool z2 = is_pow2(p->Pz);
    if (!is_pow2(p->Px)) xs = {0};
    if (z2 && dm && p->Pz >= 32 && p->Pz <= 512) zs.push_back(1);
    if (z2 && dm && p->Pz == 512) zs.push_back(2);  // 256 threads: the product stage uses every thread
    if (z2 && dm && p->Pz >= 64 && p->Pz <= 512) zs.push_back(3);  // persistent, pipelined
    if (z2 && dm && p->Pz >= 32 && p->Pz <= 512) zs.push_back(4);   // half tile, two CTAs per SM
    if (z2 && dm && p->Pz >= 32 && p->Pz <= 128) zs.push_back(8);   // 8-point second stage, two CTAs per SM
    if (z2 && p->Pz >= 32 && p->Pz <= 256) zs.push_back(5);   // persistent, TMA-staged input (DM and SP)
    if (dm && p->ntile) {  // persistent, TMA input and tensor tiles, FP32: 8 or 4 columns per tile
        zs.push_back(6);
        zs.push_back(7);
    }
    if (p->Py == 32 || p->Py == 128 || p->Py == 512) ys.push_back(1);
    if (p->Py == 512 || p->Py == 1024) ys.push_back(2);  // three-stage, more CTAs per SM
    if (p->Py == 512 || p->Py == 1024) ys.push_back(3);  // forward pass by the TMA pipeline
    const size_t bytes = 3 * (size_t)ncell(p) * elem_size(p);
    void *M = nullptr, *H = nullptr;
    DEMAG_CUDA(dmalloc(&M, bytes));
    if (dmalloc(&H, bytes) != cudaSuccess) {
        dfree(M);
        return fail(DEMAG_ERR_OOM, "autotune buffers");
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(M, 0, bytes, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool timing = p->timing, graphs = p->use_graphs;
    p->timing = false;
    p->use_graphs = false;  // variants are timed by direct launches
    double best = 1e30;
    int bz = 0, by = 0, bx = 1;
    demag_status rs = DEMAG_OK;
    for (int x : xs)
    for (int z : zs)
        for (int y : ys) {
            p->zvariant = z;
            p->yvariant = y;
            p->xvariant = x;
            // field + energy: the x-inverse forms differ most in the energy's epilogue
            for (int w = 0; w < 2 && rs == DEMAG_OK; ++w) rs = run_job(p, plain_job(M, H, p->e_dev), stream);
            cudaEventRecord(e0, st);
            for (int r = 0; r < 5 && rs == DEMAG_OK; ++r) rs = run_job(p, plain_job(M, H, p->e_dev), stream);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rs == DEMAG_OK && ms / 5 < best) { best = ms / 5; bz = z; by = y; bx = x; }
        }
    p->timing = timing;
    p->use_graphs = graphs;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(M);
    dfree(H);
    if (rs != DEMAG_OK) return rs;
    p->zvariant = bz;
    p->yvariant = by;
    p->xvariant = bx;
    p->tuned = true;
    if (best_ms) *best_ms = best;
    if (use_cache) tune_store(key, bz, by, bx, best);
    return DEMAG_OK;
}

demag_status demag_tune_padding(int nx, int ny, int nz, double dx, double dy, double dz, demag_prec prec,
                                int use_cache, demag_options *best, double *ms_best, double *ms_pow2, void *stream)
{
    if (!best) return fail(DEMAG_ERR_INVALID_ARG, "best is NULL");
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1) return fail(DEMAG_ERR_INVALID_ARG, "grid sizes must be >= 1");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(DEMAG_ERR_CUDA, "no CUDA device");
    }
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (auto &c : name)
        if (c == ' ') c = '_';
    char key[256];
    snprintf(key, sizeof key, "pad1|%s|%s|%dx%dx%d", name.c_str(), prec == DEMAG_F32 ? "f32" : "f64", nx, ny, nz);
    const std::string kbest = std::string(key) + "|best", kpow2 = std::string(key) + "|pow2";
    int c0, c1, c2, q0, q1, q2;
    double mb = 0, mp = 0;
    if (use_cache && tune_lookup(kbest, c0, c1, c2, mb) && tune_lookup(kpow2, q0, q1, q2, mp)) {
        memset(best, 0, sizeof *best);
        best->px = c0; best->py = c1; best->pz = c2;
        if (ms_best) *ms_best = mb;
        if (ms_pow2) *ms_pow2 = mp;
        return DEMAG_OK;
    }
    // candidate lengths per axis: the power of two first
    std::vector<int> cand[3];
    for (int a = 0; a < 3; ++a) {
        cand[a].push_back(default_pad(n[a]));
        if (smooth_pad(n[a]) != cand[a][0]) cand[a].push_back(smooth_pad(n[a]));
    }
    double tbest = 1e30, tpow2 = -1;
    int bP[3] = {0, 0, 0};
    for (int i : cand[0])
        for (int j : cand[1])
            for (int k : cand[2]) {
                demag_options o;
                memset(&o, 0, sizeof o);
                o.px = i; o.py = j; o.pz = k;
                demag_plan_t p = nullptr;
                demag_status s = demag_plan_create_ex(nx, ny, nz, dx, dy, dz, prec, &o, &p);
                double ms = 0;
                if (s == DEMAG_OK) s = zero_spectrum_for_timing(p, (cudaStream_t)stream);
                if (s == DEMAG_OK) s = demag_autotune(p, use_cache, &ms, stream);
                demag_plan_destroy(p);
                if (s != DEMAG_OK) return s;
                if (i == cand[0][0] && j == cand[1][0] && k == cand[2][0]) tpow2 = ms;
                if (ms < tbest) {
                    tbest = ms;
                    bP[0] = i; bP[1] = j; bP[2] = k;
                }
            }
    memset(best, 0, sizeof *best);
    best->px = bP[0]; best->py = bP[1]; best->pz = bP[2];
    if (ms_best) *ms_best = tbest;
    if (ms_pow2) *ms_pow2 = tpow2;
    if (use_cache) {
        tune_store(kbest, bP[0], bP[1], bP[2], tbest);
        tune_store(kpow2, cand[0][0], cand[1][0], cand[2][0], tpow2);
    }
    g_err.clear();
    return DEMAG_OK;
}

demag_status demag_set_spectral_energy(demag_plan_t p, int enable)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    p->spectral_energy = enable != 0;
    return DEMAG_OK;
}

demag_status demag_get_variants(demag_plan_t p, int *z, int *y)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    if (z) *z = p->zvariant;
    if (y) *y = p->yvariant;
    return DEMAG_OK;
}

demag_status demag_set_variants(demag_plan_t p, int z, int y)
{
    PlanScope scope_(p);
    if (!p || z < 0 || z > 8 || y < 0 || y > 3) return fail(DEMAG_ERR_INVALID_ARG, "bad plan or variant");
    p->zvariant = z;
    p->yvariant = y;
    return DEMAG_OK;
}

demag_status demag_get_x_variant(demag_plan_t p, int *x)
{
    PlanScope scope_(p);
    if (!p || !x) return fail(DEMAG_ERR_INVALID_ARG, "NULL argument");
    *x = p->xvariant;
    return DEMAG_OK;
}

demag_status demag_set_x_variant(demag_plan_t p, int x)
{
    PlanScope scope_(p);
    if (!p || x < 0 || x > 2) return fail(DEMAG_ERR_INVALID_ARG, "bad plan or variant");
    p->xvariant = x;
    return DEMAG_OK;
}

demag_status demag_check_pipeline(demag_plan_t p)
{
    PlanScope scope_(p);
    if (!p) return fail(DEMAG_ERR_INVALID_ARG, "plan is NULL");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(DEMAG_ERR_CUDA, "cannot select the plan's device");
    DEMAG_CUDA(cudaDeviceSynchronize());
    const int e = Passes<float>::pipe_error_take() | Passes<double>::pipe_error_take();
    if (e) return fail(DEMAG_ERR_TIMEOUT, "a pipelined x pass gave up waiting for a bulk copy");
    std::vector<std::pair<void *, GuardBlock>> blocks;
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        blocks.assign(g_guards.begin(), g_guards.end());
    }
    if (blocks.empty()) return DEMAG_OK;
    unsigned int *bad = nullptr;
    DEMAG_CUDA(cudaMalloc(&bad, sizeof(unsigned int) * 2 * blocks.size()));
    DEMAG_CUDA(cudaMemset(bad, 0, sizeof(unsigned int) * 2 * blocks.size()));
    for (size_t q = 0; q < blocks.size(); ++q) {
        const unsigned char *b = static_cast<const unsigned char *>(blocks[q].second.base);
        k_guard_scan<<<8, 256>>>(b, (int)kGuardBytes, bad + 2 * q);
        k_guard_scan<<<8, 256>>>(b + kGuardBytes + blocks[q].second.bytes, (int)kGuardBytes, bad + 2 * q + 1);
    }
    std::vector<unsigned int> h(2 * blocks.size());
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpy(h.data(), bad, sizeof(unsigned int) * h.size(), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    if (ce != cudaSuccess) return fail(DEMAG_ERR_CUDA, std::string("guard scan: ") + cudaGetErrorString(ce));
    for (size_t q = 0; q < blocks.size(); ++q)
        if (h[2 * q] || h[2 * q + 1]) {
            char msg[160];
            snprintf(msg, sizeof msg, "guard zone %s debug allocation #%ld (%zu bytes) overwritten (%u bytes)",
                     h[2 * q] ? "before" : "after", blocks[q].second.serial, blocks[q].second.bytes,
                     h[2 * q] ? h[2 * q] : h[2 * q + 1]);
            return fail(DEMAG_ERR_GUARD, msg);
        }
    return DEMAG_OK;
}

long demag_debug_guard_count(void)
{
    std::lock_guard<std::mutex> lk(g_guard_mu);
    return (long)g_guards.size();
}

demag_status demag_debug_poke_guard(void)
{
    void *base = nullptr;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(g_guard_mu);
        long best = -1;
        for (const auto &kv : g_guards)
            if (kv.second.serial > best) {
                best = kv.second.serial;
                base = kv.second.base;
                bytes = kv.second.bytes;
            }
    }
    if (!base) return fail(DEMAG_ERR_INVALID_ARG, "no debug allocation is live");
    DEMAG_CUDA(cudaMemset(static_cast<unsigned char *>(base) + kGuardBytes + bytes, 0x5A, 1));
    return DEMAG_OK;
}

}  // extern "C"
