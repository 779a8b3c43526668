// Batched stray field of many independent grids (magnetization states) of
// uneven sizes: every state has its own plan (geometry, tensor spectrum,
// spectra), and one call evaluates all of them.
//
// Persistent mode: a single
// kernel launch works through a queue of (pass, state, tile) items in
// pass-major order. An item of pass p waits until all tiles of pass p - 1 of
// its state are done (per-(pass, state) completion counters). Waits are
// bounded by a cycle budget; a wait that runs out sets an error flag and
// every CTA leaves the loop, so the launch always ends. Intermediate spectra
// are read with L1-bypassing loads because other CTAs of the same launch
// wrote them. The counter reset and the launch are captured once in a CUDA
// graph that each call replays.
//
// Pass-batched mode (the default where the persistent tile functions cover
// every state): one launch per pass covers that pass's tiles of every state,
// the six launches are captured once into a CUDA graph and replayed; the
// stream order of the launches replaces the persistent kernel's waits, and
// each launch holds only its own pass's tile functions (fewer registers, more
// CTAs per SM than the single persistent kernel).
//
// Branch mode: each state's five-kernel pipeline is captured on its own
// stream into one CUDA graph (independent branches run concurrently).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "fft2.cuh"
#include "plan.h"

namespace demag {

namespace {

constexpr int kPasses = 6;
constexpr int kThreads = 256;  // FP32 tile functions all use 256 threads
constexpr double kMu0 = 4e-7 * 3.14159265358979323846;

// Tiles and shared memory of each pass for a state, or false if the
// persistent kernel has no tile function for its sizes.
struct PassGeom {
    int tiles[kPasses];
    size_t smem[kPasses];
};

template <int L> constexpr size_t x_smem()
{
    if constexpr (L >= 64) return (size_t)XShape<float, L>::TR * XShape<float, L>::RS * 8;
    else return (size_t)swsize(L * TileShape<float, L>::TC) * 8;
}
template <int L> constexpr int x_rows()
{
    if constexpr (L >= 64) return XShape<float, L>::TR;
    else return TileShape<float, L>::TC;
}

bool x_geom(int L, int &rows_per_tile, size_t &sm)
{
    switch (L) {
    case 16: rows_per_tile = x_rows<16>(); sm = x_smem<16>(); return true;
    case 32: rows_per_tile = x_rows<32>(); sm = x_smem<32>(); return true;
    case 64: rows_per_tile = x_rows<64>(); sm = x_smem<64>(); return true;
    case 128: rows_per_tile = x_rows<128>(); sm = x_smem<128>(); return true;
    case 256: rows_per_tile = x_rows<256>(); sm = x_smem<256>(); return true;
    case 512: rows_per_tile = x_rows<512>(); sm = x_smem<512>(); return true;
    }
    return false;
}

bool y_geom(int L, int &cols_per_tile, size_t &sm)
{
    switch (L) {
    case 8: case 16: cols_per_tile = kThreads; sm = 0; return true;
    case 32: cols_per_tile = ColShape<float, 32>::TC; sm = swsize(32 * cols_per_tile) * 8; return true;
    case 64: cols_per_tile = ColShape<float, 64>::TC; sm = swsize(64 * cols_per_tile) * 8; return true;
    case 128: cols_per_tile = ColShape<float, 128>::TC; sm = swsize(128 * cols_per_tile) * 8; return true;
    case 256: cols_per_tile = ColShape<float, 256>::TC; sm = swsize(256 * cols_per_tile) * 8; return true;
    case 512: cols_per_tile = ColShape<float, 512>::TC; sm = swsize(512 * cols_per_tile) * 8; return true;
    }
    return false;
}

// z tiles of the batch kernels: the 8-point second stage (variant 8) for
// lengths 32..128, the two-stage variant 0 otherwise.
template <int L> constexpr int kBatchZV = (L >= 32 && L <= 128) ? 8 : 0;

template <int L> constexpr size_t z_smem()
{
    using Sh = ZShape<float, L, kBatchZV<L>>;
    return 3 * swsize(L * Sh::TC) * 8 + (size_t)(L / 2 + 1) * 6 * Sh::TC * 4;
}

bool z_geom(int L, int &cols_per_tile, size_t &sm)
{
    switch (L) {
    case 4: case 8: case 16: cols_per_tile = kThreads; sm = 0; return true;
    case 32: cols_per_tile = ZShape<float, 32, kBatchZV<32>>::TC; sm = z_smem<32>(); return true;
    case 64: cols_per_tile = ZShape<float, 64, kBatchZV<64>>::TC; sm = z_smem<64>(); return true;
    case 128: cols_per_tile = ZShape<float, 128, kBatchZV<128>>::TC; sm = z_smem<128>(); return true;
    case 256: cols_per_tile = ZShape<float, 256, kBatchZV<256>>::TC; sm = z_smem<256>(); return true;
    }
    return false;
}

bool pass_geom(const demag_plan *p, PassGeom &g)
{
    const int rows = 3 * p->nz * p->ny;
    int per;
    if (!x_geom(p->Px / 2, per, g.smem[0])) return false;
    g.tiles[0] = (rows + per - 1) / per;
    g.tiles[4] = g.tiles[0];
    g.smem[4] = g.smem[0];
    if (p->Py == 1) {
        g.tiles[1] = g.tiles[3] = 0;
        g.smem[1] = g.smem[3] = 0;
    } else {
        if (!y_geom(p->Py, per, g.smem[1])) return false;
        g.tiles[1] = g.tiles[3] = (3 * p->nz * p->Kx + per - 1) / per;
        g.smem[3] = g.smem[1];
    }
    if (!z_geom(p->Pz, per, g.smem[2])) return false;
    g.tiles[2] = (p->Py * p->Kx + per - 1) / per;
    g.tiles[5] = 1;
    g.smem[5] = 0;
    return true;
}

// --------------------------------------------------------------- device side
__device__ void energy_tile(const BatchState &st)
{
    __shared__ double ss[kThreads], sc[kThreads];
    const int n = st.ntiles[4];
    double s = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        const double v = __ldcg(&st.partials[i]);
        const double t = s + v;
        c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const double a = ss[threadIdx.x], b = ss[threadIdx.x + w];
            const double t = a + b;
            const double e = fabs(a) >= fabs(b) ? (a - t) + b : (b - t) + a;
            ss[threadIdx.x] = t;
            sc[threadIdx.x] += sc[threadIdx.x + w] + e;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && st.E) *st.E = st.efactor * (ss[0] + sc[0]);
}

template <int PASS>
__device__ __forceinline__ void run_item_t(const BatchState &st, int tile, unsigned char *sm)
{
    const int nx = st.nx, ny = st.ny, nz = st.nz, Px = st.Px, Py = st.Py, Pz = st.Pz, Kx = st.Kx, Kxp = st.Kxp;
    const int rows = 3 * nz * ny;
    (void)rows; (void)Pz; (void)nx;
    switch (PASS) {
    case 0: {
        XIn<float> a;
        a.in = st.M; a.in_rs = nx; a.wcell = nullptr; a.wscalar = 1.f; a.rows_per_comp = nz * ny;
        switch (Px / 2) {
        case 16: k_x_fwd_tile<float, 16, false>(a, rows, nx, st.S1, Kxp, st.tw[0], tile, sm); break;
        case 32: k_x_fwd_tile<float, 32, false>(a, rows, nx, st.S1, Kxp, st.tw[0], tile, sm); break;
        case 64: k_x_fwd2_tile<float, 64, true, false>(a, rows, nx, st.S1, Kxp, st.tw[0], tile, sm); break;
        case 128: k_x_fwd2_tile<float, 128, true, false>(a, rows, nx, st.S1, Kxp, st.tw[0], tile, sm); break;
        case 256: k_x_fwd2_tile<float, 256, true, false>(a, rows, nx, st.S1, Kxp, st.tw[0], tile, sm); break;
        case 512: k_x_fwd2_tile<float, 512, true, false>(a, rows, nx, st.S1, Kxp, st.tw[0], tile, sm); break;
        }
        break;
    }
    case 1:
    case 3: {
        const bool inv = PASS == 3;
        const float2 *in = inv ? st.S2 : st.S1;
        float2 *out = inv ? st.S1 : st.S2;
        const int64_t iss = inv ? (int64_t)Py * Kxp : (int64_t)ny * Kxp, oss = inv ? (int64_t)ny * Kxp : (int64_t)Py * Kxp;
        const int nin = inv ? Py : ny, nout = inv ? ny : Py;
        const int ncols = 3 * nz * Kx;
#define DEMAG_YCASE1(LL)                                                                                      \
    case LL:                                                                                                  \
        if (inv) k_col1_tile<float, LL, true, true>(in, out, ncols, Kx, iss, Kxp, nin, oss, Kxp, nout, tile, sm); \
        else k_col1_tile<float, LL, false, true>(in, out, ncols, Kx, iss, Kxp, nin, oss, Kxp, nout, tile, sm);  \
        break;
#define DEMAG_YCASE2(LL)                                                                                      \
    case LL:                                                                                                  \
        if (inv)                                                                                              \
            k_col2_tile<float, LL, true, false, true, true>(in, out, ncols, Kx, iss, Kxp, nin, oss, Kxp, nout,   \
                                                            st.tw[1], 1, tile, sm);                             \
        else                                                                                                  \
            k_col2_tile<float, LL, false, true, false, true>(in, out, ncols, Kx, iss, Kxp, nin, oss, Kxp, nout,  \
                                                             st.tw[1], 1, tile, sm);                            \
        break;
        switch (Py) {
            DEMAG_YCASE1(8) DEMAG_YCASE1(16) DEMAG_YCASE2(32) DEMAG_YCASE2(64) DEMAG_YCASE2(128)
            DEMAG_YCASE2(256) DEMAG_YCASE2(512)
        }
#undef DEMAG_YCASE1
#undef DEMAG_YCASE2
        break;
    }
    case 2: {
        const int ncols = Py * Kx;
        const int64_t ss = Kxp, rs = (int64_t)Py * Kxp, cs = (int64_t)nz * Py * Kxp;
        switch (Pz) {
        case 4: k_z_conv1_tile<float, 4, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, tile, sm); break;
        case 8: k_z_conv1_tile<float, 8, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, tile, sm); break;
        case 16: k_z_conv1_tile<float, 16, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, tile, sm); break;
        case 32: k_z_conv2_tile<float, 32, kBatchZV<32>, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, st.tw[2], 1, tile, sm); break;
        case 64: k_z_conv2_tile<float, 64, kBatchZV<64>, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, st.tw[2], 1, tile, sm); break;
        case 128: k_z_conv2_tile<float, 128, kBatchZV<128>, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, st.tw[2], 1, tile, sm); break;
        case 256: k_z_conv2_tile<float, 256, kBatchZV<256>, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, st.tw[2], 1, tile, sm); break;
        }
        break;
    }
    case 4: {
        XOut<float> o;
        o.out = st.H; o.out_rs = nx; o.scale = 1.f / ((float)Px * Py * Pz); o.oscale = 1.f; o.wcell = nullptr;
        o.gdev = nullptr; o.Mref = st.M; o.mscale = 1.f; o.partials = st.partials; o.rows_per_comp = nz * ny;
        switch (Px / 2) {
        case 16: k_x_inv_tile<float, 16, true>(st.S1, Kxp, rows, nx, o, st.tw[0], tile, sm); break;
        case 32: k_x_inv_tile<float, 32, true>(st.S1, Kxp, rows, nx, o, st.tw[0], tile, sm); break;
        case 64: k_x_inv2_tile<float, 64, true>(st.S1, Kxp, rows, nx, o, st.tw[0], tile, sm); break;
        case 128: k_x_inv2_tile<float, 128, true>(st.S1, Kxp, rows, nx, o, st.tw[0], tile, sm); break;
        case 256: k_x_inv2_tile<float, 256, true>(st.S1, Kxp, rows, nx, o, st.tw[0], tile, sm); break;
        case 512: k_x_inv2_tile<float, 512, true>(st.S1, Kxp, rows, nx, o, st.tw[0], tile, sm); break;
        }
        break;
    }
    case 5:
        energy_tile(st);
        break;
    }
}

__device__ void run_item(const BatchState &st, int pass, int tile, unsigned char *sm)
{
    switch (pass) {
    case 0: run_item_t<0>(st, tile, sm); break;
    case 1: run_item_t<1>(st, tile, sm); break;
    case 2: run_item_t<2>(st, tile, sm); break;
    case 3: run_item_t<3>(st, tile, sm); break;
    case 4: run_item_t<4>(st, tile, sm); break;
    case 5: run_item_t<5>(st, tile, sm); break;
    }
}

// One tile of pass PASS for a state whose transform length of that pass is
// the compile-time L (x: Px/2, y: Py, z: Pz).
template <int PASS, int L>
__device__ __forceinline__ void run_item_L(const BatchState &st, int tile, unsigned char *sm)
{
    const int nx = st.nx, ny = st.ny, nz = st.nz, Px = st.Px, Py = st.Py, Pz = st.Pz, Kx = st.Kx, Kxp = st.Kxp;
    const int rows = 3 * nz * ny;
    (void)Px; (void)Pz;
    if constexpr (PASS == 0) {
        XIn<float> a;
        a.in = st.M; a.in_rs = nx; a.wcell = nullptr; a.wscalar = 1.f; a.rows_per_comp = nz * ny;
        if constexpr (L <= 32) k_x_fwd_tile<float, L, false>(a, rows, nx, st.S1, Kxp, st.tw[0], tile, sm);
        else k_x_fwd2_tile<float, L, true, false>(a, rows, nx, st.S1, Kxp, st.tw[0], tile, sm);
    } else if constexpr (PASS == 1 || PASS == 3) {
        constexpr bool inv = PASS == 3;
        const float2 *in = inv ? st.S2 : st.S1;
        float2 *out = inv ? st.S1 : st.S2;
        const int64_t iss = inv ? (int64_t)Py * Kxp : (int64_t)ny * Kxp, oss = inv ? (int64_t)ny * Kxp : (int64_t)Py * Kxp;
        const int nin = inv ? Py : ny, nout = inv ? ny : Py;
        const int ncols = 3 * nz * Kx;
        if constexpr (L <= 16) {
            k_col1_tile<float, L, inv, true>(in, out, ncols, Kx, iss, Kxp, nin, oss, Kxp, nout, tile, sm);
        } else if constexpr (inv) {
            k_col2_tile<float, L, true, false, true, true>(in, out, ncols, Kx, iss, Kxp, nin, oss, Kxp, nout, st.tw[1], 1,
                                                           tile, sm);
        } else {
            k_col2_tile<float, L, false, true, false, true>(in, out, ncols, Kx, iss, Kxp, nin, oss, Kxp, nout, st.tw[1],
                                                            1, tile, sm);
        }
    } else if constexpr (PASS == 2) {
        const int ncols = Py * Kx;
        const int64_t ss = Kxp, rs = (int64_t)Py * Kxp, cs = (int64_t)nz * Py * Kxp;
        if constexpr (L <= 16) k_z_conv1_tile<float, L, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, tile, sm);
        else k_z_conv2_tile<float, L, kBatchZV<L>, true>(st.S2, ncols, Kx, ss, rs, cs, nz, st.nhat, Py, Kx, st.tw[2], 1,
                                                        tile, sm);
    } else if constexpr (PASS == 4) {
        XOut<float> o;
        o.out = st.H; o.out_rs = nx; o.scale = 1.f / ((float)Px * Py * Pz); o.oscale = 1.f; o.wcell = nullptr;
        o.gdev = nullptr; o.Mref = st.M; o.mscale = 1.f; o.partials = st.partials; o.rows_per_comp = nz * ny;
        if constexpr (L <= 32) k_x_inv_tile<float, L, true>(st.S1, Kxp, rows, nx, o, st.tw[0], tile, sm);
        else k_x_inv2_tile<float, L, true>(st.S1, Kxp, rows, nx, o, st.tw[0], tile, sm);
    } else {
        energy_tile(st);
    }
}

// Pass-batched mode: one launch of pass PASS per transform length L covers
// that pass's tiles of every state with that length (CTA b: item b of the
// group; its state by binary search of the group's prefix sums gstart over
// its m states gstate). The launches follow one another on the stream, so no
// dependency waits are needed, and each launch carries one tile function.
template <int PASS, int L>
__global__ void __launch_bounds__(kThreads) k_batch_pass(BatchDesc d, const int *__restrict__ gstate,
                                                         const int *__restrict__ gstart, int m)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int item = blockIdx.x;
    int lo = 0, hi = m - 1;
    while (lo < hi) {  // last group entry with start <= item
        const int mid = (lo + hi + 1) >> 1;
        if (gstart[mid] <= item) lo = mid; else hi = mid - 1;
    }
    run_item_L<PASS, L>(d.states[gstate[lo]], item - gstart[lo], smraw);
}

__global__ void __launch_bounds__(kThreads, 1) k_batch(BatchDesc d)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_item, s_pass, s_state, s_stop;
    const int n = d.n;
    for (;;) {
        if (threadIdx.x == 0) {
            int stop = *(volatile int *)d.error;
            int item = stop ? d.total : atomicAdd(d.counter, 1);
            int pass = 0, state = 0;
            if (item < d.total) {
                // pass-major item order: start[p (n+1) + s]
                while (pass + 1 < kPasses && item >= d.start[(pass + 1) * (n + 1)]) ++pass;
                int lo = 0, hi = n - 1;
                const int *row = d.start + pass * (n + 1);
                while (lo < hi) {  // last state with start <= item
                    const int mid = (lo + hi + 1) >> 1;
                    if (row[mid] <= item) lo = mid; else hi = mid - 1;
                }
                state = lo;
                if (pass > 0) {
                    // wait (bounded) until the previous pass of this state is complete
                    const int need = d.states[state].ntiles[pass - 1];
                    volatile int *cnt = d.done + (pass - 1) * n + state;
                    const long long t0 = clock64();
                    while (*cnt < need) {
                        if (*(volatile int *)d.error) { stop = 1; break; }
                        if (clock64() - t0 > d.timeout_cycles) {
                            atomicExch(d.error, 1);
                            stop = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                    __threadfence();
                }
            } else {
                stop = 1;
            }
            s_item = item;
            s_pass = pass;
            s_state = state;
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        const int pass = s_pass, state = s_state;
        const int tile = s_item - d.start[pass * (n + 1) + state];
        run_item(d.states[state], pass, tile, smraw);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(d.done + pass * n + state, 1);
    }
}

}  // namespace
}  // namespace demag

using demag::BatchDesc;
using demag::BatchState;

struct demag_batch {
    int n;
    demag_prec prec;
    int device;
    std::vector<demag_plan_t> plans;
    int mode;            // 0 persistent, 1 graph of branches
    bool persistent_ok;
    std::string why_not_persistent;
    // persistent
    std::vector<BatchState> hs;
    std::vector<int> hstart;
    BatchState *ds;
    int *dstart, *dcounter, *ddone, *derror;
    double *dE, *dpartials;
    int total;
    size_t smem;
    int grid;
    long long timeout_cycles;
    bool states_dirty;
    cudaGraphExec_t pexec;
    // pass-batched (one launch per pass and transform length over all states)
    struct Group {
        int pass, L, m, items;
        size_t smem;
        int off;  // into dgroups: m state indices, then m + 1 prefix sums
    };
    std::vector<Group> groups;
    int *dgroups;
    int pass_total[6];
    double tuned_ms[3];  // last autotune: persistent, branches, pass-batched (1e30: not run)
    size_t pass_smem[6];
    cudaGraphExec_t qexec;
    bool timing;
    cudaEvent_t tev[7];
    double pass_ms[6];
    long pass_n;
    // branches
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaEvent_t fork;
    cudaGraphExec_t bexec;
    std::vector<const void *> bM;
    std::vector<void *> bH;
    // last pointers given
    std::vector<const void *> curM;
    std::vector<void *> curH;
    long launches;
    // creation inputs (to rebuild the plans with another padding)
    std::vector<int> dims;
    std::vector<double> cells;
    int pad_mode;
};

namespace {

demag_status bfail(demag_status s, const std::string &m)
{
    demag::set_last_error(m);
    return s;
}

bool dev_ptr_ok(const void *p, int dev)
{
    if (!p || ((uintptr_t)p & 15u)) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

size_t field_bytes(const demag_plan_t p) { return 3 * (size_t)p->nx * p->ny * p->nz * (p->prec == DEMAG_F32 ? 4 : 8); }

void free_batch(demag_batch *b)
{
    if (b->pexec) cudaGraphExecDestroy(b->pexec);
    if (b->qexec) cudaGraphExecDestroy(b->qexec);
    if (b->bexec) cudaGraphExecDestroy(b->bexec);
    for (auto e : b->tev)
        if (e) cudaEventDestroy(e);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->events) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->ds);
    cudaFree(b->dstart);
    cudaFree(b->dcounter);
    cudaFree(b->ddone);
    cudaFree(b->derror);
    cudaFree(b->dE);
    cudaFree(b->dpartials);
    cudaFree(b->dgroups);
    for (auto p : b->plans) demag_plan_destroy(p);
    delete b;
}

demag_status build_persistent(demag_batch *b)
{
    const int n = b->n;
    if (b->prec != DEMAG_F32) {
        b->why_not_persistent = "the persistent kernel is built for FP32";
        return DEMAG_OK;
    }
    std::vector<demag::PassGeom> geo(n);
    size_t smem = 0;
    size_t npart = 0;
    for (int i = 0; i < n; ++i) {
        if (!demag::pass_geom(b->plans[i], geo[i])) {
            b->why_not_persistent = "state " + std::to_string(i) + " has transform lengths outside the persistent kernel";
            return DEMAG_OK;
        }
        for (int k = 0; k < demag::kPasses; ++k)
            if (geo[i].tiles[k] > 0 && geo[i].smem[k] > smem) smem = geo[i].smem[k];
        npart += geo[i].tiles[4];
    }
    if (smem > 227 * 1024) {
        b->why_not_persistent = "shared memory beyond one CTA";
        return DEMAG_OK;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&b->dpartials, sizeof(double) * npart)) != cudaSuccess) return bfail(DEMAG_ERR_OOM, "batch partials");
    if ((e = cudaMalloc(&b->dE, sizeof(double) * n)) != cudaSuccess) return bfail(DEMAG_ERR_OOM, "batch energies");
    b->hs.resize(n);
    size_t poff = 0;
    for (int i = 0; i < n; ++i) {
        const demag_plan_t p = b->plans[i];
        BatchState &s = b->hs[i];
        memset(&s, 0, sizeof(s));
        s.S1 = (float2 *)p->S1;
        s.S2 = (float2 *)p->S2;
        s.nhat = p->nhat32;
        for (int a = 0; a < 3; ++a) s.tw[a] = p->tw32[a];
        s.partials = b->dpartials + poff;
        poff += geo[i].tiles[4];
        s.E = b->dE + i;
        s.nx = p->nx; s.ny = p->ny; s.nz = p->nz;
        s.Px = p->Px; s.Py = p->Py; s.Pz = p->Pz; s.Kx = p->Kx; s.Kxp = p->Kxp;
        for (int k = 0; k < demag::kPasses; ++k) s.ntiles[k] = geo[i].tiles[k];
        s.efactor = -0.5 * demag::kMu0 * p->dx * p->dy * p->dz;
    }
    b->hstart.assign(demag::kPasses * (n + 1), 0);
    int acc = 0;
    for (int k = 0; k < demag::kPasses; ++k) {
        for (int i = 0; i < n; ++i) {
            b->hstart[k * (n + 1) + i] = acc;
            acc += geo[i].tiles[k];
        }
        b->hstart[k * (n + 1) + n] = acc;
    }
    b->total = acc;
    for (int k = 0; k < demag::kPasses; ++k) {
        b->pass_total[k] = b->hstart[k * (n + 1) + n] - b->hstart[k * (n + 1)];
        b->pass_smem[k] = 0;
        for (int i = 0; i < n; ++i)
            if (geo[i].tiles[k] > 0 && geo[i].smem[k] > b->pass_smem[k]) b->pass_smem[k] = geo[i].smem[k];
    }
    // pass-batched groups: per pass, the states of one transform length
    {
        std::vector<int> host;
        b->groups.clear();
        for (int k = 0; k < demag::kPasses; ++k) {
            std::vector<int> lens;
            for (int i = 0; i < n; ++i) {
                if (geo[i].tiles[k] <= 0) continue;
                const demag_plan_t pl = b->plans[i];
                const int L = (k == 0 || k == 4) ? pl->Px / 2 : (k == 1 || k == 3) ? pl->Py : (k == 2 ? pl->Pz : 0);
                if (std::find(lens.begin(), lens.end(), L) == lens.end()) lens.push_back(L);
            }
            std::sort(lens.begin(), lens.end());
            for (int L : lens) {
                demag_batch::Group g;
                g.pass = k; g.L = L; g.m = 0; g.items = 0; g.smem = 0;
                g.off = (int)host.size();
                std::vector<int> st, pre;
                pre.push_back(0);
                for (int i = 0; i < n; ++i) {
                    if (geo[i].tiles[k] <= 0) continue;
                    const demag_plan_t pl = b->plans[i];
                    const int Li = (k == 0 || k == 4) ? pl->Px / 2 : (k == 1 || k == 3) ? pl->Py : (k == 2 ? pl->Pz : 0);
                    if (Li != L) continue;
                    st.push_back(i);
                    pre.push_back(pre.back() + geo[i].tiles[k]);
                    if (geo[i].smem[k] > g.smem) g.smem = geo[i].smem[k];
                }
                g.m = (int)st.size();
                g.items = pre.back();
                host.insert(host.end(), st.begin(), st.end());
                host.insert(host.end(), pre.begin(), pre.end());
                b->groups.push_back(g);
            }
        }
        if (cudaMalloc(&b->dgroups, sizeof(int) * (host.size() + 1)) != cudaSuccess)
            return bfail(DEMAG_ERR_OOM, "batch groups");
        cudaMemcpy(b->dgroups, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice);
    }
    if (cudaMalloc(&b->ds, sizeof(BatchState) * n) != cudaSuccess) return bfail(DEMAG_ERR_OOM, "batch states");
    if (cudaMalloc(&b->dstart, sizeof(int) * b->hstart.size()) != cudaSuccess) return bfail(DEMAG_ERR_OOM, "batch table");
    if (cudaMalloc(&b->dcounter, sizeof(int)) != cudaSuccess) return bfail(DEMAG_ERR_OOM, "batch counter");
    if (cudaMalloc(&b->ddone, sizeof(int) * demag::kPasses * n) != cudaSuccess) return bfail(DEMAG_ERR_OOM, "batch counters");
    if (cudaMalloc(&b->derror, sizeof(int)) != cudaSuccess) return bfail(DEMAG_ERR_OOM, "batch flag");
    cudaMemset(b->derror, 0, sizeof(int));
    cudaMemcpy(b->dstart, b->hstart.data(), sizeof(int) * b->hstart.size(), cudaMemcpyHostToDevice);
    // opt in to the whole per-block shared memory (other batches launch the
    // same kernel with other sizes; the occupancy follows each launch's size)
    {
        int optin = 0;
        cudaFuncAttributes fa;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, demag::k_batch);
        if (e == cudaSuccess && smem + fa.sharedSizeBytes > (size_t)optin) {
            b->why_not_persistent = "the persistent kernel's shared memory exceeds the per-block limit";
            return DEMAG_OK;
        }
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(demag::k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
    }
    if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch kernel smem: ") + cudaGetErrorString(e));
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, demag::k_batch, demag::kThreads, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (per_sm < 1) {
        b->why_not_persistent = "the persistent kernel does not fit on an SM";
        return DEMAG_OK;
    }
    b->grid = per_sm * sms;
    b->smem = smem;
    b->persistent_ok = true;
    b->states_dirty = true;
    return DEMAG_OK;
}

demag_status launch_persistent(demag_batch *b, cudaStream_t st)
{
    const int n = b->n;
    if (b->states_dirty) {
        for (int i = 0; i < n; ++i) {
            b->hs[i].M = (const float *)b->curM[i];
            b->hs[i].H = (float *)b->curH[i];
        }
        // from pageable memory: staged before the call returns
        cudaError_t e = cudaMemcpyAsync(b->ds, b->hs.data(), sizeof(BatchState) * n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch states upload: ") + cudaGetErrorString(e));
        b->states_dirty = false;
    }
    if (!b->pexec) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return bfail(DEMAG_ERR_CUDA, "capture stream");
        BatchDesc d;
        d.states = b->ds; d.n = n; d.start = b->dstart; d.total = b->total;
        d.counter = b->dcounter; d.done = b->ddone; d.error = b->derror;
        d.timeout_cycles = b->timeout_cycles;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(b->dcounter, 0, sizeof(int), cs);
            cudaMemsetAsync(b->ddone, 0, sizeof(int) * demag::kPasses * n, cs);
            demag::k_batch<<<b->grid, demag::kThreads, b->smem, cs>>>(d);
            e = cudaStreamEndCapture(cs, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->pexec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            b->pexec = nullptr;
            return bfail(DEMAG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaGraphLaunch(b->pexec, st);
    if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    b->launches += 1;
    return DEMAG_OK;
}

template <int PASS, int L>
cudaError_t group_launch(demag_batch *b, const BatchDesc &d, const demag_batch::Group &g, cudaStream_t st)
{
    static int done_for = -1;  // opt in to the per-block shared memory once per device
    if (done_for != b->device) {
        int optin = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, demag::k_batch_pass<PASS, L>);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(demag::k_batch_pass<PASS, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
        done_for = b->device;
    }
    demag::k_batch_pass<PASS, L><<<g.items, demag::kThreads, g.smem, st>>>(d, b->dgroups + g.off,
                                                                           b->dgroups + g.off + g.m, g.m);
    return cudaGetLastError();
}

cudaError_t launch_group(demag_batch *b, const BatchDesc &d, const demag_batch::Group &g, cudaStream_t st)
{
    if (g.items <= 0) return cudaSuccess;
#define DEMAG_G(P, LL) \
    case LL: return group_launch<P, LL>(b, d, g, st);
    switch (g.pass) {
    case 0:
        switch (g.L) { DEMAG_G(0, 16) DEMAG_G(0, 32) DEMAG_G(0, 64) DEMAG_G(0, 128) DEMAG_G(0, 256) DEMAG_G(0, 512) }
        break;
    case 1:
        switch (g.L) { DEMAG_G(1, 8) DEMAG_G(1, 16) DEMAG_G(1, 32) DEMAG_G(1, 64) DEMAG_G(1, 128) DEMAG_G(1, 256) DEMAG_G(1, 512) }
        break;
    case 2:
        switch (g.L) { DEMAG_G(2, 4) DEMAG_G(2, 8) DEMAG_G(2, 16) DEMAG_G(2, 32) DEMAG_G(2, 64) DEMAG_G(2, 128) DEMAG_G(2, 256) }
        break;
    case 3:
        switch (g.L) { DEMAG_G(3, 8) DEMAG_G(3, 16) DEMAG_G(3, 32) DEMAG_G(3, 64) DEMAG_G(3, 128) DEMAG_G(3, 256) DEMAG_G(3, 512) }
        break;
    case 4:
        switch (g.L) { DEMAG_G(4, 16) DEMAG_G(4, 32) DEMAG_G(4, 64) DEMAG_G(4, 128) DEMAG_G(4, 256) DEMAG_G(4, 512) }
        break;
    case 5:
        return group_launch<5, 0>(b, d, g, st);
    }
#undef DEMAG_G
    return cudaErrorInvalidValue;
}

// The pass-batched launches on st, pass by pass (each pass's length groups
// one after another); with timing, an event before each pass and after the
// last (tev[0..6]).
cudaError_t pass_launches(demag_batch *b, cudaStream_t st, bool events)
{
    BatchDesc d;
    memset(&d, 0, sizeof d);
    d.states = b->ds; d.n = b->n; d.start = b->dstart; d.total = b->total;
    cudaError_t e = cudaSuccess;
    size_t gi = 0;
    for (int k = 0; k < demag::kPasses && e == cudaSuccess; ++k) {
        if (events) cudaEventRecord(b->tev[k], st);
        for (; gi < b->groups.size() && b->groups[gi].pass == k && e == cudaSuccess; ++gi)
            e = launch_group(b, d, b->groups[gi], st);
    }
    if (events && e == cudaSuccess) cudaEventRecord(b->tev[6], st);
    return e;
}

demag_status launch_passes(demag_batch *b, cudaStream_t st)
{
    const int n = b->n;
    if (b->states_dirty) {
        for (int i = 0; i < n; ++i) {
            b->hs[i].M = (const float *)b->curM[i];
            b->hs[i].H = (float *)b->curH[i];
        }
        cudaError_t e = cudaMemcpyAsync(b->ds, b->hs.data(), sizeof(BatchState) * n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch states upload: ") + cudaGetErrorString(e));
        b->states_dirty = false;
    }
    if (b->timing) {
        // direct launches with an event around each pass, read at the next call
        if (!b->tev[0])
            for (auto &ev : b->tev)
                if (cudaEventCreate(&ev) != cudaSuccess) return bfail(DEMAG_ERR_CUDA, "batch timing events");
        cudaError_t e = pass_launches(b, st, true);
        if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch pass launch: ") + cudaGetErrorString(e));
        cudaEventSynchronize(b->tev[6]);
        for (int k = 0; k < demag::kPasses; ++k) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, b->tev[k], b->tev[k + 1]) == cudaSuccess) b->pass_ms[k] += ms;
        }
        b->pass_n += 1;
        b->launches += (long)b->groups.size();
        return DEMAG_OK;
    }
    if (!b->qexec) {
        // a first run outside the capture (kernel attributes, lazy loading)
        cudaError_t e = pass_launches(b, st, false);
        if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch pass launch: ") + cudaGetErrorString(e));
        b->launches += (long)b->groups.size();
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return bfail(DEMAG_ERR_CUDA, "capture stream");
        cudaStreamSynchronize(st);
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = pass_launches(b, cs, false);
            e = cudaStreamEndCapture(cs, &g);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->qexec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            b->qexec = nullptr;
            return bfail(DEMAG_ERR_CUDA, std::string("batch pass graph: ") + cudaGetErrorString(e));
        }
        return DEMAG_OK;
    }
    cudaError_t e = cudaGraphLaunch(b->qexec, st);
    if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    b->launches += 1;
    return DEMAG_OK;
}

demag_status launch_branches(demag_batch *b, cudaStream_t st)
{
    const int n = b->n;
    bool same = b->bexec && b->bM == b->curM && b->bH == b->curH;
    if (!same) {
        if (b->bexec) { cudaGraphExecDestroy(b->bexec); b->bexec = nullptr; }
        if (b->streams.empty()) {
            b->streams.resize(n);
            b->events.resize(n);
            for (int i = 0; i < n; ++i) {
                if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming) != cudaSuccess)
                    return bfail(DEMAG_ERR_CUDA, "batch streams");
            }
            if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
                return bfail(DEMAG_ERR_CUDA, "batch event");
        }
        // run once outside capture (kernel attributes, lazy loading)
        for (int i = 0; i < n; ++i) {
            demag_status s = demag_field_energy(b->plans[i], b->curM[i], b->curH[i], b->dE ? b->dE + i : b->plans[i]->e_dev, st);
            if (s != DEMAG_OK) return s;
        }
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return bfail(DEMAG_ERR_CUDA, "capture stream");
        cudaStreamSynchronize(st);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        demag_status s = DEMAG_OK;
        if (e == cudaSuccess) {
            cudaEventRecord(b->fork, cs);
            for (int i = 0; i < n && s == DEMAG_OK; ++i) {
                cudaStreamWaitEvent(b->streams[i], b->fork, 0);
                const bool timing = b->plans[i]->timing;
                b->plans[i]->timing = false;
                s = demag_field_energy(b->plans[i], b->curM[i], b->curH[i], b->dE ? b->dE + i : b->plans[i]->e_dev,
                                       b->streams[i]);
                b->plans[i]->timing = timing;
                cudaEventRecord(b->events[i], b->streams[i]);
                cudaStreamWaitEvent(cs, b->events[i], 0);
            }
            e = cudaStreamEndCapture(cs, &g);
        }
        if (e == cudaSuccess && s == DEMAG_OK) e = cudaGraphInstantiate(&b->bexec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (s != DEMAG_OK) return s;
        if (e != cudaSuccess) {
            b->bexec = nullptr;
            return bfail(DEMAG_ERR_CUDA, std::string("batch branch graph: ") + cudaGetErrorString(e));
        }
        b->bM = b->curM;
        b->bH = b->curH;
    }
    cudaError_t e = cudaGraphLaunch(b->bexec, st);
    if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    b->launches += 1;
    return DEMAG_OK;
}

}  // namespace

extern "C" {

demag_status demag_batch_create(int n, const int *dims, const double *cells, demag_prec prec, demag_batch_t *out)
{
    return demag_batch_create_ex(n, dims, cells, prec, nullptr, out);
}

demag_status demag_batch_create_ex(int n, const int *dims, const double *cells, demag_prec prec,
                                   const demag_options *opt, demag_batch_t *out)
{
    if (!out) return bfail(DEMAG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (opt && (opt->px || opt->py || opt->pz))
        return bfail(DEMAG_ERR_INVALID_ARG, "batch options take a pad_mode only (no explicit lengths)");
    if (n < 1 || !dims || !cells) return bfail(DEMAG_ERR_INVALID_ARG, "need n >= 1 and the size arrays");
    demag_batch *b = new demag_batch();
    b->n = n;
    b->prec = prec;
    b->dims.assign(dims, dims + 3 * n);
    b->cells.assign(cells, cells + 3 * n);
    b->pad_mode = opt ? opt->pad_mode : DEMAG_PAD_POW2;
    b->timeout_cycles = 4000000000LL;  // ~2 s at 2 GHz; normal waits take microseconds
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bfail(DEMAG_ERR_CUDA, "no CUDA device");
    }
    b->plans.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        demag_status s = demag_plan_create_ex(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], cells[3 * i],
                                              cells[3 * i + 1], cells[3 * i + 2], prec, opt, &b->plans[i]);
        if (s == DEMAG_OK) s = demag_tensor_setup(b->plans[i], nullptr);
        if (s != DEMAG_OK) {
            demag::set_last_error(std::string("state ") + std::to_string(i) + ": " + demag_last_error(nullptr));
            free_batch(b);
            return s;
        }
    }
    demag_status s = build_persistent(b);
    if (s != DEMAG_OK) {
        free_batch(b);
        return s;
    }
    b->mode = b->persistent_ok ? 2 : 1;
    b->curM.assign(n, nullptr);
    b->curH.assign(n, nullptr);
    *out = b;
    return DEMAG_OK;
}

demag_status demag_batch_set_mode(demag_batch_t b, int mode)
{
    if (!b || mode < 0 || mode > 2) return bfail(DEMAG_ERR_INVALID_ARG, "bad batch or mode");
    if (mode != 1 && !b->persistent_ok) return bfail(DEMAG_ERR_UNSUPPORTED, b->why_not_persistent);
    b->mode = mode;
    return DEMAG_OK;
}

demag_status demag_batch_set_timeout(demag_batch_t b, double seconds, int stall_state)
{
    if (!b || !(seconds > 0)) return bfail(DEMAG_ERR_INVALID_ARG, "bad batch or timeout");
    int mhz = 0;
    cudaDeviceGetAttribute(&mhz, cudaDevAttrClockRate, b->device);  // kHz
    const double hz = mhz > 0 ? mhz * 1e3 : 2e9;
    b->timeout_cycles = (long long)(seconds * hz);
    if (b->pexec) { cudaGraphExecDestroy(b->pexec); b->pexec = nullptr; }
    if (b->persistent_ok) {
        // test hook: a state whose first pass never completes (its waiters
        // need one more tile than exists), so the bounded wait runs out
        for (int i = 0; i < b->n; ++i) b->hs[i].ntiles[0] = 0;
        demag::PassGeom g;
        for (int i = 0; i < b->n; ++i) {
            demag::pass_geom(b->plans[i], g);
            b->hs[i].ntiles[0] = g.tiles[0] + (i == stall_state ? 1 : 0);
        }
        b->states_dirty = true;
    }
    return DEMAG_OK;
}

demag_status demag_batch_field(demag_batch_t b, const void *const *M, void *const *H, double *E_dev, void *stream)
{
    if (!b || !M || !H) return bfail(DEMAG_ERR_INVALID_ARG, "NULL argument");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) return bfail(DEMAG_ERR_INVALID_ARG, "the batch lives on another device");
    bool changed = false;
    for (int i = 0; i < b->n; ++i)
        if (M[i] != b->curM[i] || H[i] != b->curH[i]) { changed = true; break; }
    if (changed) {
        for (int i = 0; i < b->n; ++i) {
            const size_t bytes = field_bytes(b->plans[i]);
            if (!dev_ptr_ok(M[i], b->device) || !dev_ptr_ok(H[i], b->device))
                return bfail(DEMAG_ERR_INVALID_ARG, "state " + std::to_string(i) + ": M and H must be 16-byte aligned device memory");
            const uintptr_t x = (uintptr_t)M[i], y = (uintptr_t)H[i];
            if (x < y + bytes && y < x + bytes) return bfail(DEMAG_ERR_INVALID_ARG, "state " + std::to_string(i) + ": H overlaps M");
        }
        for (int i = 0; i < b->n; ++i) { b->curM[i] = M[i]; b->curH[i] = H[i]; }
        b->states_dirty = true;
    }
    if (E_dev) {
        cudaPointerAttributes a;
        if (((uintptr_t)E_dev & 7u) != 0 || cudaPointerGetAttributes(&a, E_dev) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return bfail(DEMAG_ERR_INVALID_ARG, "E_dev must be 8-byte aligned device memory");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->dE && cudaMalloc(&b->dE, sizeof(double) * b->n) != cudaSuccess) return bfail(DEMAG_ERR_OOM, "batch energies");
    demag_status s = b->mode == 0 ? launch_persistent(b, st) : (b->mode == 2 ? launch_passes(b, st) : launch_branches(b, st));
    if (s != DEMAG_OK) return s;
    if (E_dev) {
        cudaError_t e = cudaMemcpyAsync(E_dev, b->dE, sizeof(double) * b->n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return bfail(DEMAG_ERR_CUDA, std::string("batch energies copy: ") + cudaGetErrorString(e));
    }
    return DEMAG_OK;
}

demag_status demag_batch_status(demag_batch_t b, void *stream)
{
    if (!b) return bfail(DEMAG_ERR_INVALID_ARG, "batch is NULL");
    if (!b->derror) return DEMAG_OK;
    int flag = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&flag, b->derror, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return bfail(DEMAG_ERR_CUDA, "reading the batch status");
    if (flag) {
        cudaMemsetAsync(b->derror, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        return bfail(DEMAG_ERR_TIMEOUT, "a dependency wait of the persistent batch kernel ran out of time");
    }
    return DEMAG_OK;
}

demag_status demag_batch_info(demag_batch_t b, int *mode, int *persistent_ok, int *items, int *grid, size_t *smem)
{
    if (!b) return bfail(DEMAG_ERR_INVALID_ARG, "batch is NULL");
    if (mode) *mode = b->mode;
    if (persistent_ok) *persistent_ok = b->persistent_ok ? 1 : 0;
    if (items) *items = b->total;
    if (grid) *grid = b->grid;
    if (smem) *smem = b->smem;
    return DEMAG_OK;
}

long demag_batch_launch_count(demag_batch_t b) { return b ? b->launches : 0; }

demag_status demag_batch_set_timing(demag_batch_t b, int enable)
{
    if (!b) return bfail(DEMAG_ERR_INVALID_ARG, "batch is NULL");
    b->timing = enable != 0;
    for (int k = 0; k < 6; ++k) b->pass_ms[k] = 0;
    b->pass_n = 0;
    return DEMAG_OK;
}

demag_status demag_batch_get_timing(demag_batch_t b, double *ms, long *calls)
{
    if (!b || !ms) return bfail(DEMAG_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < 6; ++k) ms[k] = b->pass_ms[k];
    if (calls) *calls = b->pass_n;
    return DEMAG_OK;
}

demag_status demag_batch_autotune(demag_batch_t b, int use_cache, double *ms_persistent, double *ms_branches,
                                  void *stream)
{
    if (!b) return bfail(DEMAG_ERR_INVALID_ARG, "batch is NULL");
    for (int i = 0; i < b->n; ++i) {
        demag_status s = demag_autotune(b->plans[i], use_cache, nullptr, stream);
        if (s != DEMAG_OK) return s;
    }
    std::vector<void *> bufs(2 * b->n, nullptr);
    auto release = [&]() {
        for (void *q : bufs) cudaFree(q);
        for (int i = 0; i < b->n; ++i) { b->curM[i] = nullptr; b->curH[i] = nullptr; }
    };
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < b->n; ++i) {
        const size_t bytes = field_bytes(b->plans[i]);
        if (cudaMalloc(&bufs[2 * i], bytes) != cudaSuccess || cudaMalloc(&bufs[2 * i + 1], bytes) != cudaSuccess) {
            release();
            return bfail(DEMAG_ERR_OOM, "batch autotune buffers");
        }
        cudaMemsetAsync(bufs[2 * i], 0, bytes, st);
    }
    std::vector<const void *> M(b->n);
    std::vector<void *> H(b->n);
    for (int i = 0; i < b->n; ++i) { M[i] = bufs[2 * i]; H[i] = bufs[2 * i + 1]; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double t[3] = {1e30, 1e30, 1e30};
    demag_status rs = DEMAG_OK;
    const bool timing = b->timing;
    b->timing = false;
    for (int mode = 0; mode < 3 && rs == DEMAG_OK; ++mode) {
        if (mode != 1 && !b->persistent_ok) continue;
        b->mode = mode;
        for (int w = 0; w < 2 && rs == DEMAG_OK; ++w) rs = demag_batch_field(b, M.data(), H.data(), nullptr, stream);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5 && rs == DEMAG_OK; ++r) rs = demag_batch_field(b, M.data(), H.data(), nullptr, stream);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        t[mode] = ms / 5;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->timing = timing;
    release();
    if (rs != DEMAG_OK) return rs;
    int best = 1;
    for (int m = 0; m < 3; ++m)
        if (t[m] < t[best]) best = m;
    b->mode = best;
    b->tuned_ms[0] = t[0]; b->tuned_ms[1] = t[1]; b->tuned_ms[2] = t[2];
    if (ms_persistent) *ms_persistent = b->persistent_ok ? t[0] : -1.0;
    if (ms_branches) *ms_branches = t[1];
    return demag_batch_status(b, stream);
}

demag_status demag_batch_autotune_padding(demag_batch_t b, int use_cache, double *ms_pow2, double *ms_smooth,
                                          void *stream)
{
    if (!b) return bfail(DEMAG_ERR_INVALID_ARG, "batch is NULL");
    if (b->pad_mode != DEMAG_PAD_POW2 && b->pad_mode != DEMAG_PAD_SMOOTH)
        return bfail(DEMAG_ERR_UNSUPPORTED, "the batch's padding was chosen per state by timing already");
    double tp = 0, tb = 0;
    demag_status s = demag_batch_autotune(b, use_cache, &tp, &tb, stream);
    if (s != DEMAG_OK) return s;
    const double t_this = std::min(b->tuned_ms[0], std::min(b->tuned_ms[1], b->tuned_ms[2]));
    demag_options o;
    memset(&o, 0, sizeof o);
    o.pad_mode = b->pad_mode == DEMAG_PAD_POW2 ? DEMAG_PAD_SMOOTH : DEMAG_PAD_POW2;
    demag_batch_t nb = nullptr;
    s = demag_batch_create_ex(b->n, b->dims.data(), b->cells.data(), b->prec, &o, &nb);
    if (s != DEMAG_OK) return s;
    s = demag_batch_autotune(nb, use_cache, &tp, &tb, stream);
    if (s != DEMAG_OK) {
        free_batch(nb);
        return s;
    }
    const double t_other = std::min(nb->tuned_ms[0], std::min(nb->tuned_ms[1], nb->tuned_ms[2]));
    const bool was_pow2 = b->pad_mode == DEMAG_PAD_POW2;
    if (ms_pow2) *ms_pow2 = was_pow2 ? t_this : t_other;
    if (ms_smooth) *ms_smooth = was_pow2 ? t_other : t_this;
    if (t_other < t_this) std::swap(*b, *nb);  // keep the faster plans; the caller's handle stays valid
    free_batch(nb);
    return DEMAG_OK;
}

void demag_batch_destroy(demag_batch_t b)
{
    if (b) free_batch(b);
}

}  // extern "C"
