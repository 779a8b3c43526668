// Internal declarations shared by the C-ABI layer and the kernel translation
// units. Not part of the public interface (see include/demag.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "demag.h"

namespace demag {

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };

// Prologue / epilogue options of the x passes.
// Input scaling: value = in * wscalar * (wcell ? wcell[cell] : 1), where wcell
// is a per-cell weight [nz][ny][nx] shared by the three components (a
// saturation-magnetization mask).
template <typename T> struct XIn {
    const T *in;
    int64_t in_rs;
    const T *wcell;
    T wscalar;
    int rows_per_comp;  // nz * ny rows per component (to index wcell)
};
// Output: h = scale * (inverse transform). If out: out = h * oscale * w * g
// with w = wcell[cell] (or 1) and g = *gdev (or 1). If partials: the block's
// sum of mscale * w * Mref * h is written to partials[blockIdx.x].
template <typename T> struct XOut {
    T *out;
    int64_t out_rs;
    T scale;
    T oscale;
    const T *wcell;
    const double *gdev;
    const T *Mref;
    T mscale;
    double *partials;
    int rows_per_comp;
};

// Launchers of the mixed-radix passes (transform lengths with prime factors
// 2, 3, 5, 7 that are not powers of two; mixed_f32.cu / mixed_f64.cu). Same
// arguments and results as the Passes members of the same names.
template <typename T> struct MixedPasses {
    using C = typename CplxOf<T>::type;
    static cudaError_t x_fwd(int L, const XIn<T> &a, int nrows, int nvalid, C *out, int64_t out_rs, const C *twx,
                             cudaStream_t st);
    static cudaError_t x_inv(int L, const C *in, int64_t in_rs, int nrows, int nvalid, const XOut<T> &o,
                             const C *twx, cudaStream_t st);
    static int x_blocks(int L, int nrows);
    static cudaError_t col(int L, bool inv, const C *in, C *out, int ncols, int width, int64_t iss, int64_t irs,
                           int nin, int64_t oss, int64_t ors, int nout, const C *tw, int twstride, cudaStream_t st);
    static cudaError_t zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                             const T *nhat, int Py, int Kx, const C *tw, int twstride, cudaStream_t st);
    static cudaError_t sp_zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                int nout, const T *that, int Py, int Kx, const C *tw, const C *phx, const C *phy,
                                const C *phz, cudaStream_t st);
};

// Launchers of the field passes for element type T (defined in
// passes_f32.cu / passes_f64.cu). L is the transform length of the pass.
template <typename T> struct Passes {
    using C = typename CplxOf<T>::type;
    // real-to-complex along x; L = Px/2 (complex length), Px >= 2
    // variant 1: the forward pass by persistent CTAs streaming row tiles
    // with bulk asynchronous copies (where the rows allow it); variant 2: the
    // inverse pass too; otherwise the one-tile-per-CTA kernels
    static cudaError_t x_fwd(int L, const XIn<T> &a, int nrows, int nvalid, C *out, int64_t out_rs,
                             const C *twx, cudaStream_t st, int variant = 0);
    // complex-to-real along x with the XOut epilogue
    static cudaError_t x_inv(int L, const C *in, int64_t in_rs, int nrows, int nvalid, const XOut<T> &o,
                             const C *twx, cudaStream_t st, int variant = 0);
    // 1 if a bounded wait of a pipelined pass gave up since the last call (clears it)
    static int pipe_error_take();
    static int x_blocks(int L, int nrows);
    // strided column transforms (y passes, z forward of the setup)
    static cudaError_t col(int L, bool inv, const C *in, C *out, int ncols, int width, int64_t iss,
                           int64_t irs, int nin, int64_t oss, int64_t ors, int nout, const C *tw,
                           int twstride, cudaStream_t st, int variant = 0);
    template <int L, bool INV, bool PIN, bool POUT, int V>
    static cudaError_t col_launch(const C *in, C *out, int ncols, int width, int64_t iss, int64_t irs, int nin,
                                  int64_t oss, int64_t ors, int nout, const C *tw, int twstride,
                                  cudaStream_t st);
    // fused z forward, spectral product, z inverse (in place)
    static cudaError_t zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
                             int nrows, const T *nhat, int Py, int Kx, const C *tw, int twstride,
                             cudaStream_t st, int variant = 0);
    // persistent z pass streaming column tiles by TMA (FP32, L = 256 or 512, at
    // most L/2 input rows); ntile: the tile-ordered tensor copy (tile_tensor); tc:
    // columns per tile, 8 (one CTA per SM) or 4 (two CTAs per SM). With
    // partials: also the spectral energy's per-CTA sums of w(kx) m^H N^ m,
    // taken at the product; *nparts holds the room in partials on entry (the
    // grid is capped to it) and the number of sums written on return.
    // cudaErrorNotSupported when the arguments do not allow it.
    static cudaError_t zconv_ws(int L, C *S, int Kx, int Py, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                const T *ntile, const C *tw, cudaStream_t st, int tc = 8,
                                double *partials = nullptr, int *nparts = nullptr);
    // spectral energy (the Parseval form of E, no inverse passes): forward z
    // transforms and the per-CTA sums of w(kx) m^H N^ m into partials
    // (*nparts of them; for zconv_ws_energy *nparts also holds the room in
    // partials on entry, as for zconv_ws). zconv_ws_energy: the persistent TMA form (as
    // zconv_ws); zconv_energy: the two-stage / one-thread forms (power-of-two
    // L <= 512). cudaErrorNotSupported where the form does not exist.
    static cudaError_t zconv_ws_energy(int L, C *S, int Kx, int Py, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                       const T *ntile, const C *tw, double *partials, int *nparts, cudaStream_t st,
                                       int tc = 8);
    static cudaError_t zconv_energy(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
                                    int nrows, const T *nhat, int Py, int Kx, const C *tw, int twstride,
                                    double *partials, int *nparts, cudaStream_t st);
    // partial sums the spectral energy may write (0: no spectral form for L)
    static int zenergy_blocks(int L, int Py, int Kx);
    // elements of the tile-ordered tensor copy for zconv_ws (0: not used for this L)
    static size_t tile_tensor_elems(int L, int Py, int Kx);
    static cudaError_t tile_tensor(int L, const T *nhat, T *ntile, int Py, int Kx, cudaStream_t st);
    template <int L>
    static cudaError_t zconv_pipe(C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                  const T *nhat, int Py, int Kx, const C *tw, int twstride, cudaStream_t st);
    template <int L, int V>
    static cudaError_t zconv_launch(C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs, int nrows,
                                    const T *nhat, int Py, int Kx, const C *tw, int twstride, cudaStream_t st);
    // Px == 1: rows of one value; same prologue / epilogue as above
    static cudaError_t x1_fwd(const XIn<T> &a, int64_t n, C *out, cudaStream_t st);
    static cudaError_t x1_inv(const C *in, int64_t n, const XOut<T> &o, int nblocks, cudaStream_t st);
    // scalar-potential method: fused z pass (three spectra in, the potential
    // spectrum out, nout = nz + 1 node rows) and the finite-difference field
    static cudaError_t sp_zconv(int L, C *S, int ncols, int width, int64_t ss, int64_t rs, int64_t cs,
                                int nrows, int nout, const T *that, int Py, int Kx, const C *tw,
                                const C *phx, const C *phy, const C *phz, cudaStream_t st, int variant = 0);
    static cudaError_t sp_grad(const T *phi, int nx, int ny, int nz, double dx, double dy, double dz, T *H,
                               const T *Mref, double *partials, cudaStream_t st);
    static int sp_grad_blocks(int nx, int ny, int nz);
};

// One state of a batch, as the persistent batch kernel sees it (device
// memory). Pointers come from the state's plan and the caller's arrays.
struct BatchState {
    const float *M;
    float *H;
    float2 *S1, *S2;
    const float *nhat;
    const float2 *tw[3];
    double *partials;
    double *E;
    int nx, ny, nz, Px, Py, Pz, Kx, Kxp;
    int ntiles[6];  // tiles of each pass (x fwd, y fwd, z, y inv, x inv, energy)
    double efactor; // -(mu0/2) V
};

// Shared description of one batch launch (kernel argument).
struct BatchDesc {
    BatchState *states;
    int n;
    const int *start;  // [6][n+1] first item of (pass, state); start[6*(n+1)-1] = total
    int total;
    int *counter;      // next item to claim
    int *done;         // [6][n] finished tiles
    int *error;        // set to 1 when a wait gives up
    long long timeout_cycles;
};

// Tensor setup kernels (tensor.cu).
cudaError_t tensor_octant(double *out, int nx, int ny, int nz, double dx, double dy, double dz,
                          cudaStream_t st);
cudaError_t tensor_wrap(const double *oct, int comp, int nx, int ny, int nz, int Px, int Py,
                        int Pz, double *out, cudaStream_t st);
cudaError_t tensor_extract(const double2 *S, int comp, int Px, int Py, int Pz, int Kxp,
                           double *nhat64, float *nhat32, unsigned long long *imag_max,
                           cudaStream_t st);
// Sets the calling thread's demag_last_error() message (api.cu).
void set_last_error(const std::string &msg);

// Energy from n FP64 partials: *E = factor * sum (deterministic, several
// CTAs). scratch: kFinalizeScratch doubles of device memory per plan (the
// CTA results and a counter the kernel leaves at zero; zero-initialised).
constexpr int kFinalizeBlocks = 64;
constexpr int kFinalizeScratch = 2 * kFinalizeBlocks + 1;
cudaError_t energy_finalize(const double *partials, int n, double factor, double *E, double *scratch,
                            cudaStream_t st);

// Scalar-potential kernel setup (tensor.cu): octant of the cell kernel S at
// half-integer offsets [3][nz][ny][nx], its wrapped node grid, and the real
// tables T_j of its spectrum (phase exp(-pi i sum k/P) removed).
cudaError_t sp_octant(double *out, int nx, int ny, int nz, double dx, double dy, double dz, cudaStream_t st);
cudaError_t sp_wrap(const double *oct, int comp, int nx, int ny, int nz, int Px, int Py, int Pz, double *out,
                    cudaStream_t st);
cudaError_t sp_extract(const double2 *S, int comp, int Px, int Py, int Pz, int Kxp, double *t64, float *t32,
                       unsigned long long *imag_max, cudaStream_t st);

}  // namespace demag

// The opaque plan.
struct demag_plan {
    char last_err[320];  // message of the latest failed call on this plan (plain bytes: the struct is zeroed)
    int method;  // demag_method: DM (tensor) or SP (scalar potential)
    int nx, ny, nz;
    double dx, dy, dz;
    demag_prec prec;
    int Px, Py, Pz, Kx, Kxp;
    int device;
    size_t device_bytes;
    // spectra: S1 [3][nz][ny][Kxp], S2 [3][nz][Py][Kxp] (S2 == S1 when Py == 1)
    void *S1, *S2;
    // tensor spectrum [6][Pz/2+1][Py/2+1][Kx] (SP: kernel tables [3][...])
    double *nhat64;
    float *nhat32;
    // tile-ordered copy of nhat32 for the persistent TMA z pass (z variant 6;
    // FP32 tensor-method plans whose z length it supports), else null
    float *ntile;
    size_t ntile_bytes;
    // SP: half-sample phase factors exp(-pi i k / P) per axis, k < P
    double2 *ph64[3];
    float2 *ph32[3];
    // forward twiddle tables W_P^m, m < P, per axis
    double2 *tw64[3];
    float2 *tw32[3];
    // energy: per-block partial sums and plan-owned outputs
    double *partials;
    int npartials;
    double *e_dev;
    // host-buffer entry point buffers
    void *dM, *dH;
    // asynchronous host entry point: kAsyncSlots device slots, copy streams,
    // events (three slots: the upload of call n + 2 does not wait for the
    // download of call n, so uploads and downloads run at the same time)
    static constexpr int kAsyncSlots = 3;
    void *aM[kAsyncSlots], *aH[kAsyncSlots];
    double *aE[kAsyncSlots];  // per-slot energy of the streamed host entry
    cudaStream_t s_in, s_out;
    cudaEvent_t ev_in[kAsyncSlots], ev_done[kAsyncSlots], ev_out[kAsyncSlots];
    bool out_recorded[kAsyncSlots];
    int slot;
    bool async_ready;
    bool setup_done;
    double imag_max;
    // tuning choices (kernel variants), set by demag_autotune or defaults
    int zvariant;
    int yvariant;
    int xvariant;
    bool tuned;
    // energy without a field by the spectral (Parseval) sum where the z
    // length allows it (on by default; demag_set_spectral_energy)
    bool spectral_energy;
    // timing
    bool timing;
    void *ring;  // per-kernel timing events (api.cu)
    double pass_ms[8];
    long pass_n[8];
    long launches;
    // CUDA-graph replay of whole calls (api.cu): cache of captured pipelines
    bool use_graphs;
    void *graphs;
};
