/*
 * demag.h - C ABI of the GB300 (sm_103a) FFT demagnetization-tensor library.
 *
 * The library computes the micromagnetic stray field of the demagnetization-
 * tensor method (DM) of Abert et al., "Numerical Methods for the Stray-Field
 * Calculation" (arXiv 1204.4302):
 *
 *   H(r) = -sum_r' N(r - r') M(r')                         (Sec. 3.1, Eq. "demag")
 *
 * on a regular nx x ny x nz grid of cells of edges dx, dy, dz, evaluated as a
 * zero-padded 3-D FFT convolution (Sec. 3.1, Eq. "convolution": an element-
 * wise 3x3 matrix-vector product in Fourier space). N is the cell-averaged
 * demagnetization tensor (homogeneously magnetized cells, field averaged over
 * each cell, Sec. 5.1), positive definite at the origin with trace 1. The
 * paper writes H = N * M with the opposite sign convention for N; both
 * describe the same field.
 *
 * Conventions shared by all entry points
 *  - Layout: M, H and every other field are structure-of-arrays
 *    [3][nz][ny][nx], C order, x fastest, components (x, y, z).
 *  - Element type: float for DEMAG_F32 plans, double for DEMAG_F64 plans.
 *    DEMAG_F32 runs the FFTs and the spectral product in FP32 with an FP64
 *    tensor setup; DEMAG_F64 runs everything in FP64.
 *  - Units: M and H in A/m, energies in J, cell edges in m (any consistent
 *    length unit works for the field: N is dimensionless). mu0 = 4 pi 1e-7.
 *  - Pointers named "device" must be device memory of the plan's GPU, at
 *    least 16-byte aligned, not overlapping each other. The caller keeps
 *    ownership of every pointer it passes; the plan owns its own buffers.
 *  - Streams: a cudaStream_t passed as void*; NULL means the legacy default
 *    stream. Calls are asynchronous on that stream unless stated otherwise.
 *  - Errors: every call returns a status and never aborts. On failure a
 *    message is kept per thread, readable with demag_last_error(NULL). A plan is
 *    not thread safe: use one plan per host thread or serialise calls.
 */
#ifndef DEMAG_H
#define DEMAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct demag_plan *demag_plan_t;

typedef enum {
    DEMAG_OK = 0,
    DEMAG_ERR_INVALID_ARG = 1, /* bad size, null or misaligned pointer, aliasing */
    DEMAG_ERR_NOT_SETUP = 2,   /* demag_tensor_setup() has not run on this plan */
    DEMAG_ERR_OOM = 3,         /* device or pinned host allocation failed */
    DEMAG_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has it) */
    DEMAG_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    DEMAG_ERR_UNSUPPORTED = 6, /* size or option outside what is built */
    DEMAG_ERR_GUARD = 7        /* a guard zone of a debug allocation was overwritten */
} demag_status;

typedef enum { DEMAG_F32 = 0, DEMAG_F64 = 1 } demag_prec;

/* Stray-field method of a plan (paper Sec. 3.1): the demagnetization-tensor
 * convolution (DM) or the scalar-potential convolution with a finite-
 * difference gradient (SP). */
typedef enum { DEMAG_METHOD_DM = 0, DEMAG_METHOD_SP = 1 } demag_method;

/* Choice of padded lengths where demag_options leaves one at 0. */
typedef enum {
    DEMAG_PAD_POW2 = 0,   /* smallest power of two >= 2n - 1 */
    DEMAG_PAD_SMOOTH = 1, /* smallest even length >= 2n - 1 whose prime factors
                             are 2, 3, 5 and 7 (mixed-radix passes; DM only) */
    DEMAG_PAD_TUNED = 2   /* the lengths demag_tune_padding picks (DM only; the
                             plan creation then launches kernels and
                             synchronises, unless the choice is cached) */
} demag_pad_mode;

/* Optional plan settings; zero-initialise and set what you need. */
typedef struct {
    /* Padded FFT lengths per axis. 0 selects one by pad_mode (1 when n == 1).
     * An explicit length must be >= 2n - 1 and at most 1024: for DM plans a
     * power of two or an even product of 2, 3, 5 and 7; for SP plans a power
     * of two >= 2n. Every such period gives the same field up to rounding
     * (the zero-padded convolution is exact for each). Lengths that are not
     * powers of two run the mixed-radix passes. */
    int px, py, pz;
    int pad_mode; /* demag_pad_mode */
} demag_options;

/* Tensor-spectrum files: the one-time FP64 setup (Sec. 3.1: computed once per
 * geometry) written to disk and read back instead of recomputed.
 * demag_plan_save writes a set-up plan's method, precision, sizes, cell
 * edges, padded lengths and its spectrum tables (FP32 or FP64, the plan's
 * precision) with an FNV-1a checksum, in the byte order of the writing
 * machine; synchronises. DEMAG_ERR_NOT_SETUP before demag_tensor_setup.
 * demag_plan_load validates the whole file on the host (magic, version,
 * sizes, padded lengths, table size, checksum; DEMAG_ERR_INVALID_ARG with
 * the reason otherwise) before it touches a device, then creates the plan on
 * the current device ready to use (no demag_tensor_setup needed). */
demag_status demag_plan_save(demag_plan_t plan, const char *path);
demag_status demag_plan_load(const char *path, demag_plan_t *out);

/* Test hook for the error paths: with n >= 1 the n-th next device allocation
 * made by plan creation, tensor setup, the host-buffer entry points or the
 * autotuner fails as if the device were out of memory (the call returns
 * DEMAG_ERR_OOM and frees what it had allocated); 0 disarms it. */
void demag_debug_fail_alloc(long n);

/* Debug allocations: with DEMAG_DEBUG=1 in the environment, every device
 * buffer that plan creation, tensor setup, the host-buffer entry points or
 * the autotuner allocate gets a 4 KB guard zone before and after it, filled
 * with the byte 0xA5 (the buffer itself stays 256-byte aligned). A kernel
 * that writes past either end of such a buffer overwrites a guard byte;
 * demag_check_pipeline then scans the guard zones of every live debug
 * allocation (one kernel per zone) and returns DEMAG_ERR_GUARD naming the
 * first overwritten one. Reads past the ends are not detected. Without the
 * variable the allocations are plain. demag_debug_guard_count returns the
 * number of live debug allocations; demag_debug_poke_guard overwrites one
 * byte of the trailing guard zone of the most recent one from the host (a
 * test of the scan itself) and returns DEMAG_ERR_INVALID_ARG when there is
 * none. */
long demag_debug_guard_count(void);
demag_status demag_debug_poke_guard(void);

/* Sizes of a plan, as chosen at creation. */
typedef struct {
    int nx, ny, nz;          /* physical grid */
    int px, py, pz;          /* padded FFT lengths */
    int kx;                  /* px/2 + 1 stored x frequencies */
    int prec;                /* demag_prec */
    size_t device_bytes;     /* device memory held by the plan */
    int launches_per_field;  /* kernels one demag_field call launches */
    double tensor_imag_max;  /* largest |imaginary part| of the tensor spectrum
                                after setup (exactly 0 in exact arithmetic: the
                                wrapped tensor is even or odd per axis; for SP
                                plans, of the kernel tables after removing the
                                half-cell phase) */
    int method;              /* demag_method */
    double dx, dy, dz;       /* cell edges */
    int energy_in_z;         /* 1: a field call with the energy takes the
                                energy's spectral sum in its z pass (FP32
                                plan, persistent z form, z length 256 or 512,
                                spectral route on), so its last pass does not
                                read M; 0: the last pass sums M.H */
} demag_info;

/* Create a plan for an nx x ny x nz grid with cell edges dx, dy, dz.
 * Allocates the plan's device buffers on the current CUDA device (two
 * spectra, the tensor spectrum, twiddle tables); launches nothing.
 * Sizes: 1 <= n <= 512 per axis (padded length <= 1024).
 * Returns DEMAG_ERR_INVALID_ARG for non-positive sizes or edges,
 * DEMAG_ERR_UNSUPPORTED for sizes beyond the limit, DEMAG_ERR_OOM if the
 * device allocation fails. *out is NULL on failure. */
demag_status demag_plan_create(int nx, int ny, int nz, double dx, double dy, double dz,
                               demag_prec prec, demag_plan_t *out);

/* Padded lengths a DM plan of an nx x ny x nz grid takes with these options
 * (NULL: powers of two), written to P[0..2]; no device is touched. The same
 * argument checks as demag_plan_create_ex; DEMAG_PAD_TUNED returns
 * DEMAG_ERR_UNSUPPORTED (its lengths come from timing: demag_tune_padding). */
demag_status demag_padded_lengths(int nx, int ny, int nz, const demag_options *opt, int *P);

/* Same, with options (may be NULL). */
demag_status demag_plan_create_ex(int nx, int ny, int nz, double dx, double dy, double dz,
                                  demag_prec prec, const demag_options *opt,
                                  demag_plan_t *out);

/* Scalar-potential plan (paper Sec. 3.1, Eqs. "scpot", "convolution" and
 * "field"): the potential phi = S * M of the magnetization at the grid nodes
 * (cell corners), S(R) = (1/4pi) Int_cell grad_u (1/|R - u|) du the vector
 * kernel of one homogeneously magnetized cell, as a zero-padded FFT
 * convolution; then H = -grad phi per cell as the cell average of -grad of
 * the trilinear interpolant of the 8 corner potentials,
 *   H_x = -(1/(4 dx)) sum over the cell's 4 x-edges of phi(x+) - phi(x-)
 * (likewise y, z). This discretisation reproduces the SP energies the paper
 * prints for its cube and thin-film states. It costs one inverse transform
 * instead of three; the field is an approximation of the DM field with a
 * finite-difference error (largest at the surfaces).
 * Padded lengths: powers of two >= 2n (node-minus-cell offsets take 2n
 * values); opt (may be NULL) can ask for larger ones, or with pad_mode
 * DEMAG_PAD_SMOOTH for the smallest even lengths >= 2n with prime factors
 * 2, 3, 5, 7 (mixed-radix passes; explicit lengths may be either kind;
 * DEMAG_PAD_TUNED: DEMAG_ERR_UNSUPPORTED). Sizes: nx, ny <= 512, nz <= 256
 * (padded z <= 512). Same buffers and errors as demag_plan_create_ex.
 * Entry points that accept an SP plan: demag_tensor_setup (computes the
 * kernel spectrum), demag_field, demag_field_energy, demag_energy,
 * demag_field_host(_async), demag_sp_potential, demag_plan_info,
 * demag_autotune, timing and launch counts. demag_field_adjoint and
 * demag_energy_grad return DEMAG_ERR_UNSUPPORTED (the discrete SP operator is
 * not self-adjoint and its adjoint is not built); batches are DM only. In
 * FP32 the potential carries the FFT's rounding relative to its own size and
 * the differences divide it by one cell edge, so the field's rounding error
 * relative to its largest value is about eps32 log2(PxPyPz) A / 8, with
 * A = max|phi| / (max|H| min(d)): 4e-7 for a random 256^3 state (A = 1.4),
 * 2e-5 for a uniformly magnetized 256^3 cube (A = 55). */
demag_status demag_plan_create_sp(int nx, int ny, int nz, double dx, double dy, double dz,
                                  demag_prec prec, const demag_options *opt, demag_plan_t *out);

/* Node potential of an SP plan: phi[nz+1][ny+1][nx+1] (device, element type
 * of the plan, node (i, j, k) at (i dx, j dy, k dz) from the grid's corner,
 * x fastest), phi = S * M (paper Eq. "scpot"; units of M times length). phi
 * must not overlap M. DEMAG_ERR_INVALID_ARG for a DM plan. Asynchronous. */
demag_status demag_sp_potential(demag_plan_t plan, const void *M, void *phi, void *stream);

/* Tensor setup, once per geometry (paper Sec. 4: the convolution kernel
 * depends only on geometry and discretisation). Evaluates the six tensor
 * components N_xx..N_yz in FP64 on the device for every offset of the grid
 * (closed form for touching cells, Gauss-Legendre quadrature of the point
 * kernel at intermediate range, a multipole expansion of the cell average
 * far away), places them at wrapped offsets of the padded grid and stores
 * the (real) 3-D spectrum. Allocates and frees temporary device memory;
 * blocks until done. Idempotent. */
demag_status demag_tensor_setup(demag_plan_t plan, void *stream);

/* H = -N * M (paper Sec. 3.1, Eq. "demag"). M, H: device, [3][nz][ny][nx] of
 * the plan's element type; H must not alias M. Needs demag_tensor_setup().
 * Asynchronous: launches demag_info.launches_per_field kernels on stream. */
demag_status demag_field(demag_plan_t plan, const void *M, void *H, void *stream);

/* Adjoint of M -> H applied to G (same layout). The tensor is symmetric
 * (N_ij = N_ji) and even (N(-r) = N(r)), so the operator is self-adjoint and
 * this equals demag_field(G). Used for gradients: d/dM of sum(G . H(M)). */
demag_status demag_field_adjoint(demag_plan_t plan, const void *G, void *out, void *stream);

/* Field and energy E = -(mu0/2) V sum_cells M.H (paper Sec. 2, the stray-
 * field energy, in SI units; V = dx dy dz). H: device output as above.
 * E_dev: device pointer to one double receiving E. The per-block partial sums
 * are formed in the field's last pass (sum of M.H), or, where
 * demag_info.energy_in_z says so, in its z pass as the spectral sum of
 * demag_energy (equal up to rounding: Parseval's identity), and summed in
 * FP64 with compensation. Asynchronous. */
demag_status demag_field_energy(demag_plan_t plan, const void *M, void *H, double *E_dev,
                                void *stream);

/* Energy only: computes E for M without storing H, synchronises the stream
 * and writes E to *E_out (host). By default (demag_set_spectral_energy) the
 * energy is taken in Fourier space (Parseval's identity applied to the
 * paper's Sec. 2 energy: E = (mu0/2) (V / (Px Py Pz)) sum_k w(kx) M^H N^ M
 * over the half spectrum, w = 1 for kx = 0 and kx = Px/2, else 2), in the z
 * pass right after the forward transforms, so the inverse passes do not run;
 * plans whose z length has no spectral form (1024, lengths that are not
 * powers of two) run the field pipeline and sum M.H in its last pass. */
demag_status demag_energy(demag_plan_t plan, const void *M, double *E_out, void *stream);

/* Route of energies computed without a field (demag_energy, and
 * demag_energy_grad with G = NULL): enable != 0 (the default) takes the
 * spectral sum where the plan allows it, 0 always runs the field pipeline.
 * Both give E within rounding; the spectral route skips the y and x inverse
 * passes. The same switch decides whether field calls with the energy take
 * the spectral sum in the persistent z pass (demag_info.energy_in_z) or the
 * sum of M.H in their last pass. Tensor-method plans only (scalar-potential
 * plans always run their own pipeline). */
demag_status demag_set_spectral_energy(demag_plan_t plan, int enable);

/* Energy and its gradient for a magnetization given as M = Ms * w * m, with m
 * the reduced magnetization [3][nz][ny][nx] (device), w an optional per-cell
 * weight [nz][ny][nx] (device, e.g. a 0/1 mask of the body; NULL = 1) and Ms
 * the saturation magnetization (A/m). All in the same kernels as the field:
 *   E    = -(mu0/2) V sum M.H                       (paper Sec. 2)
 *   grad = g * dE/dm = -g mu0 V Ms w H               (the operator is
 *          self-adjoint, so the adjoint of the field map is the field map)
 * E_dev (device double) and grad (device, layout of m, not aliasing m or w)
 * are each optional but not both NULL. gscale_dev: optional device double g
 * (the upstream gradient of E); NULL means g = 1. Asynchronous. */
demag_status demag_energy_grad(demag_plan_t plan, const void *m, const void *w, double Ms,
                               double *E_dev, void *grad, const double *gscale_dev, void *stream);

/* End-to-end call with host buffers: copies M (host, [3][nz][ny][nx]) to the
 * device, computes H and copies it back to H_host, then synchronises the
 * stream. Page-locked host memory gives full copy bandwidth; pageable memory
 * works too. Uses plan-owned device buffers allocated at the first call. */
demag_status demag_field_host(demag_plan_t plan, const void *M_host, void *H_host, void *stream);

/* Streaming variant of demag_field_host for sequences of host-resident
 * states: returns without synchronising. The upload runs on a copy stream,
 * the field on `stream`, the download on a second copy stream, through three
 * rotating device slots, so consecutive calls overlap one call's download
 * and a later call's upload with each other and with the fields. The caller
 * must keep M_host unchanged and must not read H_host until
 * demag_host_wait() returns; page-locked buffers are needed for the copies
 * to overlap. Device buffers (three input and three output fields) are
 * allocated at the first call. */
demag_status demag_field_host_async(demag_plan_t plan, const void *M_host, void *H_host, void *stream);

/* Same, with the energy E = -(mu0/2) V sum M.H of each call written to
 * *E_host (a host double, page-locked for the copies to overlap), valid after
 * demag_host_wait() like H_host. E_host NULL: as demag_field_host_async. */
demag_status demag_field_energy_host_async(demag_plan_t plan, const void *M_host, void *H_host, double *E_host,
                                           void *stream);

/* Waits for every upload and download issued by demag_field_host_async and
 * demag_field_energy_host_async. */
demag_status demag_host_wait(demag_plan_t plan);

/* Plan sizes and memory. */
demag_status demag_plan_info(demag_plan_t plan, demag_info *info);

/* Per-kernel timing of the field pipeline with CUDA events recorded on the
 * launch stream around each kernel (off by default). demag_get_timing fills
 * ms[i] with the summed milliseconds of pass i and counts[i] with its number
 * of launches since the last reset, for i < n (n <= 8; pass order: x forward,
 * y forward, z convolution, y inverse, x inverse, energy finalise). Reading
 * synchronises on the recorded events. */
demag_status demag_set_timing(demag_plan_t plan, int enable);
demag_status demag_get_timing(demag_plan_t plan, double *ms, long *counts, int n);

/* Energy E = -(mu0/2) dx dy dz sum M.H of a field pair the caller already
 * holds, without any memory allocation. The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory where they
 * need the energy, for example code that runs while a stream is captured
 * into a CUDA graph in the global capture mode (where cudaMalloc is
 * illegal), hosts that hand out device memory only through their own pool,
 * and tight loops in which an allocation, which can synchronise the device,
 * is not acceptable. No plan is needed.
 *   nx, ny, nz, dx, dy, dz: grid and cell edges (V = dx dy dz);
 *   prec: element type of M and H (DEMAG_F32 float, DEMAG_F64 double);
 *   M, H: device, [3][nz][ny][nx], 16-byte aligned, on the current device;
 *   E_dev: device double receiving E (8-byte aligned).
 * The per-block partial sums live in one fixed 512 KB device array owned by
 * the library (a file-scope __device__ array that every GPU loading the
 * library holds until the process exits). It fits 3 nx ny nz <= 65536 * 8192
 * values (178956970 cells); larger grids return DEMAG_ERR_UNSUPPORTED.
 * Every call on a device shares that array and leaves its last contents
 * there; each call overwrites every slot it reads, so nothing needs clearing.
 * Calls that overlap on the GPU (e.g. on two streams at once) race on it:
 * order them on one stream or with events.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and may load the
 * library's kernels; make that first call before any stream capture. The
 * address is kept per device together with the id of the device's context,
 * and looked up again (the next call doing the set-up once more) after the
 * context changed, e.g. after cudaDeviceReset.
 * Asynchronous; no cudaMalloc, cudaFree or other allocating call.
 * Returns DEMAG_ERR_INVALID_ARG for bad sizes, precision or pointers,
 * DEMAG_ERR_UNSUPPORTED beyond the capacity (checked before any product of
 * the sizes is formed) and DEMAG_ERR_CUDA if the set-up or one of its own
 * launches fails; an error left pending by earlier, unrelated work is not
 * reported as this call's failure and is not cleared. demag_last_error(NULL) is
 * not updated by this call. */
demag_status demag_energy_noalloc(int nx, int ny, int nz, double dx, double dy, double dz,
                                  demag_prec prec, const void *M, const void *H, double *E_dev,
                                  void *stream);

/* ------------------------------------------------------------------ batches
 * Many independent magnetization states on grids of uneven sizes, evaluated
 * together (each state is one DM stray-field problem of paper Sec. 3.1 with
 * its own geometry and tensor). */
typedef struct demag_batch *demag_batch_t;

/* n states; dims: 3n ints (nx, ny, nz per state); cells: 3n doubles (dx, dy,
 * dz). Creates one plan per state and runs every tensor setup (blocking),
 * then prepares the persistent batch kernel when the precision is DEMAG_F32
 * and every padded length is supported by it (x: 32..1024, y: 8..512,
 * z: 4..256); otherwise the batch uses branch mode. */
demag_status demag_batch_create(int n, const int *dims, const double *cells, demag_prec prec,
                                demag_batch_t *out);

/* Same, with the padding of every state chosen by opt->pad_mode (px, py, pz
 * must be 0; NULL = powers of two). States whose lengths are not all powers
 * of two run in branch mode. DEMAG_PAD_TUNED runs demag_tune_padding (cached)
 * per state. */
demag_status demag_batch_create_ex(int n, const int *dims, const double *cells, demag_prec prec,
                                   const demag_options *opt, demag_batch_t *out);

/* Fields and energies of all states. M, H: arrays of n device pointers
 * ([3][nz][ny][nx] per state, 16-byte aligned, H[i] not overlapping M[i]).
 * E_dev: optional device array of n doubles receiving each state's energy.
 * Mode 0 (persistent): one CUDA-graph launch holding a counter reset and one
 * persistent kernel that works through all (pass, state, tile) items; its
 * dependency waits are bounded (see demag_batch_set_timeout), and a wait
 * that runs out is reported by demag_batch_status. Mode 1 (branches): one
 * CUDA-graph launch of the per-state pipelines as independent branches. The
 * graphs are built at the first call and rebuilt when the pointers change.
 * Asynchronous. */
demag_status demag_batch_field(demag_batch_t batch, const void *const *M, void *const *H, double *E_dev,
                               void *stream);

/* 0 = persistent kernel, 2 = pass-batched launches (one launch per pass
 * over all states, the six captured in one graph; the default where
 * available), both DEMAG_ERR_UNSUPPORTED if the batch's sizes are outside
 * their tile functions (FP32, power-of-two lengths, x <= 1024, y <= 512,
 * z <= 256); 1 = graph of per-state branches. */
demag_status demag_batch_set_mode(demag_batch_t batch, int mode);

/* Per-pass timing of the pass-batched mode: with enable != 0 each call
 * launches the six passes directly with a CUDA event around each and waits
 * for them; demag_batch_get_timing adds up ms[k] per pass (k: x forward,
 * y forward, z, y inverse, x inverse, energy) over *calls calls since the
 * last demag_batch_set_timing. Other modes do not record. */
demag_status demag_batch_set_timing(demag_batch_t batch, int enable);
demag_status demag_batch_get_timing(demag_batch_t batch, double *ms, long *calls);

/* Limit of each dependency wait of the persistent kernel, in seconds of GPU
 * clock (default about 2 s; normal waits take microseconds). stall_state >= 0
 * is a test hook: that state's first pass is made to look one tile short, so
 * its waiters run out of time; -1 restores normal operation. */
demag_status demag_batch_set_timeout(demag_batch_t batch, double seconds, int stall_state);

/* Synchronises the stream and reports DEMAG_ERR_TIMEOUT if a wait of the
 * persistent kernel gave up since the last status call (then clears it). */
demag_status demag_batch_status(demag_batch_t batch, void *stream);

/* Mode in use, whether the persistent kernel is available, its work items,
 * grid size and dynamic shared memory (any pointer may be NULL). */
demag_status demag_batch_info(demag_batch_t batch, int *mode, int *persistent_ok, int *items, int *grid,
                              size_t *smem);

/* Autotunes every state's plan (demag_autotune), then times the persistent
 * and the branch mode on temporary fields and keeps the faster mode.
 * ms_persistent / ms_branches (may be NULL) receive the time per call of each
 * mode (-1 when the persistent mode is unavailable). Synchronises. */
demag_status demag_batch_autotune(demag_batch_t batch, int use_cache, double *ms_persistent,
                                  double *ms_branches, void *stream);

/* Padding autotuner of a batch created with power-of-two or smooth padding
 * (demag_batch_create[_ex] with pad_mode 0 or 1): runs demag_batch_autotune,
 * builds and autotunes the same states with the other padding, and keeps the
 * faster of the two (rebuilding the batch's plans in place when the other
 * wins; the handle stays valid, graphs are rebuilt at the next call, and a
 * timeout set with demag_batch_set_timeout returns to its default).
 * ms_pow2 / ms_smooth (may be NULL) receive the best time per call of each.
 * DEMAG_ERR_UNSUPPORTED for a batch created with DEMAG_PAD_TUNED.
 * Synchronises. */
demag_status demag_batch_autotune_padding(demag_batch_t batch, int use_cache, double *ms_pow2, double *ms_smooth,
                                          void *stream);

/* Graph launches made by this batch. */
long demag_batch_launch_count(demag_batch_t batch);

void demag_batch_destroy(demag_batch_t batch);

/* Number of kernels this plan has launched since creation. */
long demag_launch_count(demag_plan_t plan);

/* CUDA-graph replay (default off). When on, each distinct call of this plan
 * (the same pointers, scales and kernel variants) is captured once into a
 * CUDA graph on a private stream and later calls replay it with one graph
 * launch on the caller's stream; up to 4 calls are kept (least recently used
 * evicted). Results are the same; small grids, whose calls are bound by
 * launch overhead, get faster. Calls with per-kernel timing on, and the
 * autotuner's timings, launch directly. Disabling frees the graphs. */
demag_status demag_set_graphs(demag_plan_t plan, int enable);

/* Autotuner: times the kernel variants that exist for this plan's sizes (the
 * z-, y- and x-pass forms, demag_set_variants) with CUDA events on the plan's
 * own sizes (five timed field + energy calls after two warm-up calls each, on
 * stream: the x-inverse forms differ most in the energy's epilogue) and keeps
 * the fastest. With use_cache != 0 a previous result for the same GPU,
 * precision and sizes is reused from the cache file (DEMAG_TUNE_CACHE,
 * default $HOME/.cache/demag_tune.txt) and a new result is appended to it.
 * best_ms (may be NULL) receives the time of one field + energy call with the
 * chosen variants. Allocates and frees two temporary fields; synchronises. */
demag_status demag_autotune(demag_plan_t plan, int use_cache, double *best_ms, void *stream);

/* Padding autotuner for DM plans of an nx x ny x nz grid. Every axis can be
 * padded to the smallest power of two >= 2n - 1 or to the smallest even
 * length >= 2n - 1 with prime factors 2, 3, 5, 7 (mixed-radix passes); the
 * field is the same up to rounding. Each distinct combination (at most 8)
 * is created, autotuned (demag_autotune) and timed on the current device
 * (with a zero tensor spectrum: the passes do the same work whatever it
 * holds, and no FP64 tensor setup is spent on plans that are only timed); the fastest lengths are written to best->px, py, pz (pad_mode 0).
 * ms_best / ms_pow2 (may be NULL) receive the time per field call of the
 * chosen and of the all-power-of-two lengths. use_cache != 0 reuses and
 * appends results in the autotuner's cache file, keyed by GPU, precision and
 * sizes. Errors as demag_plan_create_ex and demag_tensor_setup. Synchronises. */
demag_status demag_tune_padding(int nx, int ny, int nz, double dx, double dy, double dz, demag_prec prec,
                                int use_cache, demag_options *best, double *ms_best, double *ms_pow2,
                                void *stream);

/* Current variant choice, and a way to set it by hand.
 * z: 0 = two-stage fused pass, 1 = half-width tile, 2 = 256-thread tile
 *    (z length 512 only), 3 = persistent pipelined pass (z lengths 64..512),
 *    4 = variant 0's layout on half the columns with two CTAs per SM,
 *    5 = persistent CTAs whose input columns arrive by TMA tensor copies
 *    while the previous tile is transformed (z lengths 32..512; the
 *    autotuner tries it up to 256, where it is the fastest),
 *    6 = FP32 only: one persistent CTA per SM streams 8-column tiles whose
 *    input rows arrive by a TMA tensor copy and whose tensor block arrives by
 *    one bulk copy from a tile-ordered copy of the tensor spectrum (built at
 *    setup, about the size of the spectrum), both one tile ahead; the
 *    length-512 transforms run as 2 x 16 x 16 with packed FP32x2 butterflies
 *    (z length 512, at most 256 input rows), 7 = as 6 with 4-column tiles and
 *    two CTAs per SM, 8 = variant 0 with an 8-point second stage (8 complex
 *    values per component and thread across the product, half the registers
 *    and shared memory) and two CTAs per SM (z lengths 32..128).
 * y: 0 = two-stage column transform, 1 = swapped radix order (y lengths 32,
 *    128, 512), 2 = three-stage transform with more CTAs per SM (y lengths
 *    512 and 1024), 3 = as 2, with the forward pass by persistent CTAs that
 *    receive their column tiles by TMA tensor copies (two tiles in flight).
 *    A variant that does not exist for the plan's lengths runs as variant 0.
 *    Out-of-range values: DEMAG_ERR_INVALID_ARG. */
demag_status demag_get_variants(demag_plan_t plan, int *z, int *y);
demag_status demag_set_variants(demag_plan_t plan, int z, int y);

/* x-pass variant: 0 = one CTA per tile of rows; 1 (default) = the forward
 * pass by persistent CTAs that stream their row tiles through shared memory
 * with bulk asynchronous copies (TMA) on mbarriers, two tiles in flight, where
 * the rows are contiguous 16-byte multiples (nx % 4 == 0, no cell weight),
 * else as 0; 2 = the inverse pass pipelined the same way too. The autotuner
 * times all three. Out-of-range x: DEMAG_ERR_INVALID_ARG. */
demag_status demag_get_x_variant(demag_plan_t plan, int *x);
demag_status demag_set_x_variant(demag_plan_t plan, int x);

/* The pipelined x passes wait for their bulk copies with a bound (about two
 * seconds); if a wait gives up, the kernel waits (bounded) for its copies in
 * flight, records the failure and returns, leaving that call's output
 * incomplete. This call synchronises the device and returns
 * DEMAG_ERR_TIMEOUT if that happened since the last check (and clears it);
 * with debug allocations live (DEMAG_DEBUG=1, see demag_debug_guard_count) it
 * then scans their guard zones and returns DEMAG_ERR_GUARD if one was
 * overwritten; else DEMAG_OK. */
demag_status demag_check_pipeline(demag_plan_t plan);

/* ------------------------------------------------------------------------
 * Tensor-grid method (TG, paper Sec. 3.2) for magnetization in CP format
 * (App. A): M^(p)[k][j][i] = sum_m lam[p][m] Ux[p][m][i] Uy[p][m][j] Uz[p][m][k].
 * The potential at the cell centres is the block sum of mode products of
 * Eq. "sumpot": 1/|r|^3 written as a Gaussian integral (Eq. "transform") and
 * integrated by a sinc rule in t (tau = e^t; rule error ~1e-15 for FP64
 * plans, ~2e-9 for FP32 plans), with the Gaussian matrices of Eqs. "Dmat"
 * and "gs" in closed form (FP64 setup). The field is H = -grad Phi by
 * second-order differences (central inside, one-sided at the first and last
 * cell of each axis), and the energy is E = -(mu0/2) V sum M.H with M rebuilt
 * from its factors. Cost per call: O(R r (nx^2 + ny^2 + nz^2)) for the
 * factors and O(R r nx ny nz) for the dense potential (R sinc terms), instead
 * of a convolution over the padded grid. */
typedef struct demag_tg_plan *demag_tg_plan_t;

/* Plan for an nx x ny x nz grid (3..512 per axis: the differences need three
 * cells) of edges dx, dy, dz and CP rank 1..64. Computes the sinc rule and
 * the Gaussian tables on the device (FP64, stored in the plan's precision)
 * and synchronises. Errors as demag_plan_create. */
demag_status demag_tg_plan_create(int nx, int ny, int nz, double dx, double dy, double dz, int rank,
                                  demag_prec prec, demag_tg_plan_t *out);

/* Field and/or energy of a CP magnetization. lam: device [3][rank]; Ux:
 * device [3][rank][nx]; Uy: [3][rank][ny]; Uz: [3][rank][nz] (plan element
 * type, A/m carried by lam). H: device [3][nz][ny][nx] or NULL; E_dev: device
 * double or NULL (not both NULL). Asynchronous on stream. */
demag_status demag_tg_field_cp(demag_tg_plan_t plan, const void *lam, const void *Ux, const void *Uy,
                               const void *Uz, void *H, double *E_dev, void *stream);

/* The cell-centre potential phi [nz][ny][nx] (device) of a CP magnetization. */
demag_status demag_tg_potential_cp(demag_tg_plan_t plan, const void *lam, const void *Ux, const void *Uy,
                                   const void *Uz, void *phi, void *stream);

/* Tucker input (App. A): M^(p)[k][j][i] = sum_{a,b,c} G[p][c][b][a] A[p][a][i]
 * B[p][b][j] C[p][c][k]. Mode products pass a Tucker tensor factor by factor,
 * G x_1 (D_1 A) x_2 (D_2 B) x_3 (D_3 C), so the potential of Eq. "sumpot" is
 * the same dense contraction with first operand
 * Q[(k,j)][(l,p,a)] = sum_{b,c} G[p][c][b][a] (D_2 B)[(l,p,b)][j] (D_3 C)[(l,p,c)][k]
 * (formed once per call, nz ny x 3 R r1 values) and the x factors
 * (D_1 A)[(l,p,a)][i]. Plans for Tucker ranks r1, r2, r3 (1..16 each);
 * otherwise as demag_tg_plan_create. G: device [3][r3][r2][r1]; A [3][r1][nx],
 * B [3][r2][ny], C [3][r3][nz] (plan element type, A/m carried by G). A
 * Tucker plan takes only the _tucker calls, a CP plan only the _cp calls. */
demag_status demag_tg_plan_create_tucker(int nx, int ny, int nz, double dx, double dy, double dz, int r1, int r2,
                                         int r3, demag_prec prec, demag_tg_plan_t *out);
demag_status demag_tg_field_tucker(demag_tg_plan_t plan, const void *G, const void *A, const void *B, const void *C,
                                   void *H, double *E_dev, void *stream);
demag_status demag_tg_potential_tucker(demag_tg_plan_t plan, const void *G, const void *A, const void *B,
                                       const void *C, void *phi, void *stream);

/* The dense contraction Phi[k][j][i] = sum_K Z[K][k] Y[K][j] X[K][i] over the
 * K = 3 R rank terms (the transformed factors of Eq. "sumpot"), a GEMM of
 * nz ny rows by nx columns whose first operand is formed on the fly.
 * contraction 1 (the default of FP32 plans): on the tensor cores (tcgen05,
 * TF32 operands in shared memory, FP32 accumulators in tensor memory), each
 * product a b taken as a_hi b_hi + a_hi b_lo + a_lo b_hi with a = a_hi + a_lo
 * split into TF32 parts, which keeps FP32 accuracy. contraction 0: FP32 or
 * FP64 on the CUDA cores (the only form of FP64 plans;
 * DEMAG_ERR_UNSUPPORTED when 1 is asked of one). */
demag_status demag_tg_set_contraction(demag_tg_plan_t plan, int contraction);
demag_status demag_tg_get_contraction(demag_tg_plan_t plan, int *contraction);

/* Per-stage timing of TG calls: with enable != 0 each call records CUDA
 * events on its stream around (0) the factor transforms, (1) the operand
 * preparation of the tensor-core contraction (transposes, TF32 split; empty
 * for contraction 0), (2) the contraction, (3) the differences and energy,
 * and waits for them; demag_tg_get_timing adds up ms[0..3] over *calls
 * calls since the last demag_tg_set_timing. */
demag_status demag_tg_set_timing(demag_tg_plan_t plan, int enable);
demag_status demag_tg_get_timing(demag_tg_plan_t plan, double *ms, long *calls);

/* The tensor-core contraction waits for its operand copies and MMAs with a
 * bound (about two seconds); if a wait gives up, the kernel drains what it
 * has in flight (bounded), frees its tensor memory and returns, leaving
 * that call's potential incomplete. Synchronises the stream and returns
 * DEMAG_ERR_TIMEOUT if that happened since the last call (then clears it),
 * else DEMAG_OK. */
demag_status demag_tg_status(demag_tg_plan_t plan, void *stream);

/* ------------------------------------------------------------------------
 * Low-rank magnetization (paper Sec. 3.2, "Low-Rank Magnetization"): each
 * component M^(p) [nz][ny][nx] approximated in CP or Tucker format by
 * alternating least squares (the ALS algorithms of Kolda and Bader's tensor
 * survey, which the paper uses for both), FP64, with the relative error of
 * Eq. "relr" (Frobenius norms over the three components). The initial
 * guesses are the caller's (the paper starts from random ones). Both calls
 * allocate their workspace, run on stream and synchronise it.
 *
 * CP-ALS: per component, `iters` sweeps of the mode updates x, y, z:
 *   A <- X_(x) (C kr B) V^+, V = (C^T C) * (B^T B) (Hadamard product),
 *   lambda <- the column 2-norms, A <- A / lambda (likewise B, then C),
 * V^+ the pseudo-inverse of the symmetric V (eigenvalues at or below 1e-12 of
 * the largest dropped, so ranks beyond what the tensor holds stay defined).
 * M: device double [3][nz][ny][nx]; Ux [3][rank][nx], Uy [3][rank][ny],
 * Uz [3][rank][nz]: device double, the initial factors on entry (only Uy and
 * Uz are read) and the normalised factors on return; lam: device double
 * [3][rank] out; relerr: device double or NULL. These are the CP factors the
 * TG entry points take. Grids 1..512 per axis, rank 1..64. */
demag_status demag_cp_als(int nx, int ny, int nz, const double *M, int rank, int iters, double *lam, double *Ux,
                          double *Uy, double *Uz, double *relerr, void *stream);

/* Tucker-ALS (higher-order orthogonal iteration): per component, `iters`
 * sweeps of A <- the r1 leading left singular vectors of
 * (X x_y B^T x_z C^T)_(x), then B and C likewise, and the core
 * G = X x_x A^T x_y B^T x_z C^T. A [3][r1][nx], B [3][r2][ny], C [3][r3][nz]:
 * device double, the initial factors on entry (only B and C are read) and
 * orthonormal factors on return (a direction the tensor does not hold comes
 * back as zeros); G: device double [3][r3][r2][r1] out. Ranks 1..16, at most
 * the axis length; iters >= 1. */
demag_status demag_tucker_als(int nx, int ny, int nz, const double *M, int r1, int r2, int r3, int iters,
                              double *G, double *A, double *B, double *C, double *relerr, void *stream);

/* Sinc terms R, device memory held, kernels launched so far (any may be NULL). */
demag_status demag_tg_plan_info(demag_tg_plan_t plan, int *sinc_terms, size_t *device_bytes, long *launches);

void demag_tg_plan_destroy(demag_tg_plan_t plan);

/* Destroy a plan and free its device memory (NULL is ignored). */
void demag_plan_destroy(demag_plan_t plan);

/* Error messages: with plan == NULL, the calling thread's latest one (any
 * entry point, plan-less calls included); with a plan, the latest failed call
 * on that plan ("" if none). */
const char *demag_last_error(demag_plan_t plan);

/* Name of a status code. */
const char *demag_status_string(demag_status s);

#ifdef __cplusplus
}
#endif
#endif /* DEMAG_H */
