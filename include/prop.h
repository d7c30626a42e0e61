/*
 * prop.h -- C ABI of the GB300 (sm_103a) volumetric PROPELLER library.
 *
 * The method (Ghosh, Wetzstein, Pilanci, Fridovich-Keil, CVPR 2024) lifts a
 * 2-D image to a complex volume V(x, f) over space and a spectral axis
 * (Sec. 4.1) so that off-resonance becomes a per-bin translation along each
 * blade's readout direction (Sec. 3, Eq. 2).  Blade b then measures
 *
 *     y_b(k) = s * sum_f sum_x V_t(b)(x, f) exp(-2 pi i k.(x + Delta_f d_b)),
 *
 * with s = 1/N, x on the integer grid {-N/2..N/2-1}^2, d_b = (cos th_b,
 * sin th_b), and k on the blade's rotated Cartesian lines
 * k = k_r d_b + k_p d_b^perp, k_r = (j - R/2)/N, k_p = (l - L/2)/N
 * (Sec. 4.2 "Blur" samples the Fourier transform on the blade; Sec. 7
 * "Limitations" asks for the non-uniform, blade-aligned version computed
 * here).  The volume is recovered by Adam (Sec. 4.3) on
 *     L(V) = sum |A V - y|^2 + tv_xy TV_xy(V) + tv_t TV_t(V),
 * TV smoothed and anisotropic: sum sqrt(|d|^2 + tv_eps^2) over forward
 * differences d along x1, x2 (TV_xy) and frames (TV_t), no wrap-around.
 *
 * The operator is evaluated by a Kaiser-Bessel NUFFT (oversampling 2, kernel
 * width 6): deapodise, zero-pad to 2N x 2N, 2-D FFT per spectral bin, then a
 * 6x6-tap interpolation at every blade sample fused with the displacement
 * phase exp(-2 pi i k_r Delta_f) and the sum over bins.  Its relative error
 * against the exact sum is about 1e-5; A^H is the exact adjoint of the
 * approximate A (same tables), so <A x, y> = <x, A^H y> to FP32 rounding.
 *
 * Layouts (row-major, interleaved complex64 = two floats re, im):
 *   V      [T][N][N][Nf]   index ((t*N + i2)*N + i1)*Nf + f, x_a = i_a - N/2
 *   y, r   [B][L][R]       index (b*L + l)*R + j
 *   image  [T][N][N]
 *
 * Conventions for every call:
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls on device buffers return
 *     without synchronising unless stated.
 *   - `*_dev` pointers are device memory owned by the caller, 16-byte
 *     aligned, on the plan's device.  `*_host` pointers are host memory owned
 *     by the caller.
 *   - Argument errors are detected on the host before any work is enqueued
 *     and return PROP_ERR_INVALID_ARG.  CUDA errors return PROP_ERR_CUDA;
 *     an asynchronous fault of an earlier call surfaces at a later call.
 *     Nothing aborts or throws across the ABI; prop_last_error() gives a
 *     message for the last non-OK status of the calling thread.
 *   - A plan owns its device tables and workspace.  Calls on one plan must
 *     not overlap in time (one stream at a time); different plans are
 *     independent.  The caller's current CUDA device is restored on return.
 */
#ifndef PROP_H
#define PROP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PROP_API __attribute__((visibility("default")))
#else
#define PROP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum prop_status {
  PROP_OK = 0,
  PROP_ERR_INVALID_ARG = 1,
  PROP_ERR_OOM = 2,
  PROP_ERR_CUDA = 3,
  PROP_ERR_TIMEOUT = 4,
  PROP_ERR_BUSY = 5,
  PROP_ERR_NOT_READY = 6,
  PROP_ERR_CANCELLED = 7,
  PROP_ERR_UNIMPLEMENTED = 8
} prop_status;

typedef struct prop_plan_s* prop_plan;

/* Problem geometry.  All arrays are host memory, read during plan creation
 * only (the plan keeps its own copies). */
typedef struct prop_plan_desc {
  int n;                  /* image size N: multiple of 8, 16 <= N <= 512, 2N = 2^a 3^b */
  int nf;                 /* spectral bins Nf >= 1 */
  const double* delta;    /* [nf] displacement Delta_f of each bin, pixels along readout */
  int nblades;            /* B >= 1 */
  const double* theta;    /* [nblades] blade angles th_b, radians */
  int lines;              /* L >= 1, lines per blade */
  int readout;            /* R >= 1, samples per line */
  int nframes;            /* T >= 1 (1 = static) */
  const int* blade_frame; /* [nblades] frame t(b) in [0, T), or NULL = all frame 0 */
  int kb_width;           /* Kaiser-Bessel width: 0 (= 6), 6, or 8 (two orders of magnitude more
                             accurate operator, 64 instead of 36 taps per sample) */
  int bin_chunk;          /* bins per oversampled-grid pass: 0 = auto (min(Nf, 64)), else 1..64.
                             Smaller chunks recompute the grid per chunk in less memory. */
  int row_kernel;         /* row kernel of prop_reconstruct / prop_recon_step (single bin chunk):
                             0 = auto, 1 = one CTA per (image row, 16 bins),
                             2 = persistent warp-specialised (the update of one row overlaps
                             the row FFTs of its neighbours; needs 2N <= 512 and a bin stride
                             that is a multiple of 16, else plan creation fails).
                             Auto takes 2 when it is possible and there are at least 8
                             (row, 16-bin) units per SM, else 1.  Same iterates either way. */
  int device;             /* CUDA device ordinal */
} prop_plan_desc;

/* Adam + regulariser settings of prop_reconstruct (Sec. 4.3). */
typedef struct prop_recon_params {
  int iters;              /* K >= 0 Adam iterations */
  float lr, beta1, beta2, eps;   /* Adam (Kingma & Ba, bias-corrected, per real component) */
  float tv_xy, tv_t, tv_eps;     /* TV weights and smoothing epsilon (> 0) */
} prop_recon_params;

/* Build the plan: sample positions, Kaiser-Bessel weights and grid indices,
 * displacement phase table (arguments range-reduced in FP64), deapodisation
 * and FFT twiddle tables (FP64 -> FP32), the interpolation work items and
 * the spread's gather lists (balanced over the SMs), the column passes' TMA
 * tensor maps, and the device workspace.  Allocates device memory (PROP_ERR_OOM on failure).
 * On success *out receives a handle to free with prop_plan_destroy. */
PROP_API prop_status prop_plan_create(const prop_plan_desc* desc, prop_plan* out);

/* Free the plan and all its device memory (synchronises its device). NULL is a no-op. */
PROP_API prop_status prop_plan_destroy(prop_plan plan);

/* Device bytes the plan holds once prop_reconstruct has run on it (tables +
 * grid workspace + optimiser state); used for admission control. */
PROP_API prop_status prop_plan_workspace_bytes(prop_plan plan, size_t* bytes);

/* y = A V (the forward operator above).  V_dev [T][N][N][Nf] complex64 in,
 * y_dev [B][L][R] complex64 out.  Uses the plan's grid workspace. */
PROP_API prop_status prop_forward(prop_plan plan, const void* V_dev, void* y_dev, void* stream);

/* V = A^H y (the exact adjoint of prop_forward; no factor 2).
 * y_dev [B][L][R] complex64 in, V_dev [T][N][N][Nf] complex64 out. */
PROP_API prop_status prop_adjoint(prop_plan plan, const void* y_dev, void* V_dev, void* stream);

/* K full-batch Adam iterations on L(V) starting from V_dev (in/out).
 * Iteration k (1-based) evaluates L and its gradient
 *   2 A^H (A V_{k-1} - y) + tv_xy grad TV_xy + tv_t grad TV_t
 * at V_{k-1} and applies one Adam step.  Adam moments start at zero.
 * If loss_trace_host is non-NULL it receives K doubles, loss_trace[k-1] =
 * L(V_{k-1}), and the call synchronises the stream before returning;
 * otherwise it returns after enqueueing.  Allocates the optimiser state in
 * the plan on first use. */
PROP_API prop_status prop_reconstruct(prop_plan plan, const void* y_dev, const prop_recon_params* params,
                             void* V_dev, double* loss_trace_host, void* stream);

/* Several reconstructions advanced together, each stage of an iteration one
 * launch serving all of them (multi-problem launches whose CTAs are shared
 * out in proportion to each problem's work; the request server batches its
 * running requests the same way).  plans[count] (1 <= count <= 8, distinct
 * handles) must share the transform length 2N, the bin stride (Nf rounded up
 * to even), the Kaiser-Bessel width and the device, with one bin chunk each;
 * blade counts, lines, readout lengths, angles, bins, frames and data may
 * differ.  Problem r runs params[r].iters iterations of prop_reconstruct on
 * V_dev[r] (in/out) with y_dev[r]; its volume is bitwise that of
 * prop_reconstruct on its plan alone (the loss trace agrees to FP64
 * rounding: the |r|^2 block partials are grouped by the CTAs it gets).
 * loss_trace_host (may be NULL, as may its entries) as in prop_reconstruct;
 * the call synchronises only when a trace is requested.  Errors:
 * PROP_ERR_INVALID_ARG (count out of range, null or unaligned buffers, a
 * plan given twice, plans that cannot share launches, parameters out of
 * range), PROP_ERR_OOM (optimiser state on first use), PROP_ERR_CUDA. */
PROP_API prop_status prop_reconstruct_batch(const prop_plan* plans, int count, const void* const* y_dev,
                                            const prop_recon_params* params, void* const* V_dev,
                                            double* const* loss_trace_host, void* stream);

/* One Adam iteration of prop_reconstruct, out of place: V_out = the iterate
 * after step k (1-based) from V_in (the two buffers must differ; alternate
 * them between calls).  k == 1 resets the plan's Adam moments; later calls
 * continue them, so steps k = 1, 2, ... must run in order on one plan.
 * params->iters is ignored.  If loss_dev is non-NULL (device memory, one
 * double) it receives L(V_in).  Does not synchronise. */
PROP_API prop_status prop_recon_step(prop_plan plan, const void* y_dev, const prop_recon_params* params, int k,
                                     const void* V_in_dev, void* V_out_dev, double* loss_dev, void* stream);

/* ---- Bin-sharded iterations --------------------------------------------
 * The forward operator is a sum over spectral bins (Sec. 3 Eq. 2 displaces
 * and transforms every bin's layer on its own; Sec. 4.2 sums the layers), so
 * one reconstruction can be split over G plans -- one per device -- whose
 * bins partition the spectral axis into contiguous runs: plan g is created
 * with delta[f_g .. f_g+1) and holds V_g = V[..., f_g .. f_g+1).  One Adam
 * iteration k is then, on every plan g,
 *   1. prop_shard_forward(plan_g, V_g)      -> y_g = A_g V_g
 *   2. the caller sums the y_g over the plans (an all-reduce over devices),
 *      giving the same y_sum = A V everywhere;
 *   3. prop_shard_update(plan_g, y, y_sum, .., V_g -> V_g'): residual
 *      r = y_sum - y, adjoint 2 A_g^H r, TV of the plan's bins (x-y and
 *      temporal TV act on each bin separately) and Adam.
 * The iterates equal prop_reconstruct's on the whole axis up to the rounding
 * of the bin sum.  The loss of iteration k is loss_parts[0] (the data term,
 * the same on every plan) plus the sum over plans of loss_parts[1]. */

/* y_part_dev [B][L][R] = A_g V_g, the forward operator over the plan's bins
 * (flags & PROP_SHARD_ACCUMULATE: y_part_dev += A_g V_g instead, so that
 * plans on one device can sum their parts in place without a collective).
 * flags & PROP_SHARD_REUSE_ROWS skips the row transform when V_dev is the
 * V_out of the last prop_shard_update on this plan and no other call has used
 * the plan since (the update leaves that transform in the plan's workspace);
 * otherwise it is recomputed.  Does not synchronise.  Errors:
 * PROP_ERR_INVALID_ARG (null or unaligned buffers, unknown flags),
 * PROP_ERR_CUDA. */
#define PROP_SHARD_REUSE_ROWS 1
#define PROP_SHARD_ACCUMULATE 2
PROP_API prop_status prop_shard_forward(prop_plan plan, const void* V_dev, int flags, void* y_part_dev,
                                        void* stream);

/* The rest of iteration k (1-based) on the plan's bins, out of place:
 * y_dev the measured data, y_sum_dev the summed forward A V of V_{k-1}
 * (both [B][L][R]), V_in_dev = V_{k-1} of the plan's bins, V_out_dev
 * (different buffer) receives V_k.  k == 1 resets the plan's Adam moments.
 * loss_parts_dev (device, 2 doubles, may be NULL): [0] = sum |y_sum - y|^2,
 * [1] = tv_xy TV_xy + tv_t TV_t of V_{k-1} over the plan's bins.  Leaves the
 * forward row transform of V_out in the plan for prop_shard_forward.  Does
 * not synchronise.  Errors: PROP_ERR_INVALID_ARG (null or unaligned
 * buffers, V_in == V_out, k < 1, parameters out of range), PROP_ERR_OOM
 * (optimiser state on first use), PROP_ERR_CUDA. */
PROP_API prop_status prop_shard_update(prop_plan plan, const void* y_dev, const void* y_sum_dev,
                                       const prop_recon_params* params, int k, const void* V_in_dev,
                                       void* V_out_dev, double* loss_parts_dev, void* stream);

/* prop_reconstruct on host buffers: copies y_host [B][L][R] and V_host
 * (start) to the device, runs K iterations, copies V back into V_host and
 * synchronises.  Staging buffers are allocated in the plan on first use.
 * Pinned host memory gives the fastest copies. */
PROP_API prop_status prop_reconstruct_host(prop_plan plan, const void* y_host, const prop_recon_params* params,
                                  void* V_host, double* loss_trace_host, void* stream);

/* L(V) and its gradient dL/dRe V + i dL/dIm V (torch's convention for complex
 * tensors) at V_dev, without updating anything.  grad_dev [T][N][N][Nf]
 * complex64 out (may be NULL to skip it); *loss_host receives L(V) (the call
 * synchronises the stream).  Adam fields of params are ignored. */
PROP_API prop_status prop_loss_grad(prop_plan plan, const void* y_dev, const prop_recon_params* params,
                           const void* V_dev, void* grad_dev, double* loss_host, void* stream);

/* Render (Sec. 4.3, phi = 0 projection): image[t][i2][i1] = sum_{f_lo<=f<f_hi} V[t][i2][i1][f].
 * The whole range gives the final image; a lower or upper part of the
 * spectral axis gives the water-only or fat-only image (Sec. 6).
 * Requires 0 <= f_lo < f_hi <= Nf. */
PROP_API prop_status prop_render(prop_plan plan, const void* V_dev, int f_lo, int f_hi, void* image_dev,
                        void* stream);

/* Peak signal-to-noise ratio of a render against a reference image, the
 * quality figure of the paper's results (Sec. 6, Table 1), on magnitudes:
 *   PSNR = 10 log10( max|ref|^2 / mean (|image| - |ref|)^2 )  dB
 * over `frames` consecutive images [frames][N][N] complex64 (1 <= frames <= T;
 * all frames of a dynamic series together).  *psnr_host receives +inf when
 * the magnitudes agree exactly.  The sums are FP64 block partials combined
 * in block order (deterministic).  Allocates a small reduction buffer in the
 * plan on first use (PROP_ERR_OOM on failure); synchronises the stream.
 * Errors: PROP_ERR_INVALID_ARG (null or unaligned pointer, frames out of
 * range), PROP_ERR_OOM, PROP_ERR_CUDA. */
PROP_API prop_status prop_psnr(prop_plan plan, const void* image_dev, const void* ref_dev, int frames,
                               double* psnr_host, void* stream);

/* ---- Serving: continuous batching of independent reconstructions ----------
 * A server owns one device arena of hbm_budget_bytes (+ 64 MiB rounding
 * slack) allocated at creation.  Submitted requests (each a full
 * prop_reconstruct problem) wait in a FIFO queue; admission workers admit the
 * head request when fewer than max_slots requests run and its device
 * footprint (prop_plan_estimate_bytes + its data and volume) fits the budget
 * still free, build its plan inside the arena and upload its data.  A
 * scheduler thread groups the running requests by kernel class (2N, bin
 * stride, kernel width) and advances each class with batched iterations as
 * prop_reconstruct_batch does: one launch per stage serves every running
 * request of the class, whatever its blade count, frames or data; classes
 * run on their own streams and overlap, the class holding the oldest running
 * request (by submit time) on a high-priority stream so that it keeps the
 * device as a FIFO queue would give it.  Requests that arrive while others
 * run join their class's next batched iteration as soon as a slot and memory
 * free up.  A request that needs more than the whole budget fails with
 * PROP_ERR_OOM.  Results are bitwise identical to a lone prop_reconstruct of
 * the same problem.  Latency = time from prop_serve_submit to the completed
 * copy of the result back to host memory. */
typedef struct prop_server_s* prop_server;
typedef uint64_t prop_ticket;

enum { PROP_REQ_PENDING = 0, PROP_REQ_RUNNING = 1, PROP_REQ_DONE = 2, PROP_REQ_FAILED = 3,
       PROP_REQ_CANCELLED = 4 };

typedef struct prop_serve_stats_t {
  long long completed, failed, cancelled, pending, running;
  size_t reserved_bytes;      /* footprints of admitted requests */
  size_t arena_bytes_in_use;  /* bytes handed out from the arena now */
  size_t arena_peak_bytes;    /* high-water mark of the arena */
  size_t budget_bytes;
} prop_serve_stats_t;

/* Device bytes a plan for `desc` may hold after reconstructing `iters`
 * iterations (an upper bound; host-only computation, no device access). */
PROP_API prop_status prop_plan_estimate_bytes(const prop_plan_desc* desc, int iters, size_t* bytes);

/* Start a server on `device` with a device-memory budget and a slot limit. */
PROP_API prop_status prop_serve_create(size_t hbm_budget_bytes, int max_slots, int device, prop_server* out);

/* Queue one reconstruction.  desc: geometry (desc->device is ignored);
 * params: as prop_reconstruct; y_host [B][L][R] complex64 and v0_host
 * [T][N][N][Nf] complex64 (NULL = start from zero) are copied before return.
 * *out receives the request's ticket. */
PROP_API prop_status prop_serve_submit(prop_server server, const prop_plan_desc* desc,
                                       const prop_recon_params* params, const void* y_host,
                                       const void* v0_host, prop_ticket* out);

/* Current PROP_REQ_* state of a ticket (until it has been waited for). */
PROP_API prop_status prop_serve_poll(prop_server server, prop_ticket ticket, int* state);

/* Block until the request has finished (timeout_ms < 0: no limit) and
 * release its ticket.  On success v_host_out (nullable) receives the volume
 * [T][N][N][Nf], *latency_s (nullable) the submit-to-result time and
 * *final_loss (nullable) L(V_{K-1}).  Returns PROP_ERR_NOT_READY on timeout
 * (the ticket stays valid), the request's error if it failed, or
 * PROP_ERR_CANCELLED. */
PROP_API prop_status prop_serve_wait(prop_server server, prop_ticket ticket, int timeout_ms, void* v_host_out,
                                     double* latency_s, double* final_loss);

/* Ask for a request to stop: a queued request is dropped, a running one is
 * stopped after its in-flight iterations; its wait returns PROP_ERR_CANCELLED. */
PROP_API prop_status prop_serve_cancel(prop_server server, prop_ticket ticket);

/* Counters and memory use of the server. */
PROP_API prop_status prop_serve_stats(prop_server server, prop_serve_stats_t* out);

/* Cancel everything still queued or running, join the server's threads and
 * free its arena.  Unwaited tickets become invalid. */
PROP_API prop_status prop_serve_destroy(prop_server server);

/* Smoothed TV value and gradient without any device allocation (the paper has
 * no counterpart; this is a service for callers that cannot allocate device
 * memory: code running inside a memory arena owned by a host framework, a
 * real-time loop under a no-allocation rule, or a callback that must not
 * re-enter the CUDA allocator).  Needs no plan.
 *   V_dev     [nframes][n][n][nf] complex64 in (layout of V above)
 *   grad_dev  same shape, out: tv_xy grad TV_xy(V) + tv_t grad TV_t(V)
 *   loss_dev  one device double, out: tv_xy TV_xy(V) + tv_t TV_t(V)
 * with TV as defined above (forward differences, no wrap-around).  Runs on
 * the calling thread's current device; all pointers must be on it.
 * Reduction scratch lives in a file-scope __device__ array of 128 KiB + 256 B
 * (one double per image row), resident on every device that loads the
 * library until exit, so nframes * n must be <= 16384 (larger sizes return
 * PROP_ERR_INVALID_ARG with a message).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, once per device); make
 * that first call before any stream capture.  Each call clears the scratch
 * counter with cudaMemsetAsync on `stream`; it calls no allocating routine.
 * All calls share the one array, so calls that overlap on the GPU (different
 * streams, concurrent threads) race on it: serialise them.  Does not
 * synchronise. */
PROP_API prop_status prop_tv_grad_static(const void* V_dev, int nframes, int n, int nf, float tv_xy, float tv_t,
                                         float tv_eps, void* grad_dev, double* loss_dev, void* stream);

/* Stage profiling.  Stages: 0 forward row FFT, 1 forward column FFT,
 * 2 interpolation, 3 spread, 4 adjoint column FFT, 5 adjoint row FFT,
 * 6 TV + Adam (or TV gradient), 7 other (render, PSNR), 8 the fused row
 * kernel of prop_reconstruct (adjoint row FFT + TV + Adam + the next
 * iteration's forward row FFT), 9 K-Planes expansion and render, 10 K-Planes
 * parameter gradients, 11 K-Planes Adam.  While enabled, every kernel launch
 * (or group of launches) of the plan is bracketed by two CUDA events on its
 * stream. */
#define PROP_NUM_STAGES 12
PROP_API prop_status prop_profile_enable(prop_plan plan, int enable);
/* Synchronises on the recorded events, writes per-stage total milliseconds
 * and launch counts (arrays of PROP_NUM_STAGES), and clears the record. */
PROP_API prop_status prop_profile_read(prop_plan plan, double* ms_out, long long* launches_out);

/* Measured FP32 FMA throughput of `device` in TFLOP/s (2 flops per FMA):
 * the ALU ceiling against which the interpolation and spread are placed on a
 * roofline.  Times a few launches of a register-only FMA loop (8 independent
 * chains per thread, 8 blocks of 256 threads per SM, a few milliseconds each)
 * on a private stream and returns the fastest.  Synchronous; allocates and
 * frees a small device buffer.  Errors: PROP_ERR_INVALID_ARG (null tflops,
 * bad device), PROP_ERR_CUDA. */
PROP_API prop_status prop_fp32_fma_peak(int device, double* tflops);

/* Check of the device-side bounded wait that the staged kernels use
 * (interpolation, spread, TMA column FFTs, warp-specialised row kernel):
 * launches one warp that waits on an mbarrier nobody arrives at, bounded by
 * limit_cycles SM clock cycles (0 < limit_cycles <= 4e9, the kernels' own
 * bound), and reports *expired = 1 if the wait gave up and the kernel
 * returned (0 if the phase completed, which cannot happen here).  *ms (may
 * be NULL) receives the probe's duration.  The device stays usable
 * afterwards.  Synchronous; allocates and frees 4 bytes of device memory.
 * Errors: PROP_ERR_INVALID_ARG (null expired, limit out of range, bad
 * device), PROP_ERR_CUDA. */
PROP_API prop_status prop_check_bounded_wait(int device, long long limit_cycles, int* expired, double* ms);

/* ---- The paper's own forward model (Sec. 4.2-4.3) ----------------------
 *
 * Projection: blade b's image is I_b(p) = sum_f bilinear(V_t(b)(., f), p - Delta_f d_b)
 * (one sample per spectral slice along the ray tilted towards the readout
 * direction, Delta_f = h_f tan(phi); zero outside the image).  Blur: the
 * centred unitary DFT Z = U I_b (Z(k) = (1/N) sum_x I(x) e^{-2 pi i k.x},
 * k = (u - N/2)/N), masked by the blade's support M_b: the Cartesian cells
 * whose rotated coordinates rho = N k.d_b, pi = N k.d_b^perp satisfy
 * -R/2 - 1/2 <= rho < R/2 - 1/2 and -L/2 - 1/2 <= pi < L/2 - 1/2.  Uses the
 * plan's N (>= 16), Nf, Delta_f, theta_b, L, R, T and blade frames; tables
 * and a few N x N work images are allocated on first use.
 *
 * Cartesian k-space arrays are [N][N] complex64 indexed [u2][u1]; images
 * [N][N] indexed [i2][i1] (x = i - N/2); volumes as above. */
typedef struct prop_proj_params {
  int iters;                     /* K >= 0 iterations; iteration k (1-based) uses blade (k - 1) mod B */
  float lr, beta1, beta2, eps;   /* Adam */
  float w_kspace, w_image;       /* weights of the k-space and image-space data terms (Sec. 4.3) */
  float tv_xy, tv_f, tv_t;       /* smoothed TV along x1/x2, along the spectral axis, along time */
  float l1;                      /* smoothed L1 sparsity weight, l1 * sum sqrt(|V|^2 + tv_eps^2) */
  float tv_eps;                  /* smoothing epsilon (> 0) */
} prop_proj_params;

/* z = M_b U P_b V_t(b): [N][N] complex64 on the device, zero outside the
 * mask.  Errors: PROP_ERR_INVALID_ARG (null, blade out of range, N < 16),
 * PROP_ERR_OOM, PROP_ERR_CUDA.  Does not synchronise. */
PROP_API prop_status prop_proj_forward(prop_plan plan, int blade, const void* V_dev, void* z_dev, void* stream);
/* V = P_b^H U^H M_b z: frame t(b) of the volume gets the transposed
 * projection, the other frames zero.  Errors as prop_proj_forward.  Does
 * not synchronise. */
PROP_API prop_status prop_proj_adjoint(prop_plan plan, int blade, const void* z_dev, void* V_dev, void* stream);
/* Adam over the blades in turn (Sec. 4.3) on
 *   w_kspace sum_{M_b} |Z - ycart_b|^2 + w_image sum |U^H M_b Z - img_b|^2
 *   + tv_xy TV_xy + tv_f TV_f + tv_t TV_t + l1 L1,   Z = U P_b V_t(b),
 * each TV term sum sqrt(|d|^2 + tv_eps^2) over forward differences (no wrap).
 * ycart_dev: [B][N][N] Cartesian k-space data (cells outside each mask are
 * not read); img_dev: [B][N][N] blade images, or NULL for U^H M_b ycart_b.
 * V_dev: the start in, the result out.  loss_trace_host (may be NULL):
 * [iters] loss of each iteration's blade before its update.  Synchronises
 * only when a trace is requested. */
/* Errors: PROP_ERR_INVALID_ARG (null plan/ycart/V, iters < 0, Adam
 * parameters out of range, a negative or non-finite weight, tv_eps <= 0),
 * PROP_ERR_OOM (optimiser state, image spectra), PROP_ERR_CUDA. */
PROP_API prop_status prop_proj_reconstruct(prop_plan plan, const void* ycart_dev, const void* img_dev,
                                           const prop_proj_params* params, void* V_dev, double* loss_trace_host,
                                           void* stream);

/* The results section's baseline (Sec. 6): the coverage-weighted average of
 * blades blade_lo .. blade_hi-1 in k-space (each Cartesian cell averages
 * the blades whose mask holds it; uncovered cells are zero), then the
 * inverse DFT.  ycart_dev [B][N][N]; img_dev [N][N].  All blades for a
 * static series; the most recent ones before a frame for a dynamic one.
 * Errors: PROP_ERR_INVALID_ARG (null, not 0 <= blade_lo < blade_hi <= B),
 * PROP_ERR_OOM, PROP_ERR_CUDA.  Does not synchronise. */
PROP_API prop_status prop_proj_baseline(prop_plan plan, const void* ycart_dev, int blade_lo, int blade_hi,
                                        void* img_dev, void* stream);

/* ---- The dynamic K-Planes volume model (Sec. 4.1, Eq. 3) ----------------
 *
 * V(x, y, omega, t) = sum over scales s < scales of sum_k a_s,k
 * prod_c psi(p_s,c, pi_c(x, y, omega, t))_k, the six planes c = xy, x-omega,
 * x-t, y-omega, y-t, omega-t holding `features` (1..16) complex features per
 * node, interpolated bilinearly with cell-centred nodes (voxel i maps to
 * (i + 1/2) R / N - 1/2 on a spatial axis of R nodes, clamped to [0, R-1];
 * spectral and time indices are nodes).  Scale s has N >> s spatial nodes
 * (scales is 1 or 2).  Parameters: one complex64 device buffer, per scale in
 * order xy [n][n][F], xw [Nf][n][F], xt [T][n][F], yw [Nf][n][F],
 * yt [T][n][F], wt [T][Nf][F], then a [F]. */
/* Number of complex parameters of that layout. */
PROP_API prop_status prop_kplanes_param_count(prop_plan plan, int features, int scales, size_t* count);
/* V_dev [T][N][N][Nf] = the model rendered on the volume grid.  Does not synchronise. */
PROP_API prop_status prop_kplanes_render(prop_plan plan, int features, int scales, const void* params_dev,
                                         void* V_dev, void* stream);
/* grad_dev (same layout as the parameters) = dL/dRe z + i dL/dIm z for every
 * parameter z, given gV_dev = dL/dRe V + i dL/dIm V.  Every sum is taken in a
 * fixed order (partial sums over the spectral axis, over time and over the
 * image, then fixed-order second passes and the transposed interpolation; no
 * atomics), so the result is bitwise reproducible.  The render and the
 * gradients use a workspace in the plan (the planes expanded to the volume's
 * resolution and the partial sums, about (T N^2 + N^2 Nf) * features * scales
 * complex values), allocated on first use (PROP_ERR_OOM on failure).  Does
 * not synchronise. */
PROP_API prop_status prop_kplanes_vjp(prop_plan plan, int features, int scales, const void* params_dev,
                                      const void* gV_dev, void* grad_dev, void* stream);
/* Adam on the model's parameters (in place) for the loss of prop_reconstruct
 * (non-uniform data term + TV of the rendered volume): per iteration render,
 * loss and grad V, transpose, Adam.  loss_trace_host as in prop_reconstruct.
 * Allocates and frees Adam state for the parameters; synchronises.  Errors:
 * PROP_ERR_INVALID_ARG (null, features/scales out of range, parameters out of
 * range), PROP_ERR_OOM, PROP_ERR_CUDA. */
PROP_API prop_status prop_kplanes_reconstruct(prop_plan plan, const void* y_dev, const prop_recon_params* params,
                                              int features, int scales, void* kp_params_dev, double* loss_trace_host,
                                              void* stream);

/* Message for the last non-OK status returned on the calling thread ("" if none). */
PROP_API const char* prop_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PROP_H */
