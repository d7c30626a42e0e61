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
  int n;                  /* image size N: multiple of 8, 8 <= N <= 512, 2N = 2^a 3^b */
  int nf;                 /* spectral bins Nf >= 1 */
  const double* delta;    /* [nf] displacement Delta_f of each bin, pixels along readout */
  int nblades;            /* B >= 1 */
  const double* theta;    /* [nblades] blade angles th_b, radians */
  int lines;              /* L >= 1, lines per blade */
  int readout;            /* R >= 1, samples per line */
  int nframes;            /* T >= 1 (1 = static) */
  const int* blade_frame; /* [nblades] frame t(b) in [0, T), or NULL = all frame 0 */
  int kb_width;           /* interpolation kernel width: 0 (default) or 6 */
  int bin_chunk;          /* bins per oversampled-grid pass: 0 = auto (min(Nf, 32)), else 1..64.
                             Smaller chunks recompute the grid per chunk in less memory. */
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
 * and FFT twiddle tables (FP64 -> FP32), spread tile lists, and the
 * device workspace.  Allocates device memory (PROP_ERR_OOM on failure).
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

/* One Adam iteration of prop_reconstruct, out of place: V_out = the iterate
 * after step k (1-based) from V_in (the two buffers must differ; alternate
 * them between calls).  k == 1 resets the plan's Adam moments; later calls
 * continue them, so steps k = 1, 2, ... must run in order on one plan.
 * params->iters is ignored.  If loss_dev is non-NULL (device memory, one
 * double) it receives L(V_in).  Does not synchronise. */
PROP_API prop_status prop_recon_step(prop_plan plan, const void* y_dev, const prop_recon_params* params, int k,
                                     const void* V_in_dev, void* V_out_dev, double* loss_dev, void* stream);

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
 * 6 TV + Adam (or TV gradient), 7 other (render).  While enabled, every
 * kernel launch of the plan is bracketed by two CUDA events on its stream. */
#define PROP_NUM_STAGES 8
PROP_API prop_status prop_profile_enable(prop_plan plan, int enable);
/* Synchronises on the recorded events, writes per-stage total milliseconds
 * and launch counts (arrays of PROP_NUM_STAGES), and clears the record. */
PROP_API prop_status prop_profile_read(prop_plan plan, double* ms_out, long long* launches_out);

/* Message for the last non-OK status returned on the calling thread ("" if none). */
PROP_API const char* prop_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PROP_H */
