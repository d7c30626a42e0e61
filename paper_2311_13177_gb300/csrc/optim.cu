// Fused smoothed-TV gradient + Adam update, the TV/loss reduction, and the
// spectral-sum render.
//
// Sec. 4.3 optimises the volume with Adam on the data term plus total
// variation in space and (for dynamic series) time.  Per complex voxel V(x):
//   TV terms sqrt(|d|^2 + eps^2) over forward differences d along x1, x2 and
//   t (no wrap-around); the gradient of one term with respect to its upper
//   end is d / sqrt(|d|^2 + eps^2) and minus that for its lower end;
//   g = gscale * A^H r + tv_xy grad TV_xy + tv_t grad TV_t;
//   per real component: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
//   V -= (lr / (1 - b1^k)) m / (sqrt(v) / sqrt(1 - b2^k) + eps).
// The update reads Vin and writes Vout (ping-pong), because neighbours of a
// voxel are read by other threads.  One thread per complex voxel, bins
// fastest, so warps read and write contiguous runs.
#include "prop_internal.cuh"
#include "tv_adam.cuh"

namespace prop {
namespace {

constexpr int kOptThreads = 256;
constexpr int kSeg = 1024;  // values per work unit

__device__ double block_sum_d(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

struct OptArgs {
  const float2* Vin;
  const float2* g;
  float2* m;
  float2* v;
  float2* out;  // Vout (Adam) or grad (gradient only)
  double* partials;
  unsigned int* counter;
  const double* data_loss;
  double* loss_out;
  long nvox;
  int N, Nf, T;
  AdamArgs p;
};

template <bool ADAM>
__global__ void __launch_bounds__(kOptThreads) opt_kernel(OptArgs a) {
  // Work unit: a segment of kSeg consecutive values of one image row (t, i2);
  // a row holds N * Nf values (i1, f).
  const float eps2 = a.p.tv_eps * a.p.tv_eps;
  const int rowlen = a.N * a.Nf;
  const int segs = (rowlen + kSeg - 1) / kSeg;
  const long nseg = (long)a.T * a.N * segs;
  float local = 0.f;
  for (long sgi = blockIdx.x; sgi < nseg; sgi += gridDim.x) {
    const long row = sgi / segs;
    const int seg = (int)(sgi - row * segs);
    const int i2 = (int)(row % a.N);
    const int t = (int)(row / a.N);
    const long rbase = row * rowlen;
    for (int e = seg * kSeg + threadIdx.x; e < min(rowlen, (seg + 1) * kSeg); e += blockDim.x) {
      const long idx = rbase + e;
      const int i1 = e / a.Nf;
      const float2 x = a.Vin[idx];
      float2 gxy, gt;
      local = __fadd_rn(local, voxel_tv(a.Vin, (size_t)idx, x, i1, i2, t, a.N, a.Nf, a.T, a.p.tv_xy, a.p.tv_t,
                                        eps2, &gxy, &gt));
      const float2 g = total_grad(a.g[idx], gxy, gt, a.p);
      if constexpr (ADAM) {
        float2 mm = a.m[idx], vv = a.v[idx];
        const float2 nx = adam_voxel(x, g, mm, vv, a.p);
        a.m[idx] = mm;
        a.v[idx] = vv;
        a.out[idx] = nx;
      } else {
        a.out[idx] = g;
      }
    }
  }
  if (a.partials) finish_loss(local, a.partials, a.counter, a.data_loss, a.loss_out);
}

__global__ void render_kernel(const float2* V, float2* img, long npix, int Nf, int lo, int hi) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (long)gridDim.x * blockDim.x) {
    const float2* v = V + p * Nf;
    float2 s = make_float2(0.f, 0.f);
    for (int f = lo; f < hi; ++f) {
      const float2 x = v[f];
      s.x += x.x;
      s.y += x.y;
    }
    img[p] = s;
  }
}

// PSNR partials: each block writes (sum (|a| - |b|)^2, max |b|^2) of its
// grid-stride share; the last block to arrive combines them in block order
// and writes 10 log10(peak^2 / mse).
__global__ void __launch_bounds__(kOptThreads) psnr_kernel(const float2* a, const float2* b, long count,
                                                           double* scratch, int cap, double* out) {
  double se = 0.0, pk = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const float2 x = a[i], r = b[i];
    const double ma = sqrt((double)x.x * x.x + (double)x.y * x.y);
    const double mr2 = (double)r.x * r.x + (double)r.y * r.y;
    const double d = ma - sqrt(mr2);
    se += d * d;
    pk = fmax(pk, mr2);
  }
  __shared__ double sh[32];
  __shared__ bool last;
  se = block_sum_d(se, sh);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pk = fmax(pk, __shfl_xor_sync(0xffffffffu, pk, o));
  __shared__ double shm[32];
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = pk;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, shm[w]);
    scratch[2 * blockIdx.x] = se;
    scratch[2 * blockIdx.x + 1] = m;
    __threadfence();
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + 2 * cap);
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s = 0.0, m = 0.0;
    for (int i = 0; i < (int)gridDim.x; ++i) {
      s += __ldcg(&scratch[2 * i]);
      m = fmax(m, __ldcg(&scratch[2 * i + 1]));
    }
    const double mse = s / (double)count;
    *out = mse > 0.0 ? 10.0 * log10(m / mse) : __longlong_as_double(0x7ff0000000000000LL);
    *reinterpret_cast<unsigned int*>(scratch + 2 * cap) = 0u;
  }
}

unsigned opt_blocks(const Plan& p, const Reducer* red) {
  const long segs = ((long)p.N * p.Nf + kSeg - 1) / kSeg;
  long need = (long)p.T * p.N * segs;
  long cap = red ? std::min<long>(red->capacity, 16384) : 16384;
  return (unsigned)std::max<long>(1, std::min(need, cap));
}

OptArgs make_args(const Plan& p, const float2* Vin, const float2* g, float2* out, const AdamArgs& aa,
                  const Reducer* red, const double* data_loss, double* loss_out) {
  OptArgs a{};
  a.Vin = Vin;
  a.g = g;
  a.out = out;
  a.partials = red ? red->partials : nullptr;
  a.counter = red ? red->counter : nullptr;
  a.data_loss = data_loss;
  a.loss_out = loss_out;
  a.nvox = (long)p.vol_elems();
  a.N = p.N;
  a.Nf = p.Nf;
  a.T = p.T;
  a.p = aa;
  return a;
}

}  // namespace

cudaError_t tv_adam(const Plan& p, const float2* Vin, const float2* g, float2* m, float2* v, float2* Vout,
                    const AdamArgs& aa, const Reducer* red, const double* data_loss, double* loss_out,
                    cudaStream_t s) {
  OptArgs a = make_args(p, Vin, g, Vout, aa, red, data_loss, loss_out);
  a.m = m;
  a.v = v;
  opt_kernel<true><<<opt_blocks(p, red), kOptThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t tv_grad(const Plan& p, const float2* V, const float2* g, float2* grad, const AdamArgs& aa,
                    const Reducer* red, const double* data_loss, double* loss_out, cudaStream_t s) {
  OptArgs a = make_args(p, V, g, grad, aa, red, data_loss, loss_out);
  opt_kernel<false><<<opt_blocks(p, red), kOptThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t psnr(const Plan& p, const float2* img, const float2* ref, long count, double* out, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::max<long>(1, std::min<long>((count + kOptThreads - 1) / kOptThreads,
                                                                     (long)p.psnr_cap));
  psnr_kernel<<<blocks, kOptThreads, 0, s>>>(img, ref, count, p.psnr_scratch, p.psnr_cap, out);
  return cudaGetLastError();
}

cudaError_t render(const Plan& p, const float2* V, int f_lo, int f_hi, float2* img, cudaStream_t s) {
  const long npix = (long)p.T * p.N * p.N;
  const unsigned blocks = (unsigned)std::min<long>((npix + 255) / 256, 16384);
  render_kernel<<<blocks, 256, 0, s>>>(V, img, npix, p.Nf, f_lo, f_hi);
  return cudaGetLastError();
}

}  // namespace prop

// ---------------------------------------------------------------------------
// Allocation-free TV value and gradient: prop_tv_grad_static.
//
// For callers that cannot allocate device memory (code running inside a
// memory pool or arena owned by a host framework, under a no-allocation
// rule in a real-time loop, or in a callback that must not re-enter the CUDA
// allocator).  It computes the same smoothed TV terms as the optimiser
// kernel, one CTA per image row, and keeps its reduction scratch (one FP64
// partial per image row plus the arrival counter) in the file-scope device
// array below instead of a plan.  The array is 128 KiB + 256 B and stays
// resident on every device that loads the library until the process exits.
#include <mutex>

namespace prop {
namespace {

constexpr int kStaticRows = 16384;       // most image rows (frames * N) per call
constexpr int kStaticDevices = 64;

// [0, kStaticRows): per-row partial sums; slot kStaticRows holds the counter.
static __device__ __align__(256) double g_tv_static_scratch[kStaticRows + 32];

__global__ void __launch_bounds__(kOptThreads)
tv_grad_rows_kernel(const float2* V, float2* grad, double* scratch, double* loss_out, int N, int Nf, int T,
                    float tv_xy, float tv_t, float tv_eps) {
  const float eps2 = tv_eps * tv_eps;
  const int rowlen = N * Nf;
  const int row = blockIdx.x;  // t * N + i2
  const int i2 = row % N;
  const int t = row / N;
  const long rbase = (long)row * rowlen;
  float local = 0.f;
  for (int e = threadIdx.x; e < rowlen; e += blockDim.x) {
    const long idx = rbase + e;
    const float2 x = V[idx];
    float2 gxy, gt;
    local += voxel_tv(V, (size_t)idx, x, e / Nf, i2, t, N, Nf, T, tv_xy, tv_t, eps2, &gxy, &gt);
    grad[idx] = make_float2(fmaf(tv_xy, gxy.x, tv_t * gt.x), fmaf(tv_xy, gxy.y, tv_t * gt.y));
  }
  __shared__ double sh[32];
  __shared__ bool last;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kStaticRows);
  const double bs = block_sum_d((double)local, sh);
  if (threadIdx.x == 0) {
    scratch[row] = bs;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(&scratch[i]);
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) {
      *loss_out = s;
      *counter = 0u;
    }
  }
}

std::mutex g_static_mutex;
double* g_static_addr[kStaticDevices] = {};

}  // namespace
}  // namespace prop

extern "C" prop_status prop_tv_grad_static(const void* V_dev, int nframes, int n, int nf, float tv_xy,
                                           float tv_t, float tv_eps, void* grad_dev, double* loss_dev,
                                           void* stream) {
  using namespace prop;
  if (!V_dev || !grad_dev || !loss_dev) return fail(PROP_ERR_INVALID_ARG, "tv_grad_static: null argument");
  if (((uintptr_t)V_dev & 15u) || ((uintptr_t)grad_dev & 15u) || ((uintptr_t)loss_dev & 7u))
    return fail(PROP_ERR_INVALID_ARG, "tv_grad_static: V and grad must be 16-byte aligned, loss 8-byte aligned");
  if (V_dev == grad_dev) return fail(PROP_ERR_INVALID_ARG, "tv_grad_static: V and grad must not alias");
  if (nframes < 1 || n < 1 || nf < 1 || (long long)n * nf > (1LL << 30))
    return fail(PROP_ERR_INVALID_ARG, "tv_grad_static: nframes, n, nf must be >= 1 and n * nf <= 2^30");
  if ((long long)nframes * n > kStaticRows)
    return fail(PROP_ERR_INVALID_ARG, "tv_grad_static: nframes * n = " + std::to_string((long long)nframes * n) +
                                          " image rows exceeds the static scratch limit of " +
                                          std::to_string(kStaticRows));
  if (!(tv_eps > 0.f) || !(tv_xy >= 0.f) || !(tv_t >= 0.f))
    return fail(PROP_ERR_INVALID_ARG, "tv_grad_static: need tv_xy >= 0, tv_t >= 0, tv_eps > 0");
  int dev = 0;
  PROP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticDevices) return fail(PROP_ERR_INVALID_ARG, "tv_grad_static: device ordinal too large");
  double* scratch = nullptr;
  {
    // One-time set-up per device, with that device current: the host-side
    // name of the array is not a device address, so look the address up.
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
      void* addr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&addr, g_tv_static_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "tv_grad_static: cudaGetSymbolAddress");
      g_static_addr[dev] = static_cast<double*>(addr);
    }
    scratch = g_static_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  // The counter must start at zero; the partials are fully rewritten each call.
  PROP_CUDA(cudaMemsetAsync(scratch + kStaticRows, 0, sizeof(double), s));
  tv_grad_rows_kernel<<<nframes * n, kOptThreads, 0, s>>>((const float2*)V_dev, (float2*)grad_dev, scratch,
                                                           loss_dev, n, nf, nframes, tv_xy, tv_t, tv_eps);
  PROP_CUDA(cudaGetLastError());
  return PROP_OK;
}
