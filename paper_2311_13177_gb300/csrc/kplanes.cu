// The dynamic K-Planes volume model (Sec. 4.1, Eq. 3) on the GPU.
//
// The volume is V(x, y, omega, t) = sum over scales of sum_k a_k prod_c
// psi(p_c, pi_c(x, y, omega, t))_k over the six planes c = xy, x-omega, x-t,
// y-omega, y-t, omega-t of F-vector features, bilinearly interpolated with
// cell-centred nodes (voxel i -> (i + 1/2) R / N - 1/2 on a spatial axis of
// R nodes, clamped to [0, R - 1]; spectral and time indices are nodes);
// scale s has N >> s spatial nodes.  Parameters live in one complex64
// buffer, per scale: xy [n][n][F], xw [Nf][n][F], xt [T][n][F],
// yw [Nf][n][F], yt [T][n][F], wt [T][Nf][F], then a [F].
//
// A reconstruction iteration renders V, runs the unchanged non-uniform
// forward and adjoint passes with the TV gradient (grad V), carries grad V
// back to the parameters (grad z = sum conj(dV/dz) grad V) and applies
// Adam to every parameter.  The transpose scatters each voxel's
// contributions to the plane nodes it read with float atomics (the a
// gradient is first summed over the warp), so its sums are not in a fixed
// order: results agree with the oracle to rounding, not bit for bit.
#include "prop_internal.cuh"
#include "tv_adam.cuh"

#include <algorithm>
#include <cmath>

namespace prop {
namespace {

constexpr int kKpThreads = 256;
constexpr int kKpPlanes = 6;
constexpr int kKpMaxScales = 2;
constexpr int kKpMaxF = 16;

struct KpScale {
  size_t off[kKpPlanes];  // element offset of each plane
  size_t a;               // element offset of a
  int cols[kKpPlanes];    // columns of each plane
  int n;                  // spatial nodes per axis
};
struct KpArgs {
  int N, Nf, T, F, S;
  KpScale sc[kKpMaxScales];
};

struct Tap {
  int lo, hi;
  float w;  // weight of hi
};
__device__ __forceinline__ Tap make_tap(float u, int R) {
  u = fminf(fmaxf(u, 0.f), (float)(R - 1));
  Tap t;
  t.lo = min((int)floorf(u), max(R - 2, 0));
  t.w = u - (float)t.lo;
  t.hi = min(t.lo + 1, R - 1);
  return t;
}

__device__ __forceinline__ float2 kmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 kconj(float2 a) { return make_float2(a.x, -a.y); }

// Row and column taps of plane c for voxel (t, y, x, f): xy (y, x), xw (f, x),
// xt (t, x), yw (f, y), yt (t, y), wt (t, f).
struct KpTaps {
  Tap r[kKpPlanes], c[kKpPlanes];
};
__device__ __forceinline__ KpTaps voxel_taps(const KpArgs& a, const KpScale& S, int t, int i2, int i1, int f) {
  const float s = (float)S.n / (float)a.N;
  const Tap tx = make_tap(((float)i1 + 0.5f) * s - 0.5f, S.n);
  const Tap ty = make_tap(((float)i2 + 0.5f) * s - 0.5f, S.n);
  const Tap tw = make_tap((float)f, a.Nf);
  const Tap tt = make_tap((float)t, a.T);
  KpTaps k;
  k.r[0] = ty; k.c[0] = tx;
  k.r[1] = tw; k.c[1] = tx;
  k.r[2] = tt; k.c[2] = tx;
  k.r[3] = tw; k.c[3] = ty;
  k.r[4] = tt; k.c[4] = ty;
  k.r[5] = tt; k.c[5] = tw;
  return k;
}

__device__ __forceinline__ float2 bilerp(const float2* __restrict__ P, int cols, int F, Tap r, Tap c, int k) {
  const float2 p00 = P[((size_t)r.lo * cols + c.lo) * F + k];
  const float2 p01 = P[((size_t)r.lo * cols + c.hi) * F + k];
  const float2 p10 = P[((size_t)r.hi * cols + c.lo) * F + k];
  const float2 p11 = P[((size_t)r.hi * cols + c.hi) * F + k];
  const float w00 = (1.f - r.w) * (1.f - c.w), w01 = (1.f - r.w) * c.w, w10 = r.w * (1.f - c.w), w11 = r.w * c.w;
  return make_float2(fmaf(w11, p11.x, fmaf(w10, p10.x, fmaf(w01, p01.x, w00 * p00.x))),
                     fmaf(w11, p11.y, fmaf(w10, p10.y, fmaf(w01, p01.y, w00 * p00.y))));
}

__device__ __forceinline__ void decode(size_t idx, const KpArgs& a, int& t, int& i2, int& i1, int& f) {
  f = (int)(idx % a.Nf);
  size_t r = idx / a.Nf;
  i1 = (int)(r % a.N);
  r /= a.N;
  i2 = (int)(r % a.N);
  t = (int)(r / a.N);
}

__global__ void __launch_bounds__(kKpThreads) kp_render_kernel(const float2* __restrict__ P, KpArgs a,
                                                               float2* __restrict__ V) {
  grid_dep_wait();
  grid_dep_release();
  const size_t total = (size_t)a.T * a.N * a.N * a.Nf;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    int t, i2, i1, f;
    decode(idx, a, t, i2, i1, f);
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < a.S; ++s) {
      const KpScale& S = a.sc[s];
      const KpTaps tp = voxel_taps(a, S, t, i2, i1, f);
      for (int k = 0; k < a.F; ++k) {
        float2 prod = make_float2(1.f, 0.f);
#pragma unroll
        for (int c = 0; c < kKpPlanes; ++c) prod = kmul(prod, bilerp(P + S.off[c], S.cols[c], a.F, tp.r[c], tp.c[c], k));
        const float2 ak = P[S.a + k];
        const float2 q = kmul(prod, ak);
        acc.x += q.x;
        acc.y += q.y;
      }
    }
    V[idx] = acc;
  }
}

__device__ __forceinline__ void atomic_add_c(float2* p, float2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// G (zeroed by the caller) += the parameter gradients of the voxels' grad V.
// Whole warps run every trip (lanes past the end carry a zero gradient) so
// the warp sums of the a gradient are well defined.
__global__ void __launch_bounds__(kKpThreads) kp_vjp_kernel(const float2* __restrict__ P, KpArgs a,
                                                            const float2* __restrict__ gV, float2* __restrict__ G) {
  grid_dep_wait();
  grid_dep_release();
  const size_t total = (size_t)a.T * a.N * a.N * a.Nf;
  const int lane = threadIdx.x & 31;
  for (size_t base = (size_t)blockIdx.x * blockDim.x; base < total; base += (size_t)gridDim.x * blockDim.x) {
    const size_t idx0 = base + threadIdx.x;
    const bool valid = idx0 < total;
    const size_t idx = valid ? idx0 : 0;
    int t, i2, i1, f;
    decode(idx, a, t, i2, i1, f);
    const float2 g = valid ? gV[idx] : make_float2(0.f, 0.f);
    for (int s = 0; s < a.S; ++s) {
      const KpScale& S = a.sc[s];
      const KpTaps tp = voxel_taps(a, S, t, i2, i1, f);
      for (int k = 0; k < a.F; ++k) {
        float2 h[kKpPlanes], pre[kKpPlanes];
        float2 run = make_float2(1.f, 0.f);
#pragma unroll
        for (int c = 0; c < kKpPlanes; ++c) {
          h[c] = bilerp(P + S.off[c], S.cols[c], a.F, tp.r[c], tp.c[c], k);
          pre[c] = run;  // product of the planes before c
          run = kmul(run, h[c]);
        }
        // a gradient: conj(prod) g, summed over the warp first
        float2 ga = kmul(kconj(run), g);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
          ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
        }
        if (lane == 0) atomic_add_c(G + S.a + k, ga);
        if (!valid) continue;
        const float2 ak = P[S.a + k];
        float2 suf = make_float2(1.f, 0.f);  // product of the planes after c
#pragma unroll
        for (int c = kKpPlanes - 1; c >= 0; --c) {
          const float2 others = kmul(pre[c], suf);
          const float2 q = kmul(kconj(kmul(ak, others)), g);
          suf = kmul(suf, h[c]);
          const Tap r = tp.r[c], cc = tp.c[c];
          float2* Gc = G + S.off[c];
          const int cols = S.cols[c];
          const float w00 = (1.f - r.w) * (1.f - cc.w), w01 = (1.f - r.w) * cc.w, w10 = r.w * (1.f - cc.w),
                      w11 = r.w * cc.w;
          atomic_add_c(Gc + ((size_t)r.lo * cols + cc.lo) * a.F + k, make_float2(w00 * q.x, w00 * q.y));
          atomic_add_c(Gc + ((size_t)r.lo * cols + cc.hi) * a.F + k, make_float2(w01 * q.x, w01 * q.y));
          atomic_add_c(Gc + ((size_t)r.hi * cols + cc.lo) * a.F + k, make_float2(w10 * q.x, w10 * q.y));
          atomic_add_c(Gc + ((size_t)r.hi * cols + cc.hi) * a.F + k, make_float2(w11 * q.x, w11 * q.y));
        }
      }
    }
  }
}

// Adam on every complex parameter (real and imaginary parts separately).
__global__ void __launch_bounds__(kKpThreads) kp_adam_kernel(float2* __restrict__ P, const float2* __restrict__ G,
                                                             float2* __restrict__ m, float2* __restrict__ v,
                                                             size_t count, AdamArgs ad) {
  grid_dep_wait();
  grid_dep_release();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    float2 mm = m[i], vv = v[i];
    P[i] = adam_voxel(P[i], G[i], mm, vv, ad);
    m[i] = mm;
    v[i] = vv;
  }
}

// Layout of the parameter buffer; returns the element count.
size_t kp_layout(const Plan& p, int F, int S, KpArgs* out) {
  KpArgs a{};
  a.N = p.N;
  a.Nf = p.Nf;
  a.T = p.T;
  a.F = F;
  a.S = S;
  size_t off = 0;
  for (int s = 0; s < S; ++s) {
    KpScale& sc = a.sc[s];
    const int n = p.N >> s;
    sc.n = n;
    const int rows[kKpPlanes] = {n, p.Nf, p.T, p.Nf, p.T, p.T};
    const int cols[kKpPlanes] = {n, n, n, n, n, p.Nf};
    for (int c = 0; c < kKpPlanes; ++c) {
      sc.off[c] = off;
      sc.cols[c] = cols[c];
      off += (size_t)rows[c] * cols[c] * F;
    }
    sc.a = off;
    off += F;
  }
  if (out) *out = a;
  return off;
}

prop_status kp_check(const Plan& p, int F, int S) {
  if (F < 1 || F > kKpMaxF) return fail(PROP_ERR_INVALID_ARG, "kplanes: features must be in [1, 16]");
  if (S < 1 || S > kKpMaxScales) return fail(PROP_ERR_INVALID_ARG, "kplanes: scales must be 1 or 2");
  if ((p.N >> (S - 1)) < 2) return fail(PROP_ERR_INVALID_ARG, "kplanes: image too small for the scales");
  return PROP_OK;
}

unsigned kp_blocks(size_t count, const Plan& p) {
  return (unsigned)std::max<size_t>(1, std::min<size_t>((count + kKpThreads - 1) / kKpThreads, (size_t)16 * p.num_sms));
}

}  // namespace

}  // namespace prop

using namespace prop;

extern "C" {

prop_status prop_kplanes_param_count(prop_plan plan, int features, int scales, size_t* count) {
  if (!plan || !count) return fail(PROP_ERR_INVALID_ARG, "kplanes_param_count: null argument");
  const Plan& p = *plan->p;
  prop_status st = kp_check(p, features, scales);
  if (st != PROP_OK) return st;
  *count = kp_layout(p, features, scales, nullptr);
  return PROP_OK;
}

prop_status prop_kplanes_render(prop_plan plan, int features, int scales, const void* params_dev, void* V_dev,
                                void* stream) {
  if (!plan || !params_dev || !V_dev) return fail(PROP_ERR_INVALID_ARG, "kplanes_render: null argument");
  Plan& p = *plan->p;
  prop_status st = kp_check(p, features, scales);
  if (st != PROP_OK) return st;
  DeviceGuard g(p.device);
  KpArgs a;
  kp_layout(p, features, scales, &a);
  PROP_CUDA(launch_dep(kp_render_kernel, dim3(kp_blocks(p.vol_elems(), p)), dim3(kKpThreads), 0,
                       (cudaStream_t)stream, (const float2*)params_dev, a, (float2*)V_dev));
  return PROP_OK;
}

prop_status prop_kplanes_vjp(prop_plan plan, int features, int scales, const void* params_dev, const void* gV_dev,
                             void* grad_dev, void* stream) {
  if (!plan || !params_dev || !gV_dev || !grad_dev) return fail(PROP_ERR_INVALID_ARG, "kplanes_vjp: null argument");
  Plan& p = *plan->p;
  prop_status st = kp_check(p, features, scales);
  if (st != PROP_OK) return st;
  DeviceGuard g(p.device);
  KpArgs a;
  const size_t count = kp_layout(p, features, scales, &a);
  cudaStream_t s = (cudaStream_t)stream;
  PROP_CUDA(cudaMemsetAsync(grad_dev, 0, count * sizeof(float2), s));
  PROP_CUDA(launch_dep(kp_vjp_kernel, dim3(kp_blocks(p.vol_elems(), p)), dim3(kKpThreads), 0, s,
                       (const float2*)params_dev, a, (const float2*)gV_dev, (float2*)grad_dev));
  return PROP_OK;
}

prop_status prop_kplanes_reconstruct(prop_plan plan, const void* y_dev, const prop_recon_params* params,
                                     int features, int scales, void* kp_params_dev, double* loss_trace_host,
                                     void* stream) {
  if (!plan || !y_dev || !params || !kp_params_dev)
    return fail(PROP_ERR_INVALID_ARG, "kplanes_reconstruct: null argument");
  Plan& p = *plan->p;
  prop_status st = kp_check(p, features, scales);
  if (st != PROP_OK) return st;
  const prop_recon_params& q = *params;
  if (q.iters < 0 || !(q.lr >= 0.f) || !(q.beta1 >= 0.f && q.beta1 < 1.f) || !(q.beta2 >= 0.f && q.beta2 < 1.f) ||
      !(q.eps > 0.f) || !(q.tv_eps > 0.f) || !(q.tv_xy >= 0.f) || !(q.tv_t >= 0.f))
    return fail(PROP_ERR_INVALID_ARG, "kplanes_reconstruct: parameters out of range");
  DeviceGuard g(p.device);
  if ((st = plan_ensure_recon(&p, std::max(q.iters, 1))) != PROP_OK) return st;
  KpArgs a;
  const size_t count = kp_layout(p, features, scales, &a);
  float2* G = nullptr;
  float2* m = nullptr;
  float2* v = nullptr;
  PROP_CUDA(plan_dev_alloc(&p, (void**)&G, count * sizeof(float2)));
  cudaError_t e = plan_dev_alloc(&p, (void**)&m, count * sizeof(float2));
  if (e == cudaSuccess) e = plan_dev_alloc(&p, (void**)&v, count * sizeof(float2));
  cudaStream_t s = (cudaStream_t)stream;
  if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, count * sizeof(float2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, count * sizeof(float2), s);
  float2* P = (float2*)kp_params_dev;
  const unsigned vb = kp_blocks(p.vol_elems(), p), pb = kp_blocks(count, p);
  AdamArgs la{};
  la.tv_xy = q.tv_xy;
  la.tv_t = q.tv_t;
  la.tv_eps = q.tv_eps;
  la.gscale = 2.f;
  for (int k = 1; k <= q.iters && e == cudaSuccess && st == PROP_OK; ++k) {
    e = launch_dep(kp_render_kernel, dim3(vb), dim3(kKpThreads), 0, s, (const float2*)P, a, p.vol2);
    if (e != cudaSuccess) break;
    if ((st = loss_grad_device(p, (const float2*)y_dev, la, p.vol2, p.grad, p.loss_dev + (k - 1), s)) != PROP_OK)
      break;
    e = cudaMemsetAsync(G, 0, count * sizeof(float2), s);
    if (e == cudaSuccess)
      e = launch_dep(kp_vjp_kernel, dim3(vb), dim3(kKpThreads), 0, s, (const float2*)P, a, (const float2*)p.grad, G);
    AdamArgs ad{};
    const double bc1 = 1.0 - std::pow((double)q.beta1, k), bc2 = 1.0 - std::pow((double)q.beta2, k);
    ad.lr_t = (float)(q.lr / bc1);
    ad.inv_bc2_sqrt = (float)(1.0 / std::sqrt(bc2));
    ad.beta1 = q.beta1;
    ad.beta2 = q.beta2;
    ad.eps = q.eps;
    if (e == cudaSuccess) e = launch_dep(kp_adam_kernel, dim3(pb), dim3(kKpThreads), 0, s, P, (const float2*)G, m, v, count, ad);
  }
  if (e == cudaSuccess && st == PROP_OK && loss_trace_host && q.iters > 0) {
    e = cudaMemcpyAsync(loss_trace_host, p.loss_dev, sizeof(double) * q.iters, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the work buffers are released below
  plan_dev_free(&p, G);
  plan_dev_free(&p, m);
  plan_dev_free(&p, v);
  if (st != PROP_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "kplanes_reconstruct");
  return PROP_OK;
}

}  // extern "C"
