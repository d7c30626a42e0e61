// The paper's own forward model (Sec. 4.2-4.3) on the GPU.
//
// Projection: a ray per pixel, tilted from the spectral axis in the plane of
// that axis and the blade's readout direction, meets spectral slice f at the
// in-plane point p - Delta_f d_b; the sample there is the bilinear
// interpolation of the slice (zero outside the image), and the pixel is the
// sum over the slices.  Blur: the centred unitary 2-D DFT of the projected
// image, masked by the blade's support on the Cartesian grid.  Fit: Adam,
// one blade per iteration in turn, on w_k |M (Z - y)|^2 + w_i |U^H M Z - img|^2
// plus smoothed TV along x1, x2, the spectral axis and time, and L1.
//
// One iteration is six launches: the projection (a gather, one warp per
// pixel with the bins across the lanes), four passes of N-point transforms
// (the forward column pass fused with the mask, the residuals, the data
// loss and the data-term gradient 2 M (w_k r_k + w_i r_i); the image term is
// taken through the unitary DFT, ||U^H M Z - img||^2 = ||M (Z - U img)||^2
// + ||(1 - M) U img||^2, with the second part a per-blade constant computed
// once), and a fused update: for every voxel the transposed projection (a
// gather of the four pixels that read it, so no atomics), the TV and L1
// gradients, Adam, and the FP64 loss.
#include "prop_internal.cuh"
#include "tv_adam.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace prop {
namespace {

constexpr int kProjThreads = 256;

// Projected image of blade b, frame t: img[i2][i1] = sum_f bilinear(V_t[., ., f],
// (i1, i2) - s_f).  sh[f] = (o1, o2, w1 bits, w2 bits): along axis a the
// pixel reads taps i + o_a (weight 1 - w_a) and i + o_a + 1 (weight w_a).
// A warp takes kProjPix adjacent pixels of one row, its lanes the bins: the
// pixels share all but one of their x1 taps, so each bin loads kProjPix + 1
// values per tap row.
constexpr int kProjPix = 4;
__global__ void __launch_bounds__(kProjThreads) proj_image_kernel(const float2* __restrict__ V,
                                                                  const int4* __restrict__ sh, int N, int Nf, int t,
                                                                  float2* __restrict__ img) {
  grid_dep_wait();
  grid_dep_release();
  const int lane = threadIdx.x & 31;
  const long pix0 = ((long)blockIdx.x * (kProjThreads / 32) + (threadIdx.x >> 5)) * kProjPix;
  if (pix0 >= (long)N * N) return;  // whole warps leave together
  const int i2 = (int)(pix0 / N), i10 = (int)(pix0 - (long)i2 * N);  // N % kProjPix == 0: one row
  const float2* Vt = V + (size_t)t * N * N * Nf;
  float ax[kProjPix], ay[kProjPix];
#pragma unroll
  for (int q = 0; q < kProjPix; ++q) ax[q] = ay[q] = 0.f;
  for (int f = lane; f < Nf; f += 32) {
    const int4 o = __ldg(&sh[f]);
    const float w1 = __int_as_float(o.z), w2 = __int_as_float(o.w);
    const int j1 = i10 + o.x, j2 = i2 + o.y;
#pragma unroll
    for (int d2 = 0; d2 < 2; ++d2) {
      const int r = j2 + d2;
      if (r < 0 || r >= N) continue;
      const float c2 = d2 ? w2 : 1.f - w2;
      float2 v[kProjPix + 1];
#pragma unroll
      for (int k = 0; k <= kProjPix; ++k) {
        const int c = j1 + k;
        v[k] = (c >= 0 && c < N) ? __ldg(&Vt[((size_t)r * N + c) * Nf + f]) : make_float2(0.f, 0.f);
      }
      const float wl = c2 * (1.f - w1), wh = c2 * w1;
#pragma unroll
      for (int q = 0; q < kProjPix; ++q) {
        ax[q] = fmaf(wh, v[q + 1].x, fmaf(wl, v[q].x, ax[q]));
        ay[q] = fmaf(wh, v[q + 1].y, fmaf(wl, v[q].y, ay[q]));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kProjPix; ++q) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      ax[q] += __shfl_xor_sync(0xffffffffu, ax[q], s);
      ay[q] += __shfl_xor_sync(0xffffffffu, ay[q], s);
    }
  }
  if (lane < kProjPix) {
    float bx = ax[0], by = ay[0];
#pragma unroll
    for (int q = 1; q < kProjPix; ++q)
      if (lane == q) {
        bx = ax[q];
        by = ay[q];
      }
    img[pix0 + lane] = make_float2(bx, by);
  }
}

// Transposed projection at voxel (i2, i1, f): pixel p reads voxel p + o
// (weight 1 - w) and p + o + 1 (weight w) along each axis, so the voxel
// gathers from p = i - o (weight 1 - w) and p = i - o - 1 (weight w).
__device__ __forceinline__ float2 proj_gather(const float2* __restrict__ g, int4 o, int N, int i1, int i2) {
  const float w1 = __int_as_float(o.z), w2 = __int_as_float(o.w);
  float ax = 0.f, ay = 0.f;
#pragma unroll
  for (int d2 = 0; d2 < 2; ++d2) {
    const int p2 = i2 - o.y - d2;
    if (p2 < 0 || p2 >= N) continue;
    const float c2 = d2 ? w2 : 1.f - w2;
#pragma unroll
    for (int d1 = 0; d1 < 2; ++d1) {
      const int p1 = i1 - o.x - d1;
      if (p1 < 0 || p1 >= N) continue;
      const float w = c2 * (d1 ? w1 : 1.f - w1);
      const float2 v = g[(size_t)p2 * N + p1];
      ax = fmaf(w, v.x, ax);
      ay = fmaf(w, v.y, ay);
    }
  }
  return make_float2(ax, ay);
}

// V = P_b^H g in frame tb, zero in the other frames.
__global__ void __launch_bounds__(kProjThreads) proj_adjoint_kernel(const float2* __restrict__ g,
                                                                    const int4* __restrict__ sh, int N, int Nf, int T,
                                                                    int tb, float2* __restrict__ V) {
  grid_dep_wait();
  grid_dep_release();
  const size_t total = (size_t)T * N * N * Nf;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(idx % Nf);
    size_t r = idx / Nf;
    const int i1 = (int)(r % N);
    r /= N;
    const int i2 = (int)(r % N);
    const int t = (int)(r / N);
    V[idx] = t == tb ? proj_gather(g, __ldg(&sh[f]), N, i1, i2) : make_float2(0.f, 0.f);
  }
}

struct ProjUpdArgs {
  const float2* Vin;
  float2* Vout;
  float2* m;
  float2* v;
  const float2* gimg;  // [N][N] image-space gradient of the data term (U^H of the masked k-space gradient)
  const int4* sh;      // [Nf] shifts of the iteration's blade
  int N, Nf, T, tb;
  AdamArgs ad;         // gscale 1 (gimg already holds the factor 2 and the weights)
  float tv_f, l1;
  double* partials;
  unsigned int* counter;
  const double* data_loss;
  double* loss_out;
};

// Fused update: data gradient by the transposed projection, TV along x1, x2
// and t (the same arithmetic as the non-uniform model's update), TV along
// the spectral axis, L1, Adam, and the FP64 loss of the iterate it reads.
// Grid: (blocks per image row, T N rows); 32-bit index math within a row.
// Every neighbour load is unconditional (a missing neighbour reads the voxel
// itself and is not used), so the loads of several voxels are in flight
// together; TT: the volume has time neighbours.
template <bool TT>
__global__ void __launch_bounds__(kProjThreads) proj_update_kernel(ProjUpdArgs a) {
  grid_dep_wait();
  grid_dep_release();
  const int row = blockIdx.y;  // t N + i2
  const int i2 = row % a.N, t = row / a.N;
  const int rl = a.N * a.Nf;
  const size_t base = (size_t)row * rl;
  const size_t sx = (size_t)a.Nf, sy = (size_t)rl, st = (size_t)a.N * rl;
  const float eps2 = a.ad.tv_eps * a.ad.tv_eps;
  const bool xy = a.ad.tv_xy != 0.f;
  const bool h2p = xy && i2 + 1 < a.N, h2m = xy && i2 > 0;
  const bool htp = TT && t + 1 < a.T, htm = TT && t > 0;
  const bool data = t == a.tb;
  const float2* __restrict__ Vin = a.Vin;
  float local = 0.f;
#pragma unroll 2
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rl; e += gridDim.x * blockDim.x) {
    const int i1 = e / a.Nf;
    const int f = e - i1 * a.Nf;
    const size_t idx = base + e;
    const float2 x = Vin[idx];
    TvNbrs nb;
    nb.h1p = xy && i1 + 1 < a.N;
    nb.h1m = xy && i1 > 0;
    nb.h2p = h2p;
    nb.h2m = h2m;
    nb.htp = htp;
    nb.htm = htm;
    nb.x1p = Vin[nb.h1p ? idx + sx : idx];
    nb.x1m = Vin[nb.h1m ? idx - sx : idx];
    nb.x2p = Vin[h2p ? idx + sy : idx];
    nb.x2m = Vin[h2m ? idx - sy : idx];
    if constexpr (TT) {
      nb.tp = Vin[htp ? idx + st : idx];
      nb.tm = Vin[htm ? idx - st : idx];
    } else {
      nb.tp = nb.tm = x;
    }
    const bool hfp = a.tv_f != 0.f && f + 1 < a.Nf, hfm = a.tv_f != 0.f && f > 0;
    const float2 xfp = Vin[hfp ? idx + 1 : idx];
    const float2 xfm = Vin[hfm ? idx - 1 : idx];
    float2 mm = a.m[idx], vv = a.v[idx];
    const float2 gd = data ? proj_gather(a.gimg, __ldg(&a.sh[f]), a.N, i1, i2) : make_float2(0.f, 0.f);
    float2 gxy, gt;
    float tv = voxel_tv_nb(x, nb, a.ad.tv_xy, TT ? a.ad.tv_t : 0.f, eps2, &gxy, &gt);
    float2 gf = make_float2(0.f, 0.f);
    float mag;
    if (hfp) {
      gf = csub_rn(gf, tv_term(csub_rn(xfp, x), eps2, &mag));
      tv = fmaf(a.tv_f, mag, tv);
    }
    if (hfm) gf = cadd_rn(gf, tv_term(csub_rn(x, xfm), eps2, &mag));
    float2 gl = make_float2(0.f, 0.f);
    if (a.l1 != 0.f) {
      gl = tv_term(x, eps2, &mag);  // x / sqrt(|x|^2 + eps^2) and the smoothed modulus
      tv = fmaf(a.l1, mag, tv);
    }
    float2 g = total_grad(gd, gxy, gt, a.ad);
    g.x = fmaf(a.l1, gl.x, fmaf(a.tv_f, gf.x, g.x));
    g.y = fmaf(a.l1, gl.y, fmaf(a.tv_f, gf.y, g.y));
    local = __fadd_rn(local, tv);
    const float2 nx = adam_voxel(x, g, mm, vv, a.ad);
    a.m[idx] = mm;
    a.v[idx] = vv;
    a.Vout[idx] = nx;
  }
  finish_loss(local, a.partials, a.counter, a.data_loss, a.loss_out);
}

// c[b] = w_i sum over cells outside blade b's mask of |U img_b|^2 (one block per blade).
__global__ void __launch_bounds__(kProjThreads) proj_const_kernel(const float2* __restrict__ yimg,
                                                                  const uint8_t* __restrict__ mask, int N, float wi,
                                                                  double* __restrict__ c) {
  grid_dep_wait();
  grid_dep_release();
  __shared__ double sh[32];
  const size_t n2 = (size_t)N * N;
  const float2* yb = yimg + blockIdx.x * n2;
  const uint8_t* mb = mask + blockIdx.x * n2;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n2; i += blockDim.x)
    if (!mb[i]) s += (double)yb[i].x * yb[i].x + (double)yb[i].y * yb[i].y;
  s = block_sum_tv(s, sh);
  if (threadIdx.x == 0) c[blockIdx.x] = (double)wi * s;
}

// Coverage-weighted k-space average of blades lo .. hi-1: each cell averages
// the blades whose mask holds it (zero where none does).
__global__ void __launch_bounds__(kProjThreads) proj_baseline_kernel(const float2* __restrict__ y,
                                                                     const uint8_t* __restrict__ mask, int N, int lo,
                                                                     int hi, float2* __restrict__ out) {
  grid_dep_wait();
  grid_dep_release();
  const size_t n2 = (size_t)N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    float sx = 0.f, sy = 0.f;
    int c = 0;
    for (int b = lo; b < hi; ++b)
      if (mask[b * n2 + i]) {
        const float2 v = y[b * n2 + i];
        sx += v.x;
        sy += v.y;
        ++c;
      }
    out[i] = c > 0 ? make_float2(sx / (float)c, sy / (float)c) : make_float2(0.f, 0.f);
  }
}

// Blocks per image row of the update: about 8 voxels a thread, at most 4.
int update_row_blocks(const Plan& p) {
  const int rl = p.N * p.Nf;
  return std::max(1, std::min(4, rl / (8 * kProjThreads)));
}

// Allocates *ptr unless a previous, interrupted set-up already did.
prop_status proj_alloc(Plan& p, void** ptr, size_t bytes, const char* what) {
  if (*ptr) return PROP_OK;
  cudaError_t e = plan_dev_alloc(&p, ptr, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(PROP_ERR_OOM, std::string("cudaMalloc failed for ") + what);
  }
  p.recon_bytes += std::max<size_t>(bytes, 16);
  return PROP_OK;
}

// Rotated coordinates within 1e-9 of a half-integer are that half-integer.
double snap_half(double a) {
  const double h = std::round(2.0 * a) / 2.0;
  return std::fabs(a - h) < 1e-9 ? h : a;
}

}  // namespace

prop_status plan_ensure_proj(Plan& p, bool images) {
  prop_status st;
  if (!p.proj_ready) {
    if (p.N < 16) return fail(PROP_ERR_INVALID_ARG, "projection model: N must be at least 16");
    const int N = p.N, B = p.B, Nf = p.Nf;
    const size_t n2 = (size_t)N * N;
    // per (blade, bin) taps and weights, FP64 -> FP32
    std::vector<int4> sh((size_t)B * Nf);
    for (int b = 0; b < B; ++b) {
      const double c = std::cos(p.theta[b]), s = std::sin(p.theta[b]);
      for (int f = 0; f < Nf; ++f) {
        const double s1 = p.delta[f] * c, s2 = p.delta[f] * s;
        const double o1 = std::floor(-s1), o2 = std::floor(-s2);
        const float w1 = (float)(-s1 - o1), w2 = (float)(-s2 - o2);
        int4 v;
        v.x = (int)o1;
        v.y = (int)o2;
        std::memcpy(&v.z, &w1, sizeof(float));
        std::memcpy(&v.w, &w2, sizeof(float));
        sh[(size_t)b * Nf + f] = v;
      }
    }
    // blade supports on the Cartesian grid
    std::vector<uint8_t> mask((size_t)B * n2);
    for (int b = 0; b < B; ++b) {
      const double c = std::cos(p.theta[b]), s = std::sin(p.theta[b]);
      for (int u2 = 0; u2 < N; ++u2)
        for (int u1 = 0; u1 < N; ++u1) {
          const double c1 = u1 - N / 2.0, c2 = u2 - N / 2.0;
          const double rho = snap_half(c1 * c + c2 * s), pi = snap_half(-c1 * s + c2 * c);
          const bool in = rho >= -p.R / 2.0 - 0.5 && rho < p.R / 2.0 - 0.5 && pi >= -p.L / 2.0 - 0.5 &&
                          pi < p.L / 2.0 - 0.5;
          mask[(size_t)b * n2 + (size_t)u2 * N + u1] = in ? 1 : 0;
        }
    }
    std::vector<float2> tw(N);
    for (int m = 0; m < N; ++m) {
      const double a = -2.0 * M_PI * m / N;
      tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    const int red_u = update_row_blocks(p) * p.T * N;
    const int red_k = std::max(N / kCartCols, 32);  // the loss pass's CTAs
    if ((st = proj_alloc(p, (void**)&p.proj_shift, sh.size() * sizeof(int4), "projection shifts")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.proj_mask, mask.size(), "blade masks")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.proj_twiddle, N * sizeof(float2), "DFT twiddles")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.proj_img, n2 * sizeof(float2), "projected image")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.proj_k, n2 * sizeof(float2), "k-space work")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.proj_kg, n2 * sizeof(float2), "k-space gradient")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.proj_g, n2 * sizeof(float2), "image gradient")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.proj_const, B * sizeof(double), "image-term constants")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.red_proj_k.partials, red_k * sizeof(double), "partials")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.red_proj_k.counter, sizeof(unsigned), "counter")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.red_proj_u.partials, red_u * sizeof(double), "partials")) != PROP_OK) return st;
    if ((st = proj_alloc(p, (void**)&p.red_proj_u.counter, sizeof(unsigned), "counter")) != PROP_OK) return st;
    p.red_proj_k.capacity = red_k;
    p.red_proj_u.capacity = red_u;
    PROP_CUDA(cudaMemcpy(p.proj_shift, sh.data(), sh.size() * sizeof(int4), cudaMemcpyHostToDevice));
    PROP_CUDA(cudaMemcpy(p.proj_mask, mask.data(), mask.size(), cudaMemcpyHostToDevice));
    PROP_CUDA(cudaMemcpy(p.proj_twiddle, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice));
    PROP_CUDA(cudaMemset(p.red_proj_k.counter, 0, sizeof(unsigned)));
    PROP_CUDA(cudaMemset(p.red_proj_u.counter, 0, sizeof(unsigned)));
    PROP_CUDA(cart_fft_configure(N));
    p.proj_ready = true;
  }
  if (images && !p.proj_yimg) {
    if ((st = proj_alloc(p, (void**)&p.proj_yimg, (size_t)p.B * p.N * p.N * sizeof(float2), "image spectra")) !=
        PROP_OK)
      return st;
  }
  return PROP_OK;
}

namespace {

const int4* blade_shifts(const Plan& p, int b) { return p.proj_shift + (size_t)b * p.Nf; }
const uint8_t* blade_mask(const Plan& p, int b) { return p.proj_mask + (size_t)b * p.N * p.N; }

// Z = M_b U P_b V_t(b) into z (or, with `loss`, the data term and its k-space gradient into p.proj_kg).
prop_status proj_forward_impl(Plan& p, int b, const float2* V, float2* z, const CartLoss* loss, cudaStream_t s) {
  const long warps = (long)p.N * p.N / kProjPix;
  const unsigned blocks = (unsigned)((warps + kProjThreads / 32 - 1) / (kProjThreads / 32));
  PROP_CUDA(launch_dep(proj_image_kernel, dim3(blocks), dim3(kProjThreads), 0, s, V, blade_shifts(p, b), p.N, p.Nf,
                      p.blade_frame[b], p.proj_img));
  PROP_CUDA(cart_fft_pass(p.N, kCartRowsFwd, p.proj_img, p.proj_k, p.proj_twiddle, nullptr, nullptr, 1.f, s));
  PROP_CUDA(cart_fft_pass(p.N, kCartColsFwd, p.proj_k, loss ? p.proj_kg : z, p.proj_twiddle, blade_mask(p, b), loss,
                         1.f / (float)p.N, s));
  return PROP_OK;
}

// g = U^H M_b z (image space) into p.proj_g.
prop_status proj_kadjoint_impl(Plan& p, int b, const float2* z, cudaStream_t s) {
  PROP_CUDA(cart_fft_pass(p.N, kCartColsInv, z, p.proj_k, p.proj_twiddle, blade_mask(p, b), nullptr, 1.f, s));
  PROP_CUDA(cart_fft_pass(p.N, kCartRowsInv, p.proj_k, p.proj_g, p.proj_twiddle, nullptr, nullptr, 1.f / (float)p.N, s));
  return PROP_OK;
}

prop_status check_proj_params(const prop_proj_params* q) {
  if (!q) return fail(PROP_ERR_INVALID_ARG, "projection params are NULL");
  if (q->iters < 0) return fail(PROP_ERR_INVALID_ARG, "iters must be >= 0");
  if (!(q->lr >= 0.f) || !(q->beta1 >= 0.f && q->beta1 < 1.f) || !(q->beta2 >= 0.f && q->beta2 < 1.f) ||
      !(q->eps > 0.f))
    return fail(PROP_ERR_INVALID_ARG, "Adam parameters out of range");
  const float w[] = {q->w_kspace, q->w_image, q->tv_xy, q->tv_f, q->tv_t, q->l1};
  for (float v : w)
    if (!(v >= 0.f) || !std::isfinite(v)) return fail(PROP_ERR_INVALID_ARG, "weights must be finite and >= 0");
  if (!(q->tv_eps > 0.f)) return fail(PROP_ERR_INVALID_ARG, "tv_eps must be > 0");
  return PROP_OK;
}

}  // namespace

}  // namespace prop

using namespace prop;

extern "C" {

prop_status prop_proj_forward(prop_plan plan, int blade, const void* V_dev, void* z_dev, void* stream) {
  if (!plan || !V_dev || !z_dev) return fail(PROP_ERR_INVALID_ARG, "proj_forward: null argument");
  Plan& p = *plan->p;
  if (blade < 0 || blade >= p.B) return fail(PROP_ERR_INVALID_ARG, "proj_forward: blade out of range");
  DeviceGuard g(p.device);
  prop_status st = plan_ensure_proj(p, false);
  if (st != PROP_OK) return st;
  return proj_forward_impl(p, blade, (const float2*)V_dev, (float2*)z_dev, nullptr, (cudaStream_t)stream);
}

prop_status prop_proj_adjoint(prop_plan plan, int blade, const void* z_dev, void* V_dev, void* stream) {
  if (!plan || !V_dev || !z_dev) return fail(PROP_ERR_INVALID_ARG, "proj_adjoint: null argument");
  Plan& p = *plan->p;
  if (blade < 0 || blade >= p.B) return fail(PROP_ERR_INVALID_ARG, "proj_adjoint: blade out of range");
  DeviceGuard g(p.device);
  prop_status st = plan_ensure_proj(p, false);
  if (st != PROP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = proj_kadjoint_impl(p, blade, (const float2*)z_dev, s)) != PROP_OK) return st;
  PROP_CUDA(launch_dep(proj_adjoint_kernel, dim3((unsigned)(8 * p.num_sms)), dim3(kProjThreads), 0, s,
                      (const float2*)p.proj_g, blade_shifts(p, blade), p.N, p.Nf, p.T, p.blade_frame[blade],
                      (float2*)V_dev));
  return PROP_OK;
}

prop_status prop_proj_baseline(prop_plan plan, const void* ycart_dev, int blade_lo, int blade_hi, void* img_dev,
                               void* stream) {
  if (!plan || !ycart_dev || !img_dev) return fail(PROP_ERR_INVALID_ARG, "proj_baseline: null argument");
  Plan& p = *plan->p;
  if (blade_lo < 0 || blade_hi > p.B || blade_lo >= blade_hi)
    return fail(PROP_ERR_INVALID_ARG, "proj_baseline: need 0 <= blade_lo < blade_hi <= B");
  DeviceGuard g(p.device);
  prop_status st = plan_ensure_proj(p, false);
  if (st != PROP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  PROP_CUDA(launch_dep(proj_baseline_kernel, dim3((unsigned)(4 * p.num_sms)), dim3(kProjThreads), 0, s,
                       (const float2*)ycart_dev, (const uint8_t*)p.proj_mask, p.N, blade_lo, blade_hi, p.proj_kg));
  PROP_CUDA(cart_fft_pass(p.N, kCartColsInv, p.proj_kg, p.proj_k, p.proj_twiddle, nullptr, nullptr, 1.f, s));
  PROP_CUDA(cart_fft_pass(p.N, kCartRowsInv, p.proj_k, (float2*)img_dev, p.proj_twiddle, nullptr, nullptr,
                          1.f / (float)p.N, s));
  return PROP_OK;
}

prop_status prop_proj_reconstruct(prop_plan plan, const void* ycart_dev, const void* img_dev,
                                  const prop_proj_params* params, void* V_dev, double* loss_trace_host,
                                  void* stream) {
  if (!plan || !ycart_dev || !V_dev) return fail(PROP_ERR_INVALID_ARG, "proj_reconstruct: null argument");
  prop_status st = check_proj_params(params);
  if (st != PROP_OK) return st;
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  const prop_proj_params& q = *params;
  if ((st = plan_ensure_recon(&p, std::max(q.iters, 1))) != PROP_OK) return st;
  if ((st = plan_ensure_proj(p, img_dev != nullptr)) != PROP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n2 = (size_t)p.N * p.N;
  const size_t vbytes = p.vol_elems() * sizeof(float2);
  const float2* ycart = (const float2*)ycart_dev;
  if (img_dev) {
    // U img_b for every blade, and the image term's constant outside each mask
    for (int b = 0; b < p.B; ++b) {
      PROP_CUDA(cart_fft_pass(p.N, kCartRowsFwd, (const float2*)img_dev + b * n2, p.proj_k, p.proj_twiddle, nullptr,
                             nullptr, 1.f, s));
      PROP_CUDA(cart_fft_pass(p.N, kCartColsFwd, p.proj_k, p.proj_yimg + b * n2, p.proj_twiddle, nullptr, nullptr,
                             1.f / (float)p.N, s));
    }
    PROP_CUDA(launch_dep(proj_const_kernel, dim3((unsigned)p.B), dim3(kProjThreads), 0, s,
                        (const float2*)p.proj_yimg, (const uint8_t*)p.proj_mask, p.N, q.w_image, p.proj_const));
  }
  PROP_CUDA(cudaMemsetAsync(p.adam_m, 0, vbytes, s));
  PROP_CUDA(cudaMemsetAsync(p.adam_v, 0, vbytes, s));
  float2* cur = (float2*)V_dev;
  float2* nxt = p.vol2;
  const dim3 ugrid((unsigned)update_row_blocks(p), (unsigned)(p.T * p.N));
  if ((long)ugrid.x * ugrid.y > p.red_proj_u.capacity) return fail(PROP_ERR_INVALID_ARG, "proj_reconstruct: reduction capacity");
  for (int k = 1; k <= q.iters; ++k) {
    const int b = (k - 1) % p.B;
    CartLoss loss{};
    loss.y = ycart + b * n2;
    loss.yimg = img_dev ? p.proj_yimg + b * n2 : nullptr;
    loss.wk = q.w_kspace;
    loss.wi = q.w_image;
    loss.red = &p.red_proj_k;
    loss.loss_const = img_dev ? p.proj_const + b : nullptr;
    loss.loss_out = p.scalars + 3;
    if ((st = proj_forward_impl(p, b, cur, nullptr, &loss, s)) != PROP_OK) return st;
    if ((st = proj_kadjoint_impl(p, b, p.proj_kg, s)) != PROP_OK) return st;
    ProjUpdArgs u{};
    u.Vin = cur;
    u.Vout = nxt;
    u.m = p.adam_m;
    u.v = p.adam_v;
    u.gimg = p.proj_g;
    u.sh = blade_shifts(p, b);
    u.N = p.N;
    u.Nf = p.Nf;
    u.T = p.T;
    u.tb = p.blade_frame[b];
    const double bc1 = 1.0 - std::pow((double)q.beta1, k);
    const double bc2 = 1.0 - std::pow((double)q.beta2, k);
    u.ad.lr_t = (float)(q.lr / bc1);
    u.ad.inv_bc2_sqrt = (float)(1.0 / std::sqrt(bc2));
    u.ad.beta1 = q.beta1;
    u.ad.beta2 = q.beta2;
    u.ad.eps = q.eps;
    u.ad.tv_xy = q.tv_xy;
    u.ad.tv_t = p.T > 1 ? q.tv_t : 0.f;
    u.ad.tv_eps = q.tv_eps;
    u.ad.gscale = 1.f;
    u.tv_f = q.tv_f;
    u.l1 = q.l1;
    u.partials = p.red_proj_u.partials;
    u.counter = p.red_proj_u.counter;
    u.data_loss = p.scalars + 3;
    u.loss_out = p.loss_dev + (k - 1);
    if (p.T > 1 && q.tv_t != 0.f)
      PROP_CUDA(launch_dep(proj_update_kernel<true>, ugrid, dim3(kProjThreads), 0, s, u));
    else
      PROP_CUDA(launch_dep(proj_update_kernel<false>, ugrid, dim3(kProjThreads), 0, s, u));
    std::swap(cur, nxt);
  }
  if (cur != (float2*)V_dev) PROP_CUDA(cudaMemcpyAsync(V_dev, cur, vbytes, cudaMemcpyDeviceToDevice, s));
  if (loss_trace_host && q.iters > 0) {
    PROP_CUDA(cudaMemcpyAsync(loss_trace_host, p.loss_dev, sizeof(double) * q.iters, cudaMemcpyDeviceToHost, s));
    PROP_CUDA(cudaStreamSynchronize(s));
  }
  return PROP_OK;
}

}  // extern "C"
