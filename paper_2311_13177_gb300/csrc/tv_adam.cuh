// Per-voxel smoothed-TV gradient and Adam update, shared by the optimiser
// kernel and the fused inverse-FFT / update / forward-FFT row kernel so that
// both paths run the same arithmetic (Sec. 4.3: Adam on the data term plus
// total variation in space and, for dynamic series, time).
#pragma once

#include "prop_internal.cuh"

namespace prop {

// Every operation below is an explicitly rounded intrinsic or fmaf, so the
// compiler has no contraction left to decide: the kernels that inline these
// functions in different surroundings produce the same bits.

// d / sqrt(|d|^2 + eps^2) and sqrt(|d|^2 + eps^2)
__device__ __forceinline__ float2 tv_term(float2 d, float eps2, float* mag) {
  const float s = fmaf(d.x, d.x, fmaf(d.y, d.y, eps2));
  const float inv = rsqrtf(s);
  *mag = __fmul_rn(s, inv);
  return make_float2(__fmul_rn(d.x, inv), __fmul_rn(d.y, inv));
}
__device__ __forceinline__ float2 csub_rn(float2 a, float2 b) {
  return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
}
__device__ __forceinline__ float2 cadd_rn(float2 a, float2 b) {
  return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}

// The six neighbours of a voxel along x1, x2 and t (+ and -) and which of
// them exist: differences that would reach outside the volume are left out
// (no wrap-around).
struct TvNbrs {
  float2 x1p, x1m, x2p, x2m, tp, tm;
  bool h1p, h1m, h2p, h2m, htp, htm;
};

// TV gradients at a voxel of value x from its neighbours: forward
// differences along x1, x2 and t.  *gxy, *gt get the gradients of TV_xy and
// TV_t; the return value is this voxel's own share of the weighted TV value
// (the terms of the differences it is the lower end of).
__device__ __forceinline__ float voxel_tv_nb(float2 x, const TvNbrs& nb, float tv_xy, float tv_t, float eps2,
                                             float2* gxy_out, float2* gt_out) {
  float2 gxy = make_float2(0.f, 0.f), gt = make_float2(0.f, 0.f);
  float mag, sxy = 0.f, stt = 0.f;
  if (tv_xy != 0.f) {
    if (nb.h1p) {
      gxy = csub_rn(gxy, tv_term(csub_rn(nb.x1p, x), eps2, &mag));
      sxy = __fadd_rn(sxy, mag);
    }
    if (nb.h1m) gxy = cadd_rn(gxy, tv_term(csub_rn(x, nb.x1m), eps2, &mag));
    if (nb.h2p) {
      gxy = csub_rn(gxy, tv_term(csub_rn(nb.x2p, x), eps2, &mag));
      sxy = __fadd_rn(sxy, mag);
    }
    if (nb.h2m) gxy = cadd_rn(gxy, tv_term(csub_rn(x, nb.x2m), eps2, &mag));
  }
  if (tv_t != 0.f) {
    if (nb.htp) {
      gt = csub_rn(gt, tv_term(csub_rn(nb.tp, x), eps2, &mag));
      stt = __fadd_rn(stt, mag);
    }
    if (nb.htm) gt = cadd_rn(gt, tv_term(csub_rn(x, nb.tm), eps2, &mag));
  }
  *gxy_out = gxy;
  *gt_out = gt;
  return fmaf(tv_xy, sxy, __fmul_rn(tv_t, stt));
}

// voxel_tv_nb at voxel idx = ((t N + i2) N + i1) Nf + f of Vin (value x),
// loading the neighbours that exist.
__device__ __forceinline__ float voxel_tv(const float2* __restrict__ Vin, size_t idx, float2 x, int i1, int i2,
                                          int t, int N, int Nf, int T, float tv_xy, float tv_t, float eps2,
                                          float2* gxy_out, float2* gt_out) {
  const size_t sx = (size_t)Nf, sy = (size_t)N * Nf, st = (size_t)N * N * Nf;
  const float2 z = make_float2(0.f, 0.f);
  TvNbrs nb;
  nb.h1p = tv_xy != 0.f && i1 + 1 < N;
  nb.h1m = tv_xy != 0.f && i1 > 0;
  nb.h2p = tv_xy != 0.f && i2 + 1 < N;
  nb.h2m = tv_xy != 0.f && i2 > 0;
  nb.htp = tv_t != 0.f && t + 1 < T;
  nb.htm = tv_t != 0.f && t > 0;
  nb.x1p = nb.h1p ? Vin[idx + sx] : z;
  nb.x1m = nb.h1m ? Vin[idx - sx] : z;
  nb.x2p = nb.h2p ? Vin[idx + sy] : z;
  nb.x2m = nb.h2m ? Vin[idx - sy] : z;
  nb.tp = nb.htp ? Vin[idx + st] : z;
  nb.tm = nb.htm ? Vin[idx - st] : z;
  return voxel_tv_nb(x, nb, tv_xy, tv_t, eps2, gxy_out, gt_out);
}

// g = gscale * gd + tv_xy * gxy + tv_t * gt
__device__ __forceinline__ float2 total_grad(float2 gd, float2 gxy, float2 gt, const AdamArgs& p) {
  return make_float2(fmaf(p.gscale, gd.x, fmaf(p.tv_xy, gxy.x, __fmul_rn(p.tv_t, gt.x))),
                     fmaf(p.gscale, gd.y, fmaf(p.tv_xy, gxy.y, __fmul_rn(p.tv_t, gt.y))));
}

// Bias-corrected Adam on the real and imaginary parts; updates mm, vv and
// returns the new voxel value.
__device__ __forceinline__ float2 adam_voxel(float2 x, float2 g, float2& mm, float2& vv, const AdamArgs& p) {
  const float c1 = __fsub_rn(1.f, p.beta1), c2 = __fsub_rn(1.f, p.beta2);
  mm.x = fmaf(p.beta1, mm.x, __fmul_rn(c1, g.x));
  mm.y = fmaf(p.beta1, mm.y, __fmul_rn(c1, g.y));
  vv.x = fmaf(p.beta2, vv.x, __fmul_rn(__fmul_rn(c2, g.x), g.x));
  vv.y = fmaf(p.beta2, vv.y, __fmul_rn(__fmul_rn(c2, g.y), g.y));
  const float dx = fmaf(sqrtf(vv.x), p.inv_bc2_sqrt, p.eps);
  const float dy = fmaf(sqrtf(vv.y), p.inv_bc2_sqrt, p.eps);
  return make_float2(fmaf(-p.lr_t, __fdiv_rn(mm.x, dx), x.x), fmaf(-p.lr_t, __fdiv_rn(mm.y, dy), x.y));
}

// Block sum of one double per thread; valid in thread 0 (all threads call).
// sh holds 32 doubles.
__device__ __forceinline__ double block_sum_tv(double v, double* sh) {
  if (blockDim.x < 32) {  // narrower than a warp (length-16 transforms): no full-warp shuffles
    sh[threadIdx.x] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
      for (int i = 0; i < (int)blockDim.x; ++i) t += sh[i];
    __syncthreads();
    return t;
  }
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

// Deterministic loss: every block stores its partial TV sum, the last block
// to arrive adds them in block order plus the data term and writes the loss.
// Blocks are numbered linearly over a 2-D grid.
// vb, nblk: this block's index and the block count of the reduction (the
// launch's blocks, or the share of a multi-problem launch that serves one
// problem).
__device__ __forceinline__ void finish_loss_v(float local, double* partials, unsigned int* counter,
                                              const double* data_loss, double* loss_out, unsigned vb, unsigned nblk) {
  __shared__ double sh[32];
  __shared__ bool last;
  const double bs = block_sum_tv((double)local, sh);
  if (threadIdx.x == 0) {
    partials[vb] = bs;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = prev == nblk - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)nblk; i += blockDim.x) s += __ldcg(&partials[i]);
    s = block_sum_tv(s, sh);
    if (threadIdx.x == 0) {
      *loss_out = s + (data_loss ? __ldcg(data_loss) : 0.0);
      *counter = 0u;
    }
  }
}
__device__ __forceinline__ void finish_loss(float local, double* partials, unsigned int* counter,
                                            const double* data_loss, double* loss_out) {
  finish_loss_v(local, partials, counter, data_loss, loss_out, blockIdx.y * gridDim.x + blockIdx.x,
                gridDim.x * gridDim.y);
}

}  // namespace prop
