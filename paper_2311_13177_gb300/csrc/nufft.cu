// Type-2 interpolation (forward) and type-1 spread (adjoint) between the
// oversampled grid and the blade samples.
//
// Forward, per sample m of blade b (frame t(b), readout index j):
//   y_m = s * sum_f P[j][f] * sum_{a,c < 6} w2[a] w1[c] G_{t,f}[u2 + a][u1 + c]
// i.e. the 6x6-tap Kaiser-Bessel interpolation of every bin's grid, times
// the displacement phase exp(-2 pi i k_r Delta_f) (Sec. 3: a material
// displaced along the readout picks up a phase linear in k_r), summed over
// the bins.  Bins are the fastest axis of the grid, so the lanes of a warp
// that serve one sample read consecutive bins of the same cell (256 B per
// warp load for 32 bins).
//
// Adjoint: G'_{t,f}[cell] = sum_m w(m, cell) conj(P[j_m][f]) r_m.  The grid
// is cut into 16x16-cell tiles; each CTA owns one tile, accumulates the
// contributions of the samples listed for it (plan-time CSR, a sample is
// listed in every tile its footprint touches) in shared memory, and writes
// the finished tile once.  No global atomics; every grid cell is written by
// exactly one CTA.
#include "prop_internal.cuh"

namespace prop {
namespace {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulcf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}

struct InterpArgs {
  const float2* grid;
  const uint32_t* kb_idx;
  const float4* kb_w;
  const float2* phase;
  const int* blade_frame;
  float2* y;
  const float2* y_meas;
  double* partials;
  unsigned int* counter;
  double* sumsq_out;
  int M, LR, R, n, C, Cv, f0, Nf;
  float scale;
  int accumulate;
};

constexpr int kInterpThreads = 256;

// Sum of one double per thread; result valid in thread 0.
__device__ double block_sum(double v, double* sh) {
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

template <int LP>
__global__ void __launch_bounds__(kInterpThreads) interp_kernel(InterpArgs a) {
  constexpr int SPW = 32 / LP;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LP - 1);
  const int slot = lane / LP;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarp = ((long)gridDim.x * blockDim.x) >> 5;
  const size_t nC = (size_t)a.n * a.C;
  float sumsq = 0.f;
  for (long m0 = warp * SPW; m0 < a.M; m0 += nwarp * SPW) {
    const long m = m0 + slot;
    const bool valid = m < a.M;
    float2 tot = make_float2(0.f, 0.f);
    if (valid) {
      const uint32_t idx = __ldg(&a.kb_idx[m]);
      const int i1 = idx & 0xffff, i2 = idx >> 16;
      const float4 wa = __ldg(&a.kb_w[3 * m]), wb = __ldg(&a.kb_w[3 * m + 1]),
                   wc = __ldg(&a.kb_w[3 * m + 2]);
      const float w1[6] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y};
      const float w2[6] = {wb.z, wb.w, wc.x, wc.y, wc.z, wc.w};
      const int b = (int)(m / a.LR);
      const int j = (int)(m % a.R);
      const int t = __ldg(&a.blade_frame[b]);
      const float2* G = a.grid + (size_t)t * a.n * nC;
      int col[6], row[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        int c = i1 + q;
        col[q] = (c >= a.n ? c - a.n : c) * a.C;
        int r = i2 + q;
        row[q] = r >= a.n ? r - a.n : r;
      }
      const float2* P = a.phase + (size_t)j * a.Nf + a.f0;
      for (int f = sub; f < a.Cv; f += LP) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const float2* Gr = G + (size_t)row[q] * nC + f;
          float2 ra = make_float2(0.f, 0.f);
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const float2 g = __ldg(Gr + col[c]);
            ra.x = fmaf(w1[c], g.x, ra.x);
            ra.y = fmaf(w1[c], g.y, ra.y);
          }
          acc.x = fmaf(w2[q], ra.x, acc.x);
          acc.y = fmaf(w2[q], ra.y, acc.y);
        }
        const float2 ph = __ldg(P + f);
        const float2 z = cmulf(ph, acc);
        tot.x += z.x;
        tot.y += z.y;
      }
    }
#pragma unroll
    for (int o = LP / 2; o > 0; o >>= 1) {
      tot.x += __shfl_xor_sync(0xffffffffu, tot.x, o);
      tot.y += __shfl_xor_sync(0xffffffffu, tot.y, o);
    }
    if (valid && sub == 0) {
      float2 v = make_float2(tot.x * a.scale, tot.y * a.scale);
      if (a.accumulate) {
        const float2 old = a.y[m];
        v.x += old.x;
        v.y += old.y;
      } else if (a.y_meas) {
        const float2 ym = __ldg(&a.y_meas[m]);
        v.x -= ym.x;
        v.y -= ym.y;
      }
      a.y[m] = v;
      sumsq = fmaf(v.x, v.x, fmaf(v.y, v.y, sumsq));
    }
  }
  if (a.partials) {
    __shared__ double sh[32];
    __shared__ bool last;
    const double bs = block_sum((double)sumsq, sh);
    if (threadIdx.x == 0) {
      a.partials[blockIdx.x] = bs;
      __threadfence();
      const unsigned prev = atomicAdd(a.counter, 1u);
      last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double s = 0.0;
      for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(&a.partials[i]);
      s = block_sum(s, sh);
      if (threadIdx.x == 0) {
        *a.sumsq_out = s;
        *a.counter = 0u;
      }
    }
  }
}

struct SpreadArgs {
  float2* grid;
  const uint32_t* kb_idx;
  const float4* kb_w;
  const float2* phase;
  const int* tile_off;
  const int* tile_samples;
  const float2* r;
  int n, tps, C, Cv, f0, Nf, R;
};

constexpr int kSpreadThreads = 256;

template <int LP>
__global__ void __launch_bounds__(kSpreadThreads) spread_kernel(SpreadArgs a) {
  extern __shared__ float sacc[];  // [2][kTile*kTile][C]: real plane, imaginary plane
  constexpr int NG = 32 / LP;      // tap-row groups per warp
  constexpr int CELLS = kTile * kTile;
  const int C = a.C;
  float* acc_re = sacc;
  float* acc_im = sacc + CELLS * C;
  const int tile = blockIdx.x;
  const int tpp = a.tps * a.tps;
  const int t = tile / tpp;
  const int tr = (tile / a.tps) % a.tps;
  const int tc = tile % a.tps;
  const int r0 = tr * kTile, c0 = tc * kTile;
  for (int i = threadIdx.x; i < 2 * CELLS * C; i += blockDim.x) sacc[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LP - 1);
  const int grp = lane / LP;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const int beg = __ldg(&a.tile_off[tile]), end = __ldg(&a.tile_off[tile + 1]);
  for (int e = beg + warp; e < end; e += nwarp) {
    const int m = __ldg(&a.tile_samples[e]);
    const uint32_t idx = __ldg(&a.kb_idx[m]);
    const int i1 = idx & 0xffff, i2 = idx >> 16;
    const float4 wa = __ldg(&a.kb_w[3 * (size_t)m]), wb = __ldg(&a.kb_w[3 * (size_t)m + 1]),
                 wc = __ldg(&a.kb_w[3 * (size_t)m + 2]);
    const float w1[6] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y};
    const float w2[6] = {wb.z, wb.w, wc.x, wc.y, wc.z, wc.w};
    const int j = m % a.R;
    const float2 rm = __ldg(&a.r[m]);
    const float2* P = a.phase + (size_t)j * a.Nf + a.f0;
    int lc[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      int c = i1 + q;
      c = c >= a.n ? c - a.n : c;
      lc[q] = c - c0;
    }
    for (int f = sub; f < a.Cv; f += LP) {
      const float2 cf = cmulcf(__ldg(P + f), rm);  // conj(P) * r
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        if (q % NG != grp) continue;
        int rr = i2 + q;
        rr = (rr >= a.n ? rr - a.n : rr) - r0;
        if (rr < 0 || rr >= kTile) continue;
        const float wr = w2[q];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          if (lc[c] < 0 || lc[c] >= kTile) continue;
          const float w = wr * w1[c];
          const int cell = rr * kTile + lc[c];
          atomicAdd(&acc_re[cell * C + f], w * cf.x);
          atomicAdd(&acc_im[cell * C + f], w * cf.y);
        }
      }
    }
  }
  __syncthreads();
  // Write the finished tile: cell rows are runs of kTile * C complex values.
  const size_t nC = (size_t)a.n * C;
  float2* G = a.grid + (size_t)t * a.n * nC;
  for (int i = threadIdx.x; i < CELLS * C; i += blockDim.x) {
    const int cell = i / C, f = i % C;
    const int rr = cell / kTile, cc = cell % kTile;
    G[(size_t)(r0 + rr) * nC + (size_t)(c0 + cc) * C + f] = make_float2(acc_re[i], acc_im[i]);
  }
}

int lanes_for(int Cv) {
  int lp = 1;
  while (lp < Cv && lp < 32) lp <<= 1;
  return lp;
}

}  // namespace

cudaError_t nufft_configure(int chunk) {
  const int smem = 2 * kTile * kTile * chunk * (int)sizeof(float);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(spread_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(spread_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(spread_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(spread_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(spread_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  return cudaFuncSetAttribute(spread_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t interp(const Plan& p, int f0, int nbins, float2* y, const float2* y_meas, bool accumulate,
                   const Reducer* red, double* sumsq, cudaStream_t s) {
  InterpArgs a{};
  a.grid = p.grid;
  a.kb_idx = p.kb_idx;
  a.kb_w = p.kb_w;
  a.phase = p.phase;
  a.blade_frame = p.blade_frame_d;
  a.y = y;
  a.y_meas = y_meas;
  a.partials = red ? red->partials : nullptr;
  a.counter = red ? red->counter : nullptr;
  a.sumsq_out = sumsq;
  a.M = p.M;
  a.LR = p.L * p.R;
  a.R = p.R;
  a.n = p.n;
  a.C = p.chunk;
  a.Cv = nbins;
  a.f0 = f0;
  a.Nf = p.Nf;
  a.scale = 1.0f / (float)p.N;
  a.accumulate = accumulate ? 1 : 0;
  const int lp = lanes_for(nbins);
  const long samples_per_block = (long)(kInterpThreads / 32) * (32 / lp);
  long blocks = (p.M + samples_per_block - 1) / samples_per_block;
  long cap = red ? std::min<long>(red->capacity, 16384) : 16384;
  if (blocks > cap) blocks = cap;
  dim3 grid((unsigned)blocks);
  switch (lp) {
    case 1: interp_kernel<1><<<grid, kInterpThreads, 0, s>>>(a); break;
    case 2: interp_kernel<2><<<grid, kInterpThreads, 0, s>>>(a); break;
    case 4: interp_kernel<4><<<grid, kInterpThreads, 0, s>>>(a); break;
    case 8: interp_kernel<8><<<grid, kInterpThreads, 0, s>>>(a); break;
    case 16: interp_kernel<16><<<grid, kInterpThreads, 0, s>>>(a); break;
    default: interp_kernel<32><<<grid, kInterpThreads, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t spread(const Plan& p, int f0, int nbins, const float2* r, cudaStream_t s) {
  SpreadArgs a{};
  a.grid = p.grid;
  a.kb_idx = p.kb_idx;
  a.kb_w = p.kb_w;
  a.phase = p.phase;
  a.tile_off = p.tile_off;
  a.tile_samples = p.tile_samples;
  a.r = r;
  a.n = p.n;
  a.tps = p.tiles_per_side;
  a.C = p.chunk;
  a.Cv = nbins;
  a.f0 = f0;
  a.Nf = p.Nf;
  a.R = p.R;
  const size_t smem = (size_t)2 * kTile * kTile * p.chunk * sizeof(float);
  const int lp = lanes_for(nbins);
  dim3 grid((unsigned)(p.T * p.tiles_per_side * p.tiles_per_side));
  switch (lp) {
    case 1: spread_kernel<1><<<grid, kSpreadThreads, smem, s>>>(a); break;
    case 2: spread_kernel<2><<<grid, kSpreadThreads, smem, s>>>(a); break;
    case 4: spread_kernel<4><<<grid, kSpreadThreads, smem, s>>>(a); break;
    case 8: spread_kernel<8><<<grid, kSpreadThreads, smem, s>>>(a); break;
    case 16: spread_kernel<16><<<grid, kSpreadThreads, smem, s>>>(a); break;
    default: spread_kernel<32><<<grid, kSpreadThreads, smem, s>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace prop
