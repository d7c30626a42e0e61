// Type-2 interpolation (forward) and type-1 spread (adjoint) between the
// oversampled grid and the blade samples.
//
// Forward, per sample m of blade b (frame t(b), readout index j):
//   y_m = s * sum_f P[j][f] * sum_{a,c < W} w2[a] w1[c] G_{t,f}[u2 + a][u1 + c]
// i.e. the W x W-tap Kaiser-Bessel interpolation of every bin's grid, times
// the displacement phase exp(-2 pi i k_r Delta_f) (Sec. 3: a material
// displaced along the readout picks up a phase linear in k_r), summed over
// the bins.  Bins are the fastest axis of the grid, so the lanes of a warp
// that serve one sample read consecutive bins of the same cell (256 B per
// warp load for 32 bins).  Samples are visited in the plan's tile-sorted
// order, so the warps of one CTA gather from one compact grid region.
//
// Adjoint: G'_{t,f}[cell] = sum_m w(m, cell) conj(P[j_m][f]) r_m.  The
// phased residual contrib[m][f] = conj(P[j_m][f]) r_m is formed once per
// sample (fused into the interpolation when the grid holds every bin), then
// every cell gathers its plan-time list of (sample, weight) pairs in a fixed
// order: no atomics, every cell written exactly once, bitwise reproducible.
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
  const int* order;
  const float2* phase;
  const int* blade_frame;
  float2* y;
  const float2* y_meas;
  float2* contrib;  // non-null: also write conj(P) * final value per bin
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

template <int LP, int W>
__global__ void __launch_bounds__(kInterpThreads, 3) interp_kernel(InterpArgs a) {
  constexpr int SPW = 32 / LP;
  constexpr int WQ = W / 2;  // float4 of weights per sample
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LP - 1);
  const int slot = lane / LP;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarp = ((long)gridDim.x * blockDim.x) >> 5;
  const size_t nC = (size_t)a.n * a.C;
  float sumsq = 0.f;
  for (long i0 = warp * SPW; i0 < a.M; i0 += nwarp * SPW) {
    const long idx = i0 + slot;
    const bool valid = idx < a.M;
    float2 tot = make_float2(0.f, 0.f);
    int m = 0, j = 0;
    if (valid) {
      m = __ldg(&a.order[idx]);
      const uint32_t packed = __ldg(&a.kb_idx[m]);
      const int i1 = packed & 0xffff, i2 = packed >> 16;
      float w[2 * W];
#pragma unroll
      for (int q = 0; q < WQ; ++q) {
        const float4 v = __ldg(&a.kb_w[(size_t)WQ * m + q]);
        w[4 * q] = v.x;
        w[4 * q + 1] = v.y;
        w[4 * q + 2] = v.z;
        w[4 * q + 3] = v.w;
      }
      const int b = m / a.LR;
      j = m % a.R;
      const int t = __ldg(&a.blade_frame[b]);
      const float2* G = a.grid + (size_t)t * a.n * nC;
      int col[W];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const int c = i1 + q;
        col[q] = (c >= a.n ? c - a.n : c) * a.C;
      }
      const float2* P = a.phase + (size_t)j * a.Nf + a.f0;
      for (int f = sub; f < a.Cv; f += LP) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < W; ++q) {
          int r = i2 + q;
          r = r >= a.n ? r - a.n : r;
          const float2* Gr = G + (size_t)r * nC + f;
          float2 ra = make_float2(0.f, 0.f);
#pragma unroll
          for (int c = 0; c < W; ++c) {
            const float2 g = __ldg(Gr + col[c]);
            ra.x = fmaf(w[c], g.x, ra.x);
            ra.y = fmaf(w[c], g.y, ra.y);
          }
          acc.x = fmaf(w[W + q], ra.x, acc.x);
          acc.y = fmaf(w[W + q], ra.y, acc.y);
        }
        const float2 z = cmulf(__ldg(P + f), acc);
        tot.x += z.x;
        tot.y += z.y;
      }
    }
#pragma unroll
    for (int o = LP / 2; o > 0; o >>= 1) {
      tot.x += __shfl_xor_sync(0xffffffffu, tot.x, o);
      tot.y += __shfl_xor_sync(0xffffffffu, tot.y, o);
    }
    float2 v = make_float2(tot.x * a.scale, tot.y * a.scale);
    if (valid && sub == 0) {
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
    if (a.contrib) {
      // broadcast the final value of this sample to its lanes, phase it per bin
      v.x = __shfl_sync(0xffffffffu, v.x, slot * LP);
      v.y = __shfl_sync(0xffffffffu, v.y, slot * LP);
      if (valid) {
        const float2* P = a.phase + (size_t)j * a.Nf + a.f0;
        float2* out = a.contrib + (size_t)m * a.C;
        for (int f = sub; f < a.Cv; f += LP) out[f] = cmulcf(__ldg(P + f), v);
      }
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

// contrib[m][f] = conj(P[j_m][f0 + f]) r_m, LP lanes per sample.
template <int LP>
__global__ void __launch_bounds__(256) phase_expand_kernel(const float2* r, const float2* phase, float2* contrib,
                                                            int M, int R, int Nf, int C, int Cv, int f0) {
  constexpr int SPW = 32 / LP;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LP - 1);
  const int slot = lane / LP;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarp = ((long)gridDim.x * blockDim.x) >> 5;
  for (long m = warp * SPW + slot; m < M; m += nwarp * SPW) {
    const float2 v = __ldg(&r[m]);
    const float2* P = phase + (size_t)(m % R) * Nf + f0;
    float2* out = contrib + (size_t)m * C;
    for (int f = sub; f < Cv; f += LP) out[f] = cmulcf(__ldg(P + f), v);
  }
}

// G'[cell][f] = sum over the cell's (m, w) list of w * contrib[m][f]; LP lanes per cell.
template <int LP>
__global__ void __launch_bounds__(256) spread_gather_kernel(float2* grid, const float2* contrib, const int* cell_off,
                                                             const int2* cell_ent, long ncell, int C, int Cv) {
  constexpr int CPW = 32 / LP;
  constexpr int QMAX = LP == 32 ? (kMaxChunk + 31) / 32 : 1;  // LP covers the chunk stride C
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LP - 1);
  const int slot = lane / LP;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarp = ((long)gridDim.x * blockDim.x) >> 5;
  const int nq = (C + LP - 1) / LP;
  for (long c = warp * CPW + slot; c < ncell; c += nwarp * CPW) {
    float2 acc[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) acc[q] = make_float2(0.f, 0.f);
    const int beg = __ldg(&cell_off[c]), end = __ldg(&cell_off[c + 1]);
    for (int e = beg; e < end; ++e) {
      const int2 en = __ldg(&cell_ent[e]);
      const float w = __int_as_float(en.y);
      const float2* cm = contrib + (size_t)en.x * C;
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int f = sub + LP * q;
        if (q < nq && f < Cv) {
          const float2 v = __ldg(cm + f);
          acc[q].x = fmaf(w, v.x, acc[q].x);
          acc[q].y = fmaf(w, v.y, acc[q].y);
        }
      }
    }
    float2* out = grid + (size_t)c * C;
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int f = sub + LP * q;
      if (q < nq && f < C) out[f] = f < Cv ? acc[q] : make_float2(0.f, 0.f);
    }
  }
}

int lanes_for(int Cv) {
  int lp = 1;
  while (lp < Cv && lp < 32) lp <<= 1;
  return lp;
}

unsigned grid_for(long items, long per_block, long cap) {
  long b = (items + per_block - 1) / per_block;
  return (unsigned)std::max<long>(1, std::min(b, cap));
}

template <int W>
cudaError_t launch_interp(int lp, const InterpArgs& a, dim3 grid, cudaStream_t s) {
  switch (lp) {
    case 1: interp_kernel<1, W><<<grid, kInterpThreads, 0, s>>>(a); break;
    case 2: interp_kernel<2, W><<<grid, kInterpThreads, 0, s>>>(a); break;
    case 4: interp_kernel<4, W><<<grid, kInterpThreads, 0, s>>>(a); break;
    case 8: interp_kernel<8, W><<<grid, kInterpThreads, 0, s>>>(a); break;
    case 16: interp_kernel<16, W><<<grid, kInterpThreads, 0, s>>>(a); break;
    default: interp_kernel<32, W><<<grid, kInterpThreads, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t nufft_configure(int) { return cudaSuccess; }

cudaError_t interp(const Plan& p, int f0, int nbins, float2* y, const float2* y_meas, bool accumulate,
                   const Reducer* red, double* sumsq, float2* contrib, cudaStream_t s) {
  InterpArgs a{};
  a.grid = p.grid;
  a.kb_idx = p.kb_idx;
  a.kb_w = p.kb_w;
  a.order = p.order;
  a.phase = p.phase;
  a.blade_frame = p.blade_frame_d;
  a.y = y;
  a.y_meas = y_meas;
  a.contrib = contrib;
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
  const long per_block = (long)(kInterpThreads / 32) * (32 / lp);
  const long cap = red ? std::min<long>(red->capacity, 16384) : 16384;
  dim3 grid(grid_for(p.M, per_block, cap));
  return p.W == 8 ? launch_interp<8>(lp, a, grid, s) : launch_interp<6>(lp, a, grid, s);
}

cudaError_t spread(const Plan& p, int f0, int nbins, const float2* r, bool contrib_ready, cudaStream_t s) {
  const int lp = lanes_for(nbins);
  if (!contrib_ready) {
    dim3 g(grid_for(p.M, 8L * (32 / lp), 16384));
    switch (lp) {
#define PE(L) \
  case L: phase_expand_kernel<L><<<g, 256, 0, s>>>(r, p.phase, p.contrib, p.M, p.R, p.Nf, p.chunk, nbins, f0); break;
      PE(1) PE(2) PE(4) PE(8) PE(16)
      default: phase_expand_kernel<32><<<g, 256, 0, s>>>(r, p.phase, p.contrib, p.M, p.R, p.Nf, p.chunk, nbins, f0);
#undef PE
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const long ncell = (long)p.T * p.n * p.n;
  const int lpg = lanes_for(p.chunk);
  dim3 g(grid_for(ncell, 8L * (32 / lpg), 65535));
  switch (lpg) {
#define SG(L) \
  case L: spread_gather_kernel<L><<<g, 256, 0, s>>>(p.grid, p.contrib, p.cell_off, p.cell_ent, ncell, p.chunk, nbins); break;
    SG(1) SG(2) SG(4) SG(8) SG(16)
    default: spread_gather_kernel<32><<<g, 256, 0, s>>>(p.grid, p.contrib, p.cell_off, p.cell_ent, ncell, p.chunk, nbins);
#undef SG
  }
  return cudaGetLastError();
}

}  // namespace prop
