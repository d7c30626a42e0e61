// Type-2 interpolation (forward) and type-1 spread (adjoint) between the
// oversampled grid and the blade samples.
//
// Forward, per sample m of blade b (frame t(b), readout index j):
//   y_m = s * sum_f P[j][f] * sum_{a,c < W} w2[a] w1[c] G_{t,f}[u2 + a][u1 + c]
// i.e. the W x W-tap Kaiser-Bessel interpolation of every bin's grid, times
// the displacement phase exp(-2 pi i k_r Delta_f) (Sec. 3: a material
// displaced along the readout picks up a phase linear in k_r), summed over
// the bins.  Samples are processed in tile-sorted work items; a persistent
// CTA per SM streams each item's grid tile plus halo into shared memory with
// TMA bulk copies (double-buffered, completion on an mbarrier) while it
// computes the previous item.  Bins are the fastest axis, so the lanes that
// serve one sample read consecutive bins of a cell (conflict-free).
//
// Adjoint: G'_{t,f}[cell] = sum_m w(m, cell) conj(P[j_m][f]) r_m.  The
// phased residual contrib[m][f] = conj(P[j_m][f]) r_m is formed once per
// sample (fused into the interpolation when the grid holds every bin), then
// every grid cell gathers its plan-time list of (sample, weight) pairs in a
// fixed order: no atomics, every cell written exactly once, bitwise
// reproducible.
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

// --- TMA bulk copy and mbarrier helpers (inline PTX, sm_90+ forms) ---------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Contiguous global -> shared copy by the TMA engine; bytes and both
// addresses must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2 s of SM clock (no legitimate copy takes
// that long) and reports false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > 4000000000LL) return false;
  return true;
}

struct InterpArgs {
  const float2* grid;
  const uint32_t* kb_idx;  // in interpolation (sorted) order
  const float4* kb_w;      // in interpolation (sorted) order
  const int* order;        // sorted position -> sample index m
  const int4* items;
  const float2* phase;
  float2* y;
  const float2* y_meas;
  float2* contrib;  // non-null: also write conj(P) * final value per bin
  double* partials;
  unsigned int* counter;
  double* sumsq_out;
  int* err;  // set to 1 when a bounded wait expires
  int n_items, R, n, C, Cv, f0, Nf;
  int TI, tps, nbuf;
  float scale;
  int accumulate;
};

constexpr int kInterpThreads = 512;

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

// Deterministic grid reduction: each block's partial, summed by the last block.
__device__ void reduce_to(double local, double* partials, unsigned int* counter, double* out) {
  __shared__ double sh[32];
  __shared__ bool last;
  const double bs = block_sum(local, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(&partials[i]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      *out = s;
      *counter = 0u;
    }
  }
}

struct ItemGeom {
  int t, r0, c0, start, count;
};

__device__ __forceinline__ ItemGeom item_geom(const InterpArgs& a, int item) {
  const int4 it = __ldg(&a.items[item]);
  const int tpp = a.tps * a.tps;
  ItemGeom g;
  g.t = it.x / tpp;
  const int rem = it.x - g.t * tpp;
  g.r0 = (rem / a.tps) * a.TI;
  g.c0 = (rem % a.tps) * a.TI;
  g.start = it.y;
  g.count = it.z;
  return g;
}

// Thread 0: stream item `item`'s tile + halo (HW rows of HW cells x C bins,
// wrapped modulo n) into `dst`, completing on `bar`.
template <int W>
__device__ void issue_tile(const InterpArgs& a, int item, float2* dst, uint64_t* bar) {
  const ItemGeom g = item_geom(a, item);
  const int HW = a.TI + W - 1;
  const size_t nC = (size_t)a.n * a.C;
  const float2* G = a.grid + (size_t)g.t * a.n * nC;
  mbar_expect_tx(bar, (uint32_t)((size_t)HW * HW * a.C * sizeof(float2)));
  const int run1 = min(HW, a.n - g.c0);
  for (int q = 0; q < HW; ++q) {
    int gr = g.r0 + q;
    gr = gr >= a.n ? gr - a.n : gr;
    float2* d = dst + (size_t)q * HW * a.C;
    bulk_g2s(d, G + (size_t)gr * nC + (size_t)g.c0 * a.C, (uint32_t)(run1 * a.C * sizeof(float2)), bar);
    if (run1 < HW)
      bulk_g2s(d + (size_t)run1 * a.C, G + (size_t)gr * nC, (uint32_t)((HW - run1) * a.C * sizeof(float2)), bar);
  }
}

// CS > 0: the bin stride C is the compile-time CS (so every shared-memory and
// tap offset folds into an immediate); CS == 0: runtime stride.  LP lanes
// serve one sample, each lane a bin f = sub + LP q.
template <int LP, int CS, int W>
__global__ void __launch_bounds__(kInterpThreads, 1) interp_kernel(InterpArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int SPW = 32 / LP;
  constexpr int WQ = W / 2;                           // float4 of weights per sample
  constexpr int QB = CS > 0 ? (CS + LP - 1) / LP : 0;  // bins per lane (compile-time case)
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const int sub = lane & (LP - 1);
  const int slot = lane / LP;
  const int C = CS > 0 ? CS : a.C;
  const int TI = CS > 0 ? (CS <= 32 ? 16 : 8) : a.TI;
  const int HW = TI + W - 1;
  const size_t tile_elems = (size_t)HW * HW * C;
  float2* bufs = reinterpret_cast<float2*>(smem_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + a.nbuf * tile_elems * sizeof(float2));
  __shared__ int s_abort;
  if (threadIdx.x == 0) {
    for (int b = 0; b < a.nbuf; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int b = 0; b < a.nbuf; ++b) {
      const int item = blockIdx.x + b * gridDim.x;
      if (item < a.n_items) issue_tile<W>(a, item, bufs + b * tile_elems, &bar[b]);
    }

  float sumsq = 0.f;
  int k = 0;
  for (int item = blockIdx.x; item < a.n_items; item += gridDim.x, ++k) {
    const int b = k % a.nbuf;
    const uint32_t parity = (uint32_t)((k / a.nbuf) & 1);
    if (!mbar_wait_bounded(&bar[b], parity)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    const float2* tile = bufs + b * tile_elems;
    const ItemGeom g = item_geom(a, item);

    // Warp-cooperative metadata prefetch: lane L holds the sample handled in
    // round L / SPW at slot L % SPW (an item has at most nwarp * 32 samples).
    const int sL = warp * SPW + (lane % SPW) + (lane / SPW) * nwarp * SPW;
    int mL = 0, jL = 0;
    uint32_t pL = 0;
    float wL[2 * W];
#pragma unroll
    for (int q = 0; q < 2 * W; ++q) wL[q] = 0.f;
    if (sL < g.count) {
      const int si = g.start + sL;
      mL = __ldg(&a.order[si]);
      pL = __ldg(&a.kb_idx[si]);
#pragma unroll
      for (int q = 0; q < WQ; ++q) {
        const float4 v = __ldg(&a.kb_w[(size_t)WQ * si + q]);
        wL[4 * q] = v.x;
        wL[4 * q + 1] = v.y;
        wL[4 * q + 2] = v.z;
        wL[4 * q + 3] = v.w;
      }
      jL = mL % a.R;
    }

    for (int rnd = 0; warp * SPW + rnd * nwarp * SPW < g.count; ++rnd) {
      const int s = warp * SPW + rnd * nwarp * SPW + slot;
      const bool valid = s < g.count;
      const int src = rnd * SPW + slot;
      const int m = __shfl_sync(0xffffffffu, mL, src);
      const int j = __shfl_sync(0xffffffffu, jL, src);
      const uint32_t packed = __shfl_sync(0xffffffffu, pL, src);
      float w[2 * W];
#pragma unroll
      for (int q = 0; q < 2 * W; ++q) w[q] = __shfl_sync(0xffffffffu, wL[q], src);
      float2 tot = make_float2(0.f, 0.f);
      const float2* P = a.phase + (size_t)j * a.Nf + a.f0;
      if (valid) {
        const int lc = (int)(packed & 0xffff) - g.c0;  // the first tap lies in the tile
        const int lr = (int)(packed >> 16) - g.r0;
        const float2* base = tile + ((size_t)lr * HW + lc) * C + sub;
        // W independent row sums (x1 weights), then the x2 weights; with a
        // compile-time stride every offset below is an immediate.
        auto tap_sum = [&](const float2* p) {
          float2 racc[W];
#pragma unroll
          for (int q = 0; q < W; ++q) {
            racc[q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < W; ++c) {
              const float2 gv = p[(q * HW + c) * C];
              racc[q].x = fmaf(w[c], gv.x, racc[q].x);
              racc[q].y = fmaf(w[c], gv.y, racc[q].y);
            }
          }
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < W; ++q) {
            acc.x = fmaf(w[W + q], racc[q].x, acc.x);
            acc.y = fmaf(w[W + q], racc[q].y, acc.y);
          }
          return acc;
        };
        if constexpr (CS > 0) {
#pragma unroll
          for (int qb = 0; qb < QB; ++qb) {
            const int f = sub + LP * qb;
            if (f < a.Cv) {
              const float2 z = cmulf(__ldg(P + f), tap_sum(base + LP * qb));
              tot.x += z.x;
              tot.y += z.y;
            }
          }
        } else {
          for (int f = sub; f < a.Cv; f += LP) {
            const float2 z = cmulf(__ldg(P + f), tap_sum(base + (f - sub)));
            tot.x += z.x;
            tot.y += z.y;
          }
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
          float2* out = a.contrib + (size_t)m * C;
          for (int f = sub; f < a.Cv; f += LP) out[f] = cmulcf(__ldg(P + f), v);
        }
      }
    }
    __syncthreads();  // every read of this buffer is done
    if (threadIdx.x == 0) {
      const int next = item + a.nbuf * gridDim.x;
      if (next < a.n_items) issue_tile<W>(a, next, bufs + b * tile_elems, &bar[b]);
    }
  }
  if (s_abort && threadIdx.x == 0) {
    atomicExch(a.err, 1);
    // let any copy still in flight into this CTA's buffers land (bounded)
    for (int kk = k + 1; kk < k + a.nbuf; ++kk) {
      const int item = blockIdx.x + kk * gridDim.x;
      if (item < a.n_items) mbar_wait_bounded(&bar[kk % a.nbuf], (uint32_t)((kk / a.nbuf) & 1));
    }
  }
  if (a.partials) reduce_to((double)sumsq, a.partials, a.counter, a.sumsq_out);
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

// Cell gather: G'[cell][f] = sum over the cell's (offset, w) list of
// w * contrib[offset + f].  LP lanes per cell, each lane QB bins; CS > 0 fixes
// the stride at compile time.  Cells are taken in the plan's patch-major
// order (one table lookup, no index arithmetic) and list entries are
// consumed four at a time for memory-level parallelism.
template <int LP, int CS>
__global__ void __launch_bounds__(256) spread_gather_kernel(float2* grid, const float2* contrib, const int* cell_ids,
                                                             const int* cell_off, const int2* cell_ent,
                                                             const int2* items, int n_items, int Crt, int Cv) {
  constexpr int CPW = 32 / LP;
  constexpr int QB = CS > 0 ? (CS + LP - 1) / LP : 2;  // runtime stride: LP >= C/2
  const int C = CS > 0 ? CS : Crt;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LP - 1);
  const int slot = lane / LP;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const int nq = CS > 0 ? QB : (C + LP - 1) / LP;
  const float2* cbase = contrib + sub;
  for (int itm = blockIdx.x; itm < n_items; itm += gridDim.x) {
    const int2 range = __ldg(&items[itm]);
    for (int i = range.x + warp * CPW + slot; i < range.y; i += nwarp * CPW) {
      const int c = __ldg(&cell_ids[i]);
      float2 acc[QB];
#pragma unroll
      for (int q = 0; q < QB; ++q) acc[q] = make_float2(0.f, 0.f);
      const int beg = __ldg(&cell_off[i]), end = __ldg(&cell_off[i + 1]);
      int e = beg;
      for (; e + 4 <= end; e += 4) {
        int2 en[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) en[u] = __ldg(&cell_ent[e + u]);
#pragma unroll
        for (int q = 0; q < QB; ++q) {
          if (q < nq && sub + LP * q < Cv) {
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldg(cbase + en[u].x + LP * q);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float w = __int_as_float(en[u].y);
              acc[q].x = fmaf(w, v[u].x, acc[q].x);
              acc[q].y = fmaf(w, v[u].y, acc[q].y);
            }
          }
        }
      }
      for (; e < end; ++e) {
        const int2 en = __ldg(&cell_ent[e]);
        const float w = __int_as_float(en.y);
#pragma unroll
        for (int q = 0; q < QB; ++q) {
          if (q < nq && sub + LP * q < Cv) {
            const float2 v = __ldg(cbase + en.x + LP * q);
            acc[q].x = fmaf(w, v.x, acc[q].x);
            acc[q].y = fmaf(w, v.y, acc[q].y);
          }
        }
      }
      float2* out = grid + (size_t)c * C + sub;
#pragma unroll
      for (int q = 0; q < QB; ++q) {
        const int f = sub + LP * q;
        if (q < nq && f < C) out[LP * q] = f < Cv ? acc[q] : make_float2(0.f, 0.f);
      }
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
cudaError_t launch_interp(int lp, int cs, const InterpArgs& a, dim3 grid, size_t smem, cudaStream_t s) {
  // compile-time strides for the common chunk widths (full lane use), runtime otherwise
  if (cs == 32 && lp == 32) interp_kernel<32, 32, W><<<grid, kInterpThreads, smem, s>>>(a);
  else if (cs == 64 && lp == 32) interp_kernel<32, 64, W><<<grid, kInterpThreads, smem, s>>>(a);
  else if (cs == 16 && lp == 16) interp_kernel<16, 16, W><<<grid, kInterpThreads, smem, s>>>(a);
  else if (cs == 8 && lp == 8) interp_kernel<8, 8, W><<<grid, kInterpThreads, smem, s>>>(a);
  else {
    switch (lp) {
      case 1: interp_kernel<1, 0, W><<<grid, kInterpThreads, smem, s>>>(a); break;
      case 2: interp_kernel<2, 0, W><<<grid, kInterpThreads, smem, s>>>(a); break;
      case 4: interp_kernel<4, 0, W><<<grid, kInterpThreads, smem, s>>>(a); break;
      case 8: interp_kernel<8, 0, W><<<grid, kInterpThreads, smem, s>>>(a); break;
      case 16: interp_kernel<16, 0, W><<<grid, kInterpThreads, smem, s>>>(a); break;
      default: interp_kernel<32, 0, W><<<grid, kInterpThreads, smem, s>>>(a); break;
    }
  }
  return cudaGetLastError();
}

template <class K>
cudaError_t allow_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <int W>
cudaError_t configure_interp(int optin) {
  cudaError_t e;
  if ((e = allow_smem(interp_kernel<32, 32, W>, optin))) return e;
  if ((e = allow_smem(interp_kernel<32, 64, W>, optin))) return e;
  if ((e = allow_smem(interp_kernel<16, 16, W>, optin))) return e;
  if ((e = allow_smem(interp_kernel<8, 8, W>, optin))) return e;
  if ((e = allow_smem(interp_kernel<1, 0, W>, optin))) return e;
  if ((e = allow_smem(interp_kernel<2, 0, W>, optin))) return e;
  if ((e = allow_smem(interp_kernel<4, 0, W>, optin))) return e;
  if ((e = allow_smem(interp_kernel<8, 0, W>, optin))) return e;
  if ((e = allow_smem(interp_kernel<16, 0, W>, optin))) return e;
  return allow_smem(interp_kernel<32, 0, W>, optin);
}

}  // namespace

cudaError_t nufft_configure(int smem_optin) {
  cudaError_t e = configure_interp<6>(smem_optin);
  if (e != cudaSuccess) return e;
  return configure_interp<8>(smem_optin);
}

int interp_buffers(const Plan& p) {
  const int HW = p.interp_tile + p.W - 1;
  const size_t tile = (size_t)HW * HW * p.cs * sizeof(float2);
  // two buffers when they fit next to the barriers and the static shared memory
  return 2 * tile + 1024 <= (size_t)p.smem_optin ? 2 : 1;
}

cudaError_t interp(const Plan& p, int f0, int nbins, float2* y, const float2* y_meas, bool accumulate,
                   const Reducer* red, double* sumsq, float2* contrib, cudaStream_t s) {
  InterpArgs a{};
  a.grid = p.grid;
  a.kb_idx = p.kb_idx;
  a.kb_w = p.kb_w;
  a.order = p.order;
  a.items = p.items;
  a.phase = p.phase;
  a.y = y;
  a.y_meas = y_meas;
  a.contrib = contrib;
  a.partials = red ? red->partials : nullptr;
  a.counter = red ? red->counter : nullptr;
  a.sumsq_out = sumsq;
  a.err = p.status_dev;
  a.n_items = p.n_items;
  a.R = p.R;
  a.n = p.n;
  a.C = p.cs;
  a.Cv = nbins;
  a.f0 = f0;
  a.Nf = p.Nf;
  a.scale = 1.0f / (float)p.N;
  a.accumulate = accumulate ? 1 : 0;
  a.TI = p.interp_tile;
  a.tps = p.n / p.interp_tile;
  a.nbuf = interp_buffers(p);
  if (p.n_items == 0) return cudaSuccess;
  const int HW = p.interp_tile + p.W - 1;
  const size_t smem = (size_t)a.nbuf * HW * HW * p.cs * sizeof(float2) + 2 * sizeof(uint64_t);
  const int blocks = std::min(p.n_items, p.num_sms);
  if (red && red->capacity < blocks) return cudaErrorInvalidValue;
  const int lp = lanes_for(nbins);
  dim3 grid((unsigned)blocks);
  return p.W == 8 ? launch_interp<8>(lp, p.cs, a, grid, smem, s) : launch_interp<6>(lp, p.cs, a, grid, smem, s);
}

cudaError_t spread(const Plan& p, int f0, int nbins, const float2* r, bool contrib_ready, cudaStream_t s) {
  const int lp = lanes_for(nbins);
  if (!contrib_ready) {
    dim3 g(grid_for(p.M, 8L * (32 / lp), 16384));
    switch (lp) {
#define PE(L) \
  case L: phase_expand_kernel<L><<<g, 256, 0, s>>>(r, p.phase, p.contrib, p.M, p.R, p.Nf, p.cs, nbins, f0); break;
      PE(1) PE(2) PE(4) PE(8) PE(16)
      default: phase_expand_kernel<32><<<g, 256, 0, s>>>(r, p.phase, p.contrib, p.M, p.R, p.Nf, p.cs, nbins, f0);
#undef PE
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int lpg = lanes_for(p.cs);
  dim3 g((unsigned)std::max(1, std::min(p.n_sitems, 65535)));
#define SG(L, CSV)                                                                                          \
  spread_gather_kernel<L, CSV><<<g, 256, 0, s>>>(p.grid, p.contrib, p.cell_ids, p.cell_off, p.cell_ent, p.sitems, \
                                                  p.n_sitems, p.cs, nbins)
  if (p.cs == 32) SG(32, 32);
  else if (p.cs == 64) SG(32, 64);
  else if (p.cs == 16) SG(16, 16);
  else if (p.cs == 8) SG(8, 8);
  else {
    switch (lpg) {
      case 1: SG(1, 0); break;
      case 2: SG(2, 0); break;
      case 4: SG(4, 0); break;
      case 8: SG(8, 0); break;
      case 16: SG(16, 0); break;
      default: SG(32, 0); break;
    }
  }
#undef SG
  return cudaGetLastError();
}

}  // namespace prop
