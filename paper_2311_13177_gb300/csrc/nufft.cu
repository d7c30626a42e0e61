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
// the grid is gathered from plan-time lists in a fixed order: every group
// of kSpreadGroupRows x kSpreadGroupCols cells reads each covering sample's
// phased residual once and adds it with that sample's weight on each of its
// cells (per-cell lists where the stride or a list's length rules the
// groups out).  No atomics,
// every cell written exactly once, bitwise reproducible.
#include "prop_internal.cuh"
#include "tma.cuh"

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
  const int* cta_off;  // CTA c takes items [cta_off[c], cta_off[c + 1]) (balanced at plan time)
  int n_items, R, n, C, Cv, f0, Nf;
  int TR, TC, nct, tpf, nbuf;  // tile rows, cells per row, tiles per row of tiles and per frame
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

// Deterministic grid reduction: each block's partial, summed by the last
// block; vb, nblk: this block's index and the block count of the reduction.
__device__ void reduce_to_v(double local, double* partials, unsigned int* counter, double* out, unsigned vb,
                            unsigned nblk) {
  __shared__ double sh[32];
  __shared__ bool last;
  const double bs = block_sum(local, sh);
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
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      *out = s;
      *counter = 0u;
    }
  }
}
__device__ void reduce_to(double local, double* partials, unsigned int* counter, double* out) {
  reduce_to_v(local, partials, counter, out, blockIdx.x, gridDim.x);
}

struct ItemGeom {
  int t, r0, c0, start, count;
};

__device__ __forceinline__ ItemGeom item_geom(const InterpArgs& a, int item) {
  const int4 it = __ldg(&a.items[item]);
  ItemGeom g;
  g.t = it.x / a.tpf;
  const int rem = it.x - g.t * a.tpf;
  g.r0 = (rem / a.nct) * a.TR;
  g.c0 = (rem % a.nct) * a.TC;
  g.start = it.y;
  g.count = it.z;
  return g;
}

// Thread 0: stream item `item`'s tile + halo (TR + W - 1 rows of TC + W - 1
// cells x C bins, wrapped modulo n) into `dst`, completing on `bar`.
template <int W>
__device__ void issue_tile(const InterpArgs& a, int item, float2* dst, uint64_t* bar) {
  const ItemGeom g = item_geom(a, item);
  const int HR = a.TR + W - 1, HC = a.TC + W - 1;
  const size_t nC = (size_t)a.n * a.C;
  const float2* G = a.grid + (size_t)g.t * a.n * nC;
  mbar_expect_tx(bar, (uint32_t)((size_t)HR * HC * a.C * sizeof(float2)));
  const int run1 = min(HC, a.n - g.c0);
  for (int q = 0; q < HR; ++q) {
    int gr = g.r0 + q;
    gr = gr >= a.n ? gr - a.n : gr;
    float2* d = dst + (size_t)q * HC * a.C;
    bulk_g2s(d, G + (size_t)gr * nC + (size_t)g.c0 * a.C, (uint32_t)(run1 * a.C * sizeof(float2)), bar);
    if (run1 < HC)
      bulk_g2s(d + (size_t)run1 * a.C, G + (size_t)gr * nC, (uint32_t)((HC - run1) * a.C * sizeof(float2)), bar);
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
  const int HR = (CS > 0 ? interp_tile_rows(CS, W) : a.TR) + W - 1;
  const int HC = (CS > 0 ? interp_tile_cols(CS, W) : a.TC) + W - 1;
  const size_t tile_elems = (size_t)HR * HC * C;
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
        const float2* base = tile + ((size_t)lr * HC + lc) * C + sub;
        // W independent row sums (x1 weights), then the x2 weights; with a
        // compile-time stride every offset below is an immediate.
        auto tap_sum = [&](const float2* p) {
          float2 racc[W];
#pragma unroll
          for (int q = 0; q < W; ++q) {
            racc[q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < W; ++c) {
              const float2 gv = p[(q * HC + c) * C];
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

constexpr int kInterpConsumers = 16;                          // compute warps per CTA
constexpr int kInterp2Threads = 32 * (kInterpConsumers + 1);  // plus one producer warp

// Interpolation for the compile-time bin strides CS in {8, 16, 32, 64}.
// Warp kInterpConsumers is the producer: its lane 0 streams item k's tile
// into buffer k % nbuf as soon as every compute warp has released the item
// that last used that buffer ("empty" barrier, one arrival per compute
// warp), so no compute warp ever waits for another.  Compute warps take
// CS / 2 lanes per sample, each lane two adjacent bins (16-byte shared
// loads), and 64 / CS samples per warp and round.  The metadata of an item
// (sample index, packed first tap, the 2W weights) is fetched before its
// tile is awaited, one sample per lane, and handed out by shuffles.
// The work of one persistent CTA: items [it_beg, it_end); vb, vg: the CTA's
// index and the CTA count of the |r|^2 reduction.
template <int CS, int W>
__device__ __forceinline__ void interp2_body(const InterpArgs& a, int it_beg, int it_end, unsigned vb, unsigned vg) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NCW = kInterpConsumers;
  constexpr int LPS = CS / 2;   // lanes per sample
  constexpr int SPW = 32 / LPS; // samples per warp and round
  constexpr int HR = interp_tile_rows(CS, W) + W - 1;  // staged rows
  constexpr int HC = interp_tile_cols(CS, W) + W - 1;  // staged cells per row
  constexpr int WQ = W / 2;
  constexpr int MPL = (kInterpItem + NCW * SPW - 1) / (NCW * SPW) * SPW;  // samples per warp per item
  static_assert(MPL <= 32, "one prefetched sample per lane");
  constexpr size_t tile_elems = (size_t)HR * HC * CS;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int sub = lane % LPS;
  const int slot = lane / LPS;
  float2* bufs = reinterpret_cast<float2*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + a.nbuf * tile_elems * sizeof(float2));
  uint64_t* empty = full + a.nbuf;
  __shared__ volatile int s_abort;
  if (threadIdx.x == 0) {
    for (int b = 0; b < a.nbuf; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NCW);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  grid_dep_wait();
  grid_dep_release();

  float sumsq = 0.f;
  if (warp == NCW) {
    if (lane == 0) {
      int k = 0;
      for (int item = it_beg; item < it_end; ++item, ++k) {
        const int b = k % a.nbuf;
        if (k >= a.nbuf && !mbar_wait_bounded(&empty[b], (uint32_t)(((k / a.nbuf) - 1) & 1))) {
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        issue_tile<W>(a, item, bufs + b * tile_elems, &full[b]);
      }
      // at most one copy per buffer can be in flight: the last one issued
      for (int kk = k > a.nbuf ? k - a.nbuf : 0; kk < k; ++kk)
        mbar_wait_bounded(&full[kk % a.nbuf], (uint32_t)((kk / a.nbuf) & 1));
    }
  } else {
    const int f_lo = 2 * sub;
    const bool b0 = f_lo < a.Cv, b1 = f_lo + 1 < a.Cv;
    int k = 0;
    for (int item = it_beg; item < it_end; ++item, ++k) {
      const int b = k % a.nbuf;
      const ItemGeom g = item_geom(a, item);
      // lane L prefetches the warp's sample of round L / SPW, slot L % SPW
      const int sL = (lane / SPW) * NCW * SPW + warp * SPW + (lane % SPW);
      int mL = 0, jL = 0;
      uint32_t pL = 0;
      float2 yL = make_float2(0.f, 0.f);  // the measurement (or the partial sum so far) of the sample
      float wL[2 * W];
#pragma unroll
      for (int q = 0; q < 2 * W; ++q) wL[q] = 0.f;
      if (lane < MPL && sL < g.count) {
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
        if (a.accumulate)
          yL = a.y[mL];
        else if (a.y_meas)
          yL = __ldg(&a.y_meas[mL]);
      }
      if (!mbar_wait_bounded(&full[b], (uint32_t)((k / a.nbuf) & 1))) s_abort = 1;
      if (s_abort) break;
      const float2* tile = bufs + b * tile_elems;

      for (int rnd = 0; rnd * NCW * SPW + warp * SPW < g.count; ++rnd) {
        const int s = rnd * NCW * SPW + warp * SPW + slot;
        const bool valid = s < g.count;
        const int src = rnd * SPW + slot;
        const int m = __shfl_sync(0xffffffffu, mL, src);
        const int j = __shfl_sync(0xffffffffu, jL, src);
        const uint32_t packed = __shfl_sync(0xffffffffu, pL, src);
        const float2 yprev = make_float2(__shfl_sync(0xffffffffu, yL.x, src), __shfl_sync(0xffffffffu, yL.y, src));
        float w[2 * W];
#pragma unroll
        for (int q = 0; q < 2 * W; ++q) w[q] = __shfl_sync(0xffffffffu, wL[q], src);
        const float2* P = a.phase + (size_t)j * a.Nf + a.f0 + f_lo;
        float2 P0 = make_float2(0.f, 0.f), P1 = make_float2(0.f, 0.f);
        if (valid && b0) P0 = __ldg(P);
        if (valid && b1) P1 = __ldg(P + 1);
        float2 tot = make_float2(0.f, 0.f);
        if (valid) {
          const int lc = (int)(packed & 0xffff) - g.c0;
          const int lr = (int)(packed >> 16) - g.r0;
          const float4* base = reinterpret_cast<const float4*>(tile + ((size_t)lr * HC + lc) * CS + f_lo);
          // row sums over the x1 taps, folded into the x2 sum row by row
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int q = 0; q < W; ++q) {
            float4 rs = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < W; ++c) {
              const float4 gv = base[(q * HC + c) * (CS / 2)];
              rs.x = fmaf(w[c], gv.x, rs.x);
              rs.y = fmaf(w[c], gv.y, rs.y);
              rs.z = fmaf(w[c], gv.z, rs.z);
              rs.w = fmaf(w[c], gv.w, rs.w);
            }
            acc.x = fmaf(w[W + q], rs.x, acc.x);
            acc.y = fmaf(w[W + q], rs.y, acc.y);
            acc.z = fmaf(w[W + q], rs.z, acc.z);
            acc.w = fmaf(w[W + q], rs.w, acc.w);
          }
          const float2 z0 = cmulf(P0, make_float2(acc.x, acc.y));
          const float2 z1 = cmulf(P1, make_float2(acc.z, acc.w));
          tot = make_float2(z0.x + z1.x, z0.y + z1.y);
        }
#pragma unroll
        for (int o = LPS / 2; o > 0; o >>= 1) {
          tot.x += __shfl_xor_sync(0xffffffffu, tot.x, o);
          tot.y += __shfl_xor_sync(0xffffffffu, tot.y, o);
        }
        float2 v = make_float2(tot.x * a.scale, tot.y * a.scale);
        if (a.accumulate) {
          v.x += yprev.x;
          v.y += yprev.y;
        } else if (a.y_meas) {
          v.x -= yprev.x;
          v.y -= yprev.y;
        }
        if (valid && sub == 0) {
          a.y[m] = v;
          sumsq = fmaf(v.x, v.x, fmaf(v.y, v.y, sumsq));
        }
        if (a.contrib && valid) {
          // every lane of the sample holds the same reduced value
          const float2 c0 = cmulcf(P0, v), c1 = cmulcf(P1, v);
          reinterpret_cast<float4*>(a.contrib + (size_t)m * CS)[sub] = make_float4(c0.x, c0.y, c1.x, c1.y);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
    }
  }
  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicExch(a.err, 1);
  if (a.partials) reduce_to_v((double)sumsq, a.partials, a.counter, a.sumsq_out, vb, vg);
}

template <int CS, int W>
__global__ void __launch_bounds__(kInterp2Threads, 1) interp2_kernel(InterpArgs a) {
  interp2_body<CS, W>(a, a.cta_off[blockIdx.x], a.cta_off[blockIdx.x + 1], blockIdx.x, gridDim.x);
}

// Kernel parameter of the interpolation over a batch of problems.
struct MultiInterp {
  InterpArgs a[kMaxBatch];
  int plan_ctas[kMaxBatch];      // CTAs each problem's items were balanced over
  int nreq;
  int cta_begin[kMaxBatch + 1];  // CTA ranges of the problems
};

// One launch for several problems with the same bin stride and kernel
// width: CTA b serves problem r (cta_begin[r] <= b < cta_begin[r + 1]) as
// its CTA v of c = cta_begin[r + 1] - cta_begin[r] and takes the items the
// problem's plan balanced over its CTAs v P / c .. (v + 1) P / c - 1, so every
// sample is computed as in the problem's own launch.
template <int CS, int W>
__global__ void __launch_bounds__(kInterp2Threads, 1) interp2_multi_kernel(const __grid_constant__ MultiInterp m) {
  int r = 0;
  while (r + 1 < m.nreq && (int)blockIdx.x >= m.cta_begin[r + 1]) ++r;
  const int v = (int)blockIdx.x - m.cta_begin[r], c = m.cta_begin[r + 1] - m.cta_begin[r];
  const int P = m.plan_ctas[r];
  const InterpArgs& a = m.a[r];
  interp2_body<CS, W>(a, a.cta_off[(long)v * P / c], a.cta_off[(long)(v + 1) * P / c], (unsigned)v, (unsigned)c);
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

// Residual of a forward pass summed elsewhere (over the bins of several
// plans): r = y_sum - y_meas, the FP64 sum of |r|^2 (block partials, the last
// block sums them in block order), and with contrib the phased residual
// conj(P[j][f0 + f]) r per bin for the spread.  LP lanes per sample.
template <int LP>
__global__ void __launch_bounds__(256) resid_expand_kernel(const float2* y_sum, const float2* y_meas, float2* r,
                                                            const float2* phase, float2* contrib, int M, int R,
                                                            int Nf, int C, int Cv, int f0, double* partials,
                                                            unsigned int* counter, double* sumsq_out) {
  constexpr int SPW = 32 / LP;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LP - 1);
  const int slot = lane / LP;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarp = ((long)gridDim.x * blockDim.x) >> 5;
  double local = 0.0;
  for (long m = warp * SPW + slot; m < M; m += nwarp * SPW) {
    const float2 a = __ldg(&y_sum[m]), b = __ldg(&y_meas[m]);
    const float2 v = make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
    if (sub == 0) {
      r[m] = v;
      local += (double)v.x * v.x + (double)v.y * v.y;
    }
    if (contrib) {
      const float2* P = phase + (size_t)(m % R) * Nf + f0;
      float2* out = contrib + (size_t)m * C;
      for (int f = sub; f < Cv; f += LP) out[f] = cmulcf(__ldg(P + f), v);
    }
  }
  reduce_to(local, partials, counter, sumsq_out);
}

// --- Spread: cell gather over the plan's item blobs ------------------------
//
// An item's blob: int2 cells[ncp] (cell index, end of its list relative to
// the first entry; ncp = ncells rounded up to even), then int2 entries[nent]
// (offset m * cs of a phased-residual row, weight bits).  Every list holds a
// multiple of four entries, so a list is consumed four entries (two 16-byte
// loads) at a time without predication, in list order.

// Gather of one cell by the CS / 2 lanes of its group, two adjacent bins
// per lane: returns sum_e w_e contrib[off_e + 2 sub .. + 1].
__device__ __forceinline__ float4 gather_cell2(const int4* ent, int beg4, int end4, const float2* cbase) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
  for (int e = beg4; e < end4; e += 2) {  // e counts entry pairs
    const int4 q0 = ent[e], q1 = ent[e + 1];
    const float4 v0 = __ldg(reinterpret_cast<const float4*>(cbase + q0.x));
    const float4 v1 = __ldg(reinterpret_cast<const float4*>(cbase + q0.z));
    const float4 v2 = __ldg(reinterpret_cast<const float4*>(cbase + q1.x));
    const float4 v3 = __ldg(reinterpret_cast<const float4*>(cbase + q1.z));
    const float w0 = __int_as_float(q0.y), w1 = __int_as_float(q0.w);
    const float w2 = __int_as_float(q1.y), w3 = __int_as_float(q1.w);
    acc.x = fmaf(w0, v0.x, acc.x);
    acc.y = fmaf(w0, v0.y, acc.y);
    acc.z = fmaf(w0, v0.z, acc.z);
    acc.w = fmaf(w0, v0.w, acc.w);
    acc.x = fmaf(w1, v1.x, acc.x);
    acc.y = fmaf(w1, v1.y, acc.y);
    acc.z = fmaf(w1, v1.z, acc.z);
    acc.w = fmaf(w1, v1.w, acc.w);
    acc.x = fmaf(w2, v2.x, acc.x);
    acc.y = fmaf(w2, v2.y, acc.y);
    acc.z = fmaf(w2, v2.z, acc.z);
    acc.w = fmaf(w2, v2.w, acc.w);
    acc.x = fmaf(w3, v3.x, acc.x);
    acc.y = fmaf(w3, v3.y, acc.y);
    acc.z = fmaf(w3, v3.z, acc.z);
    acc.w = fmaf(w3, v3.w, acc.w);
  }
  return acc;
}

// All cells of one item, CS / 2 lanes per cell; `cells` points at the blob
// (shared or global memory).
template <int CS>
__device__ __forceinline__ void gather_item2(const int2* cells, int ncells, int ncp, int warp, int nwarp, int lane,
                                             float2* grid, const float2* contrib, int Cv) {
  constexpr int LPC = CS / 2;
  constexpr int CPW = 32 / LPC;
  const int sub = lane % LPC, slot = lane / LPC;
  const int4* ent = reinterpret_cast<const int4*>(cells + ncp);
  const float2* cbase = contrib + 2 * sub;
  for (int i0 = warp * CPW; i0 < ncells; i0 += nwarp * CPW) {
    const int i = i0 + slot;
    const bool ok = i < ncells;
    int cid = 0, beg = 0, end = 0;
    if (ok) {
      const int2 ce = cells[i];
      cid = ce.x;
      end = ce.y;
      beg = i > 0 ? cells[i - 1].y : 0;
    }
    float4 o = gather_cell2(ent, beg >> 1, end >> 1, cbase);
    if (ok) {
      if (2 * sub >= Cv) o.x = o.y = 0.f;
      if (2 * sub + 1 >= Cv) o.z = o.w = 0.f;
      reinterpret_cast<float4*>(grid + (size_t)cid * CS)[sub] = o;
    }
  }
}

// Grouped gather (plan lists built per 2 x 2-cell group): the CS / 2 lanes
// of a group own two adjacent bins each and fetch every listed sample's
// phased-residual row once (one 16-byte load a lane), adding it with the
// entry's four weights to the four cells of the group held in registers.
// A row is read once per group instead of once per covered cell, and each
// cell still sums its own terms in ascending sample order (zero weights add
// exact zeros), as a per-cell list would.  Entries come in batches of eight
// with the eight row loads in flight together (then a last batch of four:
// every list holds a multiple of four).  Warps claim groups from a
// shared counter.  `base` points at the item's blob in shared memory.
template <int CS>
__device__ __forceinline__ void gather_groups(const int2* base, int ngroups, int nent, int lane, int* next,
                                              float2* grid, const float2* contrib, int Cv, int n) {
  constexpr int LPG = CS / 2;    // lanes per group
  constexpr int GPW = 32 / LPG;  // groups per warp
  const int sub = lane % LPG, slot = lane / LPG;
  const int ngp = (ngroups + 1) & ~1;
  const int* offs = reinterpret_cast<const int*>(base + ngp);
  const float4* wts = reinterpret_cast<const float4*>(base + ngp + nent / 2);
  const float2* cb = contrib + 2 * sub;
  auto row = [&](int off) { return __ldg(reinterpret_cast<const float4*>(cb + off)); };
  for (;;) {
    int g0 = 0;
    if (lane == 0) g0 = atomicAdd(next, GPW);
    g0 = __shfl_sync(0xffffffffu, g0, 0);
    if (g0 >= ngroups) break;
    const int g = g0 + slot;
    const bool ok = g < ngroups;
    int cell0 = 0, beg = 0, end = 0;
    if (ok) {
      const int2 ge = base[g];
      cell0 = ge.x;
      end = ge.y;
      beg = g > 0 ? base[g - 1].y : 0;
    }
    float4 acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    auto add4 = [&](int e, const float4* v) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 w = wts[e + u];
        const float wa[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[c].x = fmaf(wa[c], v[u].x, acc[c].x);
          acc[c].y = fmaf(wa[c], v[u].y, acc[c].y);
          acc[c].z = fmaf(wa[c], v[u].z, acc[c].z);
          acc[c].w = fmaf(wa[c], v[u].w, acc[c].w);
        }
      }
    };
    int e = beg;
#pragma unroll 1
    for (; e + 8 <= end; e += 8) {  // eight rows in flight
      const int4 o0 = *reinterpret_cast<const int4*>(offs + e);
      const int4 o1 = *reinterpret_cast<const int4*>(offs + e + 4);
      const float4 v0[4] = {row(o0.x), row(o0.y), row(o0.z), row(o0.w)};
      const float4 v1[4] = {row(o1.x), row(o1.y), row(o1.z), row(o1.w)};
      add4(e, v0);
      add4(e + 4, v1);
    }
    if (e < end) {  // lists hold a multiple of four entries
      const int4 o = *reinterpret_cast<const int4*>(offs + e);
      const float4 v[4] = {row(o.x), row(o.y), row(o.z), row(o.w)};
      add4(e, v);
    }
    if (ok) {
      const bool l0 = 2 * sub < Cv, l1 = 2 * sub + 1 < Cv;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float4 o = acc[c];
        if (!l0) o.x = o.y = 0.f;
        if (!l1) o.z = o.w = 0.f;
        reinterpret_cast<float4*>(grid + ((size_t)cell0 + (size_t)(c >> 1) * n + (c & 1)) * CS)[sub] = o;
      }
    }
  }
}

constexpr int kSpreadConsumers = 12;                          // gather warps per CTA (8: 4679, 10: 4764, 12: 4846, 16: 4784 it/s)
constexpr int kSpreadThreads = 32 * (kSpreadConsumers + 1);   // plus one producer warp

// Spread for the compile-time strides CS in {8, 16, 32, 64}.  Persistent
// CTAs (two per SM); the producer warp's lane 0 bulk-copies item k's blob
// into stage k % 2 once every gather warp has released the item that last
// used it, so the lists come from shared memory and only the phased-residual
// rows (mostly L1/L2 hits) are read from global memory.  Used when every
// item fits a stage (the plan checks).
// The work of one persistent CTA on items [it_beg, it_end).
template <int CS, bool GROUPED>
__device__ __forceinline__ void spread_stage_body(float2* grid, const float2* contrib, const int4* sitems,
                                                  const int2* blob, int it_beg, int it_end, int Cv, int n, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NCW = kSpreadConsumers;
  constexpr int NBUF = 2;
  int2* stage = reinterpret_cast<int2*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)NBUF * kSpreadStageInt2 * sizeof(int2));
  uint64_t* empty = full + NBUF;
  __shared__ volatile int s_abort;
  __shared__ int s_next[NBUF];  // grouped lists: next unclaimed group of the item in each stage
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NCW);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  // The producer reads only plan tables and writes shared memory: its first
  // copies go out before the predecessor kernel has finished.  The gather
  // warps read the phased residual and overwrite the grid, both shared with
  // earlier kernels, so they wait.
  if (warp == NCW) {
    grid_dep_release();
    if (lane == 0) {
      int k = 0;
      for (int item = it_beg; item < it_end; ++item, ++k) {
        const int b = k % NBUF;
        if (k >= NBUF && !mbar_wait_bounded(&empty[b], (uint32_t)(((k / NBUF) - 1) & 1))) {
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        const int4 d = __ldg(&sitems[item]);
        const uint32_t bytes = (uint32_t)d.w * (uint32_t)sizeof(int2);  // the item's blob, sized by the plan
        s_next[b] = 0;  // published to the gather warps by the barrier phase
        mbar_expect_tx(&full[b], bytes);
        bulk_g2s(stage + (size_t)b * kSpreadStageInt2, blob + d.x, bytes, &full[b]);
      }
      for (int kk = k > NBUF ? k - NBUF : 0; kk < k; ++kk)
        mbar_wait_bounded(&full[kk % NBUF], (uint32_t)((kk / NBUF) & 1));
    }
  } else {
    grid_dep_wait();
    grid_dep_release();
    int k = 0;
    for (int item = it_beg; item < it_end; ++item, ++k) {
      const int b = k % NBUF;
      const int4 d = __ldg(&sitems[item]);
      const int ncp = (d.y + 1) & ~1;
      if (!mbar_wait_bounded(&full[b], (uint32_t)((k / NBUF) & 1))) s_abort = 1;
      if (s_abort) break;
      if constexpr (GROUPED)
        gather_groups<CS>(stage + (size_t)b * kSpreadStageInt2, d.y, d.z, lane, &s_next[b], grid, contrib, Cv, n);
      else
        gather_item2<CS>(stage + (size_t)b * kSpreadStageInt2, d.y, ncp, warp, NCW, lane, grid, contrib, Cv);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
    }
  }
  __syncthreads();
  if (s_abort && threadIdx.x == 0) atomicExch(err, 1);
}

template <int CS, bool GROUPED>
__global__ void __launch_bounds__(kSpreadThreads, kSpreadCtasPerSm)
    spread_stage_kernel(float2* grid, const float2* contrib, const int4* sitems, const int2* blob,
                        const int* cta_off, int Cv, int n, int* err) {
  spread_stage_body<CS, GROUPED>(grid, contrib, sitems, blob, cta_off[blockIdx.x], cta_off[blockIdx.x + 1], Cv, n,
                                 err);
}

// Kernel parameter of the staged spread over a batch of problems.
struct SpreadArgs {
  float2* grid;
  const float2* contrib;
  const int4* sitems;
  const int2* blob;
  const int* cta_off;
  int Cv, n, plan_ctas;
  int* err;
};
struct MultiSpread {
  SpreadArgs a[kMaxBatch];
  int nreq;
  int cta_begin[kMaxBatch + 1];
};

// One launch for several problems with the same bin stride and list kind,
// CTAs mapped onto each problem's balanced item ranges as in
// interp2_multi_kernel; every cell sums its own terms in its list's order.
template <int CS, bool GROUPED>
__global__ void __launch_bounds__(kSpreadThreads, kSpreadCtasPerSm)
    spread_stage_multi_kernel(const __grid_constant__ MultiSpread m) {
  int r = 0;
  while (r + 1 < m.nreq && (int)blockIdx.x >= m.cta_begin[r + 1]) ++r;
  const int v = (int)blockIdx.x - m.cta_begin[r], c = m.cta_begin[r + 1] - m.cta_begin[r];
  const SpreadArgs& a = m.a[r];
  const int P = a.plan_ctas;
  spread_stage_body<CS, GROUPED>(a.grid, a.contrib, a.sitems, a.blob, a.cta_off[(long)v * P / c],
                                 a.cta_off[(long)(v + 1) * P / c], a.Cv, a.n, a.err);
}

// The same spread with the items claimed at run time (plans with many
// items per CTA): the producer warp's lane 0 claims the next item from the
// plan's counter when a stage frees up (one claim ahead, so the atomic's
// latency overlaps the waits) and publishes its index with the stage; when
// the items run out it completes the stage's phase without a copy and marks
// it -1.  A CTA whose items run long claims fewer; every item writes its own
// cells, so the result does not depend on which CTA took it.  claim[0]:
// items claimed, claim[1]: CTAs done; the last CTA of the launch returns
// both to 0 (seen by the next launch: kernel boundary).  A separate kernel
// from the plan-time-range one, whose code it leaves untouched (a kernel
// holding both schedules measured slower on the ranges).
template <int CS>
__global__ void __launch_bounds__(kSpreadThreads, kSpreadCtasPerSm)
    spread_claim_kernel(float2* grid, const float2* contrib, const int4* sitems, const int2* blob, int n_items,
                        int* claim, int Cv, int n, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NCW = kSpreadConsumers;
  constexpr int NBUF = 2;
  int2* stage = reinterpret_cast<int2*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)NBUF * kSpreadStageInt2 * sizeof(int2));
  uint64_t* empty = full + NBUF;
  __shared__ volatile int s_abort;
  __shared__ int s_next[NBUF];  // next unclaimed group of the item in each stage
  __shared__ int s_item[NBUF];  // the item in each stage, -1: no more items
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NCW);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  if (warp == NCW) {
    grid_dep_release();
    if (lane == 0) {
      int k = 0;
      int ahead = atomicAdd(claim, 1);
      for (;; ++k) {
        const int b = k % NBUF;
        if (k >= NBUF && !mbar_wait_bounded(&empty[b], (uint32_t)(((k / NBUF) - 1) & 1))) {
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        const int item = ahead;
        if (item >= n_items) {
          s_item[b] = -1;
          mbar_arrive(&full[b]);  // completes the phase: the end mark
          ++k;
          break;
        }
        ahead = atomicAdd(claim, 1);
        const int4 d = __ldg(&sitems[item]);
        const uint32_t bytes = (uint32_t)d.w * (uint32_t)sizeof(int2);
        s_item[b] = item;
        s_next[b] = 0;  // both published to the gather warps by the barrier phase
        mbar_expect_tx(&full[b], bytes);
        bulk_g2s(stage + (size_t)b * kSpreadStageInt2, blob + d.x, bytes, &full[b]);
      }
      // at most one copy per stage can be in flight: the last one issued
      for (int kk = k > NBUF ? k - NBUF : 0; kk < k; ++kk)
        mbar_wait_bounded(&full[kk % NBUF], (uint32_t)((kk / NBUF) & 1));
    }
  } else {
    grid_dep_wait();
    grid_dep_release();
    for (int k = 0;; ++k) {
      const int b = k % NBUF;
      if (!mbar_wait_bounded(&full[b], (uint32_t)((k / NBUF) & 1))) s_abort = 1;
      if (s_abort) break;
      const int item = s_item[b];
      if (item < 0) break;
      const int4 d = __ldg(&sitems[item]);
      gather_groups<CS>(stage + (size_t)b * kSpreadStageInt2, d.y, d.z, lane, &s_next[b], grid, contrib, Cv, n);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_abort) atomicExch(err, 1);
    if (atomicAdd(claim + 1, 1) == (int)gridDim.x - 1) {  // every claim of this CTA precedes its count
      claim[0] = 0;
      claim[1] = 0;
    }
  }
}

// Runtime bin stride (any C <= 2 LP): LP lanes per cell, bins sub and
// sub + LP, lists read from global memory.
template <int LP>
__global__ void __launch_bounds__(256) spread_global_kernel(float2* grid, const float2* contrib, const int4* sitems,
                                                            const int2* blob, int n_items, int C, int Cv) {
  constexpr int CPW = 32 / LP;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LP - 1);
  const int slot = lane / LP;
  const int warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  const bool b0 = sub < Cv, b1 = sub + LP < Cv;
  for (int itm = blockIdx.x; itm < n_items; itm += gridDim.x) {
    const int4 d = __ldg(&sitems[itm]);
    const int2* cells = blob + d.x;
    const int2* ent = cells + ((d.y + 1) & ~1);
    for (int i0 = warp * CPW; i0 < d.y; i0 += nwarp * CPW) {
      const int i = i0 + slot;
      const bool ok = i < d.y;
      int cid = 0, beg = 0, end = 0;
      if (ok) {
        const int2 ce = __ldg(&cells[i]);
        cid = ce.x;
        end = ce.y;
        beg = i > 0 ? __ldg(&cells[i - 1]).y : 0;
      }
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
      for (int e = beg; e < end; ++e) {
        const int2 en = __ldg(&ent[e]);
        const float w = __int_as_float(en.y);
        if (b0) {
          const float2 v = __ldg(contrib + en.x + sub);
          a0.x = fmaf(w, v.x, a0.x);
          a0.y = fmaf(w, v.y, a0.y);
        }
        if (b1) {
          const float2 v = __ldg(contrib + en.x + sub + LP);
          a1.x = fmaf(w, v.x, a1.x);
          a1.y = fmaf(w, v.y, a1.y);
        }
      }
      if (ok) {
        float2* out = grid + (size_t)cid * C;
        if (sub < C) out[sub] = a0;
        if (sub + LP < C) out[sub + LP] = a1;
      }
    }
  }
}

size_t spread_stage_smem() {
  return (size_t)2 * kSpreadStageInt2 * sizeof(int2) + 4 * sizeof(uint64_t);
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

bool interp2_eligible(int cs, int nbins) {
  return (cs == 8 || cs == 16 || cs == 32 || cs == 64) && 2 * nbins > cs;
}

template <int W>
cudaError_t launch_interp(int lp, int cs, const InterpArgs& a, dim3 grid, size_t smem, cudaStream_t s) {
  // compile-time strides for the common chunk widths when more than half of
  // the bins are live (two bins per lane), runtime stride otherwise
  if (interp2_eligible(cs, a.Cv)) {
    const dim3 block(kInterp2Threads);
    if (cs == 32) return launch_dep(interp2_kernel<32, W>, grid, block, smem, s, a);
    if (cs == 64) return launch_dep(interp2_kernel<64, W>, grid, block, smem, s, a);
    if (cs == 16) return launch_dep(interp2_kernel<16, W>, grid, block, smem, s, a);
    return launch_dep(interp2_kernel<8, W>, grid, block, smem, s, a);
  } else {
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
  if ((e = allow_smem(interp2_multi_kernel<32, W>, optin))) return e;
  if ((e = allow_smem(interp2_multi_kernel<64, W>, optin))) return e;
  if ((e = allow_smem(interp2_multi_kernel<16, W>, optin))) return e;
  if ((e = allow_smem(interp2_multi_kernel<8, W>, optin))) return e;
  if ((e = allow_smem(interp2_kernel<32, W>, optin))) return e;
  if ((e = allow_smem(interp2_kernel<64, W>, optin))) return e;
  if ((e = allow_smem(interp2_kernel<16, W>, optin))) return e;
  if ((e = allow_smem(interp2_kernel<8, W>, optin))) return e;
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
  if ((e = configure_interp<8>(smem_optin))) return e;
  const int st = (int)spread_stage_smem();
#define SA(CSV, GR) \
  if ((e = cudaFuncSetAttribute(spread_stage_kernel<CSV, GR>, cudaFuncAttributeMaxDynamicSharedMemorySize, st))) return e;
  SA(8, false) SA(16, false) SA(32, false) SA(64, false) SA(8, true) SA(16, true) SA(32, true) SA(64, true)
#undef SA
#define SA(CSV, GR) \
  if ((e = cudaFuncSetAttribute(spread_stage_multi_kernel<CSV, GR>, cudaFuncAttributeMaxDynamicSharedMemorySize, st))) return e;
  SA(8, false) SA(16, false) SA(32, false) SA(64, false) SA(8, true) SA(16, true) SA(32, true) SA(64, true)
#undef SA
#define SA(CSV) \
  if ((e = cudaFuncSetAttribute(spread_claim_kernel<CSV>, cudaFuncAttributeMaxDynamicSharedMemorySize, st))) return e;
  SA(8) SA(16) SA(32) SA(64)
#undef SA
  return cudaSuccess;
}

size_t interp_tile_bytes(const Plan& p) {
  return (size_t)(p.interp_tr + p.W - 1) * (p.interp_tc + p.W - 1) * p.cs * sizeof(float2);
}

int interp_buffers(const Plan& p) {
  const size_t tile = interp_tile_bytes(p);
  // two buffers when they fit next to the barriers and the static shared memory
  return 2 * tile + 1024 <= (size_t)p.smem_optin ? 2 : 1;
}

InterpArgs interp_args(const Plan& p, int f0, int nbins, float2* y, const float2* y_meas, bool accumulate,
                       const Reducer* red, double* sumsq, float2* contrib) {
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
  a.TR = p.interp_tr;
  a.TC = p.interp_tc;
  a.nct = p.n / p.interp_tc;
  a.tpf = ((p.n + p.interp_tr - 1) / p.interp_tr) * a.nct;
  a.nbuf = interp_buffers(p);
  a.cta_off = p.item_cta_off;
  return a;
}

template <int W>
cudaError_t launch_interp_multi(int cs, const MultiInterp& m, int ctas, size_t smem, cudaStream_t s) {
  const dim3 grid((unsigned)ctas), block(kInterp2Threads);
  if (cs == 32) return launch_dep(interp2_multi_kernel<32, W>, grid, block, smem, s, m);
  if (cs == 64) return launch_dep(interp2_multi_kernel<64, W>, grid, block, smem, s, m);
  if (cs == 16) return launch_dep(interp2_multi_kernel<16, W>, grid, block, smem, s, m);
  if (cs == 8) return launch_dep(interp2_multi_kernel<8, W>, grid, block, smem, s, m);
  return cudaErrorInvalidValue;
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
  a.TR = p.interp_tr;
  a.TC = p.interp_tc;
  a.nct = p.n / p.interp_tc;
  a.tpf = ((p.n + p.interp_tr - 1) / p.interp_tr) * a.nct;
  a.nbuf = interp_buffers(p);
  if (p.n_items == 0) return cudaSuccess;
  // tiles, then a full and an empty barrier per buffer
  const size_t smem = (size_t)a.nbuf * interp_tile_bytes(p) + 2 * a.nbuf * sizeof(uint64_t);
  a.cta_off = p.item_cta_off;
  // the two-bin kernel runs exactly the plan's balanced CTAs; the
  // one-bin kernel strides over the items
  const int blocks = interp2_eligible(p.cs, nbins) ? p.interp_ctas : std::min(p.n_items, p.num_sms);
  if (red && red->capacity < blocks) return cudaErrorInvalidValue;
  const int lp = lanes_for(nbins);
  dim3 grid((unsigned)blocks);
  return p.W == 8 ? launch_interp<8>(lp, p.cs, a, grid, smem, s) : launch_interp<6>(lp, p.cs, a, grid, smem, s);
}

cudaError_t interp_residual_batch(Plan* const* ps, const float2* const* y_meas, int count, cudaStream_t s) {
  if (count < 1 || count > kMaxBatch) return cudaErrorInvalidValue;
  MultiInterp m{};
  m.nreq = 0;
  Plan* mp[kMaxBatch];
  for (int r = 0; r < count; ++r) {
    Plan& p = *ps[r];
    if (p.nchunks != 1) return cudaErrorInvalidValue;
    const bool multi = interp2_eligible(p.cs, p.Nf) && p.cs == ps[0]->cs && p.W == ps[0]->W &&
                       interp_buffers(p) == interp_buffers(*ps[0]) && p.n_items > 0;
    if (!multi) {  // its own launch
      const cudaError_t e = interp(p, 0, p.Nf, p.resid, y_meas[r], false, &p.red_interp, p.scalars, p.contrib, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    mp[m.nreq] = &p;
    m.a[m.nreq] = interp_args(p, 0, p.Nf, p.resid, y_meas[r], false, &p.red_interp, p.scalars, p.contrib);
    m.plan_ctas[m.nreq] = p.interp_ctas;
    ++m.nreq;
  }
  if (m.nreq == 0) return cudaSuccess;
  long work[kMaxBatch];
  int cap[kMaxBatch];
  for (int r = 0; r < m.nreq; ++r) {
    work[r] = mp[r]->M;
    cap[r] = mp[r]->interp_ctas;
    if (mp[r]->red_interp.capacity < cap[r]) return cudaErrorInvalidValue;
  }
  const Plan& p0 = *mp[0];
  const int ctas = split_ctas(work, cap, m.nreq, std::max(m.nreq, p0.num_sms), m.cta_begin);
  const int nbuf = interp_buffers(p0);
  const size_t smem = (size_t)nbuf * interp_tile_bytes(p0) + 2 * nbuf * sizeof(uint64_t);
  return p0.W == 8 ? launch_interp_multi<8>(p0.cs, m, ctas, smem, s) : launch_interp_multi<6>(p0.cs, m, ctas, smem, s);
}

cudaError_t spread_batch(Plan* const* ps, int count, cudaStream_t s) {
  if (count < 1 || count > kMaxBatch) return cudaErrorInvalidValue;
  MultiSpread m{};
  m.nreq = 0;
  Plan* mp[kMaxBatch];
  const auto staged = [](const Plan& p) {
    return p.spread_grouped || (p.spread_staged && (p.cs == 8 || p.cs == 16 || p.cs == 32 || p.cs == 64));
  };
  for (int r = 0; r < count; ++r) {
    Plan& p = *ps[r];
    const bool multi = staged(p) && p.cs == ps[0]->cs && p.spread_grouped == ps[0]->spread_grouped &&
                       staged(*ps[0]) && p.n_sitems > 0 && !p.spread_claimed && !ps[0]->spread_claimed;
    if (!multi) {
      const cudaError_t e = spread(p, 0, p.Nf, p.resid, true, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    mp[m.nreq] = &p;
    SpreadArgs& a = m.a[m.nreq];
    a.grid = p.grid;
    a.contrib = p.contrib;
    a.sitems = p.sitems;
    a.blob = p.sblob;
    a.cta_off = p.sitem_cta_off;
    a.Cv = p.Nf;
    a.n = p.n;
    a.plan_ctas = p.spread_ctas;
    a.err = p.status_dev;
    ++m.nreq;
  }
  if (m.nreq == 0) return cudaSuccess;
  long work[kMaxBatch];
  int cap[kMaxBatch];
  for (int r = 0; r < m.nreq; ++r) {
    work[r] = (long)mp[r]->spread_entries;
    cap[r] = mp[r]->spread_ctas;
  }
  const Plan& p0 = *mp[0];
  const int ctas = split_ctas(work, cap, m.nreq, std::max(m.nreq, kSpreadCtasPerSm * p0.num_sms), m.cta_begin);
  const dim3 g((unsigned)ctas), b(kSpreadThreads);
  const size_t smem = spread_stage_smem();
#define SM(CSV, GR) return launch_dep(spread_stage_multi_kernel<CSV, GR>, g, b, smem, s, m)
  if (p0.spread_grouped) {
    if (p0.cs == 32) SM(32, true);
    if (p0.cs == 64) SM(64, true);
    if (p0.cs == 16) SM(16, true);
    SM(8, true);
  } else {
    if (p0.cs == 32) SM(32, false);
    if (p0.cs == 64) SM(64, false);
    if (p0.cs == 16) SM(16, false);
    SM(8, false);
  }
#undef SM
}

cudaError_t residual(const Plan& p, const float2* y_sum, const float2* y_meas, float2* r, bool with_contrib,
                     const Reducer& red, double* sumsq, cudaStream_t s) {
  const int nbins = std::min(p.chunk, p.Nf);
  const int lp = lanes_for(nbins);
  dim3 g(grid_for(p.M, 8L * (32 / lp), std::min(red.capacity, 16384)));
  float2* contrib = with_contrib ? p.contrib : nullptr;
  switch (lp) {
#define RE(L)                                                                                              \
  case L:                                                                                                  \
    resid_expand_kernel<L><<<g, 256, 0, s>>>(y_sum, y_meas, r, p.phase, contrib, p.M, p.R, p.Nf, p.cs, nbins, \
                                             0, red.partials, red.counter, sumsq);                          \
    break;
    RE(1) RE(2) RE(4) RE(8) RE(16)
    default:
      resid_expand_kernel<32><<<g, 256, 0, s>>>(y_sum, y_meas, r, p.phase, contrib, p.M, p.R, p.Nf, p.cs, nbins, 0,
                                                red.partials, red.counter, sumsq);
#undef RE
  }
  return cudaGetLastError();
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
  if (p.n_sitems == 0) return cudaSuccess;
  if (p.spread_grouped || (p.spread_staged && (p.cs == 8 || p.cs == 16 || p.cs == 32 || p.cs == 64))) {
    dim3 g((unsigned)p.spread_ctas);  // the CTAs the plan's ranges (or its claims) are for
    const size_t smem = spread_stage_smem();
    if (p.spread_claimed) {
#define SC(CSV)                                                                                           \
  return launch_dep(spread_claim_kernel<CSV>, g, dim3(kSpreadThreads), smem, s, p.grid, (const float2*)p.contrib, \
                    (const int4*)p.sitems, (const int2*)p.sblob, p.n_sitems, p.spread_claim, nbins, p.n,       \
                    p.status_dev)
      if (p.cs == 32) SC(32);
      if (p.cs == 64) SC(64);
      if (p.cs == 16) SC(16);
      SC(8);
#undef SC
    }
#define SS(CSV, GR)                                                                                       \
  return launch_dep(spread_stage_kernel<CSV, GR>, g, dim3(kSpreadThreads), smem, s, p.grid,                 \
                    (const float2*)p.contrib, (const int4*)p.sitems, (const int2*)p.sblob,                  \
                    (const int*)p.sitem_cta_off, nbins, p.n, p.status_dev)
    if (p.spread_grouped) {
      if (p.cs == 32) SS(32, true);
      if (p.cs == 64) SS(64, true);
      if (p.cs == 16) SS(16, true);
      SS(8, true);
    } else {
      if (p.cs == 32) SS(32, false);
      if (p.cs == 64) SS(64, false);
      if (p.cs == 16) SS(16, false);
      SS(8, false);
    }
#undef SS
  } else {
    dim3 g((unsigned)std::max(1, std::min(p.n_sitems, 65535)));
#define SG(L) spread_global_kernel<L><<<g, 256, 0, s>>>(p.grid, p.contrib, p.sitems, p.sblob, p.n_sitems, p.cs, nbins)
    switch (lanes_for((p.cs + 1) / 2)) {
      case 1: SG(1); break;
      case 2: SG(2); break;
      case 4: SG(4); break;
      case 8: SG(8); break;
      case 16: SG(16); break;
      default: SG(32); break;
    }
#undef SG
  }
  return cudaGetLastError();
}

}  // namespace prop
