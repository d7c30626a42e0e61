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
// Every plane is first expanded to the volume's resolution along its two
// axes (the interpolation done once per plane value instead of once per
// voxel), with the scale and feature index q = s F + k innermost:
//   Exy[y][x][q]  Exw[x][w][q]  Ext[t][x][q]  Eyw[y][w][q]  Eyt[t][y][q]
//   Ewt[t][w][q]  A[q] = a_s,k.
// Then V(t, y, x, w) = sum_q R_q(y, x, w) Ext(t, x)_q Eyt(t, y)_q Ewt(t, w)_q
// with R = A Exy Exw Eyw independent of t: the render walks the frames of
// each (image row, column strip) with R in registers.
//
// Gradients (grad z = sum conj(dV/dz) grad V, Sec. 4.3's Adam on the plane
// parameters) are sums of g = grad V times the other five factors over the
// two axes a plane lacks.  They are evaluated through three partial sums,
// each written once in a fixed order (no atomics, bitwise reproducible):
//   Wsum(t, y, x)_q = sum_w conj(A Exw Eyw Ewt)_q g            (omega summed)
//   Tsum(y, x, w)_q = sum_t conj(Exy Ext Eyt Ewt)_q g          (time summed)
//   Xsum(t, w)_q    = sum_y conj(Eyw)_q sum_x conj(Exw Exy Ext Eyt)_q g
// from which
//   dExy = sum_t conj(Ext Eyt) Wsum,  dExt = sum_y conj(Exy Eyt) Wsum,
//   dEyt = sum_x conj(Exy Ext) Wsum,  dExw = sum_y conj(A Eyw) Tsum,
//   dEyw = sum_x conj(A Exw) Tsum,    dEwt = conj(A) Xsum,
//   dA   = sum_(t,w) conj(Ewt) Xsum,
// and the transposed interpolation carries each expanded gradient back to
// the plane nodes.
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
constexpr int kKpYChunk = 8;                      // image rows per CTA of the gradient kernels
constexpr int kKpTB = 8;                          // frames (or rows) staged per barrier

enum { kXY = 0, kXW = 1, kXT = 2, kYW = 3, kYT = 4, kWT = 5 };

struct KpScale {
  size_t off[kKpPlanes];  // element offset of each plane in the parameter buffer
  size_t a;               // element offset of a
  int rows[kKpPlanes], cols[kKpPlanes];
  int n;                  // spatial nodes per axis
};

// Sizes, parameter layout and the offsets of the expanded planes.
struct KpArgs {
  int N, Nf, T, F, S, Q;  // Q = S F
  KpScale sc[kKpMaxScales];
  size_t e_off[kKpPlanes + 1];  // expanded planes, then A (element offsets into the E buffer)
  size_t e_count;
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
// Tap of voxel index i on an axis of R nodes spanning Nv voxels.
__device__ __forceinline__ Tap axis_tap(int i, int R, int Nv) {
  if (R == Nv) return make_tap((float)i, R);
  return make_tap(((float)i + 0.5f) * ((float)R / (float)Nv) - 0.5f, R);
}

__device__ __forceinline__ float2 kmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 kcmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 kadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// Plane c's voxel-resolution axes: (extent of the first expanded index, of the second).
__host__ __device__ inline void exp_axes(const KpArgs& a, int c, int* e0, int* e1) {
  switch (c) {
    case kXY: *e0 = a.N; *e1 = a.N; break;   // [y][x]
    case kXW: *e0 = a.N; *e1 = a.Nf; break;  // [x][w]
    case kXT: *e0 = a.T; *e1 = a.N; break;   // [t][x]
    case kYW: *e0 = a.N; *e1 = a.Nf; break;  // [y][w]
    case kYT: *e0 = a.T; *e1 = a.N; break;   // [t][y]
    default: *e0 = a.T; *e1 = a.Nf; break;   // [t][w]
  }
}

// Node (row, col) of plane c and the voxel extents along them, for expanded
// index (i0, i1): xw and yw are stored [w][.] as planes but [.][w] expanded.
struct PlaneMap {
  int vr, vc;        // voxel index along the plane's row / column axis
  int Nr, Nc;        // voxel extents of those axes
};
__device__ __forceinline__ PlaneMap plane_map(const KpArgs& a, int c, int i0, int i1) {
  PlaneMap m;
  switch (c) {
    case kXY: m.vr = i0; m.vc = i1; m.Nr = a.N; m.Nc = a.N; break;
    case kXW: m.vr = i1; m.vc = i0; m.Nr = a.Nf; m.Nc = a.N; break;
    case kXT: m.vr = i0; m.vc = i1; m.Nr = a.T; m.Nc = a.N; break;
    case kYW: m.vr = i1; m.vc = i0; m.Nr = a.Nf; m.Nc = a.N; break;
    case kYT: m.vr = i0; m.vc = i1; m.Nr = a.T; m.Nc = a.N; break;
    default: m.vr = i0; m.vc = i1; m.Nr = a.T; m.Nc = a.Nf; break;
  }
  return m;
}

// --- expansion -------------------------------------------------------------

// E[e_off[c] + (i0 * e1 + i1) * Q + q] = bilinear value of plane c (scale
// q / F, feature q % F) at voxel coordinates (i0, i1); A[q] = a.
__global__ void __launch_bounds__(kKpThreads) kp_expand_kernel(const float2* __restrict__ P, KpArgs a,
                                                               float2* __restrict__ E) {
  grid_dep_wait();
  grid_dep_release();
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < a.e_count;
       idx += (size_t)gridDim.x * blockDim.x) {
    int c = 0;
    while (c < kKpPlanes && idx >= a.e_off[c + 1]) ++c;
    const size_t rel = idx - a.e_off[c];
    const int q = (int)(rel % a.Q);
    const int s = q / a.F, k = q - s * a.F;
    const KpScale& S = a.sc[s];
    if (c == kKpPlanes) {  // the weighting vector
      E[idx] = P[S.a + k];
      continue;
    }
    int e0, e1;
    exp_axes(a, c, &e0, &e1);
    const size_t cell = rel / a.Q;
    const int i0 = (int)(cell / e1), i1 = (int)(cell % e1);
    const PlaneMap m = plane_map(a, c, i0, i1);
    const Tap r = axis_tap(m.vr, S.rows[c], m.Nr);
    const Tap cc = axis_tap(m.vc, S.cols[c], m.Nc);
    const float2* Pc = P + S.off[c];
    const int cols = S.cols[c], F = a.F;
    const float2 p00 = Pc[((size_t)r.lo * cols + cc.lo) * F + k];
    const float2 p01 = Pc[((size_t)r.lo * cols + cc.hi) * F + k];
    const float2 p10 = Pc[((size_t)r.hi * cols + cc.lo) * F + k];
    const float2 p11 = Pc[((size_t)r.hi * cols + cc.hi) * F + k];
    const float w00 = (1.f - r.w) * (1.f - cc.w), w01 = (1.f - r.w) * cc.w, w10 = r.w * (1.f - cc.w),
                w11 = r.w * cc.w;
    E[idx] = make_float2(fmaf(w11, p11.x, fmaf(w10, p10.x, fmaf(w01, p01.x, w00 * p00.x))),
                         fmaf(w11, p11.y, fmaf(w10, p10.y, fmaf(w01, p01.y, w00 * p00.y))));
  }
}

// Transpose of the expansion: node gradient of plane c = sum over the
// expanded cells that read the node of (interpolation weight x expanded
// gradient), in ascending cell order; the a gradient is copied.
__global__ void __launch_bounds__(kKpThreads) kp_contract_kernel(const float2* __restrict__ dE, KpArgs a,
                                                                 float2* __restrict__ G, size_t count) {
  grid_dep_wait();
  grid_dep_release();
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < count;
       idx += (size_t)gridDim.x * blockDim.x) {
    // locate (scale, plane, node row, node col, feature) of parameter idx
    int s = 0;
    while (s + 1 < a.S && idx >= a.sc[s + 1].off[0]) ++s;
    const KpScale& S = a.sc[s];
    if (idx >= S.a) {
      const int k = (int)(idx - S.a);
      G[idx] = dE[a.e_off[kKpPlanes] + s * a.F + k];
      continue;
    }
    int c = 0;
    while (c + 1 < kKpPlanes && idx >= S.off[c + 1]) ++c;
    const size_t rel = idx - S.off[c];
    const int k = (int)(rel % a.F);
    const size_t node = rel / a.F;
    const int rr = (int)(node / S.cols[c]), rc = (int)(node % S.cols[c]);
    const int q = s * a.F + k;
    int e0, e1;
    exp_axes(a, c, &e0, &e1);
    const PlaneMap m0 = plane_map(a, c, 0, 0);
    const int Nr = m0.Nr, Nc = m0.Nc, R = S.rows[c], C = S.cols[c];
    // voxels that can reach node rr (rc): within two node spacings
    const int r_lo = max(0, (int)floorf((rr - 2) * (float)Nr / R)), r_hi = min(Nr - 1, (int)ceilf((rr + 2) * (float)Nr / R));
    const int c_lo = max(0, (int)floorf((rc - 2) * (float)Nc / C)), c_hi = min(Nc - 1, (int)ceilf((rc + 2) * (float)Nc / C));
    float2 acc = make_float2(0.f, 0.f);
    for (int vr = r_lo; vr <= r_hi; ++vr) {
      const Tap tr = axis_tap(vr, R, Nr);
      const float wr = (tr.lo == rr ? 1.f - tr.w : 0.f) + (tr.hi == rr ? tr.w : 0.f);
      if (wr == 0.f) continue;
      for (int vc = c_lo; vc <= c_hi; ++vc) {
        const Tap tc = axis_tap(vc, C, Nc);
        const float wc = (tc.lo == rc ? 1.f - tc.w : 0.f) + (tc.hi == rc ? tc.w : 0.f);
        if (wc == 0.f) continue;
        // expanded index of (plane row voxel vr, plane col voxel vc)
        const bool swapped = (c == kXW || c == kYW);
        const int i0 = swapped ? vc : vr, i1 = swapped ? vr : vc;
        const float2 v = dE[a.e_off[c] + ((size_t)i0 * e1 + i1) * a.Q + q];
        const float w = wr * wc;
        acc.x = fmaf(w, v.x, acc.x);
        acc.y = fmaf(w, v.y, acc.y);
      }
    }
    G[idx] = acc;
  }
}

// --- render ------------------------------------------------------------------

// CTA = (column strip of XS image columns, image row y); thread = (column x,
// bin w) with w fastest; the CTA walks the frames TB at a time: the
// frames' Eyt Ewt (laid out [frame][q][w]) and Ext ([frame][q][x]) are staged
// in shared memory with one barrier per batch (double-buffered), so each
// thread has TB independent loads in flight per fill; conflict-free reads.
template <int QM>
__global__ void __launch_bounds__(kKpThreads) kp_render_kernel(const float2* __restrict__ E, KpArgs a, int XS,
                                                               int TB, float2* __restrict__ V) {
  extern __shared__ float2 kp_sm[];
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, Nf = a.Nf, N = a.N;
  const int y = blockIdx.y;
  const int xl = threadIdx.x / Nf, w = threadIdx.x - xl * Nf;
  const int x = blockIdx.x * XS + xl;
  const bool valid = xl < XS && x < N;
  const float2* Exy = E + a.e_off[kXY];
  const float2* Exw = E + a.e_off[kXW];
  const float2* Ext = E + a.e_off[kXT];
  const float2* Eyw = E + a.e_off[kYW];
  const float2* Eyt = E + a.e_off[kYT];
  const float2* Ewt = E + a.e_off[kWT];
  const float2* A = E + a.e_off[kKpPlanes];
  float2 R[QM];
#pragma unroll
  for (int q = 0; q < QM; ++q) {
    R[q] = make_float2(0.f, 0.f);
    if (valid && q < Q)
      R[q] = kmul(kmul(A[q], Exy[((size_t)y * N + x) * Q + q]),
                  kmul(Exw[((size_t)x * Nf + w) * Q + q], Eyw[((size_t)y * Nf + w) * Q + q]));
  }
  const int hsz = Nf * Q, usz = XS * Q, bsz = TB * (hsz + usz);
  for (int t0 = 0, buf = 0; t0 < a.T; t0 += TB, buf ^= 1) {
    const int nt = min(TB, a.T - t0);
    float2* H = kp_sm + buf * bsz;       // [frame][q][w]
    float2* U = H + TB * hsz;            // [frame][q][x]
    for (int e = threadIdx.x; e < hsz; e += blockDim.x) {
      const int ww = e % Nf, q = e / Nf;
      for (int tb = 0; tb < nt; ++tb)
        H[tb * hsz + e] = kmul(Eyt[((size_t)(t0 + tb) * N + y) * Q + q], Ewt[((size_t)(t0 + tb) * Nf + ww) * Q + q]);
    }
    for (int e = threadIdx.x; e < usz; e += blockDim.x) {
      const int xx = blockIdx.x * XS + e % XS, q = e / XS;
      for (int tb = 0; tb < nt; ++tb)
        U[tb * usz + e] = xx < N ? Ext[((size_t)(t0 + tb) * N + xx) * Q + q] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (valid)
      for (int tb = 0; tb < nt; ++tb) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < QM; ++q)
          if (q < Q) acc = kadd(acc, kmul(R[q], kmul(U[tb * usz + q * XS + xl], H[tb * hsz + q * Nf + w])));
        V[((((size_t)t0 + tb) * N + y) * N + x) * Nf + w] = acc;
      }
  }
}

// --- gradients ---------------------------------------------------------------
//
// Three kernels walk the frames over tiles of the volume and leave small
// fixed-order partials (summed afterwards in index order by kp_sum_kernel):
//   W kernel, CTA (strip of XS columns, chunk of kKpYChunk rows), thread (x, q):
//     Wsum(t, y, x)_q = sum_w conj(A Eyw Ewt Exw)_q g, then
//     dExy(y, x) = sum_t conj(Ext Eyt) Wsum           complete (one CTA owns (y, x))
//     dExt(t, x) = sum_y conj(Exy Eyt) Wsum           partial per row chunk
//     dEyt(t, y) = sum_x conj(Exy Ext) Wsum           partial per column strip
//   T kernel, CTA (strip, row chunk), thread (x, w):
//     Tsum(y, x, w)_q = sum_t conj(Exy Ext Eyt Ewt)_q g, then
//     dExw(x, w) = sum_y conj(A Eyw) Tsum             partial per row chunk
//     dEyw(y, w) = sum_x conj(A Exw) Tsum             partial per column strip
//   X kernel, CTA (strip, frame t), thread (w, q):
//     Xsum(t, w)_q = sum_y conj(Eyw) sum_x conj(Exw Exy Ext Eyt)_q g
//                                                     partial per column strip
//   then dEwt = conj(A) Xsum and dA = sum_(t, w) conj(Ewt) Xsum.

struct KpPart {
  float2* xt;   // [ychunks][T][N][Q]
  float2* yt;   // [xstrips_W][T][N][Q]
  float2* xw;   // [ychunks][N][Nf][Q]
  float2* yw;   // [xstrips_T][N][Nf][Q]
  float2* wt;   // [xstrips_X][T][Nf][Q]
};

__global__ void __launch_bounds__(kKpThreads) kp_wgrad_kernel(const float2* __restrict__ E, KpArgs a, int XS,
                                                              int YBW, const float2* __restrict__ gV, float2* __restrict__ dE,
                                                              KpPart part) {
  extern __shared__ float2 kp_sm[];
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, Nf = a.Nf, N = a.N;
  const int xl = threadIdx.x / Q, q = threadIdx.x - xl * Q;
  const int x = blockIdx.x * XS + xl;
  const bool valid = xl < XS && x < N;
  const int y0 = blockIdx.y * kKpYChunk, ny = min(kKpYChunk, N - y0);
  const float2* Exy = E + a.e_off[kXY];
  const float2* Exw = E + a.e_off[kXW];
  const float2* Ext = E + a.e_off[kXT];
  const float2* Eyw = E + a.e_off[kYW];
  const float2* Eyt = E + a.e_off[kYT];
  const float2* Ewt = E + a.e_off[kWT];
  const float2* A = E + a.e_off[kKpPlanes];
  float2* sEw = kp_sm;                            // [w][xl][q] Exw of the strip
  float2* sC = sEw + (size_t)Nf * XS * Q;         // [row][w][q] A Eyw(y) Ewt(t) of YBW rows of the current frame
  float2* sR = sC + (size_t)YBW * Nf * Q;         // [yi][xl][q] dEyt terms of the current frame
  for (int e = threadIdx.x; e < Nf * XS * Q; e += blockDim.x) {
    const int qq = e % Q, r = e / Q, xx = r % XS, ww = r / XS;
    const int gx = blockIdx.x * XS + xx;
    sEw[e] = gx < N ? Exw[((size_t)gx * Nf + ww) * Q + qq] : make_float2(0.f, 0.f);
  }
  float2 dxy[kKpYChunk], exy[kKpYChunk];
#pragma unroll
  for (int i = 0; i < kKpYChunk; ++i) {
    dxy[i] = make_float2(0.f, 0.f);
    exy[i] = (valid && i < ny) ? Exy[((size_t)(y0 + i) * N + x) * Q + q] : make_float2(0.f, 0.f);
  }
  for (int t = 0; t < a.T; ++t) {
    float2 dxt = make_float2(0.f, 0.f);
    const float2 ext = valid ? Ext[((size_t)t * N + x) * Q + q] : make_float2(0.f, 0.f);
    for (int yb = 0; yb < ny; yb += YBW) {
      const int nb = min(YBW, ny - yb);
      // the frame's A Eyw Ewt for YBW rows of the chunk, one barrier
      for (int e = threadIdx.x; e < Nf * Q; e += blockDim.x) {
        const int ww = e / Q, qq = e - ww * Q;
        const float2 aw = kmul(A[qq], Ewt[((size_t)t * Nf + ww) * Q + qq]);
        for (int r = 0; r < nb; ++r) sC[r * Nf * Q + e] = kmul(aw, Eyw[((size_t)(y0 + yb + r) * Nf + ww) * Q + qq]);
      }
      __syncthreads();
#pragma unroll
      for (int yi = 0; yi < kKpYChunk; ++yi) {
        if (yi < yb || yi >= yb + nb) continue;
        const int y = y0 + yi;
        if (valid) {
          const float2* g = gV + (((size_t)t * N + y) * N + x) * Nf;
          const float2* C = sC + (size_t)(yi - yb) * Nf * Q;
          float2 ws = make_float2(0.f, 0.f);
          for (int ww = 0; ww < Nf; ++ww)
            ws = kadd(ws, kcmul(kmul(C[ww * Q + q], sEw[((size_t)ww * XS + xl) * Q + q]), g[ww]));
          const float2 eyt = Eyt[((size_t)t * N + y) * Q + q];
          dxy[yi] = kadd(dxy[yi], kcmul(kmul(ext, eyt), ws));
          dxt = kadd(dxt, kcmul(kmul(exy[yi], eyt), ws));
          sR[((size_t)yi * XS + xl) * Q + q] = kcmul(kmul(exy[yi], ext), ws);
        } else if (xl < XS) {
          sR[((size_t)yi * XS + xl) * Q + q] = make_float2(0.f, 0.f);
        }
      }
      __syncthreads();  // sC is refilled for the next rows
    }
    // dEyt partial of this strip: sum the columns' terms in column order
    for (int e = threadIdx.x; e < ny * Q; e += blockDim.x) {
      const int yi = e / Q, qq = e - yi * Q;
      float2 s = make_float2(0.f, 0.f);
      for (int xx = 0; xx < XS; ++xx) s = kadd(s, sR[((size_t)yi * XS + xx) * Q + qq]);
      part.yt[(((size_t)blockIdx.x * a.T + t) * N + y0 + yi) * Q + qq] = s;
    }
    if (valid) part.xt[(((size_t)blockIdx.y * a.T + t) * N + x) * Q + q] = dxt;
    __syncthreads();  // sC and sR are rewritten for the next frame
  }
  if (valid)
    for (int yi = 0; yi < ny; ++yi) dE[a.e_off[kXY] + ((size_t)(y0 + yi) * N + x) * Q + q] = dxy[yi];
}

template <int QM>
__global__ void __launch_bounds__(kKpThreads) kp_tgrad_kernel(const float2* __restrict__ E, KpArgs a, int XS, int TB,
                                                              const float2* __restrict__ gV, KpPart part) {
  extern __shared__ float2 kp_sm[];
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, Nf = a.Nf, N = a.N;
  const int xl = threadIdx.x / Nf, w = threadIdx.x - xl * Nf;
  const int x = blockIdx.x * XS + xl;
  const bool valid = xl < XS && x < N;
  const int y0 = blockIdx.y * kKpYChunk, ny = min(kKpYChunk, N - y0);
  const float2* Exy = E + a.e_off[kXY];
  const float2* Exw = E + a.e_off[kXW];
  const float2* Ext = E + a.e_off[kXT];
  const float2* Eyw = E + a.e_off[kYW];
  const float2* Eyt = E + a.e_off[kYT];
  const float2* Ewt = E + a.e_off[kWT];
  const float2* A = E + a.e_off[kKpPlanes];
  const int hsz = Nf * Q, usz = XS * Q, bsz = TB * (hsz + usz);
  float2* sR = kp_sm + 2 * (size_t)bsz;  // [q][xl][w] dEyw terms of the current row
  float2 dxw[QM];
#pragma unroll
  for (int qq = 0; qq < QM; ++qq) dxw[qq] = make_float2(0.f, 0.f);
  int buf = 0;
  for (int yi = 0; yi < ny; ++yi) {
    const int y = y0 + yi;
    float2 acc[QM];
#pragma unroll
    for (int qq = 0; qq < QM; ++qq) acc[qq] = make_float2(0.f, 0.f);
    for (int t0 = 0; t0 < a.T; t0 += TB, buf ^= 1) {
      const int nt = min(TB, a.T - t0);
      float2* H = kp_sm + buf * bsz;  // [frame][q][w] Ewt(t)
      float2* U = H + TB * hsz;       // [frame][q][x] Exy Ext Eyt
      for (int e = threadIdx.x; e < hsz; e += blockDim.x) {
        const int ww = e % Nf, qq = e / Nf;
        for (int tb = 0; tb < nt; ++tb) H[tb * hsz + e] = Ewt[((size_t)(t0 + tb) * Nf + ww) * Q + qq];
      }
      for (int e = threadIdx.x; e < usz; e += blockDim.x) {
        const int xx = blockIdx.x * XS + e % XS, qq = e / XS;
        const float2 exy = xx < N ? Exy[((size_t)y * N + xx) * Q + qq] : make_float2(0.f, 0.f);
        for (int tb = 0; tb < nt; ++tb) {
          const int t = t0 + tb;
          U[tb * usz + e] = xx < N ? kmul(kmul(exy, Ext[((size_t)t * N + xx) * Q + qq]), Eyt[((size_t)t * N + y) * Q + qq])
                                   : make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
      if (valid)
        for (int tb = 0; tb < nt; ++tb) {
          const float2 g = gV[((((size_t)t0 + tb) * N + y) * N + x) * Nf + w];
#pragma unroll
          for (int qq = 0; qq < QM; ++qq)
            if (qq < Q) acc[qq] = kadd(acc[qq], kcmul(kmul(H[tb * hsz + qq * Nf + w], U[tb * usz + qq * XS + xl]), g));
        }
    }
    // this row's Tsum is in acc: fold it into the dExw chunk partial and
    // leave the dEyw terms for the column-order sum below
#pragma unroll
    for (int qq = 0; qq < QM; ++qq)
      if (qq < Q) {
        float2 ta = make_float2(0.f, 0.f), tb = make_float2(0.f, 0.f);
        if (valid) {
          ta = kcmul(kmul(A[qq], Eyw[((size_t)y * Nf + w) * Q + qq]), acc[qq]);
          tb = kcmul(kmul(A[qq], Exw[((size_t)x * Nf + w) * Q + qq]), acc[qq]);
        }
        dxw[qq] = kadd(dxw[qq], ta);
        if (xl < XS) sR[((size_t)qq * XS + xl) * Nf + w] = tb;
      }
    __syncthreads();
    for (int e = threadIdx.x; e < Nf * Q; e += blockDim.x) {
      const int qq = e / Nf, ww = e - qq * Nf;  // consecutive threads read consecutive bins
      float2 s = make_float2(0.f, 0.f);
      for (int xx = 0; xx < XS; ++xx) s = kadd(s, sR[((size_t)qq * XS + xx) * Nf + ww]);
      part.yw[(((size_t)blockIdx.x * N + y) * Nf + ww) * Q + qq] = s;
    }
    __syncthreads();  // sR is rewritten for the next row
  }
  if (valid) {
    float2* out = part.xw + (((size_t)blockIdx.y * N + x) * Nf + w) * Q;
#pragma unroll
    for (int qq = 0; qq < QM; ++qq)
      if (qq < Q) out[qq] = dxw[qq];
  }
}

__global__ void __launch_bounds__(kKpThreads) kp_xgrad_kernel(const float2* __restrict__ E, KpArgs a, int XS, int YB,
                                                              const float2* __restrict__ gV, KpPart part) {
  extern __shared__ float2 kp_sm[];
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, Nf = a.Nf, N = a.N;
  const int t = blockIdx.y;
  const int x0 = blockIdx.x * XS, nx = min(XS, N - x0);
  const float2* Exy = E + a.e_off[kXY];
  const float2* Exw = E + a.e_off[kXW];
  const float2* Ext = E + a.e_off[kXT];
  const float2* Eyw = E + a.e_off[kYW];
  const float2* Eyt = E + a.e_off[kYT];
  // per staged row: U [xl][q] = Exy Ext Eyt, G [xl][w] = grad V, Y [w][q] = Eyw
  const int usz = XS * Q, gsz = XS * Nf, ysz = Nf * Q, rsz = usz + gsz + ysz;
  float2* sEw = kp_sm;                          // [xl][w][q] Exw of the strip
  float2* sB = sEw + (size_t)XS * Nf * Q;       // 2 x YB staged rows
  for (int e = threadIdx.x; e < nx * Nf * Q; e += blockDim.x) sEw[e] = Exw[(size_t)x0 * Nf * Q + e];
  const int npair = Nf * Q;
  for (int pb = 0; pb < npair; pb += blockDim.x) {  // (w, q) pairs of this pass
    const int e = pb + threadIdx.x;
    const bool own = e < npair;
    const int w = own ? e / Q : 0, q = own ? e - w * Q : 0;
    float2 acc = make_float2(0.f, 0.f);
    int buf = 0;
    for (int yb = 0; yb < N; yb += YB, buf ^= 1) {
      const int nyb = min(YB, N - yb);
      float2* Bf = sB + (size_t)buf * YB * rsz;
      for (int u = threadIdx.x; u < nx * Q; u += blockDim.x) {
        const int xx = x0 + u / Q, qq = u % Q;
        const float2 ext = Ext[((size_t)t * N + xx) * Q + qq];
        for (int r = 0; r < nyb; ++r) {
          const int y = yb + r;
          Bf[(size_t)r * rsz + u] = kmul(kmul(Exy[((size_t)y * N + xx) * Q + qq], ext), Eyt[((size_t)t * N + y) * Q + qq]);
        }
      }
      for (int u = threadIdx.x; u < nx * Nf; u += blockDim.x)
        for (int r = 0; r < nyb; ++r)
          Bf[(size_t)r * rsz + usz + u] = gV[(((size_t)t * N + yb + r) * N + x0) * Nf + u];
      for (int u = threadIdx.x; u < ysz; u += blockDim.x)
        for (int r = 0; r < nyb; ++r) Bf[(size_t)r * rsz + usz + gsz + u] = Eyw[(size_t)(yb + r) * Nf * Q + u];
      __syncthreads();
      if (own)
        for (int r = 0; r < nyb; ++r) {
          const float2* Ur = Bf + (size_t)r * rsz;
          const float2* Gr = Ur + usz;
          float2 sx = make_float2(0.f, 0.f);
          for (int xx = 0; xx < nx; ++xx)
            sx = kadd(sx, kcmul(kmul(sEw[((size_t)xx * Nf + w) * Q + q], Ur[xx * Q + q]), Gr[xx * Nf + w]));
          acc = kadd(acc, kcmul(Gr[gsz + w * Q + q], sx));
        }
    }
    if (own) part.wt[(((size_t)blockIdx.x * a.T + t) * Nf + w) * Q + q] = acc;
    __syncthreads();
  }
}

// out[i] = scale(i) * sum_c part[c * len + i] over c = 0 .. nparts - 1 in
// order; scale = conj(A[i % Q]) when conj_a, else 1.
__global__ void __launch_bounds__(kKpThreads) kp_sum_kernel(const float2* __restrict__ part, int nparts, size_t len,
                                                            const float2* __restrict__ A, int Q, int conj_a,
                                                            float2* __restrict__ out) {
  grid_dep_wait();
  grid_dep_release();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int c = 0; c < nparts; ++c) s = kadd(s, part[(size_t)c * len + i]);
    out[i] = conj_a ? kcmul(A[i % Q], s) : s;
  }
}

// dEwt[t][w][q] = conj(A) Xsum and dA[q] = sum_(t, w) conj(Ewt(t, w)) Xsum,
// Xsum = the strip partials summed in strip order.  One CTA per q for dA.
__global__ void __launch_bounds__(kKpThreads) kp_dwt_kernel(const float2* __restrict__ E, KpArgs a, int nparts,
                                                            const float2* __restrict__ Xp, float2* __restrict__ dE) {
  __shared__ float2 red[kKpThreads];
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, Nf = a.Nf;
  const int q = blockIdx.x;
  const float2* Ewt = E + a.e_off[kWT];
  const float2 Aq = E[a.e_off[kKpPlanes] + q];
  float2 da = make_float2(0.f, 0.f);
  for (int tw = threadIdx.x; tw < a.T * Nf; tw += blockDim.x) {
    float2 xs = make_float2(0.f, 0.f);
    for (int c = 0; c < nparts; ++c) xs = kadd(xs, Xp[((size_t)c * a.T * Nf + tw) * Q + q]);
    dE[a.e_off[kWT] + (size_t)tw * Q + q] = kcmul(Aq, xs);
    da = kadd(da, kcmul(Ewt[(size_t)tw * Q + q], xs));
  }
  red[threadIdx.x] = da;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = kadd(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) dE[a.e_off[kKpPlanes] + q] = red[0];
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

// Layout of the parameter buffer and of the expanded planes; returns the
// parameter count.
size_t kp_layout(const Plan& p, int F, int S, KpArgs* out) {
  KpArgs a{};
  a.N = p.N;
  a.Nf = p.Nf;
  a.T = p.T;
  a.F = F;
  a.S = S;
  a.Q = S * F;
  size_t off = 0;
  for (int s = 0; s < S; ++s) {
    KpScale& sc = a.sc[s];
    const int n = p.N >> s;
    sc.n = n;
    const int rows[kKpPlanes] = {n, p.Nf, p.T, p.Nf, p.T, p.T};
    const int cols[kKpPlanes] = {n, n, n, n, n, p.Nf};
    for (int c = 0; c < kKpPlanes; ++c) {
      sc.off[c] = off;
      sc.rows[c] = rows[c];
      sc.cols[c] = cols[c];
      off += (size_t)rows[c] * cols[c] * F;
    }
    sc.a = off;
    off += F;
  }
  size_t e = 0;
  for (int c = 0; c < kKpPlanes; ++c) {
    a.e_off[c] = e;
    int e0, e1;
    exp_axes(a, c, &e0, &e1);
    e += (size_t)e0 * e1 * a.Q;
  }
  a.e_off[kKpPlanes] = e;
  a.e_count = e + a.Q;
  if (out) *out = a;
  return off;
}

prop_status kp_check(const Plan& p, int F, int S) {
  if (F < 1 || F > kKpMaxF) return fail(PROP_ERR_INVALID_ARG, "kplanes: features must be in [1, 16]");
  if (S < 1 || S > kKpMaxScales) return fail(PROP_ERR_INVALID_ARG, "kplanes: scales must be 1 or 2");
  if ((p.N >> (S - 1)) < 2) return fail(PROP_ERR_INVALID_ARG, "kplanes: image too small for the scales");
  if (p.Nf > 64) return fail(PROP_ERR_INVALID_ARG, "kplanes: at most 64 spectral bins");
  return PROP_OK;
}

unsigned kp_blocks(size_t count, const Plan& p) {
  return (unsigned)std::max<size_t>(1, std::min<size_t>((count + kKpThreads - 1) / kKpThreads, (size_t)16 * p.num_sms));
}

// Tile widths (image columns per CTA) and batch depths (frames or rows
// staged per barrier) of the frame-walking kernels.
struct KpTiles {
  int xs_r, xs_w, xs_t, xs_x;  // render (thread per (x, w)), W (x, q), T (x, w), X (strip in shared memory)
  int ns_r, ns_w, ns_t, ns_x, nch;  // strips of the render, W, T and X kernels; row chunks
  int tb_r, tb_t, yb_x, yb_w;   // frames per barrier (render, T), rows per barrier (X, W)
};
KpTiles kp_tiles(const Plan& p, int Q) {
  KpTiles k;
  const int c8 = (int)sizeof(float2);
  k.xs_r = std::max(1, std::min(std::min(p.N, 64), kKpThreads / p.Nf));
  k.xs_t = k.xs_r;
  k.xs_w = std::max(1, std::min(std::min(p.N, kKpThreads / Q), 8192 / (p.Nf * Q)));
  k.xs_x = std::max(1, std::min(8, (96 * 1024) / ((p.Nf + 2) * Q * c8)));
  k.ns_r = (p.N + k.xs_r - 1) / k.xs_r;
  k.ns_w = (p.N + k.xs_w - 1) / k.xs_w;
  k.ns_t = (p.N + k.xs_t - 1) / k.xs_t;
  k.ns_x = (p.N + k.xs_x - 1) / k.xs_x;
  k.nch = (p.N + kKpYChunk - 1) / kKpYChunk;
  const int per_frame = 2 * (p.Nf + k.xs_r) * Q * c8;  // double-buffered staging of one frame
  k.tb_r = std::max(1, std::min(kKpTB, (96 * 1024) / per_frame));
  k.tb_t = k.tb_r;
  const int xrow = k.xs_x * Q + k.xs_x * p.Nf + p.Nf * Q;  // one staged row of the X kernel
  k.yb_x = std::max(1, std::min(kKpTB, (64 * 1024) / (2 * xrow * c8)));
  k.yb_w = std::max(1, std::min(kKpYChunk, 4096 / (p.Nf * Q)));
  return k;
}
size_t smem_render(const Plan& p, const KpArgs& a, const KpTiles& k) {
  return 2 * (size_t)k.tb_r * (p.Nf + k.xs_r) * a.Q * sizeof(float2);
}
size_t smem_w(const Plan& p, const KpArgs& a, const KpTiles& k) {
  return ((size_t)p.Nf * k.xs_w * a.Q + (size_t)k.yb_w * p.Nf * a.Q + (size_t)kKpYChunk * k.xs_w * a.Q) *
         sizeof(float2);
}
size_t smem_t(const Plan& p, const KpArgs& a, const KpTiles& k) {
  return (2 * (size_t)k.tb_t * (p.Nf * a.Q + k.xs_t * a.Q) + (size_t)a.Q * k.xs_t * p.Nf) * sizeof(float2);
}
size_t smem_x(const Plan& p, const KpArgs& a, const KpTiles& k) {
  const size_t row = (size_t)k.xs_x * a.Q + (size_t)k.xs_x * p.Nf + (size_t)p.Nf * a.Q;
  return ((size_t)k.xs_x * p.Nf * a.Q + 2 * (size_t)k.yb_x * row) * sizeof(float2);
}

// Device workspace of the model (the expanded planes, their gradients and
// the gradient kernels' partials), grown on demand and kept in the plan.
struct KpWork {
  float2* E;     // expanded planes + A
  float2* dE;    // expanded gradients
  KpPart part;
};

size_t kp_part_elems(const Plan& p, const KpArgs& a, const KpTiles& k, size_t* off) {
  const size_t Q = a.Q, N = p.N, Nf = p.Nf, T = p.T;
  const size_t sz[5] = {k.nch * T * N * Q, k.ns_w * T * N * Q, k.nch * N * Nf * Q, k.ns_t * N * Nf * Q,
                        k.ns_x * T * Nf * Q};
  size_t o = 0;
  for (int i = 0; i < 5; ++i) {
    if (off) off[i] = o;
    o += sz[i];
  }
  return o;
}

KpWork kp_carve(const Plan& p, const KpArgs& a) {
  const KpTiles k = kp_tiles(p, a.Q);
  KpWork w{};
  float2* base = (float2*)p.kp_work;
  w.E = base;
  w.dE = base + a.e_count;
  float2* pb = w.dE + a.e_count;
  size_t off[5];
  kp_part_elems(p, a, k, off);
  w.part.xt = pb + off[0];
  w.part.yt = pb + off[1];
  w.part.xw = pb + off[2];
  w.part.yw = pb + off[3];
  w.part.wt = pb + off[4];
  return w;
}

prop_status kp_ensure(Plan& p, const KpArgs& a) {
  const KpTiles k = kp_tiles(p, a.Q);
  const size_t bytes = (2 * a.e_count + kp_part_elems(p, a, k, nullptr)) * sizeof(float2);
  if (p.kp_work && p.kp_work_bytes >= bytes) return PROP_OK;
  if (p.kp_work) {
    plan_dev_free(&p, p.kp_work);
    p.recon_bytes -= p.kp_work_bytes;
    p.kp_work = nullptr;
    p.kp_work_bytes = 0;
  }
  cudaError_t e = plan_dev_alloc(&p, &p.kp_work, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p.kp_work = nullptr;
    return fail(PROP_ERR_OOM, std::string("kplanes: workspace allocation of ") + std::to_string(bytes) +
                                  " bytes failed: " + cudaGetErrorString(e));
  }
  p.kp_work_bytes = bytes;
  p.recon_bytes += bytes;
  return PROP_OK;
}

// Shared memory above the default 48 KB for the frame-walking kernels.
cudaError_t kp_configure(const Plan& p, const KpArgs& a) {
  const KpTiles k = kp_tiles(p, a.Q);
  cudaError_t e = cudaSuccess;
  auto opt = [&](const void* f, size_t bytes) {
    if (e == cudaSuccess && bytes > 48 * 1024)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  const size_t sr = smem_render(p, a, k), st = smem_t(p, a, k);
  opt((const void*)kp_render_kernel<8>, sr);
  opt((const void*)kp_render_kernel<16>, sr);
  opt((const void*)kp_render_kernel<32>, sr);
  opt((const void*)kp_tgrad_kernel<8>, st);
  opt((const void*)kp_tgrad_kernel<16>, st);
  opt((const void*)kp_tgrad_kernel<32>, st);
  opt((const void*)kp_wgrad_kernel, smem_w(p, a, k));
  opt((const void*)kp_xgrad_kernel, smem_x(p, a, k));
  return e;
}

cudaError_t kp_expand(Plan& p, const KpArgs& a, const KpWork& w, const float2* P, cudaStream_t s) {
  StageScope sc(p, kStKpRender, s);
  return launch_dep(kp_expand_kernel, dim3(kp_blocks(a.e_count, p)), dim3(kKpThreads), 0, s, P, a, w.E);
}

template <int QM>
cudaError_t launch_render_q(const Plan& p, const KpArgs& a, const KpWork& w, float2* V, cudaStream_t s) {
  const KpTiles k = kp_tiles(p, a.Q);
  return launch_dep(kp_render_kernel<QM>, dim3(k.ns_r, p.N), dim3(k.xs_r * p.Nf), smem_render(p, a, k), s,
                    (const float2*)w.E, a, k.xs_r, k.tb_r, V);
}

cudaError_t kp_render(Plan& p, const KpArgs& a, const KpWork& w, float2* V, cudaStream_t s) {
  StageScope sc(p, kStKpRender, s);
  if (a.Q <= 8) return launch_render_q<8>(p, a, w, V, s);
  if (a.Q <= 16) return launch_render_q<16>(p, a, w, V, s);
  return launch_render_q<32>(p, a, w, V, s);
}

template <int QM>
cudaError_t launch_tgrad_q(const Plan& p, const KpArgs& a, const KpWork& w, const float2* gV, cudaStream_t s) {
  const KpTiles k = kp_tiles(p, a.Q);
  return launch_dep(kp_tgrad_kernel<QM>, dim3(k.ns_t, k.nch), dim3(k.xs_t * p.Nf), smem_t(p, a, k), s,
                    (const float2*)w.E, a, k.xs_t, k.tb_t, gV, w.part);
}

// Parameter gradients G from grad V, with w.E holding the expanded planes.
cudaError_t kp_vjp(Plan& p, const KpArgs& a, const KpWork& w, const float2* gV, float2* G, size_t count,
                   cudaStream_t s) {
  StageScope sc(p, kStKpVjp, s);
  const KpTiles k = kp_tiles(p, a.Q);
  const float2* A = w.E + a.e_off[kKpPlanes];
  cudaError_t e;
  e = launch_dep(kp_wgrad_kernel, dim3(k.ns_w, k.nch), dim3(k.xs_w * a.Q), smem_w(p, a, k), s, (const float2*)w.E,
                 a, k.xs_w, k.yb_w, gV, w.dE, w.part);
  if (e != cudaSuccess) return e;
  e = a.Q <= 8 ? launch_tgrad_q<8>(p, a, w, gV, s)
               : a.Q <= 16 ? launch_tgrad_q<16>(p, a, w, gV, s) : launch_tgrad_q<32>(p, a, w, gV, s);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_xgrad_kernel, dim3(k.ns_x, p.T), dim3(kKpThreads), smem_x(p, a, k), s, (const float2*)w.E, a,
                 k.xs_x, k.yb_x, gV, w.part);
  if (e != cudaSuccess) return e;
  const size_t lxt = (size_t)p.T * p.N * a.Q, lxw = (size_t)p.N * p.Nf * a.Q;
  e = launch_dep(kp_sum_kernel, dim3(kp_blocks(lxt, p)), dim3(kKpThreads), 0, s, (const float2*)w.part.xt, k.nch,
                 lxt, A, a.Q, 0, w.dE + a.e_off[kXT]);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_sum_kernel, dim3(kp_blocks(lxt, p)), dim3(kKpThreads), 0, s, (const float2*)w.part.yt, k.ns_w,
                 lxt, A, a.Q, 0, w.dE + a.e_off[kYT]);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_sum_kernel, dim3(kp_blocks(lxw, p)), dim3(kKpThreads), 0, s, (const float2*)w.part.xw, k.nch,
                 lxw, A, a.Q, 0, w.dE + a.e_off[kXW]);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_sum_kernel, dim3(kp_blocks(lxw, p)), dim3(kKpThreads), 0, s, (const float2*)w.part.yw, k.ns_t,
                 lxw, A, a.Q, 0, w.dE + a.e_off[kYW]);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_dwt_kernel, dim3(a.Q), dim3(kKpThreads), 0, s, (const float2*)w.E, a, k.ns_x,
                 (const float2*)w.part.wt, w.dE);
  if (e != cudaSuccess) return e;
  return launch_dep(kp_contract_kernel, dim3(kp_blocks(count, p)), dim3(kKpThreads), 0, s, (const float2*)w.dE, a,
                    G, count);
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
  if ((st = kp_ensure(p, a)) != PROP_OK) return st;
  PROP_CUDA(kp_configure(p, a));
  const KpWork w = kp_carve(p, a);
  cudaStream_t s = (cudaStream_t)stream;
  PROP_CUDA(kp_expand(p, a, w, (const float2*)params_dev, s));
  PROP_CUDA(kp_render(p, a, w, (float2*)V_dev, s));
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
  if ((st = kp_ensure(p, a)) != PROP_OK) return st;
  PROP_CUDA(kp_configure(p, a));
  const KpWork w = kp_carve(p, a);
  cudaStream_t s = (cudaStream_t)stream;
  PROP_CUDA(kp_expand(p, a, w, (const float2*)params_dev, s));
  PROP_CUDA(kp_vjp(p, a, w, (const float2*)gV_dev, (float2*)grad_dev, count, s));
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
  if ((st = kp_ensure(p, a)) != PROP_OK) return st;
  PROP_CUDA(kp_configure(p, a));
  const KpWork w = kp_carve(p, a);
  // Adam state and the parameter gradient: 3 x count complex values
  float2* G = nullptr;
  cudaError_t e = plan_dev_alloc(&p, (void**)&G, 3 * count * sizeof(float2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PROP_ERR_OOM, std::string("kplanes_reconstruct: Adam state allocation failed: ") +
                                  cudaGetErrorString(e));
  }
  float2* m = G + count;
  float2* v = m + count;
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemsetAsync(m, 0, 2 * count * sizeof(float2), s);
  float2* P = (float2*)kp_params_dev;
  const unsigned pb = kp_blocks(count, p);
  AdamArgs la{};
  la.tv_xy = q.tv_xy;
  la.tv_t = q.tv_t;
  la.tv_eps = q.tv_eps;
  la.gscale = 2.f;
  for (int k = 1; k <= q.iters && e == cudaSuccess && st == PROP_OK; ++k) {
    e = kp_expand(p, a, w, P, s);
    if (e == cudaSuccess) e = kp_render(p, a, w, p.vol2, s);
    if (e != cudaSuccess) break;
    if ((st = loss_grad_device(p, (const float2*)y_dev, la, p.vol2, p.grad, p.loss_dev + (k - 1), s)) != PROP_OK)
      break;
    e = kp_vjp(p, a, w, (const float2*)p.grad, G, count, s);
    AdamArgs ad{};
    const double bc1 = 1.0 - std::pow((double)q.beta1, k), bc2 = 1.0 - std::pow((double)q.beta2, k);
    ad.lr_t = (float)(q.lr / bc1);
    ad.inv_bc2_sqrt = (float)(1.0 / std::sqrt(bc2));
    ad.beta1 = q.beta1;
    ad.beta2 = q.beta2;
    ad.eps = q.eps;
    if (e == cudaSuccess) {
      StageScope sc(p, kStKpAdam, s);
      e = launch_dep(kp_adam_kernel, dim3(pb), dim3(kKpThreads), 0, s, P, (const float2*)G, m, v, count, ad);
    }
  }
  if (e == cudaSuccess && st == PROP_OK && loss_trace_host && q.iters > 0)
    e = cudaMemcpyAsync(loss_trace_host, p.loss_dev, sizeof(double) * q.iters, cudaMemcpyDeviceToHost, s);
  const cudaError_t es = cudaStreamSynchronize(s);  // the gradient and Adam state are released below
  if (e == cudaSuccess) e = es;
  plan_dev_free(&p, G);
  if (st != PROP_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "kplanes_reconstruct");
  return PROP_OK;
}

}  // extern "C"
