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
constexpr int kKpMaxQ = kKpMaxScales * kKpMaxF;  // 32
constexpr int kKpYChunk = 8;                      // image rows per partial of Xsum
constexpr int kKpXBlock = 64;                     // columns per shared-memory block in the Xsum kernel

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
// bin w) with w fastest; the CTA walks the frames, each frame's Eyt Ewt and
// Ext values staged in shared memory (double-buffered, one barrier a frame).
template <int QM>
__global__ void __launch_bounds__(kKpThreads) kp_render_kernel(const float2* __restrict__ E, KpArgs a, int XS,
                                                               float2* __restrict__ V) {
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
  const int hsz = Nf * Q, usz = XS * Q;
  for (int t = 0; t < a.T; ++t) {
    float2* H = kp_sm + (t & 1) * (hsz + usz);
    float2* U = H + hsz;
    for (int e = threadIdx.x; e < hsz; e += blockDim.x) {
      const int ww = e / Q, q = e - ww * Q;
      H[e] = kmul(Eyt[((size_t)t * N + y) * Q + q], Ewt[((size_t)t * Nf + ww) * Q + q]);
    }
    for (int e = threadIdx.x; e < usz; e += blockDim.x) {
      const int xx = blockIdx.x * XS + e / Q;
      U[e] = xx < N ? Ext[((size_t)t * N + xx) * Q + (e % Q)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (valid) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < QM; ++q)
        if (q < Q) {
          const float2 z = kmul(R[q], kmul(U[xl * Q + q], H[w * Q + q]));
          acc = kadd(acc, z);
        }
      V[(((size_t)t * N + y) * N + x) * Nf + w] = acc;
    }
  }
}

// --- gradient partial sums --------------------------------------------------

// Wsum[t][y][x][q] = sum_w conj(A Eyw Ewt Exw)_q g(t, y, x, w); CTA per (t, y)
// with C[w][q] = A Eyw(y, w) Ewt(t, w) in shared memory.
__global__ void __launch_bounds__(kKpThreads) kp_wsum_kernel(const float2* __restrict__ E, KpArgs a,
                                                             const float2* __restrict__ gV, float2* __restrict__ Ws) {
  extern __shared__ float2 kp_sm[];
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, Nf = a.Nf, N = a.N;
  const int t = blockIdx.x, y = blockIdx.y;
  const float2* Exw = E + a.e_off[kXW];
  const float2* Eyw = E + a.e_off[kYW];
  const float2* Ewt = E + a.e_off[kWT];
  const float2* A = E + a.e_off[kKpPlanes];
  for (int e = threadIdx.x; e < Nf * Q; e += blockDim.x) {
    const int w = e / Q, q = e - w * Q;
    kp_sm[e] = kmul(A[q], kmul(Eyw[((size_t)y * Nf + w) * Q + q], Ewt[((size_t)t * Nf + w) * Q + q]));
  }
  __syncthreads();
  const float2* g = gV + ((size_t)t * N + y) * N * Nf;
  float2* out = Ws + ((size_t)t * N + y) * N * Q;
  for (int e = threadIdx.x; e < N * Q; e += blockDim.x) {
    const int x = e / Q, q = e - x * Q;
    const float2* ew = Exw + (size_t)x * Nf * Q + q;
    float2 acc = make_float2(0.f, 0.f);
    for (int w = 0; w < Nf; ++w) acc = kadd(acc, kcmul(kmul(kp_sm[w * Q + q], ew[(size_t)w * Q]), g[(size_t)x * Nf + w]));
    out[e] = acc;
  }
}

// Tsum[y][x][w][q] = sum_t conj(Ewt(t, w) U3(t, y, x))_q g(t, y, x, w),
// U3 = Exy Ext Eyt; CTA = (column strip, row y), thread = (x, w), the frames
// walked with U3 and Ewt of each frame in shared memory.
template <int QM>
__global__ void __launch_bounds__(kKpThreads) kp_tsum_kernel(const float2* __restrict__ E, KpArgs a, int XS,
                                                             const float2* __restrict__ gV, float2* __restrict__ Ts) {
  extern __shared__ float2 kp_sm[];
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, Nf = a.Nf, N = a.N;
  const int y = blockIdx.y;
  const int xl = threadIdx.x / Nf, w = threadIdx.x - xl * Nf;
  const int x = blockIdx.x * XS + xl;
  const bool valid = xl < XS && x < N;
  const float2* Exy = E + a.e_off[kXY];
  const float2* Ext = E + a.e_off[kXT];
  const float2* Eyt = E + a.e_off[kYT];
  const float2* Ewt = E + a.e_off[kWT];
  float2 acc[QM];
#pragma unroll
  for (int q = 0; q < QM; ++q) acc[q] = make_float2(0.f, 0.f);
  const int hsz = Nf * Q, usz = XS * Q;
  for (int t = 0; t < a.T; ++t) {
    float2* H = kp_sm + (t & 1) * (hsz + usz);
    float2* U = H + hsz;
    for (int e = threadIdx.x; e < hsz; e += blockDim.x) H[e] = Ewt[(size_t)t * Nf * Q + e];
    for (int e = threadIdx.x; e < usz; e += blockDim.x) {
      const int xx = blockIdx.x * XS + e / Q, q = e % Q;
      U[e] = xx < N ? kmul(kmul(Exy[((size_t)y * N + xx) * Q + q], Ext[((size_t)t * N + xx) * Q + q]),
                           Eyt[((size_t)t * N + y) * Q + q])
                    : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (valid) {
      const float2 g = gV[(((size_t)t * N + y) * N + x) * Nf + w];
#pragma unroll
      for (int q = 0; q < QM; ++q)
        if (q < Q) acc[q] = kadd(acc[q], kcmul(kmul(H[w * Q + q], U[xl * Q + q]), g));
    }
  }
  if (valid) {
    float2* out = Ts + (((size_t)y * N + x) * Nf + w) * Q;
#pragma unroll
    for (int q = 0; q < QM; ++q)
      if (q < Q) out[q] = acc[q];
  }
}

// Xpart[c][t][w][q] = sum over the rows y of chunk c of conj(Eyw(y, w))_q
// sum_x conj(Exw(x, w) U3(t, y, x))_q g(t, y, x, w); CTA per (t, chunk),
// thread per (w, q), U3 of a block of columns in shared memory.
__global__ void __launch_bounds__(kKpThreads) kp_xsum_kernel(const float2* __restrict__ E, KpArgs a,
                                                             const float2* __restrict__ gV, float2* __restrict__ Xp) {
  __shared__ float2 U[kKpXBlock * kKpMaxQ];
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, Nf = a.Nf, N = a.N;
  const int t = blockIdx.x, chunk = blockIdx.y;
  const float2* Exy = E + a.e_off[kXY];
  const float2* Exw = E + a.e_off[kXW];
  const float2* Ext = E + a.e_off[kXT];
  const float2* Eyw = E + a.e_off[kYW];
  const float2* Eyt = E + a.e_off[kYT];
  const int npair = Nf * Q;
  const int y0 = chunk * kKpYChunk, y1 = min(N, y0 + kKpYChunk);
  for (int pb = 0; pb < npair; pb += blockDim.x) {  // (w, q) pairs of this pass
    const int e = pb + threadIdx.x;
    const bool own = e < npair;
    const int w = own ? e / Q : 0, q = own ? e - (e / Q) * Q : 0;
    float2 acc = make_float2(0.f, 0.f);
    for (int y = y0; y < y1; ++y) {
      float2 sx = make_float2(0.f, 0.f);
      for (int xb = 0; xb < N; xb += kKpXBlock) {
        const int nx = min(kKpXBlock, N - xb);
        __syncthreads();
        for (int u = threadIdx.x; u < nx * Q; u += blockDim.x) {
          const int xx = xb + u / Q, qq = u % Q;
          U[u] = kmul(kmul(Exy[((size_t)y * N + xx) * Q + qq], Ext[((size_t)t * N + xx) * Q + qq]),
                      Eyt[((size_t)t * N + y) * Q + qq]);
        }
        __syncthreads();
        if (own) {
          const float2* g = gV + (((size_t)t * N + y) * N + xb) * Nf + w;
          const float2* ew = Exw + ((size_t)xb * Nf + w) * Q + q;
          for (int xx = 0; xx < nx; ++xx)
            sx = kadd(sx, kcmul(kmul(ew[(size_t)xx * Nf * Q], U[xx * Q + q]), g[(size_t)xx * Nf]));
        }
      }
      if (own) acc = kadd(acc, kcmul(Eyw[((size_t)y * Nf + w) * Q + q], sx));
    }
    if (own) Xp[(((size_t)chunk * a.T + t) * Nf + w) * Q + q] = acc;
  }
}

// Second passes: the expanded gradients, each a fixed-order sum.
// dExy[y][x][q] = sum_t conj(Ext(t, x) Eyt(t, y)) Wsum(t, y, x)
__global__ void __launch_bounds__(kKpThreads) kp_dxy_kernel(const float2* __restrict__ E, KpArgs a,
                                                            const float2* __restrict__ Ws, float2* __restrict__ dE) {
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, N = a.N;
  const size_t total = (size_t)N * N * Q;
  const float2* Ext = E + a.e_off[kXT];
  const float2* Eyt = E + a.e_off[kYT];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(i % Q);
    const size_t yx = i / Q;
    const int x = (int)(yx % N), y = (int)(yx / N);
    float2 acc = make_float2(0.f, 0.f);
    for (int t = 0; t < a.T; ++t)
      acc = kadd(acc, kcmul(kmul(Ext[((size_t)t * N + x) * Q + q], Eyt[((size_t)t * N + y) * Q + q]),
                            Ws[(size_t)t * total + i]));
    dE[a.e_off[kXY] + i] = acc;
  }
}

// dExt[t][x][q] = sum_y conj(Exy(y, x) Eyt(t, y)) Wsum(t, y, x);
// dEyt[t][y][q] = sum_x conj(Exy(y, x) Ext(t, x)) Wsum(t, y, x).
__global__ void __launch_bounds__(kKpThreads) kp_dt_kernel(const float2* __restrict__ E, KpArgs a,
                                                           const float2* __restrict__ Ws, float2* __restrict__ dE) {
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, N = a.N;
  const size_t per = (size_t)a.T * N * Q;  // elements of dExt (= of dEyt)
  const float2* Exy = E + a.e_off[kXY];
  const float2* Ext = E + a.e_off[kXT];
  const float2* Eyt = E + a.e_off[kYT];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * per; i += (size_t)gridDim.x * blockDim.x) {
    const bool is_xt = i < per;
    const size_t j = is_xt ? i : i - per;
    const int q = (int)(j % Q);
    const size_t tr = j / Q;
    const int r = (int)(tr % N), t = (int)(tr / N);  // r = x (dExt) or y (dEyt)
    float2 acc = make_float2(0.f, 0.f);
    if (is_xt) {
      for (int y = 0; y < N; ++y)
        acc = kadd(acc, kcmul(kmul(Exy[((size_t)y * N + r) * Q + q], Eyt[((size_t)t * N + y) * Q + q]),
                              Ws[(((size_t)t * N + y) * N + r) * Q + q]));
      dE[a.e_off[kXT] + j] = acc;
    } else {
      for (int x = 0; x < N; ++x)
        acc = kadd(acc, kcmul(kmul(Exy[((size_t)r * N + x) * Q + q], Ext[((size_t)t * N + x) * Q + q]),
                              Ws[(((size_t)t * N + r) * N + x) * Q + q]));
      dE[a.e_off[kYT] + j] = acc;
    }
  }
}

// dExw[x][w][q] = sum_y conj(A Eyw(y, w)) Tsum(y, x, w);
// dEyw[y][w][q] = sum_x conj(A Exw(x, w)) Tsum(y, x, w).
__global__ void __launch_bounds__(kKpThreads) kp_dw_kernel(const float2* __restrict__ E, KpArgs a,
                                                           const float2* __restrict__ Ts, float2* __restrict__ dE) {
  grid_dep_wait();
  grid_dep_release();
  const int Q = a.Q, N = a.N, Nf = a.Nf;
  const size_t per = (size_t)N * Nf * Q;
  const float2* Exw = E + a.e_off[kXW];
  const float2* Eyw = E + a.e_off[kYW];
  const float2* A = E + a.e_off[kKpPlanes];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * per; i += (size_t)gridDim.x * blockDim.x) {
    const bool is_xw = i < per;
    const size_t j = is_xw ? i : i - per;
    const int q = (int)(j % Q);
    const size_t rw = j / Q;
    const int w = (int)(rw % Nf), r = (int)(rw / Nf);  // r = x (dExw) or y (dEyw)
    float2 acc = make_float2(0.f, 0.f);
    if (is_xw) {
      for (int y = 0; y < N; ++y)
        acc = kadd(acc, kcmul(Eyw[((size_t)y * Nf + w) * Q + q], Ts[(((size_t)y * N + r) * Nf + w) * Q + q]));
      dE[a.e_off[kXW] + j] = kcmul(A[q], acc);
    } else {
      for (int x = 0; x < N; ++x)
        acc = kadd(acc, kcmul(Exw[((size_t)x * Nf + w) * Q + q], Ts[(((size_t)r * N + x) * Nf + w) * Q + q]));
      dE[a.e_off[kYW] + j] = kcmul(A[q], acc);
    }
  }
}

// dEwt[t][w][q] = conj(A) Xsum(t, w) and dA[q] = sum_(t, w) conj(Ewt(t, w)) Xsum(t, w),
// Xsum = the chunk partials summed in chunk order.  One CTA per q for dA.
__global__ void __launch_bounds__(kKpThreads) kp_dwt_kernel(const float2* __restrict__ E, KpArgs a, int nchunks,
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
    for (int c = 0; c < nchunks; ++c) xs = kadd(xs, Xp[((size_t)c * a.T * Nf + tw) * Q + q]);
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
  if (p.Nf > kKpThreads) return fail(PROP_ERR_INVALID_ARG, "kplanes: at most 256 spectral bins");
  return PROP_OK;
}

unsigned kp_blocks(size_t count, const Plan& p) {
  return (unsigned)std::max<size_t>(1, std::min<size_t>((count + kKpThreads - 1) / kKpThreads, (size_t)16 * p.num_sms));
}

// Columns per CTA of the render and time-sum kernels: XS * Nf <= 256 threads.
int kp_strip(const Plan& p) { return std::max(1, std::min(p.N, kKpThreads / p.Nf)); }

int kp_ychunks(const Plan& p) { return (p.N + kKpYChunk - 1) / kKpYChunk; }

// Device workspace of the model (the expanded planes and the gradient
// partials), grown on demand and kept in the plan.
struct KpWork {
  float2* E;     // expanded planes + A
  float2* dE;    // expanded gradients
  float2* Ws;    // [T][N][N][Q]
  float2* Ts;    // [N][N][Nf][Q]
  float2* Xp;    // [chunks][T][Nf][Q]
};

KpWork kp_carve(const Plan& p, const KpArgs& a) {
  KpWork w{};
  float2* base = (float2*)p.kp_work;
  w.E = base;
  base += a.e_count;
  w.dE = base;
  base += a.e_count;
  w.Ws = base;
  base += (size_t)a.T * a.N * a.N * a.Q;
  w.Ts = base;
  base += (size_t)a.N * a.N * a.Nf * a.Q;
  w.Xp = base;
  return w;
}

size_t kp_work_elems(const Plan& p, const KpArgs& a) {
  return 2 * a.e_count + (size_t)a.T * a.N * a.N * a.Q + (size_t)a.N * a.N * a.Nf * a.Q +
         (size_t)kp_ychunks(p) * a.T * a.Nf * a.Q;
}

prop_status kp_ensure(Plan& p, const KpArgs& a) {
  const size_t bytes = kp_work_elems(p, a) * sizeof(float2);
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

template <int QM>
cudaError_t launch_render_q(const Plan& p, const KpArgs& a, const KpWork& w, float2* V, cudaStream_t s) {
  const int XS = kp_strip(p);
  const size_t smem = 2 * (size_t)(p.Nf + XS) * a.Q * sizeof(float2);
  return launch_dep(kp_render_kernel<QM>, dim3((p.N + XS - 1) / XS, p.N), dim3(XS * p.Nf), smem, s,
                    (const float2*)w.E, a, XS, V);
}

template <int QM>
cudaError_t launch_tsum_q(const Plan& p, const KpArgs& a, const KpWork& w, const float2* gV, cudaStream_t s) {
  const int XS = kp_strip(p);
  const size_t smem = 2 * (size_t)(p.Nf + XS) * a.Q * sizeof(float2);
  return launch_dep(kp_tsum_kernel<QM>, dim3((p.N + XS - 1) / XS, p.N), dim3(XS * p.Nf), smem, s,
                    (const float2*)w.E, a, XS, gV, w.Ts);
}

// Shared memory above the default 48 KB for the two frame-walking kernels.
cudaError_t kp_configure(const Plan& p, const KpArgs& a) {
  const size_t smem = 2 * (size_t)(p.Nf + kp_strip(p)) * a.Q * sizeof(float2);
  const size_t wsm = (size_t)p.Nf * a.Q * sizeof(float2);
  cudaError_t e = cudaSuccess;
  auto opt = [&](const void* k, size_t bytes) {
    if (e == cudaSuccess && bytes > 48 * 1024)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  opt((const void*)kp_render_kernel<8>, smem);
  opt((const void*)kp_render_kernel<16>, smem);
  opt((const void*)kp_render_kernel<32>, smem);
  opt((const void*)kp_tsum_kernel<8>, smem);
  opt((const void*)kp_tsum_kernel<16>, smem);
  opt((const void*)kp_tsum_kernel<32>, smem);
  opt((const void*)kp_wsum_kernel, wsm);
  return e;
}

cudaError_t kp_expand(Plan& p, const KpArgs& a, const KpWork& w, const float2* P, cudaStream_t s) {
  StageScope sc(p, kStKpRender, s);
  return launch_dep(kp_expand_kernel, dim3(kp_blocks(a.e_count, p)), dim3(kKpThreads), 0, s, P, a, w.E);
}

cudaError_t kp_render(Plan& p, const KpArgs& a, const KpWork& w, float2* V, cudaStream_t s) {
  StageScope sc(p, kStKpRender, s);
  if (a.Q <= 8) return launch_render_q<8>(p, a, w, V, s);
  if (a.Q <= 16) return launch_render_q<16>(p, a, w, V, s);
  return launch_render_q<32>(p, a, w, V, s);
}

// Parameter gradients G from grad V, with w.E holding the expanded planes.
cudaError_t kp_vjp(Plan& p, const KpArgs& a, const KpWork& w, const float2* gV, float2* G, size_t count,
                   cudaStream_t s) {
  StageScope sc(p, kStKpVjp, s);
  cudaError_t e;
  const int nch = kp_ychunks(p);
  e = launch_dep(kp_wsum_kernel, dim3(a.T, a.N), dim3(kKpThreads), (size_t)a.Nf * a.Q * sizeof(float2), s,
                 (const float2*)w.E, a, gV, w.Ws);
  if (e != cudaSuccess) return e;
  e = a.Q <= 8 ? launch_tsum_q<8>(p, a, w, gV, s)
               : a.Q <= 16 ? launch_tsum_q<16>(p, a, w, gV, s) : launch_tsum_q<32>(p, a, w, gV, s);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_xsum_kernel, dim3(a.T, nch), dim3(kKpThreads), 0, s, (const float2*)w.E, a, gV, w.Xp);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_dxy_kernel, dim3(kp_blocks((size_t)a.N * a.N * a.Q, p)), dim3(kKpThreads), 0, s,
                 (const float2*)w.E, a, (const float2*)w.Ws, w.dE);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_dt_kernel, dim3(kp_blocks(2 * (size_t)a.T * a.N * a.Q, p)), dim3(kKpThreads), 0, s,
                 (const float2*)w.E, a, (const float2*)w.Ws, w.dE);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_dw_kernel, dim3(kp_blocks(2 * (size_t)a.N * a.Nf * a.Q, p)), dim3(kKpThreads), 0, s,
                 (const float2*)w.E, a, (const float2*)w.Ts, w.dE);
  if (e != cudaSuccess) return e;
  e = launch_dep(kp_dwt_kernel, dim3(a.Q), dim3(kKpThreads), 0, s, (const float2*)w.E, a, nch,
                 (const float2*)w.Xp, w.dE);
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
