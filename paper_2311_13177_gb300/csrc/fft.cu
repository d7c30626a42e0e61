// Batched shared-memory FFTs of the oversampled grid (no cuFFT).
//
// The 2N x 2N transform of every (frame, bin) slice is done as two passes of
// 1-D transforms of length n = 2N along one axis, each CTA transforming a
// tile of kFftCols = 16 lines that are adjacent in memory, so that every
// global access of a warp covers two runs of 16 consecutive complex64
// values (2 x 128 B, fully coalesced).  Bins are the fastest axis of every
// array, so the "lines" of a pass are (u1, f) columns of the grid or the
// bins of one image row.
//
// Each 1-D transform is a mixed-radix Stockham FFT (radices 8, 4, 2, 3):
// pass p with radix R and stride Ns (product of the previous radices)
// reads R values at stride n/R, multiplies by exp(-+2 pi i r (j mod Ns) /
// (Ns R)), does an R-point DFT in registers and writes the results at
// (j / Ns) Ns R + (j mod Ns) + r Ns.  The first pass reads global memory
// directly (zero padding and deapodisation applied on the fly), the last
// pass writes global memory directly (cropping and scaling applied on the
// fly); intermediate passes exchange through shared memory in place.
// Every thread holds E = 16 (n = 2^a) or 12 (n = 3 * 2^a) values per pass.
#include <type_traits>

#include "prop_internal.cuh"
#include "tv_adam.cuh"
#include "tma.cuh"

namespace prop {
namespace {

struct RadixPlan {
  int count;
  int r[8];
};

// Radices for E values a thread (every radix divides E, so a thread holds
// whole butterflies in every pass): with E = 32, radix 32 while it divides
// and then 16; else radix 8 where E allows (E = 16 or 24), radix 4 where it
// does not (E = 12, lengths with a factor 3: half the registers of 24,
// twice the threads); then 4, 2 and the threes, a leftover factor 2 merged
// with a 3 into one radix-6 pass.
__host__ __device__ constexpr RadixPlan radix_plan(int n, int E) {
  RadixPlan p{0, {1, 1, 1, 1, 1, 1, 1, 1}};
  int m = n, threes = 0;
  while (m % 3 == 0) {
    m /= 3;
    ++threes;
  }
  while (E % 32 == 0 && threes == 0 && m % 32 == 0) {
    p.r[p.count++] = 32;
    m /= 32;
  }
  if (E % 16 == 0 && threes == 0 && m % 16 == 0 && p.count > 0) {
    p.r[p.count++] = 16;
    m /= 16;
  }
  while (E % 8 == 0 && m % 8 == 0) {
    p.r[p.count++] = 8;
    m /= 8;
  }
  while (threes > 0 && m % 4 == 0) {
    p.r[p.count++] = 4;
    m /= 4;
  }
  if (m % 4 == 0) {
    p.r[p.count++] = 4;
    m /= 4;
  }
  if (m % 2 == 0 && threes > 0) {  // a leftover 2 and a 3 make one radix-6 pass
    m /= 2;
    --threes;
    for (int i = 0; i < threes; ++i) p.r[p.count++] = 3;
    p.r[p.count++] = 6;
    return p;
  }
  if (m % 2 == 0) {
    p.r[p.count++] = 2;
    m /= 2;
  }
  for (int i = 0; i < threes; ++i) p.r[p.count++] = 3;
  return p;
}

// Twiddle tables, one per Stockham pass p >= 1 with stride NS and radix R:
// entry [k][r] (k < NS, r < R) = exp(-2 pi i r k / (NS R)), so a butterfly
// fetches its R factors with R/2 16-byte loads.  Offsets are even (every NS
// and hence every table size is even), so the tables stay 16-byte aligned.
template <int NFFT, int EV>
__host__ __device__ constexpr int tw_offset(int pass) {
  constexpr RadixPlan RP = radix_plan(NFFT, EV);
  int off = 0, ns = RP.r[0];
  for (int q = 1; q < pass; ++q) {
    off += ns * RP.r[q];
    ns *= RP.r[q];
  }
  return off;
}

// Values per thread: 16 (two radix-8 butterflies a pass), 12 for lengths
// with a factor 3 (radices 4, 2, 3).  (8 values a thread, twice the
// threads, measured slower for the column passes at n = 512.)
template <int NFFT>
constexpr int kValsPlain = (NFFT % 3 == 0) ? 12 : 16;
template <int NFFT>
constexpr int kValsFused = (NFFT % 3 == 0) ? 12 : 16;
// Values per thread of the TMA-staged column passes: 32 at n = 512 (radix
// 32 then 16: one shared-memory exchange instead of two) and 24 at n = 384
// (radices 8, 8, 6: two instead of three), with twice the registers and
// half the threads of a 16-value shape; 2N = 512: 23.9 -> 20.3 us forward,
// 24.8 -> 22.3 us adjoint; 2N = 384: 184.7 -> 153.8 us and 193.4 -> 164.7 us.
template <int NFFT>
constexpr int kValsCols = NFFT == 512 ? 32 : NFFT == 384 ? 24 : kValsPlain<NFFT>;

template <int NFFT, int EV>
struct Shape {
  static constexpr int E = EV;                 // values per thread
  static constexpr int TPL = NFFT / E;         // threads per line
  static constexpr int THREADS = TPL * kFftCols;
  static constexpr int TW = tw_offset<NFFT, EV>(radix_plan(NFFT, EV).count);  // twiddle table entries
  static constexpr size_t SMEM = (size_t)NFFT * kFftCols * sizeof(float2) + (size_t)TW * sizeof(float2);
};

// Fill the per-pass twiddle tables from the length-NFFT table exp(-2 pi i m / NFFT).
template <int NFFT, int EV>
__device__ void build_twiddles(float2* tws, const float2* __restrict__ base) {
  constexpr RadixPlan RP = radix_plan(NFFT, EV);
  int ns = RP.r[0];
  for (int p = 1; p < RP.count; ++p) {
    const int R = RP.r[p];
    const int off = tw_offset<NFFT, EV>(p);
    const int step = NFFT / (ns * R);
    for (int idx = threadIdx.x; idx < ns * R; idx += blockDim.x) {
      const int k = idx / R, r = idx - (idx / R) * R;
      tws[off + idx] = base[r * k * step];
    }
    ns *= R;
  }
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// Rounded product that is never contracted into a later add: the inputs of
// the first butterfly round the same way in every kernel that builds them.
__device__ __forceinline__ float2 cscale_rn(float2 a, float s) {
  return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s));
}
// z * (SIGN i)
template <int SIGN>
__device__ __forceinline__ float2 mul_si(float2 z) {
  return SIGN > 0 ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}

// In-register DFTs X_k = sum_q v_q exp(SIGN 2 pi i q k / R).
template <int R, int SIGN>
struct Dft;

template <int SIGN>
struct Dft<2, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int SIGN>
struct Dft<4, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = mul_si<SIGN>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <int SIGN>
struct Dft<8, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    constexpr float h = 0.70710678118654752f;  // 1/sqrt(2)
    float2 a[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = cadd(v[q], v[q + 4]);
      b[q] = csub(v[q], v[q + 4]);
    }
    // b_q *= w^q, w = exp(SIGN i pi / 4)
    {
      float2 z = b[1];
      b[1] = make_float2((z.x - SIGN * z.y) * h, (z.y + SIGN * z.x) * h);
      b[2] = mul_si<SIGN>(b[2]);
      z = b[3];
      b[3] = make_float2((-z.x - SIGN * z.y) * h, (-z.y + SIGN * z.x) * h);
    }
    Dft<4, SIGN>::run(a);
    Dft<4, SIGN>::run(b);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[2 * q] = a[q];
      v[2 * q + 1] = b[q];
    }
  }
};

template <int SIGN>
struct Dft<3, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    constexpr float s3 = 0.86602540378443865f;  // sqrt(3)/2
    float2 t = cadd(v[1], v[2]);
    float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    float2 d = mul_si<SIGN>(cscale(csub(v[1], v[2]), s3));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, d);
    v[2] = csub(m, d);
  }
};

// 6 = 2 x 3: the three-point DFTs of the even and the odd inputs, then
// X[k] = E[k] + w^k O[k] and X[k + 3] = E[k] - w^k O[k], w = exp(SIGN 2 pi i / 6).
template <int SIGN>
struct Dft<6, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    constexpr float s3 = 0.86602540378443865f;  // sqrt(3)/2
    float2 a[3] = {v[0], v[2], v[4]}, b[3] = {v[1], v[3], v[5]};
    Dft<3, SIGN>::run(a);
    Dft<3, SIGN>::run(b);
    const float2 t1 = make_float2(0.5f * b[1].x - SIGN * s3 * b[1].y, 0.5f * b[1].y + SIGN * s3 * b[1].x);
    const float2 t2 = make_float2(-0.5f * b[2].x - SIGN * s3 * b[2].y, -0.5f * b[2].y + SIGN * s3 * b[2].x);
    v[0] = cadd(a[0], b[0]);
    v[3] = csub(a[0], b[0]);
    v[1] = cadd(a[1], t1);
    v[4] = csub(a[1], t1);
    v[2] = cadd(a[2], t2);
    v[5] = csub(a[2], t2);
  }
};

// cos(2 pi m / 32) from its values on the first quadrant; sin(2 pi m / 32)
// = cos(2 pi (m - 8) / 32).  The constant factors inside the radix-16 and
// radix-32 butterflies.
__host__ __device__ constexpr double cos32(int m) {
  constexpr double q[9] = {1.0,
                           0.98078528040323044912618223613424,   // cos(pi / 16)
                           0.92387953251128675612818318939679,   // cos(pi / 8)
                           0.83146961230254523707878837761791,   // cos(3 pi / 16)
                           0.70710678118654752440084436210485,   // cos(pi / 4)
                           0.55557023301960222474283081394853,   // cos(5 pi / 16)
                           0.38268343236508977172845998403040,   // cos(3 pi / 8)
                           0.19509032201612826784828486847702,   // cos(7 pi / 16)
                           0.0};
  m &= 31;
  return m <= 8 ? q[m] : m <= 16 ? -q[16 - m] : m <= 24 ? -q[m - 16] : q[32 - m];
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }

// z * exp(SIGN 2 pi i M / R) for R dividing 32; quarter turns exactly.
template <int SIGN, int R, int M>
__device__ __forceinline__ float2 rotate(float2 z) {
  constexpr int m = (M % R) * (32 / R);  // in 32nds of a turn
  if constexpr (m == 0) {
    return z;
  } else if constexpr (m == 8) {
    return mul_si<SIGN>(z);
  } else if constexpr (m == 16) {
    return make_float2(-z.x, -z.y);
  } else if constexpr (m == 24) {
    return mul_si<-SIGN>(z);
  } else {
    constexpr float c = (float)cos32(m), sn = (float)(SIGN * sin32(m));
    return make_float2(fmaf(z.x, c, -z.y * sn), fmaf(z.x, sn, z.y * c));
  }
}

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// R = R1 R2 point DFT from R2 DFTs of R1 points and R1 of R2 points:
// with q = R2 q1 + q2 and k = k1 + R1 k2,
//   X_k = sum_q2 w_R^(q2 k1) w_R2^(q2 k2) sum_q1 x_q w_R1^(q1 k1),  w_R = exp(SIGN 2 pi i / R).
template <int R1, int R2, int SIGN>
__device__ __forceinline__ void dft_compose(float2* v) {
  constexpr int R = R1 * R2;
  float2 y[R];  // y[q2 R1 + k1]
  static_for<0, R2>([&](auto q2c) {
    constexpr int q2 = decltype(q2c)::value;
    float2 a[R1];
#pragma unroll
    for (int q1 = 0; q1 < R1; ++q1) a[q1] = v[R2 * q1 + q2];
    Dft<R1, SIGN>::run(a);
    static_for<0, R1>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      y[q2 * R1 + k1] = rotate<SIGN, R, q2 * k1>(a[k1]);
    });
  });
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    float2 b[R2];
#pragma unroll
    for (int q2 = 0; q2 < R2; ++q2) b[q2] = y[q2 * R1 + k1];
    Dft<R2, SIGN>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = b[k2];
  }
}

template <int SIGN>
struct Dft<16, SIGN> {
  __device__ __forceinline__ static void run(float2* v) { dft_compose<4, 4, SIGN>(v); }
};
template <int SIGN>
struct Dft<32, SIGN> {
  __device__ __forceinline__ static void run(float2* v) { dft_compose<8, 4, SIGN>(v); }
};

// One Stockham pass; recurses into the next pass at compile time.
// PIN: the input line is a zero-padded image line (image index i at
// position i - N/2 mod n, N = n/2, zeros elsewhere); the first pass then
// reads only the positions that hold image values, known at compile time
// for radix 8 or 4 (r < R/4 or r >= 3R/4), and never touches the padding.
// POUT likewise for a cropped output in the last pass: only the image
// positions are formed and stored.
struct NoHook {
  __device__ void operator()() const {}
};

// Barrier between passes: the whole CTA, or a named barrier over the first
// COUNT threads when only part of the CTA transforms.
struct CtaSync {
  __device__ static void sync() { __syncthreads(); }
};
template <int ID, int COUNT>
struct GroupSync {
  static_assert(COUNT % 32 == 0, "named barriers count whole warps");
  __device__ static void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory"); }
};

// `hook` runs once, on every thread, right after the barrier that follows
// the first pass (all reads of the first pass's input are then complete).
// COLS: lines a tile (the stride of the exchange buffer X[pos][col]).
template <int NFFT, int EV, int SIGN, int PI, int NS, bool PIN, bool POUT, class Sync = CtaSync, class In,
          class Out, class Hook = NoHook, int COLS = kFftCols>
__device__ __forceinline__ void fft_pass(float2* X, const float2* tws, int col, int tl, const In& in,
                                         const Out& out, const Hook& hook = Hook()) {
  constexpr RadixPlan RP = radix_plan(NFFT, EV);
  constexpr int R = RP.r[PI];
  constexpr int E = EV;
  constexpr int TPL = NFFT / EV;
  constexpr int NB = E / R;
  constexpr int STRIDE = NFFT / R;
  constexpr bool FIRST = PI == 0;
  constexpr bool LAST = PI == RP.count - 1;
  constexpr bool PRUNE_IN = FIRST && PIN && R % 4 == 0;
  constexpr bool PRUNE_OUT = LAST && POUT && R % 4 == 0;
  constexpr int Q = NFFT / 4;  // N / 2
  static_assert(E % R == 0, "radix must divide the per-thread count");
  static_assert(!(FIRST && PIN) || PRUNE_IN, "padded input needs a first radix of 32, 16, 8 or 4");
  float2 v[E];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = tl + TPL * q;
    const int k = j % NS;
    float2 w[R];
    if constexpr (NS > 1) {
      const float2* T = tws + tw_offset<NFFT, EV>(PI) + k * R;
      if constexpr (R % 2 == 0) {
#pragma unroll
        for (int h = 0; h < R / 2; ++h) {
          const float4 t = reinterpret_cast<const float4*>(T)[h];
          w[2 * h] = make_float2(t.x, t.y);
          w[2 * h + 1] = make_float2(t.z, t.w);
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) w[r] = T[r];
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int pos = j + r * STRIDE;
      float2 x;
      if constexpr (PRUNE_IN) {
        if (r < R / 4)
          x = in.at(pos + Q, col);
        else if (r >= R - R / 4)
          x = in.at(pos - 3 * Q, col);
        else
          x = make_float2(0.f, 0.f);
      } else if constexpr (FIRST) {
        x = in(pos, col);
      } else {
        x = X[pos * COLS + col];
      }
      if constexpr (NS > 1) {
        if (r > 0) x = SIGN < 0 ? cmul(x, w[r]) : cmulc(x, w[r]);
      }
      v[q * R + r] = x;
    }
    Dft<R, SIGN>::run(v + q * R);
  }
  if constexpr (!LAST) {
    if constexpr (!FIRST) Sync::sync();  // every read of this pass is done
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = tl + TPL * q;
      const int d = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) X[(d + r * NS) * COLS + col] = v[q * R + r];
    }
    Sync::sync();
    if constexpr (FIRST) hook();
    fft_pass<NFFT, EV, SIGN, PI + 1, NS * R, PIN, POUT, Sync, In, Out, Hook, COLS>(X, tws, col, tl, in, out, hook);
  } else {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = tl + TPL * q;
      const int d = (j / NS) * NS * R + (j % NS);  // = j: NS R = NFFT in the last pass
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if constexpr (PRUNE_OUT) {
          if (r < R / 4)
            out.at(d + r * NS + Q, col, v[q * R + r]);
          else if (r >= R - R / 4)
            out.at(d + r * NS - 3 * Q, col, v[q * R + r]);
        } else {
          out(d + r * NS, col, v[q * R + r]);
        }
      }
    }
  }
}

// Position p of a length-n line holds image index i = x + N/2 for
// x = p (p < N/2) or x = p - n (p >= n - N/2); other positions are padding.
__device__ __forceinline__ int image_index(int p, int N, int n) {
  const int h = N >> 1;
  if (p < h) return p + h;
  if (p >= n - h) return p - (n - h);
  return -1;
}

struct FftArgs {
  const float2* src;
  float2* dst;
  const float* deapod;
  const float2* twiddle;
  int N, n, Nf;
  int C;   // bin stride of the workspace (the plan's chunk)
  int Cv;  // valid bins in this chunk (<= C)
  int f0;
  float scale;
};

enum Kind { kFwdRows = 0, kFwdCols = 1, kAdjCols = 2, kAdjRows = 3 };

// Forward rows: V[t][i2][i1][f0 + f] * c(i1) c(i2), padded -> rows[t][i2][u1][f].
struct InFwdRows {
  const float2* V;
  const float* dp;
  int N, n, Nf, Cv, f0, fbase;
  size_t row;  // (t*N + i2)
  float c2;
  __device__ float2 at(int i1, int col) const {  // i1: image index
    const int f = fbase + col;
    if (f >= Cv) return make_float2(0.f, 0.f);
    return cscale_rn(__ldg(&V[(row * N + i1) * Nf + f0 + f]), dp[i1] * c2);
  }
};
struct OutFwdRows {
  float2* rows;
  int n, C, fbase;
  size_t row;
  __device__ void operator()(int pos, int col, float2 val) const {
    const int f = fbase + col;
    if (f < C) rows[(row * n + pos) * C + f] = val;
  }
};
// Forward columns: rows[t][i2][q], padded along i2 -> grid[t][u2][q], q = u1*C + f.
struct InFwdCols {
  const float2* rows;
  int N, n;
  size_t nq, q, t;
  __device__ float2 at(int i2, int col) const { return __ldg(&rows[(t * N + i2) * nq + q + col]); }
};
struct OutFwdCols {
  float2* grid;
  int n;
  size_t nq, q, t;
  __device__ void operator()(int pos, int col, float2 val) const {
    grid[(t * n + pos) * nq + q + col] = val;
  }
};
// Adjoint columns: grid[t][u2][q] -> inverse FFT along u2, crop -> rows[t][i2][q].
struct InAdjCols {
  const float2* grid;
  int n;
  size_t nq, q, t;
  __device__ float2 operator()(int pos, int col) const {
    return __ldg(&grid[(t * n + pos) * nq + q + col]);
  }
};
struct OutAdjCols {
  float2* rows;
  int N, n;
  size_t nq, q, t;
  __device__ void operator()(int pos, int col, float2 val) const {
    const int i2 = image_index(pos, N, n);
    if (i2 >= 0) rows[(t * N + i2) * nq + q + col] = val;
  }
  __device__ void at(int i2, int col, float2 val) const { rows[(t * N + i2) * nq + q + col] = val; }
};
// Adjoint rows: rows[t][i2][u1][f] -> inverse FFT along u1, crop,
// * scale c(i1) c(i2) -> out[t][i2][i1][f0 + f].
struct InAdjRows {
  const float2* rows;
  int n, C, Cv, fbase;
  size_t row;
  __device__ float2 operator()(int pos, int col) const {
    const int f = fbase + col;
    if (f >= Cv) return make_float2(0.f, 0.f);
    return __ldg(&rows[(row * n + pos) * C + f]);
  }
};
struct OutAdjRows {
  float2* out;
  const float* dp;
  int N, n, Nf, Cv, f0, fbase;
  size_t row;
  float c2;
  __device__ void operator()(int pos, int col, float2 val) const {
    const int f = fbase + col;
    const int i1 = image_index(pos, N, n);
    if (f < Cv && i1 >= 0) out[(row * N + i1) * Nf + f0 + f] = cscale(val, dp[i1] * c2);
  }
  __device__ void at(int i1, int col, float2 val) const {
    const int f = fbase + col;
    if (f < Cv) out[(row * N + i1) * Nf + f0 + f] = cscale(val, dp[i1] * c2);
  }
};

template <int NFFT, int KIND>
__global__ void __launch_bounds__(Shape<NFFT, kValsPlain<NFFT>>::THREADS) fft_kernel(FftArgs a) {
  constexpr int EV = kValsPlain<NFFT>;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* tw = smem + NFFT * kFftCols;
  build_twiddles<NFFT, EV>(tw, a.twiddle);
  __syncthreads();
  const int col = threadIdx.x % kFftCols;
  const int tl = threadIdx.x / kFftCols;
  if constexpr (KIND == kFwdRows) {
    const size_t row = blockIdx.y;  // t*N + i2
    const int i2 = (int)(row % a.N);
    const int fbase = blockIdx.x * kFftCols;
    InFwdRows in{a.src, a.deapod, a.N, a.n, a.Nf, a.Cv, a.f0, fbase, row, a.deapod[i2]};
    OutFwdRows out{a.dst, a.n, a.C, fbase, row};
    fft_pass<NFFT, EV, -1, 0, 1, true, false>(X, tw, col, tl, in, out);
  } else if constexpr (KIND == kFwdCols) {
    const size_t nq = (size_t)a.n * a.C;
    InFwdCols in{a.src, a.N, a.n, nq, (size_t)blockIdx.x * kFftCols, blockIdx.y};
    OutFwdCols out{a.dst, a.n, nq, (size_t)blockIdx.x * kFftCols, blockIdx.y};
    fft_pass<NFFT, EV, -1, 0, 1, true, false>(X, tw, col, tl, in, out);
  } else if constexpr (KIND == kAdjCols) {
    const size_t nq = (size_t)a.n * a.C;
    InAdjCols in{a.src, a.n, nq, (size_t)blockIdx.x * kFftCols, blockIdx.y};
    OutAdjCols out{a.dst, a.N, a.n, nq, (size_t)blockIdx.x * kFftCols, blockIdx.y};
    fft_pass<NFFT, EV, +1, 0, 1, false, true>(X, tw, col, tl, in, out);
  } else {
    const size_t row = blockIdx.y;
    const int i2 = (int)(row % a.N);
    const int fbase = blockIdx.x * kFftCols;
    InAdjRows in{a.src, a.n, a.C, a.Cv, fbase, row};
    OutAdjRows out{a.dst, a.deapod, a.N, a.n, a.Nf, a.Cv, a.f0, fbase, row, a.deapod[i2] * a.scale};
    fft_pass<NFFT, EV, +1, 0, 1, false, true>(X, tw, col, tl, in, out);
  }
}

// --- Fused row kernel: inverse row FFT -> TV + Adam -> next forward row FFT --
//
// With the whole bin range in one grid pass, the last adjoint pass (inverse
// FFT along u1, crop, deapodise, scale), the optimiser update and the first
// forward pass of the next iteration (deapodise, pad, FFT along x1) all work
// on the same (t, i2) image row and 16 bins.  One CTA does the three in
// turn: the gradient never goes to global memory, and the row workspace is
// rewritten in place (each CTA reads its slice completely before writing it).
// The arithmetic is that of the separate kernels, so the iterates are the
// same bit for bit.
struct FusedArgs {
  float2* rows;        // [T][N][n][C] in: adjoint row intermediate, out: next forward row intermediate
  const float* deapod;
  const float2* twiddle;
  const float2* Vin;
  float2* Vout;
  float2* m;
  float2* v;
  double* partials;
  unsigned int* counter;
  const double* data_loss;
  double* loss_out;
  int N, n, Nf, C, T;
  float scale;         // adjoint scale (1/N)
  AdamArgs ad;
  // warp-specialised kernel only
  int* err;            // device status word (bounded wait expired)
  int units;           // (t, i2, 16-bin) row units, unit = (t N + i2) nfb + bin group
  int nfb;             // 16-bin groups per image row
  int bh, nbox;        // tensor-copy box height and boxes per unit
};

// Kernel parameter of the fused row kernel over a batch of problems.
struct MultiFused {
  FusedArgs a[kMaxBatch];
  int fwd_tail[kMaxBatch];
  int nreq;
  int unit_begin[kMaxBatch + 1];   // unit (block) ranges of the problems
};

// Adjoint output into the CTA's gradient buffer gb[i1][col].
struct OutGrad {
  float2* gb;
  const float* dp;
  int N, n;
  float c2;
  __device__ void operator()(int pos, int col, float2 val) const {
    const int i1 = image_index(pos, N, n);
    if (i1 >= 0) gb[i1 * kFftCols + col] = cscale(val, dp[i1] * c2);
  }
  __device__ void at(int i1, int col, float2 val) const { gb[i1 * kFftCols + col] = cscale(val, dp[i1] * c2); }
};
// Forward input from the CTA's new-volume buffer vb[i1][col].
struct InNewRow {
  const float2* vb;
  const float* dp;
  int N, n;
  float c2;
  __device__ float2 at(int i1, int col) const { return cscale_rn(vb[i1 * kFftCols + col], dp[i1] * c2); }
};

// TV + Adam on the (t, i2) image row, bins fbase .. fbase + 15.  The
// nthreads threads split the row into 16 columns (one bin each) of
// nthreads / 16 runs of consecutive i1; thread tid walks its run, so the
// x1 neighbours are the previous and the next voxel of the walk and only the
// next one is loaded per step.  The adjoint gradient comes from gb[i1][col],
// the new value goes to Vout and back into gb (zero for bins >= Nf, the
// padding of the next forward row transform).  Adds this thread's TV shares
// to `local` in walk order and returns it.  Every load is unconditional
// (missing neighbours and bins >= Nf read a valid voxel whose value is then
// not used), so the loads of several steps are in flight together; TT: the
// volume has time neighbours (T > 1 and tv_t != 0).
template <bool TT>
__device__ __forceinline__ float update_row(const FusedArgs& a, float2* gb, size_t row, int i2, int t, int fbase,
                                            int tid, int nthreads, float local) {
  const float eps2 = a.ad.tv_eps * a.ad.tv_eps;
  // The volumes and moments never alias: loads of later voxels may be issued
  // ahead of the stores of earlier ones.
  const float2* __restrict__ Vin = a.Vin;
  float2* __restrict__ Vout = a.Vout;
  float2* __restrict__ mom1 = a.m;
  float2* __restrict__ mom2 = a.v;
  const int col = tid % kFftCols;
  const int runs = nthreads / kFftCols;
  const int len = (a.N + runs - 1) / runs;
  const int lo = (tid / kFftCols) * len;
  const int hi = min(a.N, lo + len);
  if (lo >= hi) return local;
  const size_t sx = (size_t)a.Nf, sy = (size_t)a.N * a.Nf, st = (size_t)a.N * a.N * a.Nf;
  const bool xy = a.ad.tv_xy != 0.f;
  const bool h2p = xy && i2 + 1 < a.N, h2m = xy && i2 > 0;
  const bool htp = TT && t + 1 < a.T, htm = TT && t > 0;
  const int f = fbase + col;
  const bool fv = f < a.Nf;
  const size_t base = row * a.N * a.Nf + (size_t)(fv ? f : a.Nf - 1);  // voxel (t, i2, 0, f)
  float2 xm = Vin[lo > 0 ? base + (size_t)(lo - 1) * sx : base];
  float2 x = Vin[base + (size_t)lo * sx];
#pragma unroll 4
  for (int i1 = lo; i1 < hi; ++i1) {
    const size_t idx = base + (size_t)i1 * sx;
    const bool more = i1 + 1 < a.N;
    const float2 xp = Vin[more ? idx + sx : idx];
    TvNbrs nb;
    nb.h1p = xy && more;
    nb.h1m = xy && i1 > 0;
    nb.h2p = h2p;
    nb.h2m = h2m;
    nb.htp = htp;
    nb.htm = htm;
    nb.x1p = xp;
    nb.x1m = xm;
    nb.x2p = Vin[h2p ? idx + sy : idx];
    nb.x2m = Vin[h2m ? idx - sy : idx];
    if constexpr (TT) {
      nb.tp = Vin[htp ? idx + st : idx];
      nb.tm = Vin[htm ? idx - st : idx];
    } else {
      nb.tp = nb.tm = x;
    }
    float2 mm = mom1[idx], vv = mom2[idx];
    float2* gp = gb + i1 * kFftCols + col;
    const float2 gd = *gp;
    float2 gxy, gt;
    const float tv = voxel_tv_nb(x, nb, a.ad.tv_xy, TT ? a.ad.tv_t : 0.f, eps2, &gxy, &gt);
    float2 nx = make_float2(0.f, 0.f);
    if (fv) {
      local = __fadd_rn(local, tv);
      const float2 g = total_grad(gd, gxy, gt, a.ad);
      nx = adam_voxel(x, g, mm, vv, a.ad);
      mom1[idx] = mm;
      mom2[idx] = vv;
      Vout[idx] = nx;
    }
    *gp = nx;
    xm = x;
    x = xp;
  }
  return local;
}

__device__ __forceinline__ float update_row_any(const FusedArgs& a, float2* gb, size_t row, int i2, int t,
                                                int fbase, int tid, int nthreads, float local) {
  if (a.T > 1 && a.ad.tv_t != 0.f) return update_row<true>(a, gb, row, i2, t, fbase, tid, nthreads, local);
  return update_row<false>(a, gb, row, i2, t, fbase, tid, nthreads, local);
}

// L2 prefetch of the update's operands for image row `row`: this row of V,
// m and v, and the neighbouring rows the TV terms read.
__device__ __forceinline__ void prefetch_update_rows(const FusedArgs& a, size_t row, int i2, int t) {
  const size_t rl = (size_t)a.N * a.Nf;
  const uint32_t rb = (uint32_t)(rl * sizeof(float2));
  prefetch_l2(a.Vin + row * rl, rb);
  prefetch_l2(a.m + row * rl, rb);
  prefetch_l2(a.v + row * rl, rb);
  if (a.ad.tv_xy != 0.f) {
    if (i2 + 1 < a.N) prefetch_l2(a.Vin + (row + 1) * rl, rb);
    if (i2 > 0) prefetch_l2(a.Vin + (row - 1) * rl, rb);
  }
  if (a.ad.tv_t != 0.f) {
    if (t + 1 < a.T) prefetch_l2(a.Vin + (row + a.N) * rl, rb);
    if (t > 0) prefetch_l2(a.Vin + (row - a.N) * rl, rb);
  }
}

// Register cap: 64 a thread (two CTAs of 512 threads per SM).
template <int NFFT>
constexpr int fused_min_blocks() {
  return 65536 / (Shape<NFFT, kValsFused<NFFT>>::THREADS * 64) > 16
             ? 16
             : 65536 / (Shape<NFFT, kValsFused<NFFT>>::THREADS * 64);
}

// The fused row kernel's work on one (image row, 16-bin group) unit: bin
// group bx of image row `row` (t N + i2); vb, nblk: the unit's index and the
// unit count of the loss reduction.
template <int NFFT, bool FWD_TAIL>
__device__ __forceinline__ void fused_rows_body(const FusedArgs& a, int bx, size_t row, unsigned vb, unsigned nblk) {
  constexpr int EV = kValsFused<NFFT>;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* tw = smem + NFFT * kFftCols;
  float2* gb = tw + Shape<NFFT, EV>::TW;  // [N][kFftCols]
  const int i2 = (int)(row % a.N);
  const int t = (int)(row / a.N);
  build_twiddles<NFFT, EV>(tw, a.twiddle);
  grid_dep_wait();
  grid_dep_release();
  // the update's operands stream into L2 while the inverse FFT runs
  if (threadIdx.x == 0) prefetch_update_rows(a, row, i2, t);
  __syncthreads();
  const int col = threadIdx.x % kFftCols;
  const int tl = threadIdx.x / kFftCols;
  const int fbase = bx * kFftCols;
  {
    InAdjRows in{a.rows, a.n, a.C, a.Nf, fbase, row};
    OutGrad out{gb, a.deapod, a.N, a.n, a.deapod[i2] * a.scale};
    fft_pass<NFFT, EV, +1, 0, 1, false, true>(X, tw, col, tl, in, out);
  }
  __syncthreads();
  const float local = update_row_any(a, gb, row, i2, t, fbase, threadIdx.x, blockDim.x, 0.f);
  if constexpr (FWD_TAIL) {
    __syncthreads();
    InNewRow in{gb, a.deapod, a.N, a.n, a.deapod[i2]};
    OutFwdRows out{a.rows, a.n, a.C, fbase, row};
    fft_pass<NFFT, EV, -1, 0, 1, true, false>(X, tw, col, tl, in, out);
  }
  finish_loss_v(local, a.partials, a.counter, a.data_loss, a.loss_out, vb, nblk);
}

template <int NFFT, bool FWD_TAIL>
__global__ void __launch_bounds__(Shape<NFFT, kValsFused<NFFT>>::THREADS, fused_min_blocks<NFFT>())
    fused_rows_kernel(FusedArgs a) {
  fused_rows_body<NFFT, FWD_TAIL>(a, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x,
                                  gridDim.x * gridDim.y);
}

// One launch of the fused row kernel for several problems of the same
// transform length (a batch of requests): block b serves problem r with
// unit_begin[r] <= b < unit_begin[r + 1], unit u = b - unit_begin[r] =
// (image row) nfb + bin group, the same unit and loss-partial order as the
// problem's own launch, so every result is the same bit for bit.
template <int NFFT>
__global__ void __launch_bounds__(Shape<NFFT, kValsFused<NFFT>>::THREADS, fused_min_blocks<NFFT>())
    fused_rows_multi_kernel(const __grid_constant__ MultiFused m) {
  int r = 0;
  while (r + 1 < m.nreq && (int)blockIdx.x >= m.unit_begin[r + 1]) ++r;
  const unsigned u = blockIdx.x - (unsigned)m.unit_begin[r];
  const unsigned nu = (unsigned)(m.unit_begin[r + 1] - m.unit_begin[r]);
  const FusedArgs& a = m.a[r];
  const int bx = (int)(u % (unsigned)a.nfb);
  const size_t row = u / (unsigned)a.nfb;
  if (m.fwd_tail[r])
    fused_rows_body<NFFT, true>(a, bx, row, u, nu);
  else
    fused_rows_body<NFFT, false>(a, bx, row, u, nu);
}

template <int NFFT>
size_t fused_smem(int N) {
  return Shape<NFFT, kValsFused<NFFT>>::SMEM + (size_t)N * kFftCols * sizeof(float2);
}

template <int NFFT>
cudaError_t launch_fused_multi(const MultiFused& m, cudaStream_t s) {
  const size_t smem = fused_smem<NFFT>(m.a[0].N);
  for (int r = 1; r < m.nreq; ++r)
    if (m.a[r].N != m.a[0].N) return cudaErrorInvalidValue;
  return launch_dep(fused_rows_multi_kernel<NFFT>, dim3((unsigned)m.unit_begin[m.nreq]),
                    dim3(Shape<NFFT, kValsFused<NFFT>>::THREADS), smem, s, m);
}

template <int NFFT>
cudaError_t launch_fused(const FusedArgs& a, bool fwd_tail, dim3 grid, cudaStream_t s) {
  const size_t smem = fused_smem<NFFT>(a.N);
  const dim3 block(Shape<NFFT, kValsFused<NFFT>>::THREADS);
  if (fwd_tail) return launch_dep(fused_rows_kernel<NFFT, true>, grid, block, smem, s, a);
  return launch_dep(fused_rows_kernel<NFFT, false>, grid, block, smem, s, a);
}

// --- Warp-specialised fused row kernel ---------------------------------------
//
// Persistent CTAs (one per SM) walk the row units u = blockIdx.x + i
// gridDim.x.  The first FT threads (the transform group, one FFT tile's
// worth) run, for i = 0, 1, ...: the inverse row FFT of unit i into
// gradient buffer i % 2, then the forward row FFT of unit i - 1 from buffer
// (i - 1) % 2; the other kUpdThreads threads (the update group) meanwhile
// apply TV + Adam to unit i - 1 .. i in place in its buffer.  The update's
// HBM stream of V, m and v thus overlaps the transforms' shared-memory work
// instead of following it.  The adjoint input of unit i + 1 is staged by a
// tensor copy as soon as the first pass of unit i has read the stage.
// Hand-offs: ready[b] (every transform thread arrives once the inverse FFT
// has written buffer b) and done[b] (every update thread arrives once it
// has rewritten buffer b); each group synchronises internally on its own
// named barrier.  A group gives up on an expired bounded wait (the status
// word is set); the other group's next wait then expires too.  The
// arithmetic is that of fused_rows_kernel, so the iterates agree bit for
// bit; the TV partial sums are per CTA.
constexpr int kUpdThreads = 512;

// Input staged in shared memory as [rows][kFftCols].
struct InTile {
  const float2* t;  // [rows][kFftCols]
  __device__ float2 at(int i, int col) const { return t[i * kFftCols + col]; }
  __device__ float2 operator()(int pos, int col) const { return t[pos * kFftCols + col]; }
};

template <int NFFT>
constexpr bool fused_ws_fits() {
  return Shape<NFFT, kValsFused<NFFT>>::THREADS % 32 == 0 && Shape<NFFT, kValsFused<NFFT>>::THREADS <= 512;
}

template <int NFFT>
constexpr size_t fused_ws_smem() {
  // stage + transform workspace [NFFT][16], two gradient buffers [N][16], twiddles, 5 mbarriers
  return (size_t)2 * NFFT * kFftCols * sizeof(float2) + (size_t)2 * (NFFT / 2) * kFftCols * sizeof(float2) +
         (size_t)Shape<NFFT, kValsFused<NFFT>>::TW * sizeof(float2) + 5 * sizeof(uint64_t);
}

template <int NFFT, bool FWD_TAIL>
__global__ void __launch_bounds__(Shape<NFFT, kValsFused<NFFT>>::THREADS + kUpdThreads, 1)
    fused_rows_ws_kernel(const __grid_constant__ CUtensorMap tin, FusedArgs a) {
  constexpr int EV = kValsFused<NFFT>;
  constexpr int FT = Shape<NFFT, EV>::THREADS;
  using FSync = GroupSync<1, FT>;
  using USync = GroupSync<2, kUpdThreads>;
  extern __shared__ __align__(128) float2 smem[];
  float2* S = smem;                          // [NFFT][16] staged adjoint input
  float2* X = S + NFFT * kFftCols;           // [NFFT][16] transform workspace
  float2* gbuf = X + NFFT * kFftCols;        // [2][N][16]
  float2* tw = gbuf + 2 * (NFFT / 2) * kFftCols;
  uint64_t* full = reinterpret_cast<uint64_t*>(tw + Shape<NFFT, EV>::TW);
  uint64_t* ready = full + 1;                // [2]
  uint64_t* done = full + 3;                 // [2]
  __shared__ volatile int s_abort_f, s_abort_u;
  const int nu = (int)blockIdx.x < a.units ? (a.units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int gsz = a.N * kFftCols;
  const uint32_t tile_bytes = (uint32_t)(NFFT * kFftCols * sizeof(float2));
  auto issue = [&](int i) {
    const int u = (int)blockIdx.x + i * (int)gridDim.x;
    const int row = u / a.nfb, fb = u - (u / a.nfb) * a.nfb;
    mbar_expect_tx(full, tile_bytes);
    for (int b = 0; b < a.nbox; ++b)
      tma_load_3d(S + (size_t)b * a.bh * kFftCols, &tin, fb * 2 * kFftCols, b * a.bh, row, full);
  };
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ready[b], FT);
      mbar_init(&done[b], kUpdThreads);
    }
    fence_mbar_init();
    s_abort_f = 0;
    s_abort_u = 0;
  }
  build_twiddles<NFFT, EV>(tw, a.twiddle);
  grid_dep_wait();
  grid_dep_release();
  int issued = 0, consumed = 0;  // tensor copies, meaningful on thread 0
  if (threadIdx.x == 0 && nu > 0) {
    issue(0);
    issued = 1;
  }
  __syncthreads();
  float local = 0.f;
  if (threadIdx.x < FT) {
    const int col = threadIdx.x % kFftCols;
    const int tl = threadIdx.x / kFftCols;
    for (int i = 0; i <= nu; ++i) {
      if (i < nu) {
        if (!mbar_wait_bounded(full, (uint32_t)(i & 1)))
          s_abort_f = 1;
        else
          ++consumed;
        FSync::sync();  // the previous forward FFT is done with X; uniform abort flag
        if (s_abort_f) break;
        const int u = (int)blockIdx.x + i * (int)gridDim.x;
        const size_t row = (size_t)(u / a.nfb);
        const int i2 = (int)(row % a.N);
        auto hook = [&]() {
          if (threadIdx.x == 0 && i + 1 < nu) {
            fence_proxy_async_smem();
            issue(i + 1);
            ++issued;
          }
        };
        InTile in{S};
        OutGrad out{gbuf + (size_t)(i & 1) * gsz, a.deapod, a.N, a.n, a.deapod[i2] * a.scale};
        fft_pass<NFFT, EV, +1, 0, 1, false, true, FSync>(X, tw, col, tl, in, out, hook);
        mbar_arrive(&ready[i & 1]);
      }
      if (i >= 1) {
        const int j = i - 1;
        if (!mbar_wait_bounded(&done[j & 1], (uint32_t)((j >> 1) & 1))) s_abort_f = 1;
        FSync::sync();  // the inverse FFT's last pass is done with X; uniform abort flag
        if (s_abort_f) break;
        if constexpr (FWD_TAIL) {
          const int u = (int)blockIdx.x + j * (int)gridDim.x;
          const size_t row = (size_t)(u / a.nfb);
          const int fbase = (u - (u / a.nfb) * a.nfb) * kFftCols;
          const int i2 = (int)(row % a.N);
          InNewRow in{gbuf + (size_t)(j & 1) * gsz, a.deapod, a.N, a.n, a.deapod[i2]};
          OutFwdRows out{a.rows, a.n, a.C, fbase, row};
          fft_pass<NFFT, EV, -1, 0, 1, true, false, FSync>(X, tw, col, tl, in, out);
        }
      }
    }
  } else {
    const int ut = threadIdx.x - FT;
    if (ut == 0 && nu > 0) {
      const size_t row = (size_t)(blockIdx.x / a.nfb);
      prefetch_update_rows(a, row, (int)(row % a.N), (int)(row / a.N));
    }
    for (int i = 0; i < nu; ++i) {
      const int u = (int)blockIdx.x + i * (int)gridDim.x;
      const size_t row = (size_t)(u / a.nfb);
      const int fbase = (u - (u / a.nfb) * a.nfb) * kFftCols;
      const int i2 = (int)(row % a.N), t = (int)(row / a.N);
      if (ut == 0 && i + 1 < nu) {
        const size_t nrow = (size_t)((u + (int)gridDim.x) / a.nfb);
        if (nrow != row) prefetch_update_rows(a, nrow, (int)(nrow % a.N), (int)(nrow / a.N));
      }
      if (!mbar_wait_bounded(&ready[i & 1], (uint32_t)((i >> 1) & 1))) s_abort_u = 1;
      USync::sync();
      if (s_abort_u) break;
      local = update_row_any(a, gbuf + (size_t)(i & 1) * gsz, row, i2, t, fbase, ut, kUpdThreads, local);
      mbar_arrive(&done[i & 1]);
    }
  }
  __syncthreads();
  if ((s_abort_f || s_abort_u) && threadIdx.x == 0) {
    atomicExch(a.err, 1);
    // let copies issued and never awaited land (bounded)
    for (int k = consumed; k < issued; ++k) mbar_wait_bounded(full, (uint32_t)(k & 1));
  }
  finish_loss(local, a.partials, a.counter, a.data_loss, a.loss_out);
}

template <int NFFT>
cudaError_t launch_fused_ws(const CUtensorMap& tm, const FusedArgs& a, bool fwd_tail, int ctas, cudaStream_t s) {
  if constexpr (fused_ws_fits<NFFT>()) {
    const dim3 grid((unsigned)ctas), block(Shape<NFFT, kValsFused<NFFT>>::THREADS + kUpdThreads);
    if (fwd_tail) return launch_dep(fused_rows_ws_kernel<NFFT, true>, grid, block, fused_ws_smem<NFFT>(), s, tm, a);
    return launch_dep(fused_rows_ws_kernel<NFFT, false>, grid, block, fused_ws_smem<NFFT>(), s, tm, a);
  } else {
    return cudaErrorInvalidValue;
  }
}

// --- Column passes staged by TMA ------------------------------------------
//
// Persistent CTAs walk the column tiles (16 adjacent (u1, bin) lines of one
// frame); the next tile for a buffer is loaded by a tensor copy as soon as
// the first pass of the tile in it has read it, so the input of the next
// tiles streams in while this one is transformed.
// Forward: the staged input is the N image rows of the row intermediate
// (padding is never stored); adjoint: the 2N grid rows.
struct ColArgs {
  float2* dst;
  const float2* twiddle;
  int* err;
  size_t nq;
  int N, n, qtiles, ntiles, bh, nbox;
};

// Kernel parameter of a column pass over a batch of problems.
struct MultiCols {
  CUtensorMap tm[kMaxBatch];       // each problem's input tensor map
  ColArgs a[kMaxBatch];
  int nreq;
  int cta_begin[kMaxBatch + 1];    // CTA ranges of the problems
};

template <int NFFT, int KIND>
constexpr int col_rows() {
  return KIND == kFwdCols ? NFFT / 2 : NFFT;
}
// Tile buffers and CTAs per SM: the forward pass stages the N image rows in
// one buffer (the next tile is requested once the first pass has read the
// current one) with two CTAs per SM; the adjoint stages all 2N rows in one
// buffer with two CTAs per SM where two such CTAs fit an SM's shared memory
// (2N <= kAdjColsTwoCtaMax), else double-buffered with one CTA per SM.
constexpr int kAdjColsTwoCtaMax = 384;
template <int NFFT, int KIND>
constexpr int col_bufs() {
  return KIND == kFwdCols || NFFT <= kAdjColsTwoCtaMax ? 1 : 2;
}
template <int NFFT, int KIND>
constexpr int col_ctas_per_sm() {
  return KIND == kFwdCols || NFFT <= kAdjColsTwoCtaMax ? 2 : 1;
}
template <int NFFT, int KIND>
constexpr size_t col_smem() {
  return (size_t)col_bufs<NFFT, KIND>() * col_rows<NFFT, KIND>() * kFftCols * sizeof(float2) +
         Shape<NFFT, kValsCols<NFFT>>::SMEM + 2 * sizeof(uint64_t);
}

// The column pass of one problem run by vg persistent CTAs, this being the
// vb-th: tile vb, vb + vg, ... ; tin is the problem's input tensor map (in
// the kernel's parameter space).
template <int NFFT, int KIND>
__device__ __forceinline__ void cols_body(const CUtensorMap* tin, const ColArgs& a, int vb, int vg) {
  constexpr int EV = kValsCols<NFFT>;
  constexpr int H = col_rows<NFFT, KIND>();
  constexpr int NB = col_bufs<NFFT, KIND>();
  extern __shared__ __align__(128) float2 smem[];
  float2* tiles = smem;                      // [NB][H][kFftCols]
  float2* X = tiles + NB * H * kFftCols;     // [NFFT][kFftCols]
  float2* tw = X + NFFT * kFftCols;
  uint64_t* full = reinterpret_cast<uint64_t*>(tw + Shape<NFFT, EV>::TW);
  __shared__ volatile int s_abort;
  const uint32_t tile_bytes = (uint32_t)(H * kFftCols * sizeof(float2));
  auto issue = [&](int tile, int b) {
    const int t = tile / a.qtiles, qt = tile - (tile / a.qtiles) * a.qtiles;
    mbar_expect_tx(&full[b], tile_bytes);
    for (int i = 0; i < a.nbox; ++i)
      tma_load_3d(tiles + ((size_t)b * H + (size_t)i * a.bh) * kFftCols, tin, qt * 2 * kFftCols, i * a.bh, t,
                  &full[b]);
  };
  if (threadIdx.x == 0) {
    for (int b = 0; b < NB; ++b) mbar_init(&full[b], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  build_twiddles<NFFT, EV>(tw, a.twiddle);
  grid_dep_wait();
  grid_dep_release();
  if (threadIdx.x == 0)
    for (int b = 0; b < NB; ++b)
      if (vb + b * vg < a.ntiles) issue(vb + b * vg, b);
  __syncthreads();
  const int col = threadIdx.x % kFftCols;
  const int tl = threadIdx.x / kFftCols;
  int k = 0;
  for (int tile = vb; tile < a.ntiles; tile += vg, ++k) {
    const int b = k % NB;
    if (!mbar_wait_bounded(&full[b], (uint32_t)((k / NB) & 1))) s_abort = 1;
    __syncthreads();  // the previous tile's last pass is done with X; all threads see s_abort
    if (s_abort) break;
    const size_t t = (size_t)(tile / a.qtiles);
    const size_t q = (size_t)(tile - (tile / a.qtiles) * a.qtiles) * kFftCols;
    const int next = tile + NB * vg;
    auto hook = [&]() {
      if (threadIdx.x == 0 && next < a.ntiles) {
        fence_proxy_async_smem();
        issue(next, b);
      }
    };
    InTile in{tiles + (size_t)b * H * kFftCols};
    if constexpr (KIND == kFwdCols) {
      OutFwdCols out{a.dst, a.n, a.nq, q, t};
      fft_pass<NFFT, EV, -1, 0, 1, true, false>(X, tw, col, tl, in, out, hook);
    } else {
      OutAdjCols out{a.dst, a.N, a.n, a.nq, q, t};
      fft_pass<NFFT, EV, +1, 0, 1, false, true>(X, tw, col, tl, in, out, hook);
    }
  }
  if (s_abort && threadIdx.x == 0) {
    atomicExch(a.err, 1);
    // let copies this CTA issued and nobody consumed land (bounded)
    for (int kk = k; kk < k + NB; ++kk)
      if (vb + kk * vg < a.ntiles) mbar_wait_bounded(&full[kk % NB], (uint32_t)((kk / NB) & 1));
  }
}

template <int NFFT, int KIND>
__global__ void __launch_bounds__(Shape<NFFT, kValsCols<NFFT>>::THREADS, col_ctas_per_sm<NFFT, KIND>())
    fft_cols_tma_kernel(const __grid_constant__ CUtensorMap tin, ColArgs a) {
  cols_body<NFFT, KIND>(&tin, a, blockIdx.x, gridDim.x);
}

// One launch of a column pass for several problems of the same transform
// length: CTA b serves problem r with cta_begin[r] <= b < cta_begin[r + 1],
// as CTA b - cta_begin[r] of cta_begin[r + 1] - cta_begin[r].  Every tile is
// transformed exactly as by the problem's own launch.
template <int NFFT, int KIND>
__global__ void __launch_bounds__(Shape<NFFT, kValsCols<NFFT>>::THREADS, col_ctas_per_sm<NFFT, KIND>())
    fft_cols_multi_kernel(const __grid_constant__ MultiCols m) {
  int r = 0;
  while (r + 1 < m.nreq && (int)blockIdx.x >= m.cta_begin[r + 1]) ++r;
  cols_body<NFFT, KIND>(&m.tm[r], m.a[r], (int)blockIdx.x - m.cta_begin[r], m.cta_begin[r + 1] - m.cta_begin[r]);
}

template <int NFFT>
cudaError_t launch(int kind, const FftArgs& a, dim3 grid, cudaStream_t s) {
  const size_t smem = Shape<NFFT, kValsPlain<NFFT>>::SMEM;
  const int threads = Shape<NFFT, kValsPlain<NFFT>>::THREADS;
  switch (kind) {
    case kFwdRows: fft_kernel<NFFT, kFwdRows><<<grid, threads, smem, s>>>(a); break;
    case kFwdCols: fft_kernel<NFFT, kFwdCols><<<grid, threads, smem, s>>>(a); break;
    case kAdjCols: fft_kernel<NFFT, kAdjCols><<<grid, threads, smem, s>>>(a); break;
    default: fft_kernel<NFFT, kAdjRows><<<grid, threads, smem, s>>>(a); break;
  }
  return cudaGetLastError();
}

template <int NFFT>
cudaError_t configure_n() {
  const int smem = (int)Shape<NFFT, kValsPlain<NFFT>>::SMEM;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(fft_kernel<NFFT, kFwdRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(fft_kernel<NFFT, kFwdCols>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(fft_kernel<NFFT, kAdjCols>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(fft_kernel<NFFT, kAdjRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  int optin = 0, dev = 0;
  if ((e = cudaGetDevice(&dev))) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
  if (col_smem<NFFT, kFwdCols>() <= (size_t)optin - 1024) {
    if ((e = cudaFuncSetAttribute(fft_cols_tma_kernel<NFFT, kFwdCols>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)col_smem<NFFT, kFwdCols>())))
      return e;
    if ((e = cudaFuncSetAttribute(fft_cols_multi_kernel<NFFT, kFwdCols>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)col_smem<NFFT, kFwdCols>())))
      return e;
  }
  if (col_smem<NFFT, kAdjCols>() <= (size_t)optin - 1024) {
    if ((e = cudaFuncSetAttribute(fft_cols_tma_kernel<NFFT, kAdjCols>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)col_smem<NFFT, kAdjCols>())))
      return e;
    if ((e = cudaFuncSetAttribute(fft_cols_multi_kernel<NFFT, kAdjCols>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)col_smem<NFFT, kAdjCols>())))
      return e;
  }
  const int fsm = (int)fused_smem<NFFT>(NFFT / 2);
  if ((e = cudaFuncSetAttribute(fused_rows_multi_kernel<NFFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm)))
    return e;
  if ((e = cudaFuncSetAttribute(fused_rows_kernel<NFFT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm)))
    return e;
  if ((e = cudaFuncSetAttribute(fused_rows_kernel<NFFT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm)))
    return e;
  if constexpr (fused_ws_fits<NFFT>()) {
    if (fused_ws_smem<NFFT>() <= (size_t)optin - 1024) {
      const int wsm = (int)fused_ws_smem<NFFT>();
      if ((e = cudaFuncSetAttribute(fused_rows_ws_kernel<NFFT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    wsm)))
        return e;
      if ((e = cudaFuncSetAttribute(fused_rows_ws_kernel<NFFT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    wsm)))
        return e;
    }
  }
  return cudaSuccess;
}

#define PROP_FFT_SIZES(X) X(16) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

cudaError_t dispatch(int n, int kind, const FftArgs& a, dim3 grid, cudaStream_t s) {
  switch (n) {
#define CASE(v) \
  case v: return launch<v>(kind, a, grid, s);
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

template <int NFFT>
cudaError_t launch_cols_tma(int kind, const CUtensorMap& tm, const ColArgs& a, int sms, cudaStream_t s) {
  const int per_sm = kind == kFwdCols ? col_ctas_per_sm<NFFT, kFwdCols>() : col_ctas_per_sm<NFFT, kAdjCols>();
  const dim3 grid((unsigned)std::max(1, std::min(a.ntiles, per_sm * sms)));
  const dim3 block(Shape<NFFT, kValsCols<NFFT>>::THREADS);
  if (kind == kFwdCols)
    return launch_dep(fft_cols_tma_kernel<NFFT, kFwdCols>, grid, block, col_smem<NFFT, kFwdCols>(), s, tm, a);
  return launch_dep(fft_cols_tma_kernel<NFFT, kAdjCols>, grid, block, col_smem<NFFT, kAdjCols>(), s, tm, a);
}

size_t cols_smem(int n, int kind) {
  switch (n) {
#define CASE(v) \
  case v: return kind == kFwdCols ? col_smem<v, kFwdCols>() : col_smem<v, kAdjCols>();
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return (size_t)1 << 30;
  }
}

int cols_per_sm(int n, int kind) {
  switch (n) {
#define CASE(v) \
  case v: return kind == kFwdCols ? col_ctas_per_sm<v, kFwdCols>() : col_ctas_per_sm<v, kAdjCols>();
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return 1;
  }
}

cudaError_t dispatch_cols_tma(int n, int kind, const CUtensorMap& tm, const ColArgs& a, int sms, cudaStream_t s) {
  switch (n) {
#define CASE(v) \
  case v: return launch_cols_tma<v>(kind, tm, a, sms, s);
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

template <int NFFT>
cudaError_t launch_cols_multi(int kind, const MultiCols& m, int ctas, cudaStream_t s) {
  const dim3 grid((unsigned)ctas), block(Shape<NFFT, kValsCols<NFFT>>::THREADS);
  if (kind == kFwdCols)
    return launch_dep(fft_cols_multi_kernel<NFFT, kFwdCols>, grid, block, col_smem<NFFT, kFwdCols>(), s, m);
  return launch_dep(fft_cols_multi_kernel<NFFT, kAdjCols>, grid, block, col_smem<NFFT, kAdjCols>(), s, m);
}

cudaError_t dispatch_cols_multi(int n, int kind, const MultiCols& m, int ctas, cudaStream_t s) {
  switch (n) {
#define CASE(v) \
  case v: return launch_cols_multi<v>(kind, m, ctas, s);
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t dispatch_fused_multi(int n, const MultiFused& m, cudaStream_t s) {
  switch (n) {
#define CASE(v) \
  case v: return launch_fused_multi<v>(m, s);
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

// Largest power of two <= 256 dividing h (the tensor copy's box height).
int box_rows(int h) {
  int b = 256;
  while (b > 1 && h % b != 0) b >>= 1;
  return b;
}

ColArgs col_args(const Plan& p, int kind) {
  ColArgs a{};
  a.dst = kind == kFwdCols ? p.grid : p.rows;
  a.twiddle = p.twiddle;
  a.err = p.status_dev;
  a.nq = (size_t)p.n * p.cs;
  a.N = p.N;
  a.n = p.n;
  a.qtiles = (int)(a.nq / kFftCols);
  a.ntiles = a.qtiles * p.T;
  a.bh = box_rows(kind == kFwdCols ? p.N : p.n);
  a.nbox = (kind == kFwdCols ? p.N : p.n) / a.bh;
  return a;
}

cudaError_t dispatch_fused(int n, const FusedArgs& a, bool fwd_tail, dim3 grid, cudaStream_t s) {
  switch (n) {
#define CASE(v) \
  case v: return launch_fused<v>(a, fwd_tail, grid, s);
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

// --- Centred unitary 2-D DFT of one N x N image (projection model) ----------
//
// Four passes of NFFT = N point transforms, kCartCols lines per CTA: forward rows,
// forward columns (scale 1/N; optionally masked, or fused with the blade's
// data term), inverse columns (input optionally masked), inverse rows (scale
// 1/N).  The centring (image index i = x + N/2, k index u = N k + N/2) is
// the index map position -> (position + N/2) mod N on every input and
// output, which is where an unshifted DFT's position 0 holds x = 0 / k = 0.
struct CartArgs {
  const float2* src;
  float2* dst;
  const float2* twiddle;  // [N] exp(-2 pi i m / N)
  const uint8_t* mask;    // [N][N] blade support, or null
  const float2* y;        // data term: [N][N] k-space data of the blade
  const float2* yimg;     // data term: [N][N] DFT of the blade's image, or null (= y)
  float wk, wi;
  double* partials;
  unsigned int* counter;
  const double* loss_const;
  double* loss_out;
  int N;
  float scale;
};

__device__ __forceinline__ int cshift(int p, int N) {
  const int q = p + (N >> 1);
  return q >= N ? q - N : q;
}
// Lines are the rows r0 + col (elements contiguous).
struct InCartRows {
  const float2* src;
  int N;
  size_t r0;
  __device__ float2 operator()(int pos, int col) const { return src[(r0 + col) * N + cshift(pos, N)]; }
};
struct OutCartRows {
  float2* dst;
  int N;
  size_t r0;
  float scale;
  __device__ void operator()(int q, int col, float2 v) const { dst[(r0 + col) * N + cshift(q, N)] = cscale(v, scale); }
};
// Lines are the columns c0 + col (elements N apart).
struct InCartCols {
  const float2* src;
  const uint8_t* mask;
  int N, c0;
  __device__ float2 operator()(int pos, int col) const {
    const size_t i = (size_t)cshift(pos, N) * N + c0 + col;
    if (mask && !mask[i]) return make_float2(0.f, 0.f);
    return src[i];
  }
};
struct OutCartCols {
  float2* dst;
  const uint8_t* mask;
  int N, c0;
  float scale;
  __device__ void operator()(int q, int col, float2 v) const {
    const size_t i = (size_t)cshift(q, N) * N + c0 + col;
    float2 z = cscale(v, scale);
    if (mask && !mask[i]) z = make_float2(0.f, 0.f);
    dst[i] = z;
  }
};
// Forward column output fused with the blade's data term: on the mask,
// r_k = Z - y, r_i = Z - yimg (the image term through the unitary DFT),
// loss += wk |r_k|^2 + wi |r_i|^2 and dst = 2 (wk r_k + wi r_i); 0 elsewhere.
struct OutCartLoss {
  float2* dst;
  const uint8_t* mask;
  const float2* y;
  const float2* yimg;
  float wk, wi;
  int N, c0;
  float scale;
  float* acc;
  __device__ void operator()(int q, int col, float2 v) const {
    const size_t i = (size_t)cshift(q, N) * N + c0 + col;
    float2 g = make_float2(0.f, 0.f);
    if (mask[i]) {
      const float2 z = cscale(v, scale);
      const float2 yy = y[i];
      const float2 yi = yimg ? yimg[i] : yy;
      const float2 rk = make_float2(z.x - yy.x, z.y - yy.y);
      const float2 ri = make_float2(z.x - yi.x, z.y - yi.y);
      *acc += wk * fmaf(rk.x, rk.x, rk.y * rk.y) + wi * fmaf(ri.x, ri.x, ri.y * ri.y);
      g = make_float2(2.f * fmaf(wk, rk.x, wi * ri.x), 2.f * fmaf(wk, rk.y, wi * ri.y));
    }
    dst[i] = g;
  }
};

template <int NFFT>
constexpr int cart_threads() {
  return NFFT / kValsPlain<NFFT> * kCartCols;
}
template <int NFFT>
constexpr size_t cart_smem() {
  return (size_t)NFFT * kCartCols * sizeof(float2) + (size_t)Shape<NFFT, kValsPlain<NFFT>>::TW * sizeof(float2);
}

template <int NFFT, int PASS>
__global__ void __launch_bounds__(cart_threads<NFFT>()) cart_fft_kernel(CartArgs a) {
  constexpr int EV = kValsPlain<NFFT>;
  constexpr int CC = kCartCols;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* tw = smem + NFFT * CC;
  build_twiddles<NFFT, EV>(tw, a.twiddle);
  grid_dep_wait();
  grid_dep_release();
  __syncthreads();
  const int col = threadIdx.x % CC;
  const int tl = threadIdx.x / CC;
  const int l0 = blockIdx.x * CC;
  if constexpr (PASS == kCartRowsFwd) {
    InCartRows in{a.src, NFFT, (size_t)l0};
    OutCartRows out{a.dst, NFFT, (size_t)l0, a.scale};
    fft_pass<NFFT, EV, -1, 0, 1, false, false, CtaSync, InCartRows, OutCartRows, NoHook, CC>(X, tw, col, tl, in, out);
  } else if constexpr (PASS == kCartColsFwd) {
    InCartCols in{a.src, nullptr, NFFT, l0};
    if (a.y) {
      float acc = 0.f;
      OutCartLoss out{a.dst, a.mask, a.y, a.yimg, a.wk, a.wi, NFFT, l0, a.scale, &acc};
      fft_pass<NFFT, EV, -1, 0, 1, false, false, CtaSync, InCartCols, OutCartLoss, NoHook, CC>(X, tw, col, tl, in,
                                                                                             out);
      finish_loss(acc, a.partials, a.counter, a.loss_const, a.loss_out);
    } else {
      OutCartCols out{a.dst, a.mask, NFFT, l0, a.scale};
      fft_pass<NFFT, EV, -1, 0, 1, false, false, CtaSync, InCartCols, OutCartCols, NoHook, CC>(X, tw, col, tl, in,
                                                                                             out);
    }
  } else if constexpr (PASS == kCartColsInv) {
    InCartCols in{a.src, a.mask, NFFT, l0};
    OutCartCols out{a.dst, nullptr, NFFT, l0, a.scale};
    fft_pass<NFFT, EV, +1, 0, 1, false, false, CtaSync, InCartCols, OutCartCols, NoHook, CC>(X, tw, col, tl, in, out);
  } else {
    InCartRows in{a.src, NFFT, (size_t)l0};
    OutCartRows out{a.dst, NFFT, (size_t)l0, a.scale};
    fft_pass<NFFT, EV, +1, 0, 1, false, false, CtaSync, InCartRows, OutCartRows, NoHook, CC>(X, tw, col, tl, in, out);
  }
}

template <int NFFT>
cudaError_t launch_cart(int pass, const CartArgs& a, cudaStream_t s) {
  const dim3 grid(NFFT / kCartCols), block(cart_threads<NFFT>());
  const size_t smem = cart_smem<NFFT>();
  switch (pass) {
    case kCartRowsFwd: return launch_dep(cart_fft_kernel<NFFT, kCartRowsFwd>, grid, block, smem, s, a);
    case kCartColsFwd: return launch_dep(cart_fft_kernel<NFFT, kCartColsFwd>, grid, block, smem, s, a);
    case kCartColsInv: return launch_dep(cart_fft_kernel<NFFT, kCartColsInv>, grid, block, smem, s, a);
    default: return launch_dep(cart_fft_kernel<NFFT, kCartRowsInv>, grid, block, smem, s, a);
  }
}

template <int NFFT>
cudaError_t configure_cart() {
  const int smem = (int)cart_smem<NFFT>();
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(cart_fft_kernel<NFFT, kCartRowsFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    return e;
  if ((e = cudaFuncSetAttribute(cart_fft_kernel<NFFT, kCartColsFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    return e;
  if ((e = cudaFuncSetAttribute(cart_fft_kernel<NFFT, kCartColsInv>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
    return e;
  return cudaFuncSetAttribute(cart_fft_kernel<NFFT, kCartRowsInv>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t dispatch_fused_ws(int n, const CUtensorMap& tm, const FusedArgs& a, bool fwd_tail, int ctas,
                              cudaStream_t s) {
  switch (n) {
#define CASE(v) \
  case v: return launch_fused_ws<v>(tm, a, fwd_tail, ctas, s);
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

bool fused_ws_size_ok(int n, size_t room) {
  switch (n) {
#define CASE(v) \
  case v: return fused_ws_fits<v>() && fused_ws_smem<v>() <= room;
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

FftArgs base_args(const Plan& p) {
  FftArgs a{};
  a.deapod = p.deapod;
  a.twiddle = p.twiddle;
  a.N = p.N;
  a.n = p.n;
  a.Nf = p.Nf;
  a.C = p.cs;
  a.Cv = p.chunk;
  a.f0 = 0;
  a.scale = 1.f;
  return a;
}

}  // namespace

cudaError_t fft_configure(int n) {
  switch (n) {
#define CASE(v) \
  case v: return configure_n<v>();
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fft_forward_rows(const Plan& p, const float2* V, int f0, cudaStream_t s) {
  FftArgs a = base_args(p);
  a.src = V;
  a.dst = p.rows;
  a.f0 = f0;
  a.Cv = std::min(p.chunk, p.Nf - f0);
  dim3 grid((a.C + kFftCols - 1) / kFftCols, p.T * p.N);
  return dispatch(p.n, kFwdRows, a, grid, s);
}

void fft_make_maps(Plan& p) {
  p.cols_tma_fwd = p.cols_tma_adj = false;
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return;
    }
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  if (p.cs % 2 != 0 || p.T > 65536) return;
  const size_t nq = (size_t)p.n * p.cs;
  auto make = [&](CUtensorMap* tm, float2* base, int h) {
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * nq), (cuuint64_t)h, (cuuint64_t)p.T};
    const cuuint64_t strides[2] = {(cuuint64_t)(2 * nq * sizeof(float)), (cuuint64_t)(2 * nq * h * sizeof(float))};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * kFftCols), (cuuint32_t)box_rows(h), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  const size_t room = (size_t)p.smem_optin - 1024;
  p.cols_tma_fwd = cols_smem(p.n, kFwdCols) <= room && make(&p.tm_rows, p.rows, p.N);
  p.cols_tma_adj = cols_smem(p.n, kAdjCols) <= room && make(&p.tm_grid, p.grid, p.n);
  // fused row kernel input: [T N][n][2 cs] floats, box = 16 bins x box_rows(n) positions of one row.
  // Automatic choice: the warp-specialised kernel pipelines the units of a
  // CTA, which pays off once every SM has several (at 3.4 units per SM the
  // per-row CTAs were faster, at 27 the warp-specialised kernel by a fifth).
  p.fused_ws = false;
  const long units = (long)((p.Nf + kFftCols - 1) / kFftCols) * p.T * p.N;
  const bool want = p.row_kernel == 2 || (p.row_kernel == 0 && units >= 8L * p.num_sms);
  if (want && p.cs % kFftCols == 0 && p.nchunks == 1 && (size_t)p.T * p.N <= 0xffffffffu &&
      fused_ws_size_ok(p.n, room)) {
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * p.cs), (cuuint64_t)p.n, (cuuint64_t)p.T * p.N};
    const cuuint64_t strides[2] = {(cuuint64_t)(2 * p.cs * sizeof(float)),
                                   (cuuint64_t)(2 * (size_t)p.cs * p.n * sizeof(float))};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * kFftCols), (cuuint32_t)box_rows(p.n), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    p.fused_ws = encode(&p.tm_fused, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p.rows, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
}

cudaError_t fft_forward_cols(const Plan& p, cudaStream_t s) {
  if (p.cols_tma_fwd) return dispatch_cols_tma(p.n, kFwdCols, p.tm_rows, col_args(p, kFwdCols), p.num_sms, s);
  FftArgs a = base_args(p);
  a.src = p.rows;
  a.dst = p.grid;
  dim3 grid(p.n * p.cs / kFftCols, p.T);
  return dispatch(p.n, kFwdCols, a, grid, s);
}

cudaError_t fft_adjoint_cols(const Plan& p, cudaStream_t s) {
  if (p.cols_tma_adj) return dispatch_cols_tma(p.n, kAdjCols, p.tm_grid, col_args(p, kAdjCols), p.num_sms, s);
  FftArgs a = base_args(p);
  a.src = p.grid;
  a.dst = p.rows;
  dim3 grid(p.n * p.cs / kFftCols, p.T);
  return dispatch(p.n, kAdjCols, a, grid, s);
}

cudaError_t fft_adjoint_rows(const Plan& p, float2* out, int f0, float scale, cudaStream_t s) {
  FftArgs a = base_args(p);
  a.src = p.rows;
  a.dst = out;
  a.f0 = f0;
  a.scale = scale;
  a.Cv = std::min(p.chunk, p.Nf - f0);
  dim3 grid((a.Cv + kFftCols - 1) / kFftCols, p.T * p.N);
  return dispatch(p.n, kAdjRows, a, grid, s);
}

namespace {
FusedArgs fused_args(const Plan& p, const float2* Vin, float2* m, float2* v, float2* Vout, const AdamArgs& aa,
                     const Reducer* red, const double* data_loss, double* loss_out) {
  FusedArgs a{};
  a.rows = p.rows;
  a.deapod = p.deapod;
  a.twiddle = p.twiddle;
  a.Vin = Vin;
  a.Vout = Vout;
  a.m = m;
  a.v = v;
  a.partials = red->partials;
  a.counter = red->counter;
  a.data_loss = data_loss;
  a.loss_out = loss_out;
  a.N = p.N;
  a.n = p.n;
  a.Nf = p.Nf;
  a.C = p.cs;
  a.T = p.T;
  a.scale = 1.0f / (float)p.N;
  a.ad = aa;
  a.err = p.status_dev;
  a.nfb = (p.Nf + kFftCols - 1) / kFftCols;
  a.units = a.nfb * p.T * p.N;
  return a;
}

// Column pass over a batch: CTAs split by tile count.
cudaError_t cols_batch(Plan* const* ps, int count, int kind, cudaStream_t s) {
  if (count < 1 || count > kMaxBatch) return cudaErrorInvalidValue;
  bool tma = true;
  for (int r = 0; r < count; ++r) {
    tma = tma && (kind == kFwdCols ? ps[r]->cols_tma_fwd : ps[r]->cols_tma_adj);
    if (ps[r]->n != ps[0]->n) return cudaErrorInvalidValue;
  }
  if (!tma) {  // untiled fallback: one launch per plan
    for (int r = 0; r < count; ++r) {
      const cudaError_t e = kind == kFwdCols ? fft_forward_cols(*ps[r], s) : fft_adjoint_cols(*ps[r], s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  MultiCols m{};
  m.nreq = count;
  long work[kMaxBatch];
  int cap[kMaxBatch];
  for (int r = 0; r < count; ++r) {
    m.tm[r] = kind == kFwdCols ? ps[r]->tm_rows : ps[r]->tm_grid;
    m.a[r] = col_args(*ps[r], kind);
    work[r] = m.a[r].ntiles;
    cap[r] = std::max(1, m.a[r].ntiles);
  }
  const int per_sm = cols_per_sm(ps[0]->n, kind);
  const int ctas = split_ctas(work, cap, count, std::max(count, per_sm * ps[0]->num_sms), m.cta_begin);
  return dispatch_cols_multi(ps[0]->n, kind, m, ctas, s);
}
}  // namespace

cudaError_t fft_forward_cols_batch(Plan* const* ps, int count, cudaStream_t s) {
  return cols_batch(ps, count, kFwdCols, s);
}
cudaError_t fft_adjoint_cols_batch(Plan* const* ps, int count, cudaStream_t s) {
  return cols_batch(ps, count, kAdjCols, s);
}

cudaError_t fused_rows_update_batch(const BatchIter* it, int count, cudaStream_t s) {
  if (count < 1 || count > kMaxBatch) return cudaErrorInvalidValue;
  MultiFused m{};
  m.nreq = 0;
  m.unit_begin[0] = 0;
  for (int r = 0; r < count; ++r) {
    const Plan& p = *it[r].p;
    if (p.nchunks != 1 || p.n != it[0].p->n) return cudaErrorInvalidValue;
    if (p.fused_ws) {  // the persistent warp-specialised kernel runs on its own
      const cudaError_t e = fused_rows_update(p, it[r].Vin, p.adam_m, p.adam_v, it[r].Vout, it[r].aa, &p.red_tv,
                                              p.scalars, it[r].loss_out, it[r].fwd_tail, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    const int q = m.nreq++;
    m.a[q] = fused_args(p, it[r].Vin, p.adam_m, p.adam_v, it[r].Vout, it[r].aa, &p.red_tv, p.scalars,
                        it[r].loss_out);
    if (m.a[q].units > p.red_tv.capacity) return cudaErrorInvalidValue;
    m.fwd_tail[q] = it[r].fwd_tail ? 1 : 0;
    m.unit_begin[q + 1] = m.unit_begin[q] + m.a[q].units;
  }
  if (m.nreq == 0) return cudaSuccess;
  return dispatch_fused_multi(it[0].p->n, m, s);
}

cudaError_t fused_rows_update(const Plan& p, const float2* Vin, float2* m, float2* v, float2* Vout,
                              const AdamArgs& aa, const Reducer* red, const double* data_loss, double* loss_out,
                              bool fwd_tail, cudaStream_t s) {
  if (p.nchunks != 1 || !red) return cudaErrorInvalidValue;
  FusedArgs a{};
  a.rows = p.rows;
  a.deapod = p.deapod;
  a.twiddle = p.twiddle;
  a.Vin = Vin;
  a.Vout = Vout;
  a.m = m;
  a.v = v;
  a.partials = red->partials;
  a.counter = red->counter;
  a.data_loss = data_loss;
  a.loss_out = loss_out;
  a.N = p.N;
  a.n = p.n;
  a.Nf = p.Nf;
  a.C = p.cs;
  a.T = p.T;
  a.scale = 1.0f / (float)p.N;
  a.ad = aa;
  a.err = p.status_dev;
  a.nfb = (p.Nf + kFftCols - 1) / kFftCols;
  a.units = a.nfb * p.T * p.N;
  if (p.fused_ws) {
    a.bh = box_rows(p.n);
    a.nbox = p.n / a.bh;
    const int ctas = std::max(1, std::min(a.units, p.num_sms));
    if (ctas > red->capacity) return cudaErrorInvalidValue;
    return dispatch_fused_ws(p.n, p.tm_fused, a, fwd_tail, ctas, s);
  }
  dim3 grid((p.Nf + kFftCols - 1) / kFftCols, p.T * p.N);
  if ((long)grid.x * grid.y > red->capacity) return cudaErrorInvalidValue;
  return dispatch_fused(p.n, a, fwd_tail, grid, s);
}


cudaError_t cart_fft_configure(int N) {
  switch (N) {
#define CASE(v) \
  case v: return configure_cart<v>();
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t cart_fft_pass(int N, int pass, const float2* src, float2* dst, const float2* twiddleN,
                          const uint8_t* mask, const CartLoss* loss, float scale, cudaStream_t s) {
  CartArgs a{};
  a.src = src;
  a.dst = dst;
  a.twiddle = twiddleN;
  a.mask = mask;
  a.N = N;
  a.scale = scale;
  if (loss) {
    if (pass != kCartColsFwd || !loss->red || !mask || loss->red->capacity < N / kCartCols) return cudaErrorInvalidValue;
    a.y = loss->y;
    a.yimg = loss->yimg;
    a.wk = loss->wk;
    a.wi = loss->wi;
    a.partials = loss->red->partials;
    a.counter = loss->red->counter;
    a.loss_const = loss->loss_const;
    a.loss_out = loss->loss_out;
  }
  switch (N) {
#define CASE(v) \
  case v: return launch_cart<v>(pass, a, s);
    PROP_FFT_SIZES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace prop
