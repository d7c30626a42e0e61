// Plan builder: validates the geometry, computes every table in FP64 on the
// host, stores them in FP32 on the device, and sizes the workspace.
//
// Tables (all from the operator y_b(k) = s sum_f P sum_x V exp(-2 pi i k.x)
// evaluated by a Kaiser-Bessel NUFFT with oversampling 2 and width 6):
//   * per sample m = (b L + l) R + j: k = k_r d_b + k_p d_b^perp, grid
//     coordinate u = 2N k (mod 2N, exact because the sum over integer x is
//     1-periodic in k), first tap floor(u) - (W/2 - 1) and the W weights per
//     axis psi(u - tap), psi(t) = I0(beta sqrt(1 - (2t/W)^2)) / I0(beta);
//   * deapodisation c(x) = I0(beta) / psihat(x / 2N) with the closed-form
//     transform psihat(xi) = W sinh(sqrt(beta^2 - (pi W xi)^2)) / sqrt(...),
//     beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8) (Beatty et al. 2005);
//   * displacement phase P[j][f] = exp(-2 pi i k_r Delta_f), the argument
//     k_r Delta_f reduced modulo 1 in FP64 before the cosine and sine
//     (Sec. 3: a displacement along the readout is a phase linear in k_r);
//   * FFT twiddles exp(-2 pi i q / 2N);
//   * interpolation order (samples sorted by grid tile) and spread gather
//     lists: for every grid cell the (sample, weight) pairs that cover it.
#include "prop_internal.cuh"

#include <cmath>
#include <cstring>
#include <algorithm>
#include <new>

namespace prop {

namespace {

// Modified Bessel function of the first kind, order 0, from its power series
// I0(z) = sum_k ((z/2)^(2k)) / (k!)^2 (all terms positive, so the partial sums
// converge monotonically; 60 terms reach double precision for z <= 40).
double bessel_i0(double z) {
  const double q = 0.25 * z * z;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 60; ++k) {
    term *= q / ((double)k * (double)k);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

bool fft_size_supported(int n) {
  static const int ok[] = {16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
  for (int v : ok)
    if (v == n) return true;
  return false;
}

// Grouped spread lists for the shared-memory staged spread kernel.  The
// grid cells of every frame are cut into 2 x 2-cell groups; a group's list
// holds every sample whose W x W footprint meets the group, in ascending m,
// as (phased-residual offset m * cs, the sample's weight w2[a] w1[b] on each
// of the group's four cells, row-major, zero where the footprint misses the
// cell).  The weights are the FP64 products rounded once, as in the
// interpolation's tables, so every cell accumulates the same terms in the
// same order as a per-cell list would.  Every list is padded to a multiple
// of four entries with (row M, zero weights), row M of the phased residual
// being kept zero.  Groups are taken in frame, 4 x 4-group patch, row-major
// order and cut into items of about equal work, each item one blob of int2
// words staged by a single bulk copy:
//   groups[ngp]      (first cell index, end of its list), ngp = ngroups rounded up to even
//   offs[nent / 2]   nent int32 offsets (nent a multiple of 4)
//   wts[2 nent]      nent float4 weights
// Returns false when one group's list alone exceeds a stage.
bool build_group_lists(const Plan& p, const std::vector<int>& first_tap, const std::vector<double>& wd,
                       std::vector<int4>& sitems, std::vector<int2>& blob) {
  const int n = p.n, W = p.W, G = kSpreadGroup, gps = n / G, PG = kSpreadGroupPatch;
  static_assert(kSpreadGroup == 2, "four weights per entry");
  const size_t LR = (size_t)p.L * p.R;
  const size_t ngroup = (size_t)p.T * gps * gps;
  auto axis_groups = [&](int first, int* out) {
    int cnt = 0;
    for (int a = 0; a < W; ++a) {
      const int g = ((first + a) % n) / G;
      bool seen = false;
      for (int k = 0; k < cnt; ++k) seen = seen || out[k] == g;
      if (!seen) out[cnt++] = g;
    }
    return cnt;
  };
  std::vector<int> gcnt(ngroup, 0);
  for (size_t m = 0; m < (size_t)p.M; ++m) {
    const size_t frame = (size_t)p.blade_frame[m / LR];
    int gr[16], gc[16];
    const int nr = axis_groups(first_tap[2 * m + 1], gr), nc = axis_groups(first_tap[2 * m], gc);
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < nc; ++b) gcnt[(frame * gps + gr[a]) * gps + gc[b]]++;
  }
  std::vector<int> glen(ngroup);
  for (size_t g = 0; g < ngroup; ++g) glen[g] = (gcnt[g] + kSpreadListPad - 1) / kSpreadListPad * kSpreadListPad;
  std::vector<int> gorder;
  gorder.reserve(ngroup);
  for (int t = 0; t < p.T; ++t)
    for (int pr = 0; pr < gps / PG; ++pr)
      for (int pc = 0; pc < gps / PG; ++pc)
        for (int r = 0; r < PG; ++r)
          for (int c = 0; c < PG; ++c) gorder.push_back((t * gps + pr * PG + r) * gps + pc * PG + c);
  std::vector<int> item_of(ngroup), first(ngroup);
  struct ItemSec { size_t offs, wts; };
  std::vector<ItemSec> secs;
  auto words = [](long ng, long ne) { return ((ng + 1) & ~1L) + ne / 2 + 2 * ne; };
  size_t i = 0;
  while (i < ngroup) {
    size_t j = i;
    long cost = 0, nent = 0;
    while (j < ngroup) {
      const int c = glen[gorder[j]];
      if (words((long)(j + 1 - i), nent + c) > kSpreadStageInt2) {
        if (j == i) return false;  // one group exceeds a stage
        break;
      }
      nent += c;
      cost += c + kSpreadGroupCost;
      ++j;
      if (cost >= kSpreadGroupItemCost) break;
    }
    const long ng = (long)(j - i), ngp = (ng + 1) & ~1L;
    const size_t at = blob.size();
    if (at + (size_t)words(ng, nent) > 0x7fffffffULL) return false;
    sitems.push_back(make_int4((int)at, (int)ng, (int)nent, (int)words(ng, nent)));
    secs.push_back({at + (size_t)ngp, at + (size_t)ngp + (size_t)nent / 2});
    blob.resize(at + (size_t)words(ng, nent), make_int2(0, 0));
    {
      int* offs = reinterpret_cast<int*>(&blob[secs.back().offs]);
      for (long q = 0; q < nent; ++q) offs[q] = (int)((size_t)p.M * p.cs);  // padding: the zero row
    }
    long e = 0;
    for (size_t q = i; q < j; ++q) {
      const int g = gorder[q];
      item_of[g] = (int)sitems.size() - 1;
      first[g] = (int)e;
      e += glen[g];
      const int t = g / (gps * gps), gr = (g / gps) % gps, gc = g % gps;
      blob[at + (q - i)] = make_int2((int)(((size_t)t * n + (size_t)gr * G) * n + (size_t)gc * G), (int)e);
    }
    i = j;
  }
  std::vector<int> cursor(ngroup, 0);
  for (size_t m = 0; m < (size_t)p.M; ++m) {
    const size_t frame = (size_t)p.blade_frame[m / LR];
    const int r0 = first_tap[2 * m + 1], c0 = first_tap[2 * m];
    int gr[16], gc[16];
    const int nr = axis_groups(r0, gr), nc = axis_groups(c0, gc);
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < nc; ++b) {
        const int g = (int)((frame * gps + gr[a]) * gps + gc[b]);
        const ItemSec& sec = secs[item_of[g]];
        const size_t e = (size_t)first[g] + cursor[g]++;
        float w[4];
        for (int ii = 0; ii < G; ++ii)
          for (int jj = 0; jj < G; ++jj) {
            const int da = (gr[a] * G + ii - r0 + n) % n, db = (gc[b] * G + jj - c0 + n) % n;
            w[ii * G + jj] = (da < W && db < W) ? (float)(wd[m * 2 * W + W + da] * wd[m * 2 * W + db]) : 0.f;
          }
        reinterpret_cast<int*>(&blob[sec.offs])[e] = (int)(m * (size_t)p.cs);
        std::memcpy(&blob[sec.wts + 2 * e], w, sizeof(w));
      }
  }
  return true;
}

struct DevAlloc {
  Plan* p;
  size_t* counter;
  template <class T>
  prop_status operator()(T** ptr, size_t count, const char* what) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = plan_dev_alloc(p, (void**)ptr, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      *ptr = nullptr;
      return fail(PROP_ERR_OOM, std::string("cudaMalloc failed for ") + what + ": " +
                                    cudaGetErrorString(e));
    }
    *counter += count * sizeof(T);
    return PROP_OK;
  }
};

template <class T>
prop_status upload(T* dst, const std::vector<T>& src) {
  PROP_CUDA(cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PROP_OK;
}

}  // namespace

cudaError_t plan_dev_alloc(Plan* p, void** ptr, size_t bytes) {
  return p->alloc ? p->alloc->allocate(ptr, bytes) : cudaMalloc(ptr, bytes);
}

void plan_dev_free(Plan* p, void* ptr) {
  if (!ptr) return;
  if (p->alloc)
    p->alloc->release(ptr);
  else
    cudaFree(ptr);
}

void plan_free(Plan* p) {
  if (!p) return;
  void* ptrs[] = {p->kb_idx, p->kb_w, p->phase, p->deapod, p->twiddle, p->blade_frame_d,
                  p->order, p->items, p->item_cta_off, p->sitems, p->sitem_cta_off, p->spread_claim, p->sblob, p->contrib, p->grid, p->rows,
                  p->resid, p->grad, p->status_dev,
                  p->vol2, p->adam_m, p->adam_v, p->loss_dev, p->scalars,
                  p->red_interp.partials, p->red_interp.counter, p->red_tv.partials,
                  p->red_tv.counter, p->stage_y, p->stage_v, p->proj_shift, p->proj_mask, p->proj_twiddle,
                  p->proj_img, p->proj_k, p->proj_kg, p->proj_g, p->proj_yimg, p->proj_const,
                  p->red_proj_k.partials, p->red_proj_k.counter, p->red_proj_u.partials, p->red_proj_u.counter,
                  p->psnr_scratch, p->kp_work};
  for (void* q : ptrs) plan_dev_free(p, q);
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  for (auto& v : p->ev_rec)
    for (auto& pr : v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  delete p;
}

prop_status plan_build(const prop_plan_desc* d, Plan** out, DeviceAllocator* alloc) {
  if (!d || !out) return fail(PROP_ERR_INVALID_ARG, "plan_create: null argument");
  *out = nullptr;
  const int N = d->n;
  if (N < 16 || N > 512 || N % 8 != 0 || !fft_size_supported(2 * N))
    return fail(PROP_ERR_INVALID_ARG,
                "plan_create: n must be a multiple of 8 in [16, 512] with 2n = 2^a 3^b (n = " +
                    std::to_string(N) + ")");
  if (d->nf < 1 || d->nf > 4096) return fail(PROP_ERR_INVALID_ARG, "plan_create: nf out of range");
  if (d->nblades < 1 || d->lines < 1 || d->readout < 1)
    return fail(PROP_ERR_INVALID_ARG, "plan_create: nblades, lines and readout must be >= 1");
  if ((long long)d->nblades * d->lines * d->readout > (1LL << 30))
    return fail(PROP_ERR_INVALID_ARG, "plan_create: too many samples");
  if ((long long)d->nblades * d->lines * d->readout * kMaxChunk >= (1LL << 31))
    return fail(PROP_ERR_INVALID_ARG, "plan_create: too many samples for 32-bit spread offsets");
  if (d->nframes < 1) return fail(PROP_ERR_INVALID_ARG, "plan_create: nframes must be >= 1");
  if (!d->delta || !d->theta) return fail(PROP_ERR_INVALID_ARG, "plan_create: delta/theta is NULL");
  if (d->kb_width != 0 && d->kb_width != 6 && d->kb_width != 8)
    return fail(PROP_ERR_INVALID_ARG, "plan_create: kb_width must be 0 (= 6), 6 or 8");
  if (d->bin_chunk < 0 || d->bin_chunk > kMaxChunk)
    return fail(PROP_ERR_INVALID_ARG, "plan_create: bin_chunk must be in [0, 64]");
  if (d->row_kernel < 0 || d->row_kernel > 2)
    return fail(PROP_ERR_INVALID_ARG, "plan_create: row_kernel must be 0, 1 or 2");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || d->device < 0 || d->device >= ndev) {
    cudaGetLastError();
    return fail(PROP_ERR_INVALID_ARG, "plan_create: no such CUDA device");
  }
  for (int f = 0; f < d->nf; ++f)
    if (!std::isfinite(d->delta[f])) return fail(PROP_ERR_INVALID_ARG, "plan_create: delta not finite");
  for (int b = 0; b < d->nblades; ++b) {
    if (!std::isfinite(d->theta[b])) return fail(PROP_ERR_INVALID_ARG, "plan_create: theta not finite");
    if (d->blade_frame && (d->blade_frame[b] < 0 || d->blade_frame[b] >= d->nframes))
      return fail(PROP_ERR_INVALID_ARG, "plan_create: blade_frame out of range");
  }

  Plan* p = new (std::nothrow) Plan();
  if (!p) return fail(PROP_ERR_OOM, "plan_create: host allocation failed");
  p->alloc = alloc;
  p->N = N;
  p->n = 2 * N;
  p->Nf = d->nf;
  p->B = d->nblades;
  p->L = d->lines;
  p->R = d->readout;
  p->T = d->nframes;
  p->M = p->B * p->L * p->R;
  p->device = d->device;
  p->W = d->kb_width == 0 ? kKbWidthDefault : d->kb_width;
  p->chunk = d->bin_chunk == 0 ? std::min(p->Nf, kMaxChunk) : std::min(d->bin_chunk, p->Nf);
  p->nchunks = (p->Nf + p->chunk - 1) / p->chunk;
  p->cs = p->chunk + (p->chunk & 1);  // even stride: staged grid rows are 16-byte runs
  p->theta.assign(d->theta, d->theta + p->B);
  p->delta.assign(d->delta, d->delta + p->Nf);
  p->blade_frame.assign(p->B, 0);
  if (d->blade_frame) p->blade_frame.assign(d->blade_frame, d->blade_frame + p->B);

  DeviceGuard guard(p->device);
  if (!guard.ok) {
    plan_free(p);
    return fail(PROP_ERR_CUDA, "plan_create: cudaSetDevice failed");
  }
  if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device) != cudaSuccess) {
    cudaGetLastError();
    plan_free(p);
    return fail(PROP_ERR_CUDA, "plan_create: device attribute query failed");
  }

  const int n = p->n;
  const int Wi = p->W;
  const double W = Wi, sigma = 2.0;
  const double beta = M_PI * std::sqrt((W / sigma) * (W / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
  const double i0b = bessel_i0(beta);

  auto psi = [&](double t) {
    double a = 2.0 * t / W;
    double r = 1.0 - a * a;
    if (r < 0.0) return 0.0;
    return bessel_i0(beta * std::sqrt(r)) / i0b;
  };

  // Per-sample grid indices and weights.
  std::vector<uint32_t> kb_idx(p->M);
  const int wq = Wi / 2;  // float4 per sample
  std::vector<float4> kb_w((size_t)p->M * wq);
  std::vector<int> first_tap(2 * (size_t)p->M);
  std::vector<double> wd((size_t)p->M * 2 * Wi);  // FP64 weights: w1[W] then w2[W]
  for (int b = 0; b < p->B; ++b) {
    const double c = std::cos(p->theta[b]), s = std::sin(p->theta[b]);
    for (int l = 0; l < p->L; ++l) {
      const double kp = ((double)l - p->L / 2.0) / N;
      for (int j = 0; j < p->R; ++j) {
        const double kr = ((double)j - p->R / 2.0) / N;
        const double k[2] = {kr * c - kp * s, kr * s + kp * c};
        const size_t m = ((size_t)b * p->L + l) * p->R + j;
        float w[16];
        int base[2];
        for (int a = 0; a < 2; ++a) {
          double u = n * k[a];
          u -= n * std::floor(u / n);
          if (u >= n) u -= n;
          if (u < 0) u = 0;
          const double fl = std::floor(u);
          const double fr = u - fl;
          const int h = Wi / 2 - 1;  // taps floor(u) - h .. floor(u) + W/2
          base[a] = ((int)fl - h + n) % n;
          for (int q = 0; q < Wi; ++q) {
            const double v = psi(fr + h - q);
            wd[m * 2 * Wi + a * Wi + q] = v;
            w[a * Wi + q] = (float)v;
          }
        }
        kb_idx[m] = (uint32_t)base[0] | ((uint32_t)base[1] << 16);
        first_tap[2 * m] = base[0];
        first_tap[2 * m + 1] = base[1];
        for (int q = 0; q < wq; ++q)
          kb_w[(size_t)wq * m + q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
      }
    }
  }

  // Deapodisation along one axis.
  std::vector<float> deapod(N);
  for (int i = 0; i < N; ++i) {
    const double xi = (double)(i - N / 2) / n;
    const double a = M_PI * W * xi;
    const double z2 = beta * beta - a * a;
    double ft;
    if (z2 > 0) {
      const double z = std::sqrt(z2);
      ft = W * std::sinh(z) / z;
    } else if (z2 < 0) {
      const double z = std::sqrt(-z2);
      ft = W * std::sin(z) / z;
    } else {
      ft = W;
    }
    deapod[i] = (float)(i0b / ft);
  }

  // Displacement phase per readout sample and bin.
  std::vector<float2> phase((size_t)p->R * p->Nf);
  for (int j = 0; j < p->R; ++j) {
    const double kr = ((double)j - p->R / 2.0) / N;
    for (int f = 0; f < p->Nf; ++f) {
      double arg = kr * p->delta[f];
      arg -= std::nearbyint(arg);
      phase[(size_t)j * p->Nf + f] = make_float2((float)std::cos(2 * M_PI * arg),
                                                 (float)-std::sin(2 * M_PI * arg));
    }
  }

  std::vector<float2> tw(n);
  for (int q = 0; q < n; ++q)
    tw[q] = make_float2((float)std::cos(2 * M_PI * q / n), (float)-std::sin(2 * M_PI * q / n));

  // Interpolation work items: samples sorted by (frame, TR x TC-cell tile of
  // their first tap), ascending m within a tile; every non-empty tile's run is
  // cut into items of at most kInterpItem samples.  One CTA per item stages
  // the tile plus its (W-1)-cell halo in shared memory.
  p->interp_tr = interp_tile_rows(p->cs, p->W);
  p->interp_tc = interp_tile_cols(p->cs, p->W);
  const int TR = p->interp_tr, TC = p->interp_tc;
  const int nrt = (n + TR - 1) / TR, nct = n / TC;  // tiles per column / per row of the grid
  const size_t ntile = (size_t)p->T * nrt * nct;
  const size_t LR = (size_t)p->L * p->R;
  std::vector<int> order(p->M);
  std::vector<int4> items;
  {
    auto tile_of = [&](size_t m) {
      const size_t frame = (size_t)p->blade_frame[m / LR];
      return (frame * nrt + first_tap[2 * m + 1] / TR) * nct + first_tap[2 * m] / TC;
    };
    std::vector<int> cnt(ntile + 1, 0);
    for (size_t m = 0; m < (size_t)p->M; ++m) cnt[tile_of(m) + 1]++;
    for (size_t t = 0; t < ntile; ++t) cnt[t + 1] += cnt[t];
    for (size_t t = 0; t < ntile; ++t) {
      // a tile's run in ceil(c / kInterpItem) items of nearly equal size
      const int c = cnt[t + 1] - cnt[t];
      const int parts = (c + kInterpItem - 1) / kInterpItem;
      for (int q = 0, s = cnt[t]; q < parts; ++q) {
        const int sz = c / parts + (q < c % parts ? 1 : 0);
        items.push_back(make_int4((int)t, s, sz, 0));
        s += sz;
      }
    }
    for (size_t m = 0; m < (size_t)p->M; ++m) order[cnt[tile_of(m)]++] = (int)m;
  }
  p->n_items = (int)items.size();
  // Static balance over the persistent CTAs (one per SM): longest item first
  // to the least loaded CTA, with an item's cost its shared-memory traffic
  // (W^2 taps of cs bins per sample plus the staged tile); each CTA's items
  // are then stored contiguously, in tile order.
  std::vector<int> cta_off;
  {
    const int P = std::max(1, std::min(p->num_sms, p->n_items));
    const long tile_cost = (long)(TR + Wi - 1) * (TC + Wi - 1) * p->cs / 16;
    auto cost = [&](const int4& it) { return (long)it.z * Wi * Wi * p->cs / 16 + tile_cost; };
    std::vector<int> idx(items.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost(items[a]) > cost(items[b]); });
    std::vector<long> load(P, 0);
    std::vector<std::vector<int>> own(P);
    for (int i : idx) {
      int best = 0;
      for (int c = 1; c < P; ++c)
        if (load[c] < load[best]) best = c;
      load[best] += cost(items[i]);
      own[best].push_back(i);
    }
    std::vector<int4> sorted;
    sorted.reserve(items.size());
    cta_off.assign(P + 1, 0);
    for (int c = 0; c < P; ++c) {
      std::sort(own[c].begin(), own[c].end());
      for (int i : own[c]) sorted.push_back(items[i]);
      cta_off[c + 1] = (int)sorted.size();
    }
    items.swap(sorted);
    p->interp_ctas = P;
  }
  // The interpolation reads the per-sample tables in this sorted order, so that
  // an item's metadata is one contiguous run.
  {
    std::vector<uint32_t> idx_s(p->M);
    std::vector<float4> w_s(kb_w.size());
    for (size_t i = 0; i < (size_t)p->M; ++i) {
      const size_t m = (size_t)order[i];
      idx_s[i] = kb_idx[m];
      for (int q = 0; q < wq; ++q) w_s[i * wq + q] = kb_w[m * wq + q];
    }
    kb_idx.swap(idx_s);
    kb_w.swap(w_s);
  }

  // Spread gather lists: for every (frame, cell) the samples whose W x W
  // footprint covers the cell, as (phased-residual offset m * cs, weight
  // w2[a] w1[b]) in ascending m.  The weight is formed in FP64 from the same
  // factors the interpolation applies, so the spread is its exact transpose.
  // Cells are listed in patch-major order (frame, 8x8-cell patch, row-major in
  // the patch) and cut into work items of about equal work (list entries plus
  // a fixed cost per written cell); patch order keeps the residual rows an
  // item reads within a small region of k-space.
  std::vector<int4> sitems;
  std::vector<int2> blob;
  const int2 pad_entry = make_int2((int)((size_t)p->M * p->cs), 0);
  p->spread_grouped = (p->cs == 8 || p->cs == 16 || p->cs == 32 || p->cs == 64) &&
                      build_group_lists(*p, first_tap, wd, sitems, blob);
  if (!p->spread_grouped) {
  sitems.clear();
  blob.clear();
  const size_t ncell = (size_t)p->T * n * n;
  std::vector<int> cell_cnt(ncell, 0);
  auto cell_of = [&](size_t m, int a, int b) {
    const size_t frame = (size_t)p->blade_frame[m / LR];
    const int r = (first_tap[2 * m + 1] + a) % n, c = (first_tap[2 * m] + b) % n;
    return (frame * n + r) * n + c;
  };
  for (size_t m = 0; m < (size_t)p->M; ++m)
    for (int a = 0; a < Wi; ++a)
      for (int b = 0; b < Wi; ++b) cell_cnt[cell_of(m, a, b)]++;
  std::vector<int> cell_ids(ncell);
  {
    const int pps = n / kSpreadPatch;
    size_t i = 0;
    for (int t = 0; t < p->T; ++t)
      for (int pr = 0; pr < pps; ++pr)
        for (int pc = 0; pc < pps; ++pc)
          for (int r = 0; r < kSpreadPatch; ++r)
            for (int c = 0; c < kSpreadPatch; ++c)
              cell_ids[i++] = (int)(((size_t)t * n + pr * kSpreadPatch + r) * n + pc * kSpreadPatch + c);
  }
  // Work items: runs of consecutive cells (patch-major order) of about equal
  // work (list entries plus a fixed cost per written cell), each stored as
  // one contiguous blob that a CTA stages into shared memory with a single
  // bulk copy:
  //   int2 cells[ncells, rounded up to even]: (cell index, end of its list
  //        relative to the item's first entry)
  //   int2 entries[nent]: the lists, one after the other
  // Every list is padded to a multiple of kSpreadListPad entries with
  // (row M, weight 0): row M of the phased-residual buffer is kept zero, so
  // a padding entry adds an exact zero and the gather runs unpredicated.  A
  // cell whose list alone exceeds the staging capacity forms an item of its
  // own and the plan then gathers from global memory.
  std::vector<int> cell_first(ncell + 1, 0);  // cell -> first entry in the item's entries
  {
    auto padded = [](int c) { return (c + kSpreadListPad - 1) / kSpreadListPad * kSpreadListPad; };
    size_t i = 0;
    while (i < ncell) {
      // choose [i, j)
      size_t j = i;
      long cost = 0, nent = 0;
      while (j < ncell) {
        const int c = padded(cell_cnt[cell_ids[j]]);
        const long ncp = (long)((j + 1 - i + 1) & ~(size_t)1);
        if (j > i && ncp + nent + c > kSpreadStageInt2) break;  // would overflow the stage
        nent += c;
        cost += c + kSpreadCellCost;
        ++j;
        if (cost >= kSpreadItemCost) break;
      }
      const size_t ncells = j - i, ncp = (ncells + 1) & ~(size_t)1;
      if ((long)ncp + nent > kSpreadStageInt2) p->spread_staged = false;  // longer than a stage: read from global
      if (blob.size() + ncp + nent > 0x7fffffffULL) {
        plan_free(p);
        return fail(PROP_ERR_INVALID_ARG, "plan_create: spread lists exceed 2^31 entries");
      }
      sitems.push_back(make_int4((int)blob.size(), (int)ncells, (int)nent, (int)(ncp + nent)));
      const size_t cells_at = blob.size(), ent_at = cells_at + ncp;
      blob.resize(ent_at + nent, pad_entry);
      long e = 0;
      for (size_t q = i; q < j; ++q) {
        const int cid = cell_ids[q];
        cell_first[cid] = (int)(ent_at + e);
        e += padded(cell_cnt[cid]);
        blob[cells_at + (q - i)] = make_int2(cid, (int)e);
      }
      if (ncp > ncells) blob[cells_at + ncells] = make_int2(0, (int)e);
      i = j;
    }
  }
  for (size_t m = 0; m < (size_t)p->M; ++m)
    for (int a = 0; a < Wi; ++a)
      for (int b = 0; b < Wi; ++b) {
        const float w = (float)(wd[m * 2 * Wi + Wi + a] * wd[m * 2 * Wi + b]);
        int wbits;
        std::memcpy(&wbits, &w, sizeof(float));
        blob[cell_first[cell_of(m, a, b)]++] = make_int2((int)(m * (size_t)p->cs), wbits);
      }
  }
  // every item's blob (its word count is the staged copy's size) lies in the
  // list array, and a staged item fits a stage
  for (const int4& it : sitems) {
    const bool staged = p->spread_grouped || p->spread_staged;
    if (it.x < 0 || it.w < 0 || (size_t)it.x + (size_t)it.w > blob.size() || (staged && it.w > kSpreadStageInt2)) {
      plan_free(p);
      return fail(PROP_ERR_INVALID_ARG, "plan_create: inconsistent spread lists");
    }
  }
  p->n_sitems = (int)sitems.size();
  p->spread_entries = blob.size();
  // Schedule of the spread items over the staged kernel's persistent CTAs
  // (two per SM).  With few items per CTA, a plan-time balance (longest
  // first to the least loaded CTA, each CTA's items then in k-space order so
  // that consecutive items share residual rows in L1) and CTA c takes
  // [off[c], off[c + 1]).  With many (kSpreadClaimMinItems per CTA or more),
  // grouped lists keep the items in k-space order and the CTAs claim them
  // from a device counter, so each CTA's share follows the items' measured
  // cost.
  std::vector<int> scta_off;
  {
    const int P = std::max(1, std::min(kSpreadCtasPerSm * p->num_sms, p->n_sitems));
    p->spread_claimed = p->spread_grouped && p->n_sitems >= kSpreadClaimMinItems * P;
    if (p->spread_claimed) {
      scta_off = {0, p->n_sitems};
    } else {
      auto cost = [&](const int4& it) {
        return (long)it.z + (long)it.y * (p->spread_grouped ? kSpreadGroupCost : kSpreadCellCost);
      };
      std::vector<int> idx(sitems.size());
      for (size_t q = 0; q < idx.size(); ++q) idx[q] = (int)q;
      std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost(sitems[a]) > cost(sitems[b]); });
      std::vector<long> load(P, 0);
      std::vector<std::vector<int>> own(P);
      for (int q : idx) {
        int best = 0;
        for (int c = 1; c < P; ++c)
          if (load[c] < load[best]) best = c;
        load[best] += cost(sitems[q]);
        own[best].push_back(q);
      }
      std::vector<int4> sorted;
      sorted.reserve(sitems.size());
      scta_off.assign(P + 1, 0);
      for (int c = 0; c < P; ++c) {
        std::sort(own[c].begin(), own[c].end());  // k-space order within a CTA
        for (int q : own[c]) sorted.push_back(sitems[q]);
        scta_off[c + 1] = (int)sorted.size();
      }
      sitems.swap(sorted);
    }
    p->spread_ctas = P;
  }
  if (blob.empty()) blob.push_back(pad_entry);

  DevAlloc tab{p, &p->table_bytes};
  DevAlloc wrk{p, &p->work_bytes};
  prop_status st;
#define TRY(x)               \
  do {                       \
    st = (x);                \
    if (st != PROP_OK) {     \
      plan_free(p);          \
      return st;             \
    }                        \
  } while (0)
  TRY(tab(&p->kb_idx, kb_idx.size(), "sample indices"));
  TRY(tab(&p->kb_w, kb_w.size(), "sample weights"));
  TRY(tab(&p->phase, phase.size(), "phase table"));
  TRY(tab(&p->deapod, deapod.size(), "deapodisation table"));
  TRY(tab(&p->twiddle, tw.size(), "twiddles"));
  TRY(tab(&p->blade_frame_d, p->blade_frame.size(), "blade frames"));
  TRY(tab(&p->order, order.size(), "interpolation order"));
  TRY(tab(&p->items, std::max<size_t>(items.size(), 1), "interpolation items"));
  TRY(tab(&p->item_cta_off, cta_off.size(), "interpolation item ranges"));
  TRY(tab(&p->sitems, std::max<size_t>(sitems.size(), 1), "spread items"));
  TRY(tab(&p->sitem_cta_off, scta_off.size(), "spread item ranges"));
  TRY(tab(&p->sblob, blob.size(), "spread lists"));
  TRY(wrk(&p->grid, (size_t)p->T * n * n * p->cs, "grid workspace"));
  TRY(wrk(&p->rows, (size_t)p->T * N * n * p->cs, "row workspace"));
  TRY(wrk(&p->contrib, (size_t)(p->M + 1) * p->cs, "phased residual"));
  TRY(upload(p->kb_idx, kb_idx));
  TRY(upload(p->kb_w, kb_w));
  TRY(upload(p->phase, phase));
  TRY(upload(p->deapod, deapod));
  TRY(upload(p->twiddle, tw));
  TRY(upload(p->blade_frame_d, p->blade_frame));
  TRY(upload(p->order, order));
  if (!sitems.empty()) TRY(upload(p->sitems, sitems));
  TRY(upload(p->sitem_cta_off, scta_off));
  TRY(upload(p->sblob, blob));
  if (!items.empty()) TRY(upload(p->items, items));
  TRY(upload(p->item_cta_off, cta_off));
  p->row_kernel = d->row_kernel;
  fft_make_maps(*p);
  if (p->row_kernel == 2 && !p->fused_ws) {
    plan_free(p);
    return fail(PROP_ERR_INVALID_ARG,
                "plan_create: row_kernel 2 needs 2N <= 512, one bin chunk and a bin stride that is a "
                "multiple of 16");
  }
  {
    cudaError_t e = fft_configure(n);
    // The interpolation may use the device's whole opt-in shared memory.
    if (e == cudaSuccess) e = nufft_configure(p->smem_optin);
    if (e != cudaSuccess) {
      plan_free(p);
      return cuda_fail(e, "kernel configuration");
    }
  }
  TRY(tab(&p->status_dev, 1, "status word"));
  if (p->spread_claimed) TRY(tab(&p->spread_claim, 2, "spread item counter"));
  {
    cudaError_t e = cudaMemset(p->status_dev, 0, sizeof(int));
    if (e == cudaSuccess && p->spread_claim) e = cudaMemset(p->spread_claim, 0, 2 * sizeof(int));
    // the zero row that padding entries of the spread lists point at
    if (e == cudaSuccess) e = cudaMemset(p->contrib + (size_t)p->M * p->cs, 0, (size_t)p->cs * sizeof(float2));
    if (e != cudaSuccess) {
      plan_free(p);
      return cuda_fail(e, "status word");
    }
  }
#undef TRY
  *out = p;
  return PROP_OK;
}

prop_status plan_ensure_recon(Plan* p, int iters) {
  DevAlloc rec{p, &p->recon_bytes};
  prop_status st;
  if (!p->recon_ready) {
    const size_t nv = p->vol_elems();
    const int fused_blocks = (p->Nf + kFftCols - 1) / kFftCols * p->T * p->N;  // fused row kernel's CTAs
    const int red_cap = std::max(std::max(1 << 15, p->n_items), fused_blocks);
    if ((st = rec(&p->resid, (size_t)p->M, "residual")) != PROP_OK) return st;
    if ((st = rec(&p->grad, nv, "gradient")) != PROP_OK) return st;
    if ((st = rec(&p->vol2, nv, "volume buffer")) != PROP_OK) return st;
    if ((st = rec(&p->adam_m, nv, "Adam m")) != PROP_OK) return st;
    if ((st = rec(&p->adam_v, nv, "Adam v")) != PROP_OK) return st;
    if ((st = rec(&p->scalars, 8, "loss scalars")) != PROP_OK) return st;
    if ((st = rec(&p->red_interp.partials, red_cap, "partials")) != PROP_OK) return st;
    if ((st = rec(&p->red_interp.counter, 1, "counter")) != PROP_OK) return st;
    if ((st = rec(&p->red_tv.partials, red_cap, "partials")) != PROP_OK) return st;
    if ((st = rec(&p->red_tv.counter, 1, "counter")) != PROP_OK) return st;
    p->red_interp.capacity = red_cap;
    p->red_tv.capacity = red_cap;
    PROP_CUDA(cudaMemset(p->red_interp.counter, 0, sizeof(unsigned int)));
    PROP_CUDA(cudaMemset(p->red_tv.counter, 0, sizeof(unsigned int)));
    p->recon_ready = true;
  }
  if (iters > p->loss_cap) {
    if (p->loss_dev) {
      plan_dev_free(p, p->loss_dev);
      p->recon_bytes -= (size_t)p->loss_cap * sizeof(double);
      p->loss_dev = nullptr;
      p->loss_cap = 0;
    }
    const int cap = std::max(iters, 64);
    if ((st = rec(&p->loss_dev, cap, "loss trace")) != PROP_OK) return st;
    p->loss_cap = cap;
  }
  return PROP_OK;
}

}  // namespace prop

namespace prop {

size_t plan_estimate_bytes(const prop_plan_desc* d, int iters) {
  if (!d || d->n < 8 || d->nf < 1 || d->nblades < 1 || d->lines < 1 || d->readout < 1 || d->nframes < 1)
    return 0;
  const size_t N = d->n, n = 2 * N, Nf = d->nf, B = d->nblades, T = d->nframes;
  const size_t M = B * (size_t)d->lines * d->readout;
  const size_t W = d->kb_width == 8 ? 8 : 6;
  const size_t chunk = d->bin_chunk == 0 ? std::min<size_t>(Nf, kMaxChunk) : std::min<size_t>(d->bin_chunk, Nf);
  const size_t cs = chunk + (chunk & 1);
  const size_t TR = (size_t)interp_tile_rows((int)cs, (int)W), TC = (size_t)interp_tile_cols((int)cs, (int)W);
  const size_t ncell = T * n * n;
  const size_t vol = T * N * N * Nf;
  const size_t interp_items = M / kInterpItem + T * ((n + TR - 1) / TR) * (n / TC) + 1;
  const size_t spread_items = (M * W * W + kSpreadCellCost * ncell) / kSpreadItemCost + 1;
  size_t b = 0;
  b += 4 * M + M * (W / 2) * 16 + (size_t)d->readout * Nf * 8 + 4 * N + 8 * n + 4 * B + 4 * M;  // sample tables
  const size_t cell_lists = 8 * (ncell + spread_items) + 8 * (M * W * W + (kSpreadListPad - 1) * std::min(ncell, M * W * W));
  const size_t group_lists = 8 * (ncell / 4) + 8 + (4 + 16) * 2 * 16 * M + 16 * (ncell / 4);  // items <= groups
  b += 16 * interp_items + 16 * spread_items + std::max(cell_lists, group_lists) + 4 * 1024;  // lists
  b += 8 * T * n * n * cs + 8 * T * N * n * cs + 8 * (M + 1) * cs;                                  // workspace
  b += 8 * M + 4 * 8 * vol + 64 + 2 * 8 * std::max<size_t>(std::max<size_t>(32768, interp_items), (Nf + 15) / 16 * T * N) + 8 +
       8 * std::max<size_t>((size_t)std::max(iters, 1), 64);                                           // optimiser
  b += 32 * 512;  // allocation rounding
  return b;
}

}  // namespace prop
