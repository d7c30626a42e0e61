// C ABI entry points (declared in include/prop.h): argument checking,
// chunk loops and the reconstruction iteration.  Every step of the
// operator, its adjoint, the loss and the optimiser runs in this library's
// kernels; the host only validates, enqueues and copies.
#include "prop_internal.cuh"

#include <cmath>
#include <algorithm>

namespace prop {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

prop_status fail(prop_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

prop_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return PROP_ERR_CUDA;
}

namespace {
cudaEvent_t take_event(Plan& p) {
  if (!p.ev_pool.empty()) {
    cudaEvent_t e = p.ev_pool.back();
    p.ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

StageScope::StageScope(Plan& plan, int st, cudaStream_t stream) : p(plan), stage(st), s(stream) {
  if (!p.profiling) return;
  a = take_event(p);
  b = take_event(p);
  if (a) cudaEventRecord(a, s);
}

StageScope::~StageScope() {
  if (!a || !b) return;
  cudaEventRecord(b, s);
  p.ev_rec[stage].emplace_back(a, b);
}

namespace {

#define PROP_LAUNCH(call)                                   \
  do {                                                      \
    cudaError_t e__ = (call);                               \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call);   \
  } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// After a synchronisation: report (and clear) an expired bounded device wait.
prop_status check_device_status(Plan& p) {
  int st = 0;
  PROP_CUDA(cudaMemcpy(&st, p.status_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    PROP_CUDA(cudaMemset(p.status_dev, 0, sizeof(int)));
    return fail(PROP_ERR_TIMEOUT, "a bounded device-side wait expired (grid tile staging did not complete)");
  }
  return PROP_OK;
}

// y = A V, or r = A V - y_meas with |r|^2 reduced into *sumsq.  rows_ready:
// p.rows already holds the forward row transform of V (single chunk only).
prop_status forward_impl(Plan& p, const float2* V, float2* y, const float2* y_meas, const Reducer* red,
                         double* sumsq, cudaStream_t s, bool rows_ready = false, bool accumulate = false) {
  if (!(rows_ready && p.nchunks == 1)) p.rows_of = nullptr;
  for (int c = 0; c < p.nchunks; ++c) {
    const int f0 = c * p.chunk;
    const int nb = std::min(p.chunk, p.Nf - f0);
    const bool last = c == p.nchunks - 1;
    if (!(rows_ready && p.nchunks == 1)) {
      StageScope sc(p, kStFwdRows, s);
      PROP_LAUNCH(fft_forward_rows(p, V, f0, s));
    }
    {
      StageScope sc(p, kStFwdCols, s);
      PROP_LAUNCH(fft_forward_cols(p, s));
    }
    {
      StageScope sc(p, kStInterp, s);
      // With a single chunk the residual is final here: also emit the spread's input.
      float2* contrib = (y_meas && p.nchunks == 1) ? p.contrib : nullptr;
      PROP_LAUNCH(interp(p, f0, nb, y, c == 0 ? y_meas : nullptr, c > 0 || accumulate, last ? red : nullptr, sumsq,
                         contrib, s));
    }
  }
  return PROP_OK;
}

// V = scale * (unscaled adjoint) of r; scale = 1/N gives A^H.
prop_status adjoint_impl(Plan& p, const float2* r, float2* V, bool contrib_ready, cudaStream_t s) {
  const float scale = 1.0f / (float)p.N;
  p.rows_of = nullptr;  // the adjoint passes overwrite the row workspace
  for (int c = 0; c < p.nchunks; ++c) {
    const int f0 = c * p.chunk;
    const int nb = std::min(p.chunk, p.Nf - f0);
    {
      StageScope sc(p, kStSpread, s);
      PROP_LAUNCH(spread(p, f0, nb, r, contrib_ready && p.nchunks == 1, s));
    }
    {
      StageScope sc(p, kStAdjCols, s);
      PROP_LAUNCH(fft_adjoint_cols(p, s));
    }
    {
      StageScope sc(p, kStAdjRows, s);
      PROP_LAUNCH(fft_adjoint_rows(p, V, f0, scale, s));
    }
  }
  return PROP_OK;
}

prop_status check_params(const prop_recon_params* q) {
  if (!q) return fail(PROP_ERR_INVALID_ARG, "params is NULL");
  if (q->iters < 0) return fail(PROP_ERR_INVALID_ARG, "iters must be >= 0");
  if (!(q->lr >= 0.f) || !(q->beta1 >= 0.f && q->beta1 < 1.f) || !(q->beta2 >= 0.f && q->beta2 < 1.f) ||
      !(q->eps > 0.f))
    return fail(PROP_ERR_INVALID_ARG, "Adam parameters out of range");
  if (!(q->tv_eps > 0.f) || !(q->tv_xy >= 0.f) || !(q->tv_t >= 0.f) || !std::isfinite(q->tv_xy) ||
      !std::isfinite(q->tv_t))
    return fail(PROP_ERR_INVALID_ARG, "TV parameters out of range (weights >= 0, tv_eps > 0)");
  return PROP_OK;
}

AdamArgs adam_args(const prop_recon_params* q, int k) {
  AdamArgs a{};
  const double bc1 = 1.0 - std::pow((double)q->beta1, k);
  const double bc2 = 1.0 - std::pow((double)q->beta2, k);
  a.lr_t = (float)(q->lr / bc1);
  a.inv_bc2_sqrt = (float)(1.0 / std::sqrt(bc2));
  a.beta1 = q->beta1;
  a.beta2 = q->beta2;
  a.eps = q->eps;
  a.tv_xy = q->tv_xy;
  a.tv_t = q->tv_t;
  a.tv_eps = q->tv_eps;
  a.gscale = 2.f;
  return a;
}

// One Adam iteration k from Vin into Vout.  With a single bin chunk the
// last adjoint pass, the update and (next_rows) the next iteration's forward
// row pass run as one fused kernel; rows_ready says that p.rows already holds
// the forward row transform of Vin (left there by the previous iteration).
prop_status step_impl(Plan& p, const float2* y, const prop_recon_params* q, int k, const float2* Vin,
                      float2* Vout, double* loss_dst, cudaStream_t s, bool rows_ready = false,
                      bool next_rows = false) {
  prop_status st;
  if (k == 1) {
    const size_t vbytes = p.vol_elems() * sizeof(float2);
    PROP_CUDA(cudaMemsetAsync(p.adam_m, 0, vbytes, s));
    PROP_CUDA(cudaMemsetAsync(p.adam_v, 0, vbytes, s));
  }
  const bool fused = p.nchunks == 1;
  if ((st = forward_impl(p, Vin, p.resid, y, &p.red_interp, p.scalars, s, rows_ready && fused)) != PROP_OK)
    return st;
  p.rows_of = nullptr;  // the adjoint passes below overwrite the row workspace
  if (fused) {
    {
      StageScope sc(p, kStSpread, s);
      PROP_LAUNCH(spread(p, 0, p.Nf, p.resid, true, s));
    }
    {
      StageScope sc(p, kStAdjCols, s);
      PROP_LAUNCH(fft_adjoint_cols(p, s));
    }
    StageScope sc(p, kStFused, s);
    PROP_LAUNCH(fused_rows_update(p, Vin, p.adam_m, p.adam_v, Vout, adam_args(q, k), &p.red_tv, p.scalars,
                                  loss_dst, next_rows, s));
    return PROP_OK;
  }
  if ((st = adjoint_impl(p, p.resid, p.grad, true, s)) != PROP_OK) return st;
  StageScope sc(p, kStOpt, s);
  PROP_LAUNCH(tv_adam(p, Vin, p.grad, p.adam_m, p.adam_v, Vout, adam_args(q, k), &p.red_tv, p.scalars,
                      loss_dst, s));
  return PROP_OK;
}

prop_status reconstruct_impl(Plan& p, const float2* y, const prop_recon_params* q, float2* V,
                             double* trace_host, cudaStream_t s) {
  prop_status st = plan_ensure_recon(&p, std::max(q->iters, 1));
  if (st != PROP_OK) return st;
  const size_t vbytes = p.vol_elems() * sizeof(float2);
  float2* cur = V;
  float2* nxt = p.vol2;
  for (int k = 1; k <= q->iters; ++k) {
    if ((st = step_impl(p, y, q, k, cur, nxt, p.loss_dev + (k - 1), s, k > 1, k < q->iters)) != PROP_OK) return st;
    std::swap(cur, nxt);
  }
  if (cur != V) PROP_CUDA(cudaMemcpyAsync(V, cur, vbytes, cudaMemcpyDeviceToDevice, s));
  if (trace_host && q->iters > 0) {
    PROP_CUDA(cudaMemcpyAsync(trace_host, p.loss_dev, sizeof(double) * q->iters, cudaMemcpyDeviceToHost, s));
    PROP_CUDA(cudaStreamSynchronize(s));
    if ((st = check_device_status(p)) != PROP_OK) return st;
  }
  return PROP_OK;
}

}  // namespace

bool batch_compatible(const Plan& a, const Plan& b) {
  return a.nchunks == 1 && b.nchunks == 1 && a.n == b.n && a.cs == b.cs && a.W == b.W && a.device == b.device;
}

prop_status batch_step(BatchMember* mb, int count, cudaStream_t s) {
  if (count < 1 || count > kMaxBatch) return fail(PROP_ERR_INVALID_ARG, "batch: 1 to 8 problems");
  Plan* ps[kMaxBatch];
  const float2* ym[kMaxBatch];
  BatchIter it[kMaxBatch];
  for (int r = 0; r < count; ++r) {
    Plan& p = *mb[r].p;
    if (!batch_compatible(p, *mb[0].p)) return fail(PROP_ERR_INVALID_ARG, "batch: plans differ in 2N, bin stride or width");
    for (int q = 0; q < r; ++q)
      if (mb[q].p == &p) return fail(PROP_ERR_INVALID_ARG, "batch: a plan appears twice (its workspace is one problem's)");
    if (mb[r].k == 1) {
      const size_t vbytes = p.vol_elems() * sizeof(float2);
      PROP_CUDA(cudaMemsetAsync(p.adam_m, 0, vbytes, s));
      PROP_CUDA(cudaMemsetAsync(p.adam_v, 0, vbytes, s));
    }
    p.rows_of = nullptr;
    if (!mb[r].rows_ready) PROP_LAUNCH(fft_forward_rows(p, mb[r].Vin, 0, s));
    ps[r] = &p;
    ym[r] = mb[r].y;
    it[r].p = &p;
    it[r].Vin = mb[r].Vin;
    it[r].Vout = mb[r].Vout;
    it[r].aa = adam_args(mb[r].q, mb[r].k);
    it[r].loss_out = mb[r].loss_dst;
    it[r].fwd_tail = mb[r].next_rows;
  }
  PROP_LAUNCH(fft_forward_cols_batch(ps, count, s));
  PROP_LAUNCH(interp_residual_batch(ps, ym, count, s));
  PROP_LAUNCH(spread_batch(ps, count, s));
  PROP_LAUNCH(fft_adjoint_cols_batch(ps, count, s));
  PROP_LAUNCH(fused_rows_update_batch(it, count, s));
  return PROP_OK;
}

prop_status loss_grad_device(Plan& p, const float2* y, const AdamArgs& a, const float2* V, float2* grad,
                             double* loss_out, cudaStream_t s) {
  prop_status st;
  if ((st = forward_impl(p, V, p.resid, y, &p.red_interp, p.scalars, s)) != PROP_OK) return st;
  if ((st = adjoint_impl(p, p.resid, p.grad, true, s)) != PROP_OK) return st;
  StageScope sc(p, kStOpt, s);
  PROP_LAUNCH(tv_grad(p, V, p.grad, grad, a, &p.red_tv, p.scalars, loss_out, s));
  return PROP_OK;
}

prop_status plan_step(Plan& p, const float2* y, const prop_recon_params* q, int k, const float2* Vin, float2* Vout,
                      double* loss_dst, cudaStream_t s, bool rows_ready, bool next_rows) {
  return step_impl(p, y, q, k, Vin, Vout, loss_dst, s, rows_ready, next_rows);
}

}  // namespace prop

using namespace prop;

extern "C" {

const char* prop_last_error(void) { return g_last_error.c_str(); }

prop_status prop_plan_create(const prop_plan_desc* desc, prop_plan* out) {
  if (!out) return fail(PROP_ERR_INVALID_ARG, "plan_create: out is NULL");
  *out = nullptr;
  Plan* p = nullptr;
  prop_status st = plan_build(desc, &p);
  if (st != PROP_OK) return st;
  prop_plan h = new (std::nothrow) prop_plan_s{p};
  if (!h) {
    plan_free(p);
    return fail(PROP_ERR_OOM, "plan_create: host allocation failed");
  }
  *out = h;
  return PROP_OK;
}

prop_status prop_plan_destroy(prop_plan plan) {
  if (!plan) return PROP_OK;
  {
    DeviceGuard g(plan->p->device);
    cudaDeviceSynchronize();
    plan_free(plan->p);
  }
  delete plan;
  return PROP_OK;
}

prop_status prop_plan_workspace_bytes(prop_plan plan, size_t* bytes) {
  if (!plan || !bytes) return fail(PROP_ERR_INVALID_ARG, "workspace_bytes: null argument");
  const Plan& p = *plan->p;
  size_t recon = p.recon_bytes;
  if (!p.recon_ready) {
    recon = (size_t)p.M * sizeof(float2) + 4 * p.vol_elems() * sizeof(float2) +
            2 * (size_t)(1 << 15) * sizeof(double) + 64 * sizeof(double) + 256;
  }
  *bytes = p.table_bytes + p.work_bytes + recon;
  return PROP_OK;
}

prop_status prop_forward(prop_plan plan, const void* V_dev, void* y_dev, void* stream) {
  if (!plan || !V_dev || !y_dev) return fail(PROP_ERR_INVALID_ARG, "forward: null argument");
  if (!aligned16(V_dev) || !aligned16(y_dev)) return fail(PROP_ERR_INVALID_ARG, "forward: buffers must be 16-byte aligned");
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  return forward_impl(p, (const float2*)V_dev, (float2*)y_dev, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

prop_status prop_adjoint(prop_plan plan, const void* y_dev, void* V_dev, void* stream) {
  if (!plan || !V_dev || !y_dev) return fail(PROP_ERR_INVALID_ARG, "adjoint: null argument");
  if (!aligned16(V_dev) || !aligned16(y_dev)) return fail(PROP_ERR_INVALID_ARG, "adjoint: buffers must be 16-byte aligned");
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  return adjoint_impl(p, (const float2*)y_dev, (float2*)V_dev, false, (cudaStream_t)stream);
}

prop_status prop_reconstruct(prop_plan plan, const void* y_dev, const prop_recon_params* params, void* V_dev,
                             double* loss_trace_host, void* stream) {
  if (!plan || !y_dev || !V_dev) return fail(PROP_ERR_INVALID_ARG, "reconstruct: null argument");
  if (!aligned16(V_dev) || !aligned16(y_dev)) return fail(PROP_ERR_INVALID_ARG, "reconstruct: buffers must be 16-byte aligned");
  prop_status st = check_params(params);
  if (st != PROP_OK) return st;
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  return reconstruct_impl(p, (const float2*)y_dev, params, (float2*)V_dev, loss_trace_host, (cudaStream_t)stream);
}

prop_status prop_recon_step(prop_plan plan, const void* y_dev, const prop_recon_params* params, int k,
                            const void* V_in_dev, void* V_out_dev, double* loss_dev, void* stream) {
  if (!plan || !y_dev || !V_in_dev || !V_out_dev) return fail(PROP_ERR_INVALID_ARG, "recon_step: null argument");
  if (V_in_dev == V_out_dev) return fail(PROP_ERR_INVALID_ARG, "recon_step: V_in and V_out must differ");
  if (k < 1) return fail(PROP_ERR_INVALID_ARG, "recon_step: k must be >= 1");
  if (!aligned16(V_in_dev) || !aligned16(V_out_dev) || !aligned16(y_dev))
    return fail(PROP_ERR_INVALID_ARG, "recon_step: buffers must be 16-byte aligned");
  prop_status st = check_params(params);
  if (st != PROP_OK) return st;
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  if ((st = plan_ensure_recon(&p, 1)) != PROP_OK) return st;
  return step_impl(p, (const float2*)y_dev, params, k, (const float2*)V_in_dev, (float2*)V_out_dev,
                   loss_dev ? loss_dev : p.scalars + 2, (cudaStream_t)stream);
}

prop_status prop_shard_forward(prop_plan plan, const void* V_dev, int flags, void* y_part_dev, void* stream) {
  if (!plan || !V_dev || !y_part_dev) return fail(PROP_ERR_INVALID_ARG, "shard_forward: null argument");
  if (!aligned16(V_dev) || !aligned16(y_part_dev))
    return fail(PROP_ERR_INVALID_ARG, "shard_forward: buffers must be 16-byte aligned");
  if (flags & ~(PROP_SHARD_REUSE_ROWS | PROP_SHARD_ACCUMULATE))
    return fail(PROP_ERR_INVALID_ARG, "shard_forward: unknown flags");
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  const bool ready = (flags & PROP_SHARD_REUSE_ROWS) && p.nchunks == 1 && p.rows_of == V_dev;
  return forward_impl(p, (const float2*)V_dev, (float2*)y_part_dev, nullptr, nullptr, nullptr,
                      (cudaStream_t)stream, ready, (flags & PROP_SHARD_ACCUMULATE) != 0);
}

prop_status prop_shard_update(prop_plan plan, const void* y_dev, const void* y_sum_dev,
                              const prop_recon_params* params, int k, const void* V_in_dev, void* V_out_dev,
                              double* loss_parts_dev, void* stream) {
  if (!plan || !y_dev || !y_sum_dev || !V_in_dev || !V_out_dev)
    return fail(PROP_ERR_INVALID_ARG, "shard_update: null argument");
  if (V_in_dev == V_out_dev) return fail(PROP_ERR_INVALID_ARG, "shard_update: V_in and V_out must differ");
  if (k < 1) return fail(PROP_ERR_INVALID_ARG, "shard_update: k must be >= 1");
  if (!aligned16(V_in_dev) || !aligned16(V_out_dev) || !aligned16(y_dev) || !aligned16(y_sum_dev) ||
      ((uintptr_t)loss_parts_dev & 7u))
    return fail(PROP_ERR_INVALID_ARG, "shard_update: buffers must be 16-byte aligned (loss_parts 8-byte)");
  prop_status st = check_params(params);
  if (st != PROP_OK) return st;
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  if ((st = plan_ensure_recon(&p, 1)) != PROP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vbytes = p.vol_elems() * sizeof(float2);
  if (k == 1) {
    PROP_CUDA(cudaMemsetAsync(p.adam_m, 0, vbytes, s));
    PROP_CUDA(cudaMemsetAsync(p.adam_v, 0, vbytes, s));
  }
  double* parts = loss_parts_dev ? loss_parts_dev : p.scalars + 4;  // [0] data term, [1] this plan's TV
  double* zero = p.scalars + 6;  // "data loss" input of the update kernels, so that they report TV alone
  PROP_CUDA(cudaMemsetAsync(zero, 0, sizeof(double), s));
  p.rows_of = nullptr;
  const bool fused = p.nchunks == 1;
  {
    StageScope sc(p, kStInterp, s);
    PROP_LAUNCH(residual(p, (const float2*)y_sum_dev, (const float2*)y_dev, p.resid, fused, p.red_interp, parts, s));
  }
  const AdamArgs aa = adam_args(params, k);
  if (fused) {
    {
      StageScope sc(p, kStSpread, s);
      PROP_LAUNCH(spread(p, 0, p.Nf, p.resid, true, s));
    }
    {
      StageScope sc(p, kStAdjCols, s);
      PROP_LAUNCH(fft_adjoint_cols(p, s));
    }
    StageScope sc(p, kStFused, s);
    PROP_LAUNCH(fused_rows_update(p, (const float2*)V_in_dev, p.adam_m, p.adam_v, (float2*)V_out_dev, aa,
                                  &p.red_tv, zero, parts + 1, true, s));
    p.rows_of = V_out_dev;
    return PROP_OK;
  }
  if ((st = adjoint_impl(p, p.resid, p.grad, false, s)) != PROP_OK) return st;
  StageScope sc(p, kStOpt, s);
  PROP_LAUNCH(tv_adam(p, (const float2*)V_in_dev, p.grad, p.adam_m, p.adam_v, (float2*)V_out_dev, aa, &p.red_tv,
                      zero, parts + 1, s));
  return PROP_OK;
}

prop_status prop_reconstruct_batch(const prop_plan* plans, int count, const void* const* y_dev,
                                   const prop_recon_params* params, void* const* V_dev, double* const* loss_trace_host,
                                   void* stream) {
  if (!plans || !y_dev || !params || !V_dev) return fail(PROP_ERR_INVALID_ARG, "reconstruct_batch: null argument");
  if (count < 1 || count > kMaxBatch) return fail(PROP_ERR_INVALID_ARG, "reconstruct_batch: count must be 1 to 8");
  int kmax = 0;
  for (int r = 0; r < count; ++r) {
    if (!plans[r] || !y_dev[r] || !V_dev[r]) return fail(PROP_ERR_INVALID_ARG, "reconstruct_batch: null argument");
    if (!aligned16(V_dev[r]) || !aligned16(y_dev[r]))
      return fail(PROP_ERR_INVALID_ARG, "reconstruct_batch: buffers must be 16-byte aligned");
    prop_status st = check_params(&params[r]);
    if (st != PROP_OK) return st;
    for (int q = 0; q < r; ++q)
      if (plans[q] == plans[r]) return fail(PROP_ERR_INVALID_ARG, "reconstruct_batch: a plan appears twice");
    if (!batch_compatible(*plans[r]->p, *plans[0]->p))
      return fail(PROP_ERR_INVALID_ARG,
                  "reconstruct_batch: the plans must share 2N, bin stride, kernel width and device, one bin chunk each");
    kmax = std::max(kmax, params[r].iters);
  }
  Plan& p0 = *plans[0]->p;
  DeviceGuard g(p0.device);
  cudaStream_t s = (cudaStream_t)stream;
  float2* cur[kMaxBatch];
  float2* nxt[kMaxBatch];
  for (int r = 0; r < count; ++r) {
    prop_status st = plan_ensure_recon(plans[r]->p, std::max(params[r].iters, 1));
    if (st != PROP_OK) return st;
    cur[r] = (float2*)V_dev[r];
    nxt[r] = plans[r]->p->vol2;
  }
  for (int k = 1; k <= kmax; ++k) {
    BatchMember mb[kMaxBatch];
    int n = 0;
    for (int r = 0; r < count; ++r) {
      if (k > params[r].iters) continue;
      Plan& p = *plans[r]->p;
      mb[n] = BatchMember{&p, (const float2*)y_dev[r], &params[r], k, cur[r], nxt[r], p.loss_dev + (k - 1), k > 1,
                          k < params[r].iters};
      ++n;
    }
    prop_status st = batch_step(mb, n, s);
    if (st != PROP_OK) return st;
    for (int r = 0; r < count; ++r)
      if (k <= params[r].iters) std::swap(cur[r], nxt[r]);
  }
  bool sync = false;
  for (int r = 0; r < count; ++r) {
    Plan& p = *plans[r]->p;
    if (cur[r] != (float2*)V_dev[r])
      PROP_CUDA(cudaMemcpyAsync(V_dev[r], cur[r], p.vol_elems() * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    if (loss_trace_host && loss_trace_host[r] && params[r].iters > 0) {
      PROP_CUDA(cudaMemcpyAsync(loss_trace_host[r], p.loss_dev, sizeof(double) * params[r].iters,
                                cudaMemcpyDeviceToHost, s));
      sync = true;
    }
  }
  if (sync) {
    PROP_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < count; ++r) {
      prop_status st = check_device_status(*plans[r]->p);
      if (st != PROP_OK) return st;
    }
  }
  return PROP_OK;
}

prop_status prop_reconstruct_host(prop_plan plan, const void* y_host, const prop_recon_params* params,
                                  void* V_host, double* loss_trace_host, void* stream) {
  if (!plan || !y_host || !V_host) return fail(PROP_ERR_INVALID_ARG, "reconstruct_host: null argument");
  prop_status st = check_params(params);
  if (st != PROP_OK) return st;
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vbytes = p.vol_elems() * sizeof(float2);
  const size_t ybytes = (size_t)p.M * sizeof(float2);
  if (!p.stage_y) {
    PROP_CUDA(plan_dev_alloc(&p, (void**)&p.stage_y, ybytes));
    p.recon_bytes += ybytes;
  }
  if (!p.stage_v) {
    PROP_CUDA(plan_dev_alloc(&p, (void**)&p.stage_v, vbytes));
    p.recon_bytes += vbytes;
  }
  PROP_CUDA(cudaMemcpyAsync(p.stage_y, y_host, ybytes, cudaMemcpyHostToDevice, s));
  PROP_CUDA(cudaMemcpyAsync(p.stage_v, V_host, vbytes, cudaMemcpyHostToDevice, s));
  st = reconstruct_impl(p, p.stage_y, params, p.stage_v, nullptr, s);
  if (st != PROP_OK) return st;
  PROP_CUDA(cudaMemcpyAsync(V_host, p.stage_v, vbytes, cudaMemcpyDeviceToHost, s));
  if (loss_trace_host && params->iters > 0)
    PROP_CUDA(cudaMemcpyAsync(loss_trace_host, p.loss_dev, sizeof(double) * params->iters,
                              cudaMemcpyDeviceToHost, s));
  PROP_CUDA(cudaStreamSynchronize(s));
  if ((st = check_device_status(p)) != PROP_OK) return st;
  return PROP_OK;
}

prop_status prop_loss_grad(prop_plan plan, const void* y_dev, const prop_recon_params* params, const void* V_dev,
                           void* grad_dev, double* loss_host, void* stream) {
  if (!plan || !y_dev || !V_dev || !loss_host) return fail(PROP_ERR_INVALID_ARG, "loss_grad: null argument");
  if (!aligned16(V_dev) || !aligned16(y_dev) || (grad_dev && !aligned16(grad_dev)))
    return fail(PROP_ERR_INVALID_ARG, "loss_grad: buffers must be 16-byte aligned");
  if (!params || !(params->tv_eps > 0.f) || !(params->tv_xy >= 0.f) || !(params->tv_t >= 0.f))
    return fail(PROP_ERR_INVALID_ARG, "loss_grad: TV parameters out of range");
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  cudaStream_t s = (cudaStream_t)stream;
  prop_status st = plan_ensure_recon(&p, 1);
  if (st != PROP_OK) return st;
  if ((st = forward_impl(p, (const float2*)V_dev, p.resid, (const float2*)y_dev, &p.red_interp, p.scalars, s)) != PROP_OK)
    return st;
  if ((st = adjoint_impl(p, p.resid, p.grad, true, s)) != PROP_OK) return st;
  AdamArgs a{};
  a.tv_xy = params->tv_xy;
  a.tv_t = params->tv_t;
  a.tv_eps = params->tv_eps;
  a.gscale = 2.f;
  float2* out = grad_dev ? (float2*)grad_dev : p.grad;
  {
    StageScope sc(p, kStOpt, s);
    PROP_LAUNCH(tv_grad(p, (const float2*)V_dev, p.grad, out, a, &p.red_tv, p.scalars, p.scalars + 1, s));
  }
  PROP_CUDA(cudaMemcpyAsync(loss_host, p.scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  PROP_CUDA(cudaStreamSynchronize(s));
  if ((st = check_device_status(p)) != PROP_OK) return st;
  return PROP_OK;
}

prop_status prop_render(prop_plan plan, const void* V_dev, int f_lo, int f_hi, void* image_dev, void* stream) {
  if (!plan || !V_dev || !image_dev) return fail(PROP_ERR_INVALID_ARG, "render: null argument");
  Plan& p = *plan->p;
  if (f_lo < 0 || f_hi > p.Nf || f_lo >= f_hi) return fail(PROP_ERR_INVALID_ARG, "render: need 0 <= f_lo < f_hi <= nf");
  DeviceGuard g(p.device);
  StageScope sc(p, kStOther, (cudaStream_t)stream);
  PROP_LAUNCH(render(p, (const float2*)V_dev, f_lo, f_hi, (float2*)image_dev, (cudaStream_t)stream));
  return PROP_OK;
}

prop_status prop_psnr(prop_plan plan, const void* image_dev, const void* ref_dev, int frames, double* psnr_host,
                      void* stream) {
  if (!plan || !image_dev || !ref_dev || !psnr_host) return fail(PROP_ERR_INVALID_ARG, "psnr: null argument");
  if (!aligned16(image_dev) || !aligned16(ref_dev))
    return fail(PROP_ERR_INVALID_ARG, "psnr: buffers must be 16-byte aligned");
  Plan& p = *plan->p;
  if (frames < 1 || frames > p.T) return fail(PROP_ERR_INVALID_ARG, "psnr: need 1 <= frames <= nframes");
  DeviceGuard g(p.device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!p.psnr_scratch) {
    const int cap = 4 * p.num_sms;
    // [2 cap] partials, then the counter word (and the result) in the last two doubles
    cudaError_t e = plan_dev_alloc(&p, (void**)&p.psnr_scratch, (2 * (size_t)cap + 2) * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      p.psnr_scratch = nullptr;
      return fail(PROP_ERR_OOM, std::string("psnr: scratch allocation failed: ") + cudaGetErrorString(e));
    }
    p.recon_bytes += (2 * (size_t)cap + 2) * sizeof(double);
    p.psnr_cap = cap;
    PROP_CUDA(cudaMemsetAsync(p.psnr_scratch + 2 * cap, 0, 2 * sizeof(double), s));
  }
  const long count = (long)frames * p.N * p.N;
  double* out = p.psnr_scratch + 2 * p.psnr_cap + 1;
  {
    StageScope sc(p, kStOther, s);
    PROP_LAUNCH(psnr(p, (const float2*)image_dev, (const float2*)ref_dev, count, out, s));
  }
  PROP_CUDA(cudaMemcpyAsync(psnr_host, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  PROP_CUDA(cudaStreamSynchronize(s));
  return PROP_OK;
}

prop_status prop_profile_enable(prop_plan plan, int enable) {
  if (!plan) return fail(PROP_ERR_INVALID_ARG, "profile_enable: null plan");
  plan->p->profiling = enable != 0;
  return PROP_OK;
}

prop_status prop_profile_read(prop_plan plan, double* ms_out, long long* launches_out) {
  if (!plan) return fail(PROP_ERR_INVALID_ARG, "profile_read: null plan");
  Plan& p = *plan->p;
  DeviceGuard g(p.device);
  for (int st = 0; st < PROP_NUM_STAGES; ++st) {
    double ms = 0.0;
    for (auto& pr : p.ev_rec[st]) {
      float t = 0.f;
      PROP_CUDA(cudaEventSynchronize(pr.second));
      PROP_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
      ms += t;
    }
    if (ms_out) ms_out[st] = ms;
    if (launches_out) launches_out[st] = (long long)p.ev_rec[st].size();
    for (auto& pr : p.ev_rec[st]) {
      p.ev_pool.push_back(pr.first);
      p.ev_pool.push_back(pr.second);
    }
    p.ev_rec[st].clear();
  }
  return PROP_OK;
}

}  // extern "C"
