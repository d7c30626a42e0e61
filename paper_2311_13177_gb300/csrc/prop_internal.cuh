// Internal declarations shared by the CUDA translation units of libprop.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/prop.h"

namespace prop {

constexpr int kKbWidthDefault = 6; // taps per axis of the Kaiser-Bessel kernel (6 or 8)
constexpr int kInterpItem = 256;   // most samples per interpolation work item
constexpr int kSpreadPatch = 8;        // spread cells are visited in 8x8-cell patches
constexpr int kSpreadCellCost = 4;     // work of writing one cell, in list entries
constexpr int kSpreadItemCost = 2048;  // target work per spread item
constexpr int kSpreadListPad = 4;      // spread lists hold a multiple of this many entries
// Shared-memory stage of one spread item, in int2 (46 KB): two CTAs of two
// stages then fit the SM's 196 KB shared-memory carve-out (48 KB stages
// need the 228 KB one), leaving about 60 KB of L1 instead of 28 KB for the
// residual rows the gathers read (static workload 72.8 -> 68.3 us).
constexpr int kSpreadStageInt2 = 5888;
constexpr int kSpreadCtasPerSm = 2;    // persistent staged-spread CTAs per SM
constexpr int kSpreadGroup = 2;        // grouped spread: 2 x 2-cell groups
constexpr int kSpreadGroupPatch = 4;   // groups are ordered in 4 x 4-group patches
// Work of writing one group, in list entries (the cost model of the spread
// items: an empty group only stores zeros; measured at the static workload,
// 1: 4744, 2: 4790, 4: 4708, 8: 4628, 16: 4423 iterations/s).
constexpr int kSpreadGroupCost = 2;
constexpr int kSpreadGroupItemCost = 2048;  // target work per grouped spread item
constexpr int kSpreadClaimMinItems = 8;  // spread items per CTA from which the CTAs claim items at run time
constexpr int kFftCols = 16;       // columns (complex lines) per FFT tile
// Lines a CTA of the projection model's image transforms: 4 (an N x N image
// is only N lines a pass, so 16-line tiles left all but N / 16 SMs idle;
// 4-line tiles still read whole 32-byte sectors along a column).
constexpr int kCartCols = 4;

// Interpolation tile (rows x cells per row) for bin stride cs and kernel
// width W: 16 x 16 up to 32 bins, 8 x 8 above.  At width 8 with 32 bins a
// 16 x 16 tile plus its 7-cell halo (23 x 23 cells, 135 KB) leaves room for
// one buffer only, so its copy could not overlap the previous tile's work;
// 12 rows of 16 (19 x 23 staged cells, 112 KB) double-buffer and stage 2.3x
// the cells they own (16 x 16: 2.1x; 8 x 8: 3.5x, which measured slower).
// Rows of tiles need not divide the grid: the last one wraps past row n - 1.
constexpr int interp_tile_rows(int cs, int W) { return cs > 32 ? 8 : (W == 8 && cs == 32 ? 12 : 16); }
constexpr int interp_tile_cols(int cs, int W) { return (void)W, cs > 32 ? 8 : 16; }

constexpr int kMaxChunk = 64;      // most bins in one grid pass
constexpr int kMaxBatch = 8;       // most problems in one multi-problem launch

// Status plumbing -----------------------------------------------------------
void set_error(const std::string& msg);
prop_status fail(prop_status s, const std::string& msg);
prop_status cuda_fail(cudaError_t e, const char* what);

#define PROP_CUDA(call)                                          \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return ::prop::cuda_fail(e__, #call); \
  } while (0)

// Restores the caller's current device when it goes out of scope.
struct DeviceGuard {
  int old = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&old) != cudaSuccess) old = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (old >= 0) cudaSetDevice(old);
  }
};

// Programmatic dependent launch -------------------------------------------
//
// The kernels of the iteration chain (column FFTs, interpolation, spread,
// fused row kernel) are launched with programmatic stream serialisation: a
// kernel may be scheduled onto SMs that its predecessor on the stream has
// already left, and runs the part of its prologue that reads only plan
// tables (barrier set-up, twiddles, staged spread lists) before the
// predecessor has finished.  Every thread of such a kernel calls
// grid_dep_wait() before it reads or writes any buffer that an earlier
// kernel of the stream may touch; grid_dep_wait() returns once the
// predecessor grid has completed and its memory operations are visible.
// grid_dep_release() then lets the successor be scheduled in turn.  For a
// kernel launched without the attribute both are no-ops.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... P, class... A>
cudaError_t launch_dep(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

// Deterministic "last block reduces" accumulator: every block writes one
// double partial, the block that arrives last sums them in index order.
struct Reducer {
  double* partials = nullptr;      // [capacity]
  unsigned int* counter = nullptr; // one word, returns to 0 after each use
  int capacity = 0;
};

// Source of a plan's device memory.  The default (null) is cudaMalloc /
// cudaFree; the request server hands out sub-ranges of one arena instead, so
// retiring a request never synchronises the device.
struct DeviceAllocator {
  virtual ~DeviceAllocator() {}
  virtual cudaError_t allocate(void** ptr, size_t bytes) = 0;
  virtual void release(void* ptr) = 0;
};

struct Plan {
  DeviceAllocator* alloc = nullptr;
  // geometry
  int N = 0, n = 0, Nf = 0, B = 0, L = 0, R = 0, T = 1, M = 0;
  int W = kKbWidthDefault;       // kernel width (taps per axis)
  int num_sms = 1;               // streaming multiprocessors of the device
  int smem_optin = 48 * 1024;    // largest opt-in shared memory per block (bytes)
  int* status_dev = nullptr;     // device status word: 1 = a bounded device wait expired
  int chunk = 0;                 // bins per grid pass
  int cs = 0;                    // bin stride of the grid workspaces (chunk rounded up to even)
  int nchunks = 0;
  int device = 0;
  std::vector<double> theta, delta;
  std::vector<int> blade_frame;

  // device tables
  uint32_t* kb_idx = nullptr;    // [M] packed (i1 | i2 << 16) first tap, mod n, in interpolation order
  float4* kb_w = nullptr;        // [M][W/2] -> 2W floats: w1[W] (x1 taps) then w2[W] (x2 taps), same order
  float2* phase = nullptr;       // [R][Nf] exp(-2 pi i k_r Delta_f)
  float* deapod = nullptr;       // [N]
  float2* twiddle = nullptr;     // [n] exp(-2 pi i k / n)
  int* blade_frame_d = nullptr;  // [B]
  int* order = nullptr;          // [M] samples sorted by grid tile (interpolation order)
  int4* items = nullptr;         // [n_items] (frame * tiles^2 + tile, first, count, 0), grouped by CTA
  int* item_cta_off = nullptr;   // [interp_ctas + 1] CTA c interpolates items [off[c], off[c + 1])
  int n_items = 0;
  int interp_ctas = 1;           // persistent interpolation CTAs the items are balanced over
  int interp_tr = 16, interp_tc = 16;  // interpolation tile: rows, cells per row
  // Spread gather: cells in patch-major order (frame, 8x8-cell patch,
  // row-major in the patch), cut into items; each item is one blob of
  // (cell, list end) pairs followed by its cells' (offset m * cs, weight
  // bits) lists, every list padded to kSpreadListPad entries with (M * cs, 0).
  int4* sitems = nullptr;        // [n_sitems] (blob offset in int2, cells or groups, entries, blob words)
  int2* sblob = nullptr;         // [spread_entries] item blobs
  int* sitem_cta_off = nullptr;  // [spread_ctas + 1] staged-spread CTA c takes items [off[c], off[c + 1])
  int* spread_claim = nullptr;   // [2]: next unclaimed spread item, CTAs done (both 0 between launches)
  bool spread_claimed = false;   // the staged-spread CTAs claim items at run time (else the ranges above)
  int n_sitems = 0;
  int spread_ctas = 1;           // persistent staged-spread CTAs (the ranges' CTA count)
  size_t spread_entries = 0;
  bool spread_staged = true;     // cell lists: every item fits a shared-memory stage
  bool spread_grouped = false;   // sblob/sitems hold grouped lists (2 x 2-cell groups), else cell lists

  // TMA tensor maps of the column passes' inputs (row workspace, grid), and
  // whether the staged column kernels run for this plan's size
  CUtensorMap tm_rows;
  CUtensorMap tm_grid;
  bool cols_tma_fwd = false, cols_tma_adj = false;
  // Row workspace seen as [T N][n][2 cs floats]: a box is the 16-bin slice
  // of one image row's n positions, the input of the warp-specialised fused
  // row kernel (used when its size and bin stride allow)
  CUtensorMap tm_fused;
  bool fused_ws = false;         // the warp-specialised row kernel runs (row_kernel rule below)
  int row_kernel = 0;            // as requested: 0 auto, 1 per-row CTAs, 2 warp-specialised

  // grid workspace (one bin chunk)
  float2* grid = nullptr;        // [T][n][n][chunk]
  float2* rows = nullptr;        // [T][N][n][chunk] row-pass intermediate
  float2* contrib = nullptr;     // [M + 1][cs] conj(P[j][f]) r_m, input of the spread; row M stays zero
  const void* rows_of = nullptr; // volume whose forward row transform p.rows holds (left by prop_shard_update)

  // projection model, the paper's own forward model (allocated on first use)
  bool proj_ready = false;
  int4* proj_shift = nullptr;      // [B][Nf] (o1, o2, w1 bits, w2 bits): along axis a pixel i reads
                                   // taps i + o_a (weight 1 - w_a) and i + o_a + 1 (weight w_a)
  uint8_t* proj_mask = nullptr;    // [B][N][N] blade support on the Cartesian k grid
  float2* proj_twiddle = nullptr;  // [N] exp(-2 pi i m / N)
  float2* proj_img = nullptr;      // [N][N] projected image
  float2* proj_k = nullptr;        // [N][N] transform work
  float2* proj_kg = nullptr;       // [N][N] k-space gradient of the data term
  float2* proj_g = nullptr;        // [N][N] its inverse DFT (image-space gradient)
  float2* proj_yimg = nullptr;     // [B][N][N] DFT of the given blade images
  double* proj_const = nullptr;    // [B] image term outside each mask
  Reducer red_proj_k, red_proj_u;

  // reconstruction state (allocated on first use)
  bool recon_ready = false;
  float2* resid = nullptr;       // [M]
  float2* grad = nullptr;        // [T][N][N][Nf] adjoint of the residual
  float2* vol2 = nullptr;        // [T][N][N][Nf] ping-pong volume
  float2* adam_m = nullptr;      // [T][N][N][Nf] (re, im) first moment
  float2* adam_v = nullptr;      // [T][N][N][Nf] (re, im) second moment
  double* loss_dev = nullptr;    // [max_iters] loss trace
  int loss_cap = 0;
  double* scalars = nullptr;     // [4] data loss, tv_xy, tv_t scratch
  Reducer red_interp, red_tv;

  // host-API staging (allocated on first use)
  float2* stage_y = nullptr;
  float2* stage_v = nullptr;

  // PSNR reduction scratch (allocated on first use): [2 * psnr_cap] FP64
  // block partials (squared magnitude error, reference peak), then the
  // arrival counter
  double* psnr_scratch = nullptr;
  int psnr_cap = 0;

  // K-Planes model workspace (expanded planes and gradient partials),
  // allocated on first use and grown on demand
  void* kp_work = nullptr;
  size_t kp_work_bytes = 0;

  size_t table_bytes = 0, work_bytes = 0, recon_bytes = 0;

  // stage profiling (prop_profile_enable)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;                  // idle events
  std::vector<std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> ev_rec =
      std::vector<std::vector<std::pair<cudaEvent_t, cudaEvent_t>>>(PROP_NUM_STAGES);

  size_t vol_elems() const { return (size_t)T * N * N * Nf; }
};

// Stage ids of prop_profile_read.
enum Stage { kStFwdRows = 0, kStFwdCols, kStInterp, kStSpread, kStAdjCols, kStAdjRows, kStOpt, kStOther, kStFused,
             kStKpRender, kStKpVjp, kStKpAdam };

// Brackets one launch with profiling events when the plan profiles.
struct StageScope {
  Plan& p;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  StageScope(Plan& plan, int st, cudaStream_t stream);
  ~StageScope();
};

// plan.cu
prop_status plan_build(const prop_plan_desc* d, Plan** out, DeviceAllocator* alloc = nullptr);
void plan_free(Plan* p);
cudaError_t plan_dev_alloc(Plan* p, void** ptr, size_t bytes);
void plan_dev_free(Plan* p, void* ptr);
prop_status plan_ensure_recon(Plan* p, int iters);
// Upper bound of the device bytes a plan for `d` holds once it has
// reconstructed (tables, workspace, optimiser state); 0 if `d` is invalid.
size_t plan_estimate_bytes(const prop_plan_desc* d, int iters);
// One Adam iteration k (1-based) from Vin into Vout; L(Vin) -> *loss_dst (device).
// rows_ready: the plan's row workspace holds the forward row transform of Vin
// (left by the previous step with next_rows); next_rows: leave the forward
// row transform of Vout there.  Both only take effect with one bin chunk.
struct AdamArgs;
// Loss L(V) (data term + TV with a.tv_xy, a.tv_t, a.tv_eps; a.gscale = 2) into
// *loss_out (device) and dL/dRe V + i dL/dIm V into grad (may be p.grad).
prop_status loss_grad_device(Plan& p, const float2* y, const AdamArgs& a, const float2* V, float2* grad,
                             double* loss_out, cudaStream_t s);
prop_status plan_step(Plan& p, const float2* y, const prop_recon_params* q, int k, const float2* Vin,
                      float2* Vout, double* loss_dst, cudaStream_t s, bool rows_ready = false,
                      bool next_rows = false);

// fft.cu: the four line-FFT passes of the 2-D (i)FFT per bin chunk.
// Forward: V chunk -> rows (deapodise, pad, FFT along x1) -> grid (pad, FFT along x2).
// Adjoint: grid -> rows (iFFT along u2, crop) -> out chunk (iFFT along u1, crop, deapodise, scale).
cudaError_t fft_forward_rows(const Plan& p, const float2* V, int f0, cudaStream_t s);
cudaError_t fft_forward_cols(const Plan& p, cudaStream_t s);
cudaError_t fft_adjoint_cols(const Plan& p, cudaStream_t s);
cudaError_t fft_adjoint_rows(const Plan& p, float2* out, int f0, float scale, cudaStream_t s);
cudaError_t fft_configure(int n);
// proj.cu: tables and workspace of the projection model; `images`: also the
// per-blade image spectra.
prop_status plan_ensure_proj(Plan& p, bool images);
// Centred unitary 2-D DFT of one N x N image, [i2][i1] <-> [u2][u1] (projection
// model): one pass of N-point transforms over the rows or the columns.
enum CartPass { kCartRowsFwd = 0, kCartColsFwd = 1, kCartColsInv = 2, kCartRowsInv = 3 };
struct CartLoss {              // blade data term fused into the forward column pass
  const float2* y;             // [N][N] k-space data of the blade
  const float2* yimg;          // [N][N] DFT of the blade's image, or null (image term against y)
  float wk, wi;                // k-space and image-space weights
  const Reducer* red;          // >= N/16 partials
  const double* loss_const;    // added to the data loss (image term outside the mask), or null
  double* loss_out;
};
// kCartColsFwd writes Z * scale masked by `mask` (when given), or with `loss`
// the data-term gradient 2 M (wk (Z - y) + wi (Z - yimg)) and the loss;
// kCartColsInv masks its input by `mask` (when given).  Rows passes and the
// inverse column pass multiply by `scale`.
cudaError_t cart_fft_pass(int N, int pass, const float2* src, float2* dst, const float2* twiddleN,
                          const uint8_t* mask, const CartLoss* loss, float scale, cudaStream_t s);
cudaError_t cart_fft_configure(int N);
// Builds the column passes' tensor maps (after the workspaces exist) and
// decides whether the staged column kernels fit this plan; never fails the
// plan (the unstaged kernels remain).
void fft_make_maps(Plan& p);

// nufft.cu
// Interpolation of the grid chunk at every blade sample, times the
// displacement phase, summed over the chunk's bins, scaled by s.
// mode 0: y = part, 1: y += part; y_meas != null subtracts the measurement
// (first chunk). With red != null the final |y|^2 is reduced into *sumsq.
// contrib != null also writes conj(P) * (final value) per bin for the spread.
cudaError_t interp(const Plan& p, int f0, int nbins, float2* y, const float2* y_meas,
                   bool accumulate, const Reducer* red, double* sumsq, float2* contrib, cudaStream_t s);
// Adjoint spread of r into the grid chunk: contrib[m][f] = conj(P[j_m][f0+f]) r_m,
// then every cell gathers sum_{(m, w) in its list} w contrib[m][f] (every cell written).
cudaError_t nufft_configure(int smem_optin);
int interp_buffers(const Plan& p);
// contrib_ready: p.contrib already holds this chunk's phased residual (fused by interp).
cudaError_t spread(const Plan& p, int f0, int nbins, const float2* r, bool contrib_ready, cudaStream_t s);
// r = y_sum - y_meas, the FP64 sum of |r|^2 into *sumsq (device, reduced with `red`), and with
// with_contrib (single bin chunk) the spread's phased residual of every bin.
cudaError_t residual(const Plan& p, const float2* y_sum, const float2* y_meas, float2* r, bool with_contrib,
                     const Reducer& red, double* sumsq, cudaStream_t s);

// optim.cu
struct AdamArgs {
  float lr_t;        // lr / (1 - beta1^k)
  float inv_bc2_sqrt;// 1 / sqrt(1 - beta2^k)
  float beta1, beta2, eps;
  float tv_xy, tv_t, tv_eps;
  float gscale;      // factor on the adjoint (2 for the squared-L2 data term)
};
// Fused smoothed-TV gradient + Adam: Vout = Adam(Vin, gscale*g + TV grads).
// Writes data + tv_xy*TV_xy + tv_t*TV_t of Vin into loss_out[0] when red != null.
cudaError_t tv_adam(const Plan& p, const float2* Vin, const float2* g, float2* m, float2* v,
                    float2* Vout, const AdamArgs& a, const Reducer* red,
                    const double* data_loss, double* loss_out, cudaStream_t s);
// grad = gscale * g + TV grads (no update); loss as above.
cudaError_t tv_grad(const Plan& p, const float2* V, const float2* g, float2* grad,
                    const AdamArgs& a, const Reducer* red, const double* data_loss,
                    double* loss_out, cudaStream_t s);
cudaError_t render(const Plan& p, const float2* V, int f_lo, int f_hi, float2* img, cudaStream_t s);
// PSNR of |img| against |ref| over `count` complex values: 10 log10(max|ref|^2 / mean (|img| - |ref|)^2)
// into *out (device); scratch: p.psnr_scratch with p.psnr_cap block partials.
cudaError_t psnr(const Plan& p, const float2* img, const float2* ref, long count, double* out, cudaStream_t s);

// Multi-problem launches (a batch of plans with the same transform length
// 2N, bin stride and kernel width, one bin chunk each): one launch per stage
// serves every plan of the batch; each plan's results are the same bit for
// bit as from its own launches.
struct BatchIter {
  Plan* p;
  const float2* Vin;    // V_{k-1}
  float2* Vout;         // V_k
  AdamArgs aa;          // Adam step k
  double* loss_out;     // L(V_{k-1})
  bool fwd_tail;        // leave the forward row transform of V_k in p->rows
};
// Splits `total` persistent CTAs over `count` problems in proportion to
// their work (every problem gets at least one and at most cap[i]);
// begin[count + 1] receives the CTA ranges; returns the CTAs used.
inline int split_ctas(const long* work, const int* cap, int count, int total, int* begin) {
  long sum = 0;
  for (int i = 0; i < count; ++i) sum += work[i] > 0 ? work[i] : 1;
  int c[kMaxBatch];
  int used = 0;
  for (int i = 0; i < count; ++i) {
    const long w = work[i] > 0 ? work[i] : 1;
    c[i] = (int)((w * (long)total) / (sum > 0 ? sum : 1));
    c[i] = c[i] < 1 ? 1 : (c[i] > cap[i] ? cap[i] : c[i]);
    used += c[i];
  }
  // hand leftover CTAs to the problems with the most work per CTA
  while (used < total) {
    int best = -1;
    double br = 0.0;
    for (int i = 0; i < count; ++i)
      if (c[i] < cap[i]) {
        const double r = (double)(work[i] > 0 ? work[i] : 1) / c[i];
        if (best < 0 || r > br) {
          best = i;
          br = r;
        }
      }
    if (best < 0) break;
    ++c[best];
    ++used;
  }
  begin[0] = 0;
  for (int i = 0; i < count; ++i) begin[i + 1] = begin[i] + c[i];
  return begin[count];
}
cudaError_t fft_forward_cols_batch(Plan* const* ps, int count, cudaStream_t s);
cudaError_t fft_adjoint_cols_batch(Plan* const* ps, int count, cudaStream_t s);
cudaError_t fused_rows_update_batch(const BatchIter* it, int count, cudaStream_t s);
// nufft.cu: the residual interpolation (each plan: its own y and measured
// data, residual into p->resid, phased residual into p->contrib, FP64 |r|^2
// into p->scalars) and the spread of p->contrib into p->grid.
cudaError_t interp_residual_batch(Plan* const* ps, const float2* const* y_meas, int count, cudaStream_t s);
cudaError_t spread_batch(Plan* const* ps, int count, cudaStream_t s);
// api.cu: one Adam iteration of every member, the stages launched once for
// the whole batch (members share 2N, bin stride and kernel width and have one
// bin chunk each; batch_compatible says whether two plans can share).
struct BatchMember {
  Plan* p;
  const float2* y;               // measured data (device)
  const prop_recon_params* q;
  int k;                         // iteration (1-based)
  const float2* Vin;
  float2* Vout;
  double* loss_dst;              // device: L(Vin)
  bool rows_ready;               // p->rows holds the forward row transform of Vin
  bool next_rows;                // leave the forward row transform of Vout in p->rows
};
bool batch_compatible(const Plan& a, const Plan& b);
prop_status batch_step(BatchMember* mb, int count, cudaStream_t s);

// fft.cu, single bin chunk only: the inverse row FFT of p.rows (the last
// adjoint pass) fused with TV + Adam (Vin -> Vout, moments m, v) and, with
// fwd_tail, the forward row FFT of Vout into p.rows for the next iteration.
// Loss as in tv_adam.
cudaError_t fused_rows_update(const Plan& p, const float2* Vin, float2* m, float2* v, float2* Vout,
                              const AdamArgs& aa, const Reducer* red, const double* data_loss, double* loss_out,
                              bool fwd_tail, cudaStream_t s);

}  // namespace prop

struct prop_plan_s {
  prop::Plan* p;
};
