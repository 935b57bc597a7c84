// Internal declarations of the SPS library: context and state structures, status handling,
// and the inline-PTX wrappers (mbarrier, TMA, tcgen05) the sm_103a kernels use.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "sps.h"

namespace sps {

// ------------------------------------------------------------------------------------------
// Status plumbing

#define SPS_CUDA_TRY(expr)                                                           \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) {                                                         \
      return ::sps::fail(ctx, _e == cudaErrorMemoryAllocation ? SPS_ERR_OOM          \
                                                              : SPS_ERR_CUDA,        \
                         std::string(#expr) + ": " + cudaGetErrorString(_e));        \
    }                                                                                \
  } while (0)

#define SPS_TRY(expr)                  \
  do {                                 \
    sps_status _s = (expr);            \
    if (_s != SPS_OK) return _s;       \
  } while (0)

// ------------------------------------------------------------------------------------------
// Device buffers owned by the context or a state. Growth only; freed in the destructor.

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  ~DevBuf();
  cudaError_t reserve(size_t nbytes);
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Encoding of X for the tensor-core path. Columns are permuted so that the columns that are not
// exact in BF16 ("continuous") come first. Each observation row holds [Xh | Xl]:
// Xh = bf16(x) in elements [0, k16), Xl = bf16(x - Xh) of the continuous columns in
// [k16, k16 + kc16) (k16, kc16: k and kc rounded up to 16), zero padding up to kx (a multiple of
// 64, the 128-byte swizzle row). Theta operand rows hold [bf16(theta log2 e) | low part] in
// [0, k16) and [k16, 2 k16), padded to kt.
struct XEncoding {
  int k = 0, kc = 0;          // covariates, continuous covariates
  int k16 = 0, kc16 = 0;      // k and kc rounded up to 16 (MMA K step)
  int kx = 0, kt = 0;         // row widths of the X and theta operands (multiples of 64)
  int bn = 0;                 // observation rows per tile; 0: no tile fits
  int cl = 1;                 // 1: one CTA per work item; 2: a CTA pair issuing 256-row MMAs,
                              // each CTA holding bn / 2 rows of every X tile (TMA box {64, bn / cl})
  int max_clusters = 0;       // co-resident clusters of the fused kernel at this shape
  int chunk_obs = 0;          // observations per work item chosen by the autotuner (0: heuristic)
  std::vector<int> perm;      // internal column j holds original column perm[j]
  DevBuf perm_dev;            // int [k]
  DevBuf invperm_dev;         // int [k]: internal column of original column i (gradient kernel)
  DevBuf Xp;                  // bf16 [n x kx]
  CUtensorMap mapX;
};

// Encoding of the first k_m covariates for batched calls of nested models: the same layout as
// XEncoding for X[:, :k_m] (continuous columns of the model first), so that a model's tiles in a
// batched launch issue exactly the MMAs, and load exactly the X bytes, of its own launch.
struct ModelEncoding {
  int k = 0, kc = 0, k16 = 0, kc16 = 0, kx = 0;
  DevBuf perm_dev;            // int [k]: internal column j holds original column perm[j]
  DevBuf Xp;                  // bf16 [n x kx]
};

// Per model of a batched launch (device table, one entry per model of the call): its X tiles'
// tensor map and the K blocks and MMA slices of its rows.
struct BatchModel {
  CUtensorMap mapX;
  int kbx;                    // K blocks of an X row
  int k16;                    // element offset of the theta low parts
  int ksh;                    // 16-wide K slices over Xh (and Th, Tl)
  int ksl;                    // over Xl
};

// A prepared launch of the batched fused kernel (loglik_split_batched_prepare): its tables are in
// device memory, so it can be launched, or captured into a graph, without host copies.
struct SplitBatchedPlan;

// Per-call scratch of the likelihood kernels.
struct LoglikScratch {
  DevBuf thetaP;              // bf16 [NC * Ppad x kt] operand rows (class-major row blocks)
  int64_t ppad_cap = 0;       // particle capacity of thetaP
  CUtensorMap mapT;
  DevBuf partial;             // FP64 partial sums [slices x Ppad]
  DevBuf flag;                // int error/timeout flag
  DevBuf theta_in, ll_out, grad_out, aux;   // staging for host-memory calls
  DevBuf gpartial;            // FP32 [n_chunks x Ppad x NC ng] gradient partial sums (tensor cores)
  CUtensorMap mapXg;          // X tiles of the gradient kernel (box rows mapXg_rows)
  int mapXg_rows = 0;
  DevBuf batch_lin;           // FP64 [M x NC x k] linear terms of the models
  DevBuf batch_models;        // BatchModel [M]
  std::shared_ptr<SplitBatchedPlan> bplan[2];   // prepared batched launches (two slots)
};

// Device-resident control block of a captured M phase: the step size h and the Philox step word
// of the next M step, the steps taken so far, the stop flag and an error code (1: Cholesky
// failure, 2: non-finite proposal log-likelihood).
struct StepCtl {
  double h;
  unsigned long long step;
  int r;
  int r_max;
  int stop;
  int err;
};

// Device-resident control of a captured C phase (one per state): the block of observations in
// progress, decided on the device from the ESS of the previous block's rows.
struct CphaseCtl {
  int64_t range[2];   // observations [s, s + b) of the block in progress
  int64_t block;      // rows of that block before the cap at the data's end (doubles up to max_rows)
  int64_t max_rows;
  int64_t n;
  int64_t P;
  int64_t t_new;      // the phase's end, once done
  int64_t row;        // the block row that the advance step reads
  int64_t blocks;     // blocks run
  double frac;        // ESS fraction of the stopping rule
  int done;
  int err;
};

// Incremented by every device-buffer (re)allocation: a captured graph whose generation differs
// may point at freed memory and is captured again.
uint64_t buffer_generation();

}  // namespace sps

struct sps_ctx {
  int device = 0;
  int num_sms = 148;
  cudaStream_t stream = nullptr;
  int64_t n = 0;
  int k = 0, C = 2, NC = 1, D = 0;
  sps_options opt;
  std::string last_error;

  // data
  sps::XEncoding enc;
  sps::DevBuf Xd;             // FP64 [n x k] original column order
  sps::DevBuf Xf;             // FP32 [n x k] original column order (FP32 path, C phase)
  sps::DevBuf y;              // int32 [n]
  sps::DevBuf xbar;           // FP64 [k] covariate means over all n observations
  std::vector<double> xbar_host;
  // linear term of the split path: lin(t) [NC x k] FP64 (original order), cached by t.
  // binary: sum_{s<t} (y_s - 1/2) x_s; C > 2: sum_{s<t, y_s = c} x_s for c = 1..C-1.
  sps::DevBuf lin;
  int64_t lin_t = -1;
  sps::DevBuf lin_prefix;     // FP64 [(n/128 + 1) x NC x k] prefix sums at 128-row boundaries
  // prior: N(mean, cov) on the D free coefficients
  int prior_kind = SPS_PRIOR_ISO;
  std::vector<double> prior_mean, prior_cov, prior_chol;
  sps::DevBuf d_prior_mean;   // FP64 [D]
  sps::DevBuf d_prior_prec;   // FP64 [D x D] (FULL) or [D] diagonal precision (ISO / DIAG)
  sps::DevBuf d_prior_chol;   // FP64 [D x D] lower Cholesky factor of cov

  sps::LoglikScratch ll;
  std::map<int, std::unique_ptr<sps::ModelEncoding>> model_enc;   // by k_m, built on first use

  // instrumentation: kernels launched on this context; CUDA events around each launch of the
  // fused log-likelihood kernel when timing is on
  int64_t launches = 0;
  bool timing = false;
  // diagnostics (sps_set_debug): wall limit of the fused kernel's bounded waits (0: 2 s) and a
  // switch that makes its TMA producer issue no copy, so that the waits run out
  uint64_t debug_timeout_ns = 0;
  int debug_stall = 0;
  bool capturing = false;                // stream capture in progress: no event records
  cudaStream_t cap_stream = nullptr;     // private non-blocking stream for graph capture (the
                                         // legacy default stream cannot be captured)
  cudaStream_t copy_stream = nullptr;    // host-memory calls: theta slices are copied here
  std::vector<cudaEvent_t> copy_events;  // one per slice, plus one ordering event
  std::vector<cudaEvent_t> hot_events;   // pairs (start, stop)
  size_t hot_used = 0;                   // events in use (2 per recorded launch)
  ~sps_ctx();
};

struct sps_state {
  sps_ctx* ctx = nullptr;
  int32_t J = 0, N = 0;
  int64_t P = 0;
  uint64_t seed = 0;
  int64_t t = 0;
  double h = 0.5;
  bool have_weights = false;      // a C phase has run since the last S phase
  bool ll_stale = false;          // ll holds C-phase sums: recompute with the M-phase kernel
  int ll_kind = -1;               // function that produced ll: 0 split, 1 FP32, 2 gradient kernel
  bool grad_valid = false;        // grad holds the log-likelihood gradient of theta at t
  uint64_t step_counter = 0;      // Philox counter word for per-step streams
  uint64_t cycle_counter = 0;
  sps::DevBuf theta, theta_prop;  // FP64 [P x D]
  sps::DevBuf ll, ll_prop;        // FP64 [P]
  sps::DevBuf lp, lp_prop;        // FP64 [P] prior log kernel
  sps::DevBuf logw;               // FP64 [P]
  sps::DevBuf logml;              // FP64 [J]
  sps::DevBuf lwbuf;              // float2 [block x P] C-phase running log weights (Kahan pairs)
  sps::DevBuf lwstate;            // float2 [P] running log weights at the start of a C-phase block
  sps::DevBuf gmax;               // FP64 [J] group maxima of logw (S-phase weight scale)
  sps::DevBuf lpl_dev;            // FP64 [block x J] per-group log-mean-exp of C-phase rows
  sps::DevBuf ess_buf;            // FP64 [block] ESS per observation of a block
  sps::DevBuf idx;                // int32 [P]
  sps::DevBuf scratch;            // moments, covariance partials, counters
  sps::DevBuf cov;                // FP64 [D x D]
  sps::DevBuf chol;               // FP64 [D x D]
  sps::DevBuf counters;           // int/unsigned counters (accepts, error flags)
  sps::DevBuf grad, grad_prop;    // FP64 [P x D] (MALA)
  sps::DevBuf zq;                 // FP32 [P x D] MALA: 1/2 L' g(theta) + z of the current proposal
  sps::DevBuf z2;                 // FP64 [P] MALA: |z|^2 of the current proposal
  std::vector<double> host_tmp;
  // captured M phase: one M step and its control kernel inside a conditional WHILE node, valid
  // while the key (prefix, kernel, precision, buffer generation and addresses) is unchanged
  cudaGraphExec_t mgraph = nullptr;
  struct MKey {
    int64_t t = -1;
    int kernel = -1, precision = -1, sig = 0;
    uint64_t gen = 0;
    const void* bufs[8] = {};
    bool operator==(const MKey& o) const {
      if (t != o.t || kernel != o.kernel || precision != o.precision || sig != o.sig || gen != o.gen) return false;
      for (int i = 0; i < 8; ++i)
        if (bufs[i] != o.bufs[i]) return false;
      return true;
    }
  } mkey;
  int64_t mgraph_launches = 0;    // kernels of one captured step (control kernel included)
  sps::DevBuf ctl;                // StepCtl
  sps::DevBuf steplog;            // FP64 [r_max x 3]: h, acceptance rate, min RNE of each step
  void* pinned = nullptr;         // page-locked host copy of an M step's counters and sums
  size_t pinned_bytes = 0;
  sps::DevBuf sigmalog;           // FP64 [r_max x D x D]: Sigma of each step (recorded schedules)
  int64_t graph_steps = 0;        // M steps run inside captured graphs
};

namespace sps {

// Record an error on ctx and return its status.
sps_status fail(sps_ctx* ctx, sps_status s, const std::string& msg);
inline sps_status fail(const sps_ctx* ctx, sps_status s, const std::string& msg) {
  return fail(const_cast<sps_ctx*>(ctx), s, msg);
}

// Build a 2D bf16 tensor map with 128-byte swizzle: rows x cols (cols contiguous, multiple of
// 64), box {64, box_rows}.
sps_status make_map_bf16(sps_ctx* ctx, CUtensorMap* map, const void* base, uint64_t rows,
                         uint64_t cols, uint32_t box_rows);

// Likelihood launchers (loglik_tc.cu, loglik_simt.cu). Device pointers, context stream.
sps_status loglik_split(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll);
// Batched nested models (see sps_loglik_batched): one fused-kernel launch for all of them; model
// m's particles at device d_theta[m] ([P_m x k_m NC]), its results to d_ll[m] ([P_m]).
// skip (optional, [M]): models whose particle tiles are skipped (their results are not
// defined); the work decomposition is the same with and without skips.
sps_status loglik_split_batched(sps_ctx* ctx, int M, const int32_t* km, const int64_t* Pm, const int64_t* tm,
                                const double* const* d_theta, double* const* d_ll, const char* skip = nullptr);
// The same call in two parts: prepare (tables and operand encodings in device memory, the launch
// shape kept in the context's plan slot 0 or 1; tiles receives each model's particle-tile range
// [x, y) of the table of prefix lengths) and launch (kernels only: no allocation, no host copy,
// so it can be captured). *ptile_table receives that table (int2 {prefix length, slot} per
// particle tile). The two slots' launches share the operand and partial-sum buffers: they must
// run one after the other.
sps_status loglik_split_batched_prepare(sps_ctx* ctx, int plan_slot, int M, const int32_t* km, const int64_t* Pm,
                                        const int64_t* tm, const double* const* d_theta, double* const* d_ll,
                                        const char* skip, std::vector<int2>* tiles, int2** ptile_table);
sps_status loglik_split_batched_launch(sps_ctx* ctx, int plan_slot);
sps_status loglik_fp32(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll);
sps_status loglik_dispatch(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll,
                           int precision);
sps_status ensure_lin(sps_ctx* ctx, int64_t t);
// Observation rows per tensor-core tile for NC = C - 1 outcomes and operand widths kx, kt.
int tc_tile_rows(int NC, int kx, int kt, int CL);
// Cluster size of the fused kernel for the context's tile shape (sets enc.cl, enc.max_clusters):
// 2 when clusters of two fit on the device, else 1; SPS_TC_CLUSTER=1 in the environment forces 1.
sps_status tc_configure_cluster(sps_ctx* ctx);
// Waves of work items of one split-precision call of P particles at prefix t on the persistent
// grid (work items / items run at once); 0 when the context has no tensor-core tile.
double tc_waves(const sps_ctx* ctx, int64_t P, int64_t t);
// Tile-shape autotuner (sps_autotune).
sps_status tc_autotune(sps_ctx* ctx, int64_t P, int64_t t, sps_tune_result* out);
// Start/stop event of one timed launch of the fused kernel (no-ops when timing is off).
void hot_begin(sps_ctx* ctx);
void hot_end(sps_ctx* ctx);
// C-phase running log weights for observations [s_lo, s_hi): d_lw[j*P + p] = d_lw_in[p] plus the
// terms of observations s_lo..s_lo+j, as Kahan pairs (s, c) of value s - c. With d_range the
// block is [d_range[0], d_range[1]) read on the device (s_lo, s_hi ignored).
sps_status cphase_increments(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t s_lo,
                             int64_t s_hi, const float2* d_lw_in, float2* d_lw, const int64_t* d_range = nullptr);
// Log-likelihood and gradient (FP32 products, FP64 sums across 32-observation tiles).
// Log-likelihood and gradient with the tensor cores (split precision; C - 1 <= 2 and covariate
// widths whose gradient accumulators fit TMEM); SPS_ERR_UNSUPPORTED otherwise, nothing launched.
sps_status loglik_grad_tc(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll, double* d_grad);
// The context's gradient function: tensor cores in split precision where supported, else the
// FP32 SIMT kernel. Deterministic for a context and shape.
sps_status loglik_grad_dispatch(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll,
                                double* d_grad);
sps_status loglik_grad_fp32(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll,
                            double* d_grad);

}  // namespace sps

// ------------------------------------------------------------------------------------------
// FP64 <-> FP32 conversions by integer operations. FP64 arithmetic and conversion instructions
// run at about 1.5-1.8 per clock per SM on this GPU (FP32: 128), so element-wise code converts
// with these and keeps FP64 instructions for reductions.

namespace sps {

// double -> float, rounding toward zero (relative error < 2^-23). Zero and values below the
// float normal range give a signed zero, values above it a signed infinity, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
  const unsigned sign = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  if (e <= 896u) return __uint_as_float(sign);                          // |d| < 2^-126
  if (e >= 1151u)                                                        // |d| >= 2^128, inf, NaN
    return __uint_as_float(sign | 0x7F800000u | ((e == 0x7FFu && ((hi & 0xFFFFFu) | lo)) ? 0x400000u : 0u));
  return __uint_as_float(sign | ((e - 896u) << 23) | m);
}

// float -> double, exact (float subnormals give a signed zero).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  unsigned hi;
  if (e == 0u) hi = sign;
  else if (e == 0xFFu) hi = sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
  else hi = sign | ((e + 896u) << 20) | (m >> 3);
  const unsigned lo = (e == 0u || e == 0xFFu) ? 0u : (m << 29);
  return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(hi) << 32) | lo));
}

}  // namespace sps

// ------------------------------------------------------------------------------------------
// Inline PTX wrappers (device). Written for sm_103a.

namespace sps {
namespace ptx {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}

// As mbar_try_wait with acquire semantics at cluster scope: for phases completed by arrives
// from the other CTA of a pair.
__device__ __forceinline__ uint32_t mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase. Gives up when *abort becomes non-zero or after
// `limit_ns` of wall time; returns false in both cases (and sets *abort on a timeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ bool mbar_wait_bounded_cluster(uint64_t* bar, uint32_t parity,
                                                          volatile int* abort, uint64_t limit_ns) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (*abort) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster: arrive (release) and wait (acquire).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---- tcgen05 ----

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, bf16 inputs, fp32 accumulate, one CTA; and the
// arrive on `bar` once all MMAs issued so far by the issuing thread have completed. Warp-wide:
// every lane of the issuing warp executes them with the same operands (so that the operands are
// computed in warp-uniform code) and only the lane with issue != 0 issues.
__device__ __forceinline__ void mma_bf16_if(uint32_t issue, uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "setp.ne.b32 q, %5, 0;\n\t"
      "@q tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(issue)
      : "memory");
}
__device__ __forceinline__ void mma_commit_if(uint32_t issue, uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "setp.ne.b32 q, %1, 0;\n\t"
      "@q tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_u32(bar)),
      "r"(issue)
      : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem desc]: A (128 rows x 16 bf16) from tensor memory, two bf16 per
// 32-bit column, row i in lane i. Warp-wide: all lanes execute it with the same operands, lanes
// with issue != 0 (one) issue.
__device__ __forceinline__ void mma_bf16_ts_if(uint32_t issue, uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "setp.ne.b32 q, %5, 0;\n\t"
      "@q tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(issue)
      : "memory");
}

// 128 TMEM lanes x 256 bits (8 columns) from the rows of a shared-memory operand tile: row i of
// the 16-element K slice described by `sdesc` (the layout an MMA reads) into lane i. Issued by
// the lanes with issue != 0 (one).
__device__ __forceinline__ void tmem_cp_128x256b_if(uint32_t issue, uint32_t taddr, uint64_t sdesc) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "setp.ne.b32 q, %2, 0;\n\t"
      "@q tcgen05.cp.cta_group::1.128x256b [%0], %1;\n\t}" ::"r"(taddr), "l"(sdesc), "r"(issue)
      : "memory");
}

// ---- CTA pairs (cta_group::2): one MMA of 256 rows over the two CTAs of a cluster ----

__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D[tmem of both CTAs] (+)= A * B^T over the CTA pair: rows 0-127 of A (and of D) in the even
// CTA, 128-255 in the odd one; each CTA holds half of B's rows. Issued by the even CTA only; the
// descriptors' shared-memory addresses are read at the same offsets in both CTAs. The commit
// arrives once on the mbarrier at the offset of `bar` in every CTA of `cta_mask` when all pair
// MMAs issued so far by the issuing thread have completed. Warp-wide, as mma_bf16_if.
__device__ __forceinline__ void mma_bf16_pair_if(uint32_t issue, uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                                 uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "setp.ne.b32 q, %5, 0;\n\t"
      "@q tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(issue)
      : "memory");
}
__device__ __forceinline__ void mma_commit_pair_if(uint32_t issue, uint64_t* bar, uint16_t cta_mask) {
  asm volatile(
      "{\n\t.reg .pred q;\n\t"
      "setp.ne.b32 q, %2, 0;\n\t"
      "@q tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;\n\t}" ::"r"(smem_u32(bar)), "h"(cta_mask), "r"(issue)
      : "memory");
}

// Address in the shared::cluster window of the variable at the offset of `p` in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

// Arrive (release at cluster scope) on an mbarrier of another CTA of the cluster.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread i of the warp gets lane (base + i).
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, float (&v)[32]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, float (&v)[16]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
// 32 lanes x 8 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld_32x32b_x8(uint32_t taddr, float (&v)[8]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with 128-byte
// swizzle: rows of 128 bytes, 8-row swizzle atoms 1024 bytes apart (stride byte offset),
// descriptor version 1, swizzle mode 2 (128B). The leading byte offset is unused in this mode.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1u) << 16;
  d |= static_cast<uint64_t>(1024u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(2u) << 61;
  return d;
}

// Instruction descriptor for kind::f16 with bf16 A/B, fp32 D, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

}  // namespace ptx
}  // namespace sps
