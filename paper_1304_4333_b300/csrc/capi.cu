// C ABI of the SPS library: context lifecycle, data encoding and the likelihood entry points.

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sps {

DevBuf::~DevBuf() {
  if (ptr) cudaFree(ptr);
}

namespace {
std::atomic<uint64_t> g_buffer_generation{0};
}

uint64_t buffer_generation() { return g_buffer_generation.load(std::memory_order_relaxed); }

cudaError_t DevBuf::reserve(size_t nbytes) {
  if (nbytes <= bytes && ptr) return cudaSuccess;
  g_buffer_generation.fetch_add(1, std::memory_order_relaxed);
  if (ptr) {
    cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  if (nbytes == 0) nbytes = 16;
  cudaError_t e = cudaMalloc(&ptr, nbytes);
  if (e == cudaSuccess) bytes = nbytes;
  else ptr = nullptr;
  return e;
}

}  // namespace sps

sps_ctx::~sps_ctx() {
  for (cudaEvent_t e : hot_events) cudaEventDestroy(e);
  for (cudaEvent_t e : copy_events) cudaEventDestroy(e);
}

namespace sps {

sps_status fail(sps_ctx* ctx, sps_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Columns with every value exactly representable in BF16 (0/1 dummies, the intercept, small
// integers) need no low part.
__global__ void nonexact_columns_kernel(const double* __restrict__ X, int64_t n, int k,
                                        int* __restrict__ nonexact, int* __restrict__ nonfinite) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= n * k) return;
  const double v = X[idx];
  if (!isfinite(v)) {
    atomicOr(nonfinite, 1);
    return;
  }
  const int col = static_cast<int>(idx % k);
  const double h = static_cast<double>(__bfloat162float(__double2bfloat16(v)));
  if (h != v) atomicOr(&nonexact[col], 1);
}

// Packed operand rows of X: [Xh over k16 | Xl over kc16 | 0], internal column order; and the
// FP32 copy in the original order.
__global__ void encode_x_kernel(const double* __restrict__ X, int64_t n, int k,
                                const int* __restrict__ perm, int k16, int kc, int kx,
                                __nv_bfloat16* __restrict__ Xp, float* __restrict__ Xf) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= n * kx) return;
  const int64_t s = idx / kx;
  const int e = static_cast<int>(idx - s * kx);
  double v = 0.0;
  if (e < k16) {
    if (e < k) v = static_cast<double>(__bfloat162float(__double2bfloat16(X[s * k + perm[e]])));
  } else if (e - k16 < kc) {
    const double x = X[s * k + perm[e - k16]];
    v = x - static_cast<double>(__bfloat162float(__double2bfloat16(x)));
  }
  Xp[idx] = __double2bfloat16(v);
  if (e < k) Xf[s * k + e] = static_cast<float>(X[s * k + e]);
}

// lin[c*k + i] = prefix[tile] + sum over the remaining rows s in [128*tile, t) of w_c(y_s) x_{s,i}.
// One warp per output: lanes take every 32nd row, then a shuffle sum (FP64).
__global__ void lin_tail_kernel(const double* __restrict__ prefix, const double* __restrict__ X,
                                const int* __restrict__ y, int k, int NC, int64_t t,
                                double* __restrict__ lin) {
  const int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (idx >= NC * k) return;
  const int c = idx / k;
  const int i = idx - c * k;
  const int64_t tile = t / 128;
  double a = 0.0;
  for (int64_t s = tile * 128 + lane; s < t; s += 32) {
    const int ys = y[s];
    const double w = (NC == 1) ? (ys == 1 ? 0.5 : -0.5) : (ys == c + 1 ? 1.0 : 0.0);
    a = fma(w, X[s * k + i], a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) lin[idx] = prefix[tile * NC * k + idx] + a;
}

sps_status to_device(sps_ctx* ctx, DevBuf& buf, const void* host, size_t bytes) {
  SPS_CUDA_TRY(buf.reserve(bytes));
  SPS_CUDA_TRY(cudaMemcpy(buf.ptr, host, bytes, cudaMemcpyHostToDevice));
  return SPS_OK;
}

// FP32 copy (the library's FP64 -> FP32 conversion) of a full prior precision matrix.
__global__ void prec_to_f32_kernel(const double* __restrict__ p, int64_t n, float* __restrict__ out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = f64_to_f32(p[i]);
}

// Lower Cholesky factor of a symmetric positive definite matrix (host FP64, row-major).
bool cholesky_host(const std::vector<double>& A, int D, std::vector<double>& L) {
  L.assign(static_cast<size_t>(D) * D, 0.0);
  for (int j = 0; j < D; ++j) {
    double s = A[j * D + j];
    for (int m = 0; m < j; ++m) s -= L[j * D + m] * L[j * D + m];
    if (!(s > 0.0) || !std::isfinite(s)) return false;
    const double d = std::sqrt(s);
    L[j * D + j] = d;
    for (int i = j + 1; i < D; ++i) {
      double r = A[i * D + j];
      for (int m = 0; m < j; ++m) r -= L[i * D + m] * L[j * D + m];
      L[i * D + j] = r / d;
    }
  }
  return true;
}

// Validate a prior for the context's D and install it: mean, covariance, host Cholesky factor,
// device mean, precision (diagonal for ISO/DIAG, full inverse for FULL) and factor. Nothing of
// the context changes when the prior is rejected.
sps_status apply_prior(sps_ctx* ctx, const sps_prior* prior) {
  const int D = ctx->D;
  if (!prior || !prior->cov_or_sd) return fail(ctx, SPS_ERR_INVALID_ARG, "prior: covariance missing");
  std::vector<double> mean(D, 0.0), cov(static_cast<size_t>(D) * D, 0.0), chol;
  if (prior->mean)
    for (int i = 0; i < D; ++i) mean[i] = prior->mean[i];
  if (prior->kind == SPS_PRIOR_ISO) {
    const double sd = prior->cov_or_sd[0];
    if (!(sd > 0.0) || !std::isfinite(sd)) return fail(ctx, SPS_ERR_INVALID_ARG, "prior: bad sd");
    for (int i = 0; i < D; ++i) cov[i * D + i] = sd * sd;
  } else if (prior->kind == SPS_PRIOR_DIAG) {
    for (int i = 0; i < D; ++i) {
      const double sd = prior->cov_or_sd[i];
      if (!(sd > 0.0) || !std::isfinite(sd)) return fail(ctx, SPS_ERR_INVALID_ARG, "prior: bad sd");
      cov[i * D + i] = sd * sd;
    }
  } else if (prior->kind == SPS_PRIOR_FULL) {
    for (int i = 0; i < D * D; ++i) cov[i] = prior->cov_or_sd[i];
  } else {
    return fail(ctx, SPS_ERR_INVALID_ARG, "prior: unknown kind");
  }
  for (double v : mean)
    if (!std::isfinite(v)) return fail(ctx, SPS_ERR_INVALID_ARG, "prior: non-finite mean");
  if (!cholesky_host(cov, D, chol)) return fail(ctx, SPS_ERR_INVALID_ARG, "prior covariance is not positive definite");
  std::vector<double> prec;
  if (prior->kind == SPS_PRIOR_FULL) {
    std::vector<double> Linv(static_cast<size_t>(D) * D, 0.0);
    for (int j = 0; j < D; ++j) {
      Linv[j * D + j] = 1.0 / chol[j * D + j];
      for (int i = j + 1; i < D; ++i) {
        double a = 0.0;
        for (int m = j; m < i; ++m) a += chol[i * D + m] * Linv[m * D + j];
        Linv[i * D + j] = -a / chol[i * D + i];
      }
    }
    prec.assign(static_cast<size_t>(D) * D, 0.0);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double a = 0.0;
        for (int m = std::max(i, j); m < D; ++m) a += Linv[m * D + i] * Linv[m * D + j];
        prec[i * D + j] = a;
      }
  } else {
    prec.resize(D);
    for (int i = 0; i < D; ++i) prec[i] = 1.0 / cov[i * D + i];
  }
  if (prior->kind == SPS_PRIOR_FULL) {
    // FP64 precision matrix followed by its FP32 conversion (read by the prior log kernel)
    const size_t dd = static_cast<size_t>(D) * D;
    SPS_CUDA_TRY(ctx->d_prior_prec.reserve(dd * sizeof(double) + dd * sizeof(float)));
    SPS_CUDA_TRY(cudaMemcpy(ctx->d_prior_prec.ptr, prec.data(), dd * sizeof(double), cudaMemcpyHostToDevice));
    prec_to_f32_kernel<<<static_cast<unsigned>((dd + 255) / 256), 256>>>(
        ctx->d_prior_prec.as<double>(), static_cast<int64_t>(dd),
        reinterpret_cast<float*>(ctx->d_prior_prec.as<double>() + dd)); ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
    SPS_CUDA_TRY(cudaDeviceSynchronize());
  } else {
    SPS_TRY(to_device(ctx, ctx->d_prior_prec, prec.data(), prec.size() * sizeof(double)));
  }
  SPS_TRY(to_device(ctx, ctx->d_prior_mean, mean.data(), D * sizeof(double)));
  SPS_TRY(to_device(ctx, ctx->d_prior_chol, chol.data(), chol.size() * sizeof(double)));
  ctx->prior_kind = prior->kind;
  ctx->prior_mean = mean;
  ctx->prior_cov = cov;
  ctx->prior_chol = chol;
  return SPS_OK;
}

// X'X [k x k] in FP64: one block per lower-triangle entry (i >= j), threads over observations.
__global__ void xtx_kernel(const double* __restrict__ X, int64_t n, int k, double* __restrict__ out) {
  __shared__ double sh[32];
  int i = 0, e = blockIdx.x;
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  const int j = e - i * (i + 1) / 2;
  double a = 0.0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) a = fma(X[t * k + i], X[t * k + j], a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += sh[w];
    out[i * k + j] = s;
    out[j * k + i] = s;
  }
}

}  // namespace

sps_status make_map_bf16(sps_ctx* ctx, CUtensorMap* map, const void* base, uint64_t rows,
                         uint64_t cols, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(ctx, SPS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t gdim[2] = {cols, rows};
  cuuint64_t gstride[1] = {cols * sizeof(__nv_bfloat16)};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim, gstride, box,
                  estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char msg[96];
    snprintf(msg, sizeof msg, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return fail(ctx, SPS_ERR_CUDA, msg);
  }
  return SPS_OK;
}

sps_status ensure_lin(sps_ctx* ctx, int64_t t) {
  if (ctx->lin_t == t) return SPS_OK;
  const int nk = ctx->NC * ctx->k;
  lin_tail_kernel<<<(nk + 3) / 4, 128, 0, ctx->stream>>>(ctx->lin_prefix.as<double>(), ctx->Xd.as<double>(),
                                                            ctx->y.as<int>(), ctx->k, ctx->NC, t,
                                                            ctx->lin.as<double>()); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  // inside a stream capture the kernel only runs if the graph does: leave the cache as it was
  if (!ctx->capturing) ctx->lin_t = t;
  return SPS_OK;
}

void hot_begin(sps_ctx* ctx) {
  if (!ctx->timing || ctx->capturing) return;
  if (ctx->hot_used + 2 > ctx->hot_events.size()) {
    for (int q = 0; q < 2; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      ctx->hot_events.push_back(e);
    }
  }
  cudaEventRecord(ctx->hot_events[ctx->hot_used], ctx->stream);
}

void hot_end(sps_ctx* ctx) {
  if (!ctx->timing || ctx->capturing || ctx->hot_used + 2 > ctx->hot_events.size()) return;
  cudaEventRecord(ctx->hot_events[ctx->hot_used + 1], ctx->stream);
  ctx->hot_used += 2;
}

sps_status loglik_dispatch(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll,
                           int precision) {
  if (precision == SPS_PREC_FP32) return loglik_fp32(ctx, d_theta, P, t, d_ll);
  if (precision == SPS_PREC_SPLIT) return loglik_split(ctx, d_theta, P, t, d_ll);
  return fail(ctx, SPS_ERR_INVALID_ARG, "unknown precision");
}

}  // namespace sps

using namespace sps;

extern "C" {

void sps_options_default(sps_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->ess_fraction = 0.5;
  o->h_init = 0.5;
  o->h_step = 0.01;
  o->h_min = 0.1;
  o->h_max = 1.0;
  o->target_accept = 0.25;
  o->rne_cycle = 0.35;
  o->rne_final = 0.9;
  o->r_max = 200;
  o->precision = SPS_PREC_SPLIT;
  o->mkernel = SPS_MKERNEL_RW;
  o->cphase_block = 64;
  o->mala_target_accept = 0.5;
  o->seed = 0;
  o->resampling = SPS_RESAMPLE_MULTINOMIAL;
  o->graphs = 1;
}

const char* sps_status_string(sps_status s) {
  switch (s) {
    case SPS_OK: return "ok";
    case SPS_ERR_INVALID_ARG: return "invalid argument";
    case SPS_ERR_CUDA: return "CUDA error";
    case SPS_ERR_OOM: return "out of device memory";
    case SPS_ERR_DEGENERATE: return "degenerate particle set (proposal covariance not positive definite)";
    case SPS_ERR_NONFINITE: return "non-finite log-likelihood";
    case SPS_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPS_ERR_STATE: return "call out of order";
    case SPS_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* sps_last_error(const sps_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

sps_status sps_get_dims(const sps_ctx* ctx, int64_t* n, int32_t* k, int32_t* C, int32_t* D) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (n) *n = ctx->n;
  if (k) *k = ctx->k;
  if (C) *C = ctx->C;
  if (D) *D = ctx->D;
  return SPS_OK;
}

sps_status sps_loglik_batched(sps_ctx* ctx, int32_t M, const int32_t* k_models, const int64_t* P_models,
                              const int64_t* t_models, const double* theta, double* ll) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (M < 1 || M > 1024 || !k_models || !P_models || !t_models || !theta || !ll)
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_loglik_batched: bad arguments");
  for (int m = 0; m < M; ++m)
    if (k_models[m] < 1 || k_models[m] > ctx->k || P_models[m] < 1 || t_models[m] < 0 || t_models[m] > ctx->n)
      return fail(ctx, SPS_ERR_INVALID_ARG, "sps_loglik_batched: bad model sizes");
  std::vector<const double*> th(M);
  std::vector<double*> out(M);
  int64_t thoff = 0, poff = 0;
  for (int m = 0; m < M; ++m) {
    th[m] = theta + thoff;
    out[m] = ll + poff;
    thoff += P_models[m] * ctx->NC * k_models[m];
    poff += P_models[m];
  }
  return loglik_split_batched(ctx, M, k_models, P_models, t_models, th.data(), out.data());
}

sps_status sps_autotune(sps_ctx* ctx, int64_t P, int64_t t, sps_tune_result* out) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (P < 1 || P > (int64_t{1} << 28) || t < 1 || t > ctx->n)
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_autotune: bad P or t");
  return tc_autotune(ctx, P, t, out);
}

sps_status sps_set_prior(sps_ctx* ctx, const sps_prior* prior) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  return apply_prior(ctx, prior);
}

sps_status sps_prior_normalize(int32_t k, int32_t n_outcomes, const double* mu, const double* Sigma,
                               double* mean_out, double* cov_out) {
  if (k < 1 || n_outcomes < 2 || !mu || !Sigma || !mean_out || !cov_out) return SPS_ERR_INVALID_ARG;
  const int C = n_outcomes, D = k * (C - 1);
  for (int a = 1; a < C; ++a)
    for (int i = 0; i < k; ++i) mean_out[(a - 1) * k + i] = mu[a * k + i] - mu[i];
  const size_t kk = static_cast<size_t>(k) * k;
  for (int a = 1; a < C; ++a)
    for (int b = 1; b < C; ++b)
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
          double v = Sigma[i * k + j];                       // Sigma_0
          if (a == b) v += Sigma[a * kk + i * k + j];        // + Sigma_a on the diagonal blocks
          cov_out[static_cast<size_t>((a - 1) * k + i) * D + (b - 1) * k + j] = v;
        }
  return SPS_OK;
}

sps_status sps_gprior(sps_ctx* ctx, double g, double* mean_out, double* cov_out) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!(g > 0.0) || !std::isfinite(g) || !mean_out || !cov_out)
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_gprior: bad arguments");
  const int k = ctx->k, C = ctx->C;
  DevBuf d;
  SPS_CUDA_TRY(d.reserve(sizeof(double) * k * k));
  xtx_kernel<<<k * (k + 1) / 2, 256, 0, ctx->stream>>>(ctx->Xd.as<double>(), ctx->n, k, d.as<double>()); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  std::vector<double> A(static_cast<size_t>(k) * k), L;
  SPS_CUDA_TRY(cudaMemcpyAsync(A.data(), d.ptr, sizeof(double) * k * k, cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (!cholesky_host(A, k, L)) return fail(ctx, SPS_ERR_DEGENERATE, "sps_gprior: X'X is singular");
  // (X'X)^-1 = L^-T L^-1 from the inverse of the Cholesky factor
  std::vector<double> Linv(static_cast<size_t>(k) * k, 0.0), S(static_cast<size_t>(k) * k, 0.0);
  for (int j = 0; j < k; ++j) {
    Linv[j * k + j] = 1.0 / L[j * k + j];
    for (int i = j + 1; i < k; ++i) {
      double a = 0.0;
      for (int m = j; m < i; ++m) a += L[i * k + m] * Linv[m * k + j];
      Linv[i * k + j] = -a / L[i * k + i];
    }
  }
  const double scale = g * static_cast<double>(ctx->n);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double a = 0.0;
      for (int m = std::max(i, j); m < k; ++m) a += Linv[m * k + i] * Linv[m * k + j];
      S[i * k + j] = scale * a;
    }
  std::vector<double> mu(static_cast<size_t>(C) * k, 0.0), Sig(static_cast<size_t>(C) * k * k);
  for (int c = 0; c < C; ++c) std::copy(S.begin(), S.end(), Sig.begin() + static_cast<size_t>(c) * k * k);
  return sps_prior_normalize(k, C, mu.data(), Sig.data(), mean_out, cov_out);
}

sps_status sps_set_stream(sps_ctx* ctx, void* stream) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return SPS_OK;
}

void sps_destroy(sps_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  delete ctx;
}

sps_status sps_set_timing(sps_ctx* ctx, int32_t on) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  ctx->timing = (on != 0);
  return SPS_OK;
}

sps_status sps_set_debug(sps_ctx* ctx, int32_t stall_producer, uint64_t timeout_ns) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  ctx->debug_stall = stall_producer != 0;
  ctx->debug_timeout_ns = timeout_ns;
  return SPS_OK;
}

sps_status sps_counters(sps_ctx* ctx, int32_t reset, int64_t* launches, int64_t* hot_launches, double* hot_ms) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  double ms = 0.0;
  for (size_t q = 0; q + 1 < ctx->hot_used; q += 2) {
    float e = 0.f;
    SPS_CUDA_TRY(cudaEventElapsedTime(&e, ctx->hot_events[q], ctx->hot_events[q + 1]));
    ms += e;
  }
  if (launches) *launches = ctx->launches;
  if (hot_launches) *hot_launches = static_cast<int64_t>(ctx->hot_used / 2);
  if (hot_ms) *hot_ms = ms;
  if (reset) {
    ctx->launches = 0;
    ctx->hot_used = 0;
  }
  return SPS_OK;
}

sps_status sps_init(sps_ctx** out, const double* X, int64_t n, int32_t k, const int32_t* y,
                    int32_t n_outcomes, const sps_prior* prior, const sps_options* opt) {
  if (!out) return SPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!X || !y || !prior || n < 1 || k < 1 || k > 256 || n_outcomes < 2 || n_outcomes > 16 ||
      n > (1LL << 31) - 256)
    return SPS_ERR_INVALID_ARG;
  for (int64_t s = 0; s < n; ++s)
    if (y[s] < 0 || y[s] >= n_outcomes) return SPS_ERR_INVALID_ARG;
  sps_ctx* ctx = new sps_ctx();
  auto bail = [&](sps_status s) {
    delete ctx;
    return s;
  };
  if (opt) ctx->opt = *opt;
  else sps_options_default(&ctx->opt);
  ctx->n = n;
  ctx->k = k;
  ctx->C = n_outcomes;
  ctx->NC = n_outcomes - 1;
  ctx->D = k * ctx->NC;
  const int NC = ctx->NC;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(SPS_ERR_CUDA);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) return bail(SPS_ERR_CUDA);
  ctx->num_sms = prop.multiProcessorCount;

  // ---- prior
  if (const sps_status ps = apply_prior(ctx, prior); ps != SPS_OK) return bail(ps);

  // ---- data
  sps_status st;
  if ((st = to_device(ctx, ctx->Xd, X, static_cast<size_t>(n) * k * sizeof(double))) != SPS_OK) return bail(st);
  if ((st = to_device(ctx, ctx->y, y, static_cast<size_t>(n) * sizeof(int32_t))) != SPS_OK) return bail(st);
  {
    DevBuf flags;
    if (flags.reserve((k + 1) * sizeof(int)) != cudaSuccess) return bail(SPS_ERR_OOM);
    cudaMemset(flags.ptr, 0, (k + 1) * sizeof(int));
    const int64_t tot = n * k;
    nonexact_columns_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256>>>(
        ctx->Xd.as<double>(), n, k, flags.as<int>(), flags.as<int>() + k); ++ctx->launches;
    std::vector<int> h(k + 1);
    if (cudaMemcpy(h.data(), flags.ptr, (k + 1) * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return bail(SPS_ERR_CUDA);
    if (h[k]) {
      ctx->last_error = "X holds non-finite values";
      return bail(SPS_ERR_INVALID_ARG);
    }
    XEncoding& enc = ctx->enc;
    enc.k = k;
    enc.perm.clear();
    for (int j = 0; j < k; ++j)
      if (h[j]) enc.perm.push_back(j);
    enc.kc = static_cast<int>(enc.perm.size());
    for (int j = 0; j < k; ++j)
      if (!h[j]) enc.perm.push_back(j);
    enc.k16 = (k + 15) / 16 * 16;
    enc.kc16 = (enc.kc + 15) / 16 * 16;
    enc.kx = (enc.k16 + enc.kc16 + 63) / 64 * 64;
    enc.kt = (2 * enc.k16 + 63) / 64 * 64;
    enc.bn = (NC <= 3) ? tc_tile_rows(NC, enc.kx, enc.kt, 1) : 0;
    if ((st = to_device(ctx, enc.perm_dev, enc.perm.data(), k * sizeof(int))) != SPS_OK) return bail(st);
    if (enc.Xp.reserve(static_cast<size_t>(n) * enc.kx * 2) != cudaSuccess ||
        ctx->Xf.reserve(static_cast<size_t>(n) * k * 4) != cudaSuccess)
      return bail(SPS_ERR_OOM);
    const int64_t tot2 = n * enc.kx;
    encode_x_kernel<<<static_cast<unsigned>((tot2 + 255) / 256), 256>>>(
        ctx->Xd.as<double>(), n, k, enc.perm_dev.as<int>(), enc.k16, enc.kc, enc.kx,
        enc.Xp.as<__nv_bfloat16>(), ctx->Xf.as<float>()); ++ctx->launches;
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(SPS_ERR_CUDA);
    if (enc.bn > 0 && (st = tc_configure_cluster(ctx)) != SPS_OK) return bail(st);
    if (enc.bn > 0 && (st = make_map_bf16(ctx, &enc.mapX, enc.Xp.ptr, n, enc.kx, enc.bn / enc.cl)) != SPS_OK)
      return bail(st);
  }
  // covariate means and prefix sums of the linear term, host FP64 in observation order
  {
    ctx->xbar_host.assign(k, 0.0);
    const int64_t ntiles = n / 128 + 1;
    std::vector<double> pre(static_cast<size_t>(ntiles) * NC * k, 0.0);
    std::vector<double> run(static_cast<size_t>(NC) * k, 0.0);
    for (int64_t s = 0; s < n; ++s) {
      if (s % 128 == 0) std::copy(run.begin(), run.end(), pre.begin() + (s / 128) * NC * k);
      const double* xs = X + s * k;
      for (int i = 0; i < k; ++i) ctx->xbar_host[i] += xs[i];
      for (int c = 0; c < NC; ++c) {
        const double w = (NC == 1) ? (y[s] == 1 ? 0.5 : -0.5) : (y[s] == c + 1 ? 1.0 : 0.0);
        if (w == 0.0) continue;
        for (int i = 0; i < k; ++i) run[c * k + i] += w * xs[i];
      }
    }
    if (n % 128 == 0) std::copy(run.begin(), run.end(), pre.begin() + (n / 128) * NC * k);
    for (int i = 0; i < k; ++i) ctx->xbar_host[i] /= static_cast<double>(n);
    if ((st = to_device(ctx, ctx->lin_prefix, pre.data(), pre.size() * sizeof(double))) != SPS_OK) return bail(st);
    if ((st = to_device(ctx, ctx->xbar, ctx->xbar_host.data(), k * sizeof(double))) != SPS_OK) return bail(st);
    if (ctx->lin.reserve(static_cast<size_t>(NC) * k * sizeof(double)) != cudaSuccess) return bail(SPS_ERR_OOM);
  }
  *out = ctx;
  return SPS_OK;
}

static sps_status check_finite_ll(sps_ctx* ctx, const double* h_ll, int64_t P) {
  for (int64_t p = 0; p < P; ++p)
    if (!std::isfinite(h_ll[p])) return fail(ctx, SPS_ERR_NONFINITE, "non-finite log-likelihood");
  return SPS_OK;
}

// Split-precision log-likelihood of host-resident particles in slices: theta is copied slice by
// slice on a second stream while the fused kernel runs on the slices already on the device, and
// each slice's results are copied back as soon as they are final. At 65 536 particles and
// k = 30 the host-to-device copy (15.7 MB) takes about twice as long as the kernel, so without
// slices the two add up; with them the call takes about the copy plus one slice's kernel.
// Results equal those of one call on all particles up to the order of the FP32/FP64 partial
// sums (the observation chunking of a launch depends on its particle count).
static constexpr int64_t kHostSlice = 16384;   // particles per slice at least
static constexpr int kMaxHostSlices = 8;

static sps_status loglik_host_sliced(sps_ctx* ctx, const double* theta, int64_t P, int64_t t, double* ll) {
  LoglikScratch& S = ctx->ll;
  const int64_t D = ctx->D;
  const int ns = static_cast<int>(std::min<int64_t>(kMaxHostSlices, P / kHostSlice));
  const int64_t per = ((P + ns - 1) / ns + 255) / 256 * 256;   // whole 256-particle tile pairs
  if (!ctx->copy_stream) {
    const cudaError_t e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      ctx->copy_stream = nullptr;
      return fail(ctx, SPS_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
  }
  while (ctx->copy_events.size() < static_cast<size_t>(ns) + 1) {
    cudaEvent_t e;
    SPS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->copy_events.push_back(e);
  }
  SPS_CUDA_TRY(S.aux.reserve(kMaxHostSlices * sizeof(int)));
  int* d_flags = S.aux.as<int>();
  double* d_theta = S.theta_in.as<double>();
  double* d_ll = S.ll_out.as<double>();
  cudaEvent_t* ev = ctx->copy_events.data();
  // the copies overwrite theta_in: they start after all earlier work on the context's stream
  SPS_CUDA_TRY(cudaEventRecord(ev[ns], ctx->stream));
  SPS_CUDA_TRY(cudaStreamWaitEvent(ctx->copy_stream, ev[ns], 0));
  auto finish = [&](sps_status st) {
    // no copy of the caller's buffer may still run when the call returns
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamSynchronize(ctx->stream);
    return st;
  };
  int used = 0;
  for (int i = 0; i < ns; ++i) {
    const int64_t off = i * per, cnt = std::min(per, P - off);
    if (cnt <= 0) break;
    const cudaError_t e = cudaMemcpyAsync(d_theta + off * D, theta + off * D, cnt * D * sizeof(double),
                                          cudaMemcpyHostToDevice, ctx->copy_stream);
    if (e != cudaSuccess) return finish(fail(ctx, SPS_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e)));
    if (cudaEventRecord(ev[i], ctx->copy_stream) != cudaSuccess)
      return finish(fail(ctx, SPS_ERR_CUDA, "cudaEventRecord"));
    ++used;
  }
  for (int i = 0; i < used; ++i) {
    const int64_t off = i * per, cnt = std::min(per, P - off);
    if (cudaStreamWaitEvent(ctx->stream, ev[i], 0) != cudaSuccess)
      return finish(fail(ctx, SPS_ERR_CUDA, "cudaStreamWaitEvent"));
    const sps_status st = loglik_split(ctx, d_theta + off * D, cnt, t, d_ll + off);
    if (st != SPS_OK) return finish(st);
    // each launch clears the timeout flag: keep this slice's flag
    cudaError_t e = cudaMemcpyAsync(d_flags + i, S.flag.ptr, sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ll + off, d_ll + off, cnt * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return finish(fail(ctx, SPS_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e)));
  }
  int flags[kMaxHostSlices] = {};
  cudaError_t e = cudaMemcpyAsync(flags, d_flags, used * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  finish(SPS_OK);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("sliced loglik: ") + cudaGetErrorString(e));
  for (int i = 0; i < used; ++i)
    if (flags[i]) return fail(ctx, SPS_ERR_TIMEOUT, "loglik kernel: bounded wait timed out");
  return check_finite_ll(ctx, ll, P);
}

sps_status sps_loglik(sps_ctx* ctx, const double* theta, int64_t P, int64_t t, double* ll,
                      int32_t precision, int32_t mem) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!theta || !ll || P < 1 || t < 0 || t > ctx->n || P > (1LL << 28))
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_loglik: bad arguments");
  if (mem == SPS_MEM_DEVICE) return loglik_dispatch(ctx, theta, P, t, ll, precision);
  if (mem != SPS_MEM_HOST) return fail(ctx, SPS_ERR_INVALID_ARG, "sps_loglik: bad mem kind");
  LoglikScratch& S = ctx->ll;
  const size_t tb = static_cast<size_t>(P) * ctx->D * sizeof(double);
  SPS_CUDA_TRY(S.theta_in.reserve(tb));
  SPS_CUDA_TRY(S.ll_out.reserve(P * sizeof(double)));
  if (precision == SPS_PREC_SPLIT && P >= 2 * kHostSlice && !ctx->capturing)
    return loglik_host_sliced(ctx, theta, P, t, ll);
  SPS_CUDA_TRY(cudaMemcpyAsync(S.theta_in.ptr, theta, tb, cudaMemcpyHostToDevice, ctx->stream));
  SPS_TRY(loglik_dispatch(ctx, S.theta_in.as<double>(), P, t, S.ll_out.as<double>(), precision));
  SPS_CUDA_TRY(cudaMemcpyAsync(ll, S.ll_out.ptr, P * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (precision == SPS_PREC_SPLIT) {
    int flag = 0;
    SPS_CUDA_TRY(cudaMemcpy(&flag, S.flag.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(ctx, SPS_ERR_TIMEOUT, "loglik kernel: bounded wait timed out");
  }
  return check_finite_ll(ctx, ll, P);
}

}  // extern "C"

extern "C" sps_status sps_loglik_grad(sps_ctx* ctx, const double* theta, int64_t P, int64_t t, double* ll,
                                      double* grad, int32_t mem) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!theta || !ll || !grad || P < 1 || t < 0 || t > ctx->n || P > (1LL << 28))
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_loglik_grad: bad arguments");
  if (mem == SPS_MEM_DEVICE) return loglik_grad_dispatch(ctx, theta, P, t, ll, grad);
  LoglikScratch& S = ctx->ll;
  const size_t tb = static_cast<size_t>(P) * ctx->D * sizeof(double);
  SPS_CUDA_TRY(S.theta_in.reserve(tb));
  SPS_CUDA_TRY(S.ll_out.reserve(P * sizeof(double)));
  SPS_CUDA_TRY(S.grad_out.reserve(tb));
  SPS_CUDA_TRY(cudaMemcpyAsync(S.theta_in.ptr, theta, tb, cudaMemcpyHostToDevice, ctx->stream));
  SPS_TRY(loglik_grad_dispatch(ctx, S.theta_in.as<double>(), P, t, S.ll_out.as<double>(), S.grad_out.as<double>()));
  SPS_CUDA_TRY(cudaMemcpyAsync(ll, S.ll_out.ptr, P * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(grad, S.grad_out.ptr, tb, cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return check_finite_ll(ctx, ll, P);
}
