// Plain FP32 SIMT log-likelihood (the baseline path) and the C-phase increment kernel; a
// register-resident variant serves models with k <= 64 and C <= 4 (k <= 32 for C > 2).
//
// Both evaluate, per particle and observation, the log probability of the observed outcome of
// the multinomial logit (Eq. 1, Sec. 2.1) in FP32: eta_c = theta_c' x_s (eta_0 = 0),
// term = eta_{y_s} - (m + log(exp(-m) + sum_c exp(eta_c - m))), m = max(0, eta_1..eta_{C-1}),
// one thread per particle, 128 particles per block, theta transposed in shared memory so that
// each thread reads its own column without bank conflicts and X rows are broadcast.
// Sums over observations are FP32 within a 32-observation tile and FP64 across tiles.

#include <algorithm>

#include "common.cuh"

namespace sps {
namespace {

constexpr int kP = 128;    // particles per block
constexpr int kTS = 32;    // observations per shared-memory tile

// Load theta [P x D] (FP64) of particles p0..p0+127 into sm[D][128] FP32.
__device__ __forceinline__ void load_theta_t(float* sm, const double* __restrict__ theta, int64_t P,
                                             int D, int64_t p0) {
  for (int idx = threadIdx.x; idx < D * kP; idx += blockDim.x) {
    const int pp = idx / D;
    const int d = idx - pp * D;
    const int64_t p = p0 + pp;
    sm[d * kP + pp] = (p < P) ? f64_to_f32(theta[p * D + d]) : 0.f;
  }
}

// Log probability of outcome yo for linear predictors eta[1..NC] (eta[0] = 0), FP32.
__device__ __forceinline__ float logit_term(const float* eta, int NC, int yo) {
  float m = 0.f;
  for (int c = 0; c < NC; ++c) m = fmaxf(m, eta[c]);
  float s = expf(-m);
  for (int c = 0; c < NC; ++c) s += expf(eta[c] - m);
  const float obs = (yo == 0) ? 0.f : eta[yo - 1];
  return obs - (m + logf(s));
}

constexpr int kMaxNC = 15;

// Running C-phase log weight kept as a Kahan pair (s, c), value s - c: one FP32 add of the term
// and three FP32 operations of compensation per observation, about FP64-accumulation accuracy
// for FP32 terms without FP64 instructions.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Each thread: particle p0 + threadIdx.x; observations [s_lo, s_hi).
// mode 0: out[blockIdx.y * P + p] = sum of terms (FP64 across tiles);
// mode 1: C-phase increments: lw_out[j * P + p] = lw_in[p] + sum_{s_lo <= s' <= s_lo + j} term,
//         as Kahan pairs.
__global__ void __launch_bounds__(kP)
fp32_terms_kernel(const double* __restrict__ theta, int64_t P, int k, int NC,
                  const float* __restrict__ X, const int* __restrict__ y, int64_t s_begin,
                  int64_t s_end, int64_t chunk, int mode, double* __restrict__ out,
                  float2* __restrict__ lw_out, const float2* __restrict__ lw_in,
                  const int64_t* __restrict__ range) {
  extern __shared__ float smf[];
  if (range) {   // a C-phase block whose observations [range[0], range[1]) are decided on the device
    s_begin = range[0];
    s_end = range[1];
    chunk = s_end - s_begin;
  }
  const int D = k * NC;
  float* th = smf;                          // [D][128]
  float* xs = th + D * kP;                  // [kTS][k]
  int* ys = reinterpret_cast<int*>(xs + kTS * k);   // [kTS]
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kP;
  const int64_t p = p0 + threadIdx.x;
  const int64_t s_lo = s_begin + static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t s_hi = (s_lo + chunk < s_end) ? s_lo + chunk : s_end;
  load_theta_t(th, theta, P, D, p0);
  double acc = 0.0;
  float ks = 0.f, kc = 0.f;
  if (mode == 1 && p < P) {
    const float2 v = lw_in[p];
    ks = v.x;
    kc = v.y;
  }
  float eta[kMaxNC];
  for (int64_t s0 = s_lo; s0 < s_hi; s0 += kTS) {
    const int ns = static_cast<int>(s_hi - s0 < kTS ? s_hi - s0 : kTS);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ns * k; idx += blockDim.x) xs[idx] = X[s0 * k + idx];
    for (int idx = threadIdx.x; idx < ns; idx += blockDim.x) ys[idx] = y[s0 + idx];
    __syncthreads();
    float tile = 0.f;
    for (int j = 0; j < ns; ++j) {
      const float* xr = xs + j * k;
      for (int c = 0; c < NC; ++c) {
        const float* tc = th + (c * k) * kP + threadIdx.x;
        float e = 0.f;
        for (int i = 0; i < k; ++i) e = fmaf(tc[i * kP], xr[i], e);
        eta[c] = e;
      }
      const float term = logit_term(eta, NC, ys[j]);
      if (mode == 1) {
        kahan_add(ks, kc, term);
        if (p < P) lw_out[(s0 - s_lo + j) * P + p] = make_float2(ks, kc);
      } else {
        tile += term;
      }
    }
    if (mode == 0) acc += f32_to_f64(tile);
  }
  if (mode == 0 && p < P) out[static_cast<int64_t>(blockIdx.y) * P + p] = acc;
}

// Register-resident variant for small models (k <= KMAX, NC = C - 1 fixed): each thread keeps
// its particle's theta in registers; X rows are staged in shared memory padded with zeros to KMAX
// and read as broadcast float4. Same arithmetic and outputs as fp32_terms_kernel.
template <int KMAX, int NC>
__global__ void __launch_bounds__(kP)
fp32_terms_reg_kernel(const double* __restrict__ theta, int64_t P, int k, const float* __restrict__ X,
                      const int* __restrict__ y, int64_t s_begin, int64_t s_end, int64_t chunk, int mode,
                      double* __restrict__ out, float2* __restrict__ lw_out, const float2* __restrict__ lw_in,
                      const int64_t* __restrict__ range) {
  __shared__ __align__(16) float xs[kTS][KMAX];
  __shared__ int ys[kTS];
  if (range) {
    s_begin = range[0];
    s_end = range[1];
    chunk = s_end - s_begin;
  }
  const int D = k * NC;
  const int64_t p = static_cast<int64_t>(blockIdx.x) * kP + threadIdx.x;
  const int64_t s_lo = s_begin + static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t s_hi = (s_lo + chunk < s_end) ? s_lo + chunk : s_end;
  float th[NC][KMAX];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int i = 0; i < KMAX; ++i) th[c][i] = (p < P && i < k) ? f64_to_f32(theta[p * D + c * k + i]) : 0.f;
  double acc = 0.0;
  float ks = 0.f, kc = 0.f;
  if (mode == 1 && p < P) {
    const float2 v = lw_in[p];
    ks = v.x;
    kc = v.y;
  }
  for (int64_t s0 = s_lo; s0 < s_hi; s0 += kTS) {
    const int ns = static_cast<int>(s_hi - s0 < kTS ? s_hi - s0 : kTS);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTS * KMAX; idx += blockDim.x) {
      const int j = idx / KMAX, i = idx - j * KMAX;
      xs[j][i] = (j < ns && i < k) ? X[(s0 + j) * k + i] : 0.f;
    }
    for (int idx = threadIdx.x; idx < ns; idx += blockDim.x) ys[idx] = y[s0 + idx];
    __syncthreads();
    float tile = 0.f;
    for (int j = 0; j < ns; ++j) {
      float eta[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) eta[c] = 0.f;
#pragma unroll
      for (int i = 0; i < KMAX; i += 4) {
        const float4 xv = *reinterpret_cast<const float4*>(&xs[j][i]);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          eta[c] = fmaf(th[c][i], xv.x, eta[c]);
          eta[c] = fmaf(th[c][i + 1], xv.y, eta[c]);
          eta[c] = fmaf(th[c][i + 2], xv.z, eta[c]);
          eta[c] = fmaf(th[c][i + 3], xv.w, eta[c]);
        }
      }
      const float term = logit_term(eta, NC, ys[j]);
      if (mode == 1) {
        kahan_add(ks, kc, term);
        if (p < P) lw_out[(s0 - s_lo + j) * P + p] = make_float2(ks, kc);
      } else {
        tile += term;
      }
    }
    if (mode == 0) acc += f32_to_f64(tile);
  }
  if (mode == 0 && p < P) out[static_cast<int64_t>(blockIdx.y) * P + p] = acc;
}

// Launch the register variant when the model fits one of its instantiations.
bool launch_reg(sps_ctx* ctx, dim3 grid, const double* theta, int64_t P, int64_t s_begin, int64_t s_end,
                int64_t chunk, int mode, double* out, float2* lw_out, const float2* lw_in,
                const int64_t* range = nullptr) {
  const int k = ctx->k, NC = ctx->NC;
  const float* X = ctx->Xf.as<float>();
  const int* y = ctx->y.as<int>();
#define SPS_REG_CASE(KM, NCM)                                                                          \
  if (NC == NCM && k <= KM) {                                                                          \
    fp32_terms_reg_kernel<KM, NCM><<<grid, kP, 0, ctx->stream>>>(theta, P, k, X, y, s_begin, s_end, chunk, \
                                                                 mode, out, lw_out, lw_in, range);     \
    ++ctx->launches;                                                                                   \
    return true;                                                                                       \
  }
  SPS_REG_CASE(8, 1)
  SPS_REG_CASE(32, 1)
  SPS_REG_CASE(64, 1)
  SPS_REG_CASE(8, 2)
  SPS_REG_CASE(32, 2)
  SPS_REG_CASE(8, 3)
  SPS_REG_CASE(32, 3)
#undef SPS_REG_CASE
  return false;
}

__global__ void sum_slices_kernel(const double* __restrict__ partial, int64_t P, int slices,
                                  double* __restrict__ ll) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= P) return;
  double s = 0.0;
  for (int q = 0; q < slices; ++q) s += partial[static_cast<int64_t>(q) * P + p];
  ll[p] = s;
}

size_t fp32_smem(int k, int NC) {
  return sizeof(float) * (static_cast<size_t>(k) * NC * kP + static_cast<size_t>(kTS) * k) +
         sizeof(int) * kTS;
}

}  // namespace

sps_status loglik_fp32(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll) {
  if (ctx->NC > kMaxNC) return fail(ctx, SPS_ERR_UNSUPPORTED, "FP32 path supports at most 16 outcomes");
  const size_t smem = fp32_smem(ctx->k, ctx->NC);
  if (smem > 200 * 1024) return fail(ctx, SPS_ERR_UNSUPPORTED, "FP32 path: k*(C-1) too large");
  const int64_t ptiles = (P + kP - 1) / kP;
  int64_t chunks = 1;
  if (t > 0) {
    const int64_t want = 8LL * ctx->num_sms;
    chunks = std::max<int64_t>(1, std::min<int64_t>((want + ptiles - 1) / ptiles, (t + kTS - 1) / kTS));
  }
  int64_t chunk = (t + chunks - 1) / chunks;
  chunk = std::max<int64_t>(kTS, (chunk + kTS - 1) / kTS * kTS);
  chunks = std::max<int64_t>(1, (t + chunk - 1) / chunk);
  SPS_CUDA_TRY(ctx->ll.partial.reserve(static_cast<size_t>(chunks) * P * sizeof(double)));
  double* partial = ctx->ll.partial.as<double>();
  dim3 grid(static_cast<unsigned>(ptiles), static_cast<unsigned>(chunks));
  if (!launch_reg(ctx, grid, d_theta, P, 0, t, chunk, 0, partial, nullptr, nullptr)) {
    SPS_CUDA_TRY(cudaFuncSetAttribute(fp32_terms_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
    fp32_terms_kernel<<<grid, kP, smem, ctx->stream>>>(d_theta, P, ctx->k, ctx->NC, ctx->Xf.as<float>(),
                                                       ctx->y.as<int>(), 0, t, chunk, 0, partial, nullptr,
                                                       nullptr, nullptr); ++ctx->launches;
  }
  SPS_CUDA_TRY(cudaGetLastError());
  sum_slices_kernel<<<static_cast<unsigned>((P + 255) / 256), 256, 0, ctx->stream>>>(
      partial, P, t > 0 ? static_cast<int>(chunks) : 0, d_ll); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

sps_status cphase_increments(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t s_lo,
                             int64_t s_hi, const float2* d_lw_in, float2* d_lw, const int64_t* d_range) {
  const size_t smem = fp32_smem(ctx->k, ctx->NC);
  if (ctx->NC > kMaxNC || smem > 200 * 1024)
    return fail(ctx, SPS_ERR_UNSUPPORTED, "C phase: k*(C-1) too large");
  const int64_t ptiles = (P + kP - 1) / kP;
  dim3 grid(static_cast<unsigned>(ptiles), 1);
  if (!launch_reg(ctx, grid, d_theta, P, s_lo, s_hi, s_hi - s_lo, 1, nullptr, d_lw, d_lw_in, d_range)) {
    SPS_CUDA_TRY(cudaFuncSetAttribute(fp32_terms_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
    fp32_terms_kernel<<<grid, kP, smem, ctx->stream>>>(d_theta, P, ctx->k, ctx->NC, ctx->Xf.as<float>(),
                                                       ctx->y.as<int>(), s_lo, s_hi, s_hi - s_lo, 1, nullptr,
                                                       d_lw, d_lw_in, d_range); ++ctx->launches;
  }
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps

// ------------------------------------------------------------------------------------------
// Gradient of the log-likelihood, d ll / d theta_c = sum_{s<=t} (1[y_s = c] - p_{s,c}) x_s (the
// derivative of Eq. 1 summed over observations). One thread per particle, 64 particles per
// block; residual-times-covariate products accumulate in FP32 over a 32-observation tile (in
// shared memory, [D][64]) and are added to FP64 accumulators once per tile.

namespace sps {
namespace {

constexpr int kGP = 64;

__global__ void __launch_bounds__(kGP)
grad_fp32_kernel(const double* __restrict__ theta, int64_t P, int k, int NC, const float* __restrict__ X,
                 const int* __restrict__ y, int64_t t, int64_t chunk, double* __restrict__ llp,
                 double* __restrict__ gp) {
  extern __shared__ double smd[];
  const int D = k * NC;
  double* g64 = smd;                                   // [D][64]
  float* th = reinterpret_cast<float*>(g64 + D * kGP); // [D][64]
  float* g32 = th + D * kGP;                           // [D][64]
  float* xs = g32 + D * kGP;                           // [kTS][k]
  int* ys = reinterpret_cast<int*>(xs + kTS * k);      // [kTS]
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kGP;
  const int64_t p = p0 + threadIdx.x;
  const int64_t s_lo = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t s_hi = (s_lo + chunk < t) ? s_lo + chunk : t;
  for (int idx = threadIdx.x; idx < D * kGP; idx += blockDim.x) {
    const int pp = idx / D, d = idx - pp * D;
    th[d * kGP + pp] = (p0 + pp < P) ? static_cast<float>(theta[(p0 + pp) * D + d]) : 0.f;
  }
  for (int d = 0; d < D; ++d) {
    g64[d * kGP + threadIdx.x] = 0.0;
    g32[d * kGP + threadIdx.x] = 0.f;
  }
  double acc = 0.0;
  float eta[kMaxNC], pr[kMaxNC];
  for (int64_t s0 = s_lo; s0 < s_hi; s0 += kTS) {
    const int ns = static_cast<int>(s_hi - s0 < kTS ? s_hi - s0 : kTS);
    __syncthreads();
    for (int idx = threadIdx.x; idx < ns * k; idx += blockDim.x) xs[idx] = X[s0 * k + idx];
    for (int idx = threadIdx.x; idx < ns; idx += blockDim.x) ys[idx] = y[s0 + idx];
    __syncthreads();
    float tile = 0.f;
    for (int j = 0; j < ns; ++j) {
      const float* xr = xs + j * k;
      float m = 0.f;
      for (int c = 0; c < NC; ++c) {
        const float* tc = th + (c * k) * kGP + threadIdx.x;
        float e = 0.f;
        for (int i = 0; i < k; ++i) e = fmaf(tc[i * kGP], xr[i], e);
        eta[c] = e;
        m = fmaxf(m, e);
      }
      float z = expf(-m);
      for (int c = 0; c < NC; ++c) {
        pr[c] = expf(eta[c] - m);
        z += pr[c];
      }
      const float inv = 1.f / z;
      const int yo = ys[j];
      tile += ((yo == 0) ? 0.f : eta[yo - 1]) - (m + logf(z));
      for (int c = 0; c < NC; ++c) {
        const float r = ((yo == c + 1) ? 1.f : 0.f) - pr[c] * inv;
        float* gc = g32 + (c * k) * kGP + threadIdx.x;
        for (int i = 0; i < k; ++i) gc[i * kGP] = fmaf(r, xr[i], gc[i * kGP]);
      }
    }
    acc += static_cast<double>(tile);
    for (int d = 0; d < D; ++d) {
      g64[d * kGP + threadIdx.x] += static_cast<double>(g32[d * kGP + threadIdx.x]);
      g32[d * kGP + threadIdx.x] = 0.f;
    }
  }
  if (p < P) {
    llp[static_cast<int64_t>(blockIdx.y) * P + p] = acc;
    double* go = gp + (static_cast<int64_t>(blockIdx.y) * P + p) * D;
    for (int d = 0; d < D; ++d) go[d] = g64[d * kGP + threadIdx.x];
  }
}

// Register-resident gradient for small models (k <= KMAX, NC = C - 1 fixed): each thread keeps
// its particle's theta and its FP32 gradient sums over a 128-observation tile in registers; the
// tile sums go to FP64 accumulators in shared memory once per tile (FP64 work per observation
// D / 128). X rows are staged in shared memory padded with zeros to KMAX (broadcast float4).
// Same outputs as grad_fp32_kernel: per chunk FP64 log-likelihood and gradient partials.
constexpr int kGR = 128;   // particles per block
constexpr int kGT = 128;   // observations per tile

template <int KMAX, int NC>
__global__ void __launch_bounds__(kGR)
grad_reg_kernel(const double* __restrict__ theta, int64_t P, int k, const float* __restrict__ X,
                const int* __restrict__ y, int64_t t, int64_t chunk, double* __restrict__ llp,
                double* __restrict__ gp) {
  __shared__ __align__(16) float xs[kGT][KMAX];
  __shared__ int ys[kGT];
  extern __shared__ double g64[];   // [D][kGR]
  const int D = k * NC;
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kGR;
  const int64_t p = p0 + threadIdx.x;
  const int64_t s_lo = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t s_hi = (s_lo + chunk < t) ? s_lo + chunk : t;
  float th[NC][KMAX];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int i = 0; i < KMAX; ++i) th[c][i] = (p < P && i < k) ? f64_to_f32(theta[p * D + c * k + i]) : 0.f;
  for (int d = 0; d < D; ++d) g64[d * kGR + threadIdx.x] = 0.0;
  double acc = 0.0;
  for (int64_t s0 = s_lo; s0 < s_hi; s0 += kGT) {
    const int ns = static_cast<int>(s_hi - s0 < kGT ? s_hi - s0 : kGT);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kGT * KMAX; idx += blockDim.x) {
      const int j = idx / KMAX, i = idx - j * KMAX;
      xs[j][i] = (j < ns && i < k) ? X[(s0 + j) * k + i] : 0.f;
    }
    for (int idx = threadIdx.x; idx < ns; idx += blockDim.x) ys[idx] = y[s0 + idx];
    __syncthreads();
    float gt[NC][KMAX];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < KMAX; ++i) gt[c][i] = 0.f;
    // log-sum-exp arguments z_j = e^-m + sum_c e^(eta_c - m) (in [1, C]) multiplied over 8
    // observations before one logarithm; m = max(0, eta_c)
    float tile = 0.f, zprod = 1.f;
    for (int j = 0; j < ns; ++j) {
      float xr[KMAX];
#pragma unroll
      for (int i = 0; i < KMAX; i += 4) {
        const float4 xv = *reinterpret_cast<const float4*>(&xs[j][i]);
        xr[i] = xv.x;
        xr[i + 1] = xv.y;
        xr[i + 2] = xv.z;
        xr[i + 3] = xv.w;
      }
      float eta[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;   // four chains for the FMA latency
#pragma unroll
        for (int i = 0; i < KMAX; i += 4) {
          a0 = fmaf(th[c][i], xr[i], a0);
          a1 = fmaf(th[c][i + 1], xr[i + 1], a1);
          a2 = fmaf(th[c][i + 2], xr[i + 2], a2);
          a3 = fmaf(th[c][i + 3], xr[i + 3], a3);
        }
        eta[c] = (a0 + a1) + (a2 + a3);
      }
      const int yo = ys[j];
      float r[NC];
      float obs = 0.f, m;
      if constexpr (NC == 1) {
        // p = sigmoid(eta) from e = e^-|eta|; z = 1 + e, m = max(eta, 0)
        const float e = __expf(-fabsf(eta[0]));
        const float inv = __fdividef(1.f, 1.f + e);
        const float pr = eta[0] >= 0.f ? inv : e * inv;
        m = fmaxf(eta[0], 0.f);
        zprod *= 1.f + e;
        r[0] = ((yo == 1) ? 1.f : 0.f) - pr;
        obs = (yo == 1) ? eta[0] : 0.f;
      } else {
        m = 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) m = fmaxf(m, eta[c]);
        float pr[NC];
        float z = __expf(-m);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          pr[c] = __expf(eta[c] - m);
          z += pr[c];
        }
        const float inv = __fdividef(1.f, z);
        zprod *= z;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          r[c] = ((yo == c + 1) ? 1.f : 0.f) - pr[c] * inv;
          obs = (yo == c + 1) ? eta[c] : obs;
        }
      }
      tile += obs - m;
      if ((j & 7) == 7) {
        tile -= logf(zprod);
        zprod = 1.f;
      }
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int i = 0; i < KMAX; ++i) gt[c][i] = fmaf(r[c], xr[i], gt[c][i]);
    }
    tile -= logf(zprod);
    acc += f32_to_f64(tile);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < KMAX; ++i)
        if (i < k) g64[(c * k + i) * kGR + threadIdx.x] += f32_to_f64(gt[c][i]);
  }
  if (p < P) llp[static_cast<int64_t>(blockIdx.y) * P + p] = acc;
  __syncthreads();
  // gradient partials of the block's particles, written element by element (coalesced)
  const int np = static_cast<int>(P - p0 < kGR ? P - p0 : kGR);
  double* go = gp + (static_cast<int64_t>(blockIdx.y) * P + p0) * D;
  for (int q = threadIdx.x; q < np * D; q += blockDim.x) {
    const int pp = q / D, d = q - pp * D;
    go[q] = g64[d * kGR + pp];
  }
}

bool launch_grad_reg(sps_ctx* ctx, dim3 grid, const double* theta, int64_t P, int64_t t, int64_t chunk,
                     double* llp, double* gp) {
  const int k = ctx->k, NC = ctx->NC;
  const size_t smem = sizeof(double) * static_cast<size_t>(k) * NC * kGR;
#define SPS_GRAD_CASE(KM, NCM)                                                                              \
  if (NC == NCM && k <= KM) {                                                                               \
    cudaFuncSetAttribute(grad_reg_kernel<KM, NCM>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                         static_cast<int>(smem));                                                            \
    grad_reg_kernel<KM, NCM><<<grid, kGR, smem, ctx->stream>>>(theta, P, k, ctx->Xf.as<float>(),            \
                                                               ctx->y.as<int>(), t, chunk, llp, gp);        \
    ++ctx->launches;                                                                                        \
    return true;                                                                                            \
  }
  SPS_GRAD_CASE(8, 1)
  SPS_GRAD_CASE(32, 1)
  SPS_GRAD_CASE(64, 1)
  SPS_GRAD_CASE(8, 2)
  SPS_GRAD_CASE(32, 2)
  SPS_GRAD_CASE(8, 3)
#undef SPS_GRAD_CASE
  return false;
}

__global__ void grad_sum_kernel(const double* __restrict__ llp, const double* __restrict__ gp, int64_t P, int D,
                                int slices, double* __restrict__ ll, double* __restrict__ grad) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= P * (D + 1)) return;
  if (idx < P) {
    double s = 0.0;
    for (int q = 0; q < slices; ++q) s += llp[q * P + idx];
    ll[idx] = s;
  } else {
    const int64_t e = idx - P;   // p * D + d
    double s = 0.0;
    for (int q = 0; q < slices; ++q) s += gp[q * P * D + e];
    grad[e] = s;
  }
}

}  // namespace

sps_status loglik_grad_fp32(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll,
                            double* d_grad) {
  const int D = ctx->D, k = ctx->k;
  if (ctx->NC > kMaxNC) return fail(ctx, SPS_ERR_UNSUPPORTED, "gradient: at most 16 outcomes");
  {
    // register-resident kernel when the model fits one of its instantiations
    const int64_t ptiles = (P + kGR - 1) / kGR;
    int64_t chunks = 1;
    if (t > 0) {
      const int64_t want = 4LL * ctx->num_sms;
      const int64_t cap = std::max<int64_t>(1, (int64_t{1} << 26) / (P * (D + 1)));
      chunks = std::max<int64_t>(1, std::min<int64_t>({(want + ptiles - 1) / ptiles, (t + kGT - 1) / kGT, cap}));
    }
    int64_t chunk = std::max<int64_t>(kGT, ((t + chunks - 1) / chunks + kGT - 1) / kGT * kGT);
    chunks = std::max<int64_t>(1, (t + chunk - 1) / chunk);
    SPS_CUDA_TRY(ctx->ll.partial.reserve(sizeof(double) * chunks * P));
    SPS_CUDA_TRY(ctx->ll.aux.reserve(sizeof(double) * chunks * P * D));
    const dim3 grid(static_cast<unsigned>(ptiles), static_cast<unsigned>(chunks));
    if (launch_grad_reg(ctx, grid, d_theta, P, t, chunk, ctx->ll.partial.as<double>(), ctx->ll.aux.as<double>())) {
      SPS_CUDA_TRY(cudaGetLastError());
      const int64_t tot = P * (D + 1);
      grad_sum_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, ctx->stream>>>(
          ctx->ll.partial.as<double>(), ctx->ll.aux.as<double>(), P, D, t > 0 ? static_cast<int>(chunks) : 0, d_ll,
          d_grad); ++ctx->launches;
      SPS_CUDA_TRY(cudaGetLastError());
      return SPS_OK;
    }
  }
  const size_t smem = sizeof(double) * D * kGP + sizeof(float) * (2 * static_cast<size_t>(D) * kGP + kTS * k) +
                      sizeof(int) * kTS;
  if (smem > 220 * 1024) return fail(ctx, SPS_ERR_UNSUPPORTED, "gradient: k*(C-1) too large");
  const int64_t ptiles = (P + kGP - 1) / kGP;
  int64_t chunks = 1;
  if (t > 0) {
    const int64_t want = 4LL * ctx->num_sms;
    const int64_t cap = std::max<int64_t>(1, (int64_t{1} << 26) / (P * (D + 1)));
    chunks = std::max<int64_t>(1, std::min<int64_t>({(want + ptiles - 1) / ptiles, (t + kTS - 1) / kTS, cap}));
  }
  int64_t chunk = std::max<int64_t>(kTS, ((t + chunks - 1) / chunks + kTS - 1) / kTS * kTS);
  chunks = std::max<int64_t>(1, (t + chunk - 1) / chunk);
  SPS_CUDA_TRY(ctx->ll.partial.reserve(sizeof(double) * chunks * P));
  SPS_CUDA_TRY(ctx->ll.aux.reserve(sizeof(double) * chunks * P * D));
  SPS_CUDA_TRY(cudaFuncSetAttribute(grad_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
  dim3 grid(static_cast<unsigned>(ptiles), static_cast<unsigned>(chunks));
  grad_fp32_kernel<<<grid, kGP, smem, ctx->stream>>>(d_theta, P, k, ctx->NC, ctx->Xf.as<float>(), ctx->y.as<int>(),
                                                     t, chunk, ctx->ll.partial.as<double>(), ctx->ll.aux.as<double>()); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  const int64_t tot = P * (D + 1);
  grad_sum_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, ctx->stream>>>(
      ctx->ll.partial.as<double>(), ctx->ll.aux.as<double>(), P, D, t > 0 ? static_cast<int>(chunks) : 0, d_ll, d_grad); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
