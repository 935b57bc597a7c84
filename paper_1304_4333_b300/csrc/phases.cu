// Simulator phases of the SPS library (Algorithms 1-3 of Sec. 2): particle state, the C phase
// with the ESS rule (Eq. 14), the S phase (multinomial resampling within groups), the M phase
// (random-walk Metropolis with Sigma = h V, Algorithm 2 step 2), group moments, NSE and RNE
// (Eqs. 3-10), and the sps_run driver.
//
// Random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by the state's seed, with
// counter (index, stream, step_lo, step_hi): every draw is a pure function of its position, so
// runs are reproducible and independent of launch configuration.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "common.cuh"

namespace sps {
namespace {

// ------------------------------------------------------------------------------ Philox

constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;

enum Stream : uint32_t { kStreamInit = 1, kStreamPropose = 2, kStreamAccept = 3, kStreamResample = 4 };

__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kWeyl0;
      k1 += kWeyl1;
    }
    const uint32_t hi0 = __umulhi(kMul0, c.x), lo0 = kMul0 * c.x;
    const uint32_t hi1 = __umulhi(kMul1, c.z), lo1 = kMul1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t idx, uint32_t stream, uint64_t step) {
  return philox(make_uint4(idx, stream, static_cast<uint32_t>(step), static_cast<uint32_t>(step >> 32)),
                static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// FP64 uniform on [0, 1): the top 53 bits of (hi:lo) times 2^-53.
__device__ __forceinline__ double uniform53(uint32_t lo, uint32_t hi) {
  const uint64_t b = ((static_cast<uint64_t>(hi) << 32) | lo) >> 11;
  return static_cast<double>(b) * 0x1.0p-53;
}

// Two FP32 standard normals by the Box-Muller transform of two 24-bit uniforms.
__device__ __forceinline__ float2 normals2(uint32_t a, uint32_t b) {
  const float u1 = (static_cast<float>(a >> 8) + 1.0f) * 0x1.0p-24f;   // (0, 1]
  const float u2 = static_cast<float>(b >> 8) * 0x1.0p-24f;            // [0, 1)
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(r * c, r * s);
}

__global__ void philox_kernel(uint32_t k0, uint32_t k1, uint4 ctr, int64_t count, uint4* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= count) return;
  uint4 c = ctr;
  c.x += static_cast<uint32_t>(i);
  out[i] = philox(c, k0, k1);
}

// ------------------------------------------------------------------------------ reductions

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum / max (blockDim a multiple of 32, <= 1024); result valid in every thread.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
    t = warp_sum(t);
    if (l == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}
__device__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : -INFINITY;
  if (w == 0) {
    t = warp_max(t);
    if (l == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// ------------------------------------------------------------------------------ prior

// Prior log kernel -(1/2) (theta - mu)' Prec (theta - mu); prec is diagonal [D] unless full.
// FP32 element-wise (d = f32(theta) - f32(mu)) and FP32 sums: the same deterministic function
// for every particle and proposal, so Metropolis ratios stay exact for it; its relative error
// (about 1e-7) is far below the posterior's scale.
constexpr int kMaxD = 155;   // covariance kernel: <= 48 moment entries per thread

__device__ double prior_log_kernel(const double* th, const double* mu, const double* prec, int D, bool full) {
  float a = 0.f;
  if (!full) {
    for (int i = 0; i < D; ++i) {
      const float d = f64_to_f32(th[i]) - f64_to_f32(mu[i]);
      a = fmaf(d * d, f64_to_f32(prec[i]), a);
    }
  } else {
    // full precision matrix: its FP32 copy follows the FP64 one; the centred coordinates are
    // converted once (the values and the order of operations are those of the plain loops)
    const float* p32 = reinterpret_cast<const float*>(prec + static_cast<size_t>(D) * D);
    float d[kMaxD];
    for (int j = 0; j < D; ++j) d[j] = f64_to_f32(th[j]) - f64_to_f32(mu[j]);
    for (int i = 0; i < D; ++i) {
      const float* pi = p32 + static_cast<size_t>(i) * D;
      float r = 0.f;
      for (int j = 0; j < D; ++j) r = fmaf(pi[j], d[j], r);
      a = fmaf(d[i], r, a);
    }
  }
  return -0.5 * f32_to_f64(a);
}

// Algorithm 1 step 1: theta_p = mu + L0 z, z iid N(0, 1) (FP64 Box-Muller from Philox).
__global__ void prior_init_kernel(uint64_t seed, int64_t P, int D, const double* __restrict__ mu,
                                  const double* __restrict__ L0, const double* __restrict__ prec, bool full,
                                  double* __restrict__ theta, double* __restrict__ lp, double* __restrict__ zbuf) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= P) return;
  double* z = zbuf + p * D;
  for (int d = 0; d < D; d += 2) {
    const uint4 r = draw(seed, static_cast<uint32_t>(p * ((D + 1) / 2) + d / 2), kStreamInit, 0);
    const double u1 = 1.0 - uniform53(r.x, r.y);   // (0, 1]
    const double u2 = uniform53(r.z, r.w);
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z[d] = rad * c;
    if (d + 1 < D) z[d + 1] = rad * s;
  }
  double* th = theta + p * D;
  for (int i = 0; i < D; ++i) {
    double a = mu[i];
    if (full) {
      for (int j = 0; j <= i; ++j) a = fma(L0[i * D + j], z[j], a);
    } else {
      a = fma(L0[i * D + i], z[i], a);
    }
    th[i] = a;
  }
  lp[p] = prior_log_kernel(th, mu, prec, D, full);
}

__global__ void prior_lp_kernel(const double* __restrict__ theta, int64_t P, int D, const double* __restrict__ mu,
                                const double* __restrict__ prec, bool full, double* __restrict__ lp) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= P) return;
  lp[p] = prior_log_kernel(theta + p * D, mu, prec, D, full);
}

// ------------------------------------------------------------------------------ C phase

// A running log weight as a pair (s, c) of value s - c: the C phase's Kahan pairs, or an FP64
// value split into its FP32 truncation and the FP32 remainder.
struct LwPair {
  float s, c;
};
__device__ __forceinline__ LwPair load_lw(const float2* __restrict__ r, int64_t p) {
  const float2 v = r[p];
  return {v.x, v.y};
}
__device__ __forceinline__ LwPair load_lw(const double* __restrict__ r, int64_t p) {
  const double v = r[p];
  const float hi = f64_to_f32(v);
  return {hi, f64_to_f32(f32_to_f64(hi) - v)};
}

__device__ float block_max_f(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  float t = (threadIdx.x < nw) ? sh[threadIdx.x] : -INFINITY;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (l == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// ESS(s) of rows of running log weights (Eq. 14), in two kernels. Block (row, part) reads its
// slice of the row once: each thread keeps an online maximum m of s and the FP32 sums of
// e = exp((s - m) - c) and e^2, rescaled when m grows (s - m is exact near the maximum, where
// the weights matter); the block rescales its threads to the block maximum and sums in FP64.
// The merge rescales the parts to the row maximum and returns (sum e)^2 / sum e^2.
constexpr int kEssParts = 8;

// range (optional): a C-phase block decided on the device; rows past its length are skipped.
template <class InT>
__global__ void ess_part_kernel(const InT* __restrict__ lw, int64_t P, double* __restrict__ parts,
                                const int64_t* __restrict__ range) {
  __shared__ float shf[33];
  __shared__ double sh[33];
  if (range && static_cast<int64_t>(blockIdx.x) >= range[1] - range[0]) return;
  const InT* row = lw + static_cast<int64_t>(blockIdx.x) * P;
  const int64_t per = (P + gridDim.y - 1) / gridDim.y;
  const int64_t lo = blockIdx.y * per, hi = min(P, lo + per);
  float m = -INFINITY, s1 = 0.f, s2 = 0.f;
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
    const LwPair v = load_lw(row, p);
    if (v.s > m) {
      const float f = (m > -INFINITY) ? __expf(m - v.s) : 0.f;
      s1 *= f;
      s2 *= f * f;
      m = v.s;
    }
    const float e = __expf((v.s - m) - v.c);
    s1 += e;
    s2 = fmaf(e, e, s2);
  }
  const float M = block_max_f(m, shf);
  const float f = (m > -INFINITY) ? __expf(m - M) : 0.f;
  const double t1 = block_sum(f32_to_f64(s1 * f), sh);
  const double t2 = block_sum(f32_to_f64(s2 * f * f), sh);
  if (threadIdx.x == 0) {
    double* o = parts + (static_cast<int64_t>(blockIdx.x) * gridDim.y + blockIdx.y) * 3;
    o[0] = f32_to_f64(M);
    o[1] = t1;
    o[2] = t2;
  }
}

__global__ void ess_merge_kernel(const double* __restrict__ parts, int rows, int nparts, double* __restrict__ ess,
                                 const int64_t* __restrict__ range) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (range) rows = static_cast<int>(range[1] - range[0]);
  if (r >= rows) return;
  const double* q = parts + static_cast<int64_t>(r) * nparts * 3;
  float M = -INFINITY;
  for (int i = 0; i < nparts; ++i) M = fmaxf(M, f64_to_f32(q[3 * i]));   // the part maxima are FP32 values
  double s1 = 0.0, s2 = 0.0;
  for (int i = 0; i < nparts; ++i) {
    const float mi = f64_to_f32(q[3 * i]);
    if (mi == -INFINITY) continue;
    const double f = f32_to_f64(__expf(mi - M));
    s1 += f * q[3 * i + 1];
    s2 += f * f * q[3 * i + 2];
  }
  ess[r] = (s2 > 0.0) ? s1 * s1 / s2 : 0.0;
}

// The stopping rule of a captured C phase (Algorithm 2 step 1, as cphase_impl applies it on the
// host): the first row j of the block with ESS / P below the fraction, or the data's last
// observation, ends the phase at t = s + j + 1 (row j is read into the log weights); otherwise
// the last row becomes the running state and the next block, of twice the rows up to max_rows,
// starts at s + b. Sets the model's conditional node (another block while not done). One thread.
__global__ void cphase_scan_kernel(CphaseCtl* __restrict__ cc, const double* __restrict__ ess,
                                   cudaGraphConditionalHandle more) {
  const int64_t s = cc->range[0], b = cc->range[1] - cc->range[0];
  int done = 0;
  for (int64_t j = 0; j < b; ++j) {
    const int64_t sj = s + j + 1;
    if (ess[j] / static_cast<double>(cc->P) < cc->frac || sj == cc->n) {
      cc->row = j;
      cc->t_new = sj;
      done = 1;
      break;
    }
  }
  cc->blocks += 1;
  if (!done) {
    cc->row = b - 1;
    const int64_t s2 = s + b;
    const int64_t blk = (cc->block * 2 < cc->max_rows) ? cc->block * 2 : cc->max_rows;
    cc->block = blk;
    cc->range[0] = s2;
    cc->range[1] = s2 + ((blk < cc->n - s2) ? blk : cc->n - s2);
  }
  cc->done = done;
  cudaGraphSetConditional(more, done ? 0u : 1u);
}

// After the scan: the stop row to FP64 log weights (as lw_to_f64_kernel), else the block's last
// row to the running state (as the host's device-to-device copy).
__global__ void cphase_advance_kernel(const CphaseCtl* __restrict__ cc, const float2* __restrict__ rows, int64_t P,
                                      float2* __restrict__ lwstate, double* __restrict__ logw) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= P) return;
  const float2 v = rows[cc->row * P + p];
  if (cc->done) logw[p] = f32_to_f64(v.x) - f32_to_f64(v.y);
  else lwstate[p] = v;
}

// Loop condition of the captured C phases of several models: another block while any model's
// phase goes on. cc[M] counts the loop's iterations: at its max_rows (a bound no data reaches)
// the loop ends with err = 1.
__global__ void cphase_continue_kernel(CphaseCtl* __restrict__ cc, int M, cudaGraphConditionalHandle cond) {
  int any = 0;
  for (int m = 0; m < M; ++m) any |= cc[m].done ? 0 : 1;
  const int64_t it = ++cc[M].row;
  if (any && it >= cc[M].max_rows) {
    cc[M].err = 1;
    any = 0;
  }
  cudaGraphSetConditional(cond, any ? 1u : 0u);
}

// logw[p] = value of the Kahan pair row[p] in FP64.
__global__ void lw_to_f64_kernel(const float2* __restrict__ row, int64_t P, double* __restrict__ logw) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= P) return;
  const float2 v = row[p];
  logw[p] = f32_to_f64(v.x) - f32_to_f64(v.y);
}

// Per-group log N^-1 sum_n exp(lw_jn) of each row of C-phase running log weights (Kahan pairs):
// out[r * J + j]; block (row, group), FP32 exponentials of (s - m) - c with an online maximum,
// FP64 block sums. Differences of consecutive rows are the log predictive likelihoods.
__global__ void row_group_lme_kernel(const float2* __restrict__ rows, int64_t P, int N, double* __restrict__ out) {
  __shared__ float shf[33];
  __shared__ double sh[33];
  const float2* g = rows + static_cast<int64_t>(blockIdx.x) * P + static_cast<int64_t>(blockIdx.y) * N;
  float m = -INFINITY, s1 = 0.f;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const float2 v = g[n];
    if (v.x > m) {
      s1 *= (m > -INFINITY) ? __expf(m - v.x) : 0.f;
      m = v.x;
    }
    s1 += __expf((v.x - m) - v.y);
  }
  const float M = block_max_f(m, shf);
  const double t = block_sum(f32_to_f64(s1 * ((m > -INFINITY) ? __expf(m - M) : 0.f)), sh);
  if (threadIdx.x == 0)
    out[static_cast<int64_t>(blockIdx.x) * gridDim.y + blockIdx.y] = f32_to_f64(M) + log(t / static_cast<double>(N));
}

// Per-group log N^-1 sum_n exp(logw_jn) in FP64, in two kernels: block (group, part) writes its
// slice's maximum and sum of exp(logw - maximum); the merge (thread per group) rescales the
// parts, writes lme_j, adds it to logml_j and records the group maximum.
constexpr int kLmeParts = 8;

__global__ void group_lme_part_kernel(const double* __restrict__ logw, int N, double* __restrict__ parts) {
  __shared__ double sh[33];
  const double* row = logw + static_cast<int64_t>(blockIdx.x) * N;
  const int per = (N + gridDim.y - 1) / gridDim.y;
  const int lo = blockIdx.y * per, hi = min(N, lo + per);
  double m = -INFINITY;
  for (int n = lo + threadIdx.x; n < hi; n += blockDim.x) m = fmax(m, row[n]);
  m = block_max(m, sh);
  double s = 0.0;
  if (m > -INFINITY)
    for (int n = lo + threadIdx.x; n < hi; n += blockDim.x) s += exp(row[n] - m);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    double* o = parts + (static_cast<int64_t>(blockIdx.x) * gridDim.y + blockIdx.y) * 2;
    o[0] = m;
    o[1] = s;
  }
}

__global__ void group_lme_merge_kernel(const double* __restrict__ parts, int J, int nparts, int N,
                                       double* __restrict__ lme, double* __restrict__ logml,
                                       double* __restrict__ gmax) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  const double* q = parts + static_cast<int64_t>(j) * nparts * 2;
  double M = -INFINITY;
  for (int i = 0; i < nparts; ++i) M = fmax(M, q[2 * i]);
  double S = 0.0;
  for (int i = 0; i < nparts; ++i)
    if (q[2 * i] > -INFINITY) S += q[2 * i + 1] * exp(q[2 * i] - M);
  const double v = M + log(S / static_cast<double>(N));
  lme[j] = v;
  if (logml) logml[j] += v;
  if (gmax) gmax[j] = M;
}

__global__ void add_kernel(double* __restrict__ a, const double* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) a[i] += b[i];
}

// ------------------------------------------------------------------------------ S phase

constexpr int kMaxN = 4096;
constexpr int kResThreads = 1024;
constexpr int kResBlocks = 4;   // blocks per group, each drawing N / kResBlocks of the indices

// Multinomial resampling within groups by an integer CDF (S phase, Algorithm 1), two kernels.
// q_p = floor(w_p 2^40) with w_p = exp(logw_p - max of its group) (mode 0, FP64) or the given
// w_p (mode 1).
__global__ void resample_q_kernel(const double* __restrict__ src, int mode, int N, int64_t P,
                                  const double* __restrict__ gmax, unsigned long long* __restrict__ q) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= P) return;
  const double w = (mode == 0) ? exp(src[p] - gmax[p / N]) : src[p];
  q[p] = static_cast<unsigned long long>(floor(ldexp(w, 40)));
}

// Block (group j, slice b): c = inclusive uint64 prefix sums of the group's q (every block of the
// group builds the same table), then for the draws i of its slice tau_i = min(floor(u_i Q), Q - 1)
// and idx_i = first n with c_n > tau_i. Sets *flag when the group's Q is zero.
__global__ void __launch_bounds__(kResThreads)
resample_kernel(const unsigned long long* __restrict__ qv, int N, const double* __restrict__ u_given,
                uint64_t seed, uint64_t step, int* __restrict__ idx, int* __restrict__ flag) {
  __shared__ unsigned long long c[kMaxN];
  __shared__ unsigned long long part[kResThreads];
  const int j = blockIdx.x;
  const unsigned long long* q = qv + static_cast<int64_t>(j) * N;
  // each thread owns a contiguous run of ceil(N / threads) elements
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int n0 = threadIdx.x * per;
  unsigned long long run = 0;
  for (int k = 0; k < per; ++k) {
    const int n = n0 + k;
    if (n < N) {
      run += q[n];
      c[n] = run;
    }
  }
  part[threadIdx.x] = run;
  __syncthreads();
  // inclusive scan of the per-thread totals (Hillis-Steele over <= 1024 values)
  for (int o = 1; o < static_cast<int>(blockDim.x); o <<= 1) {
    const unsigned long long v = (threadIdx.x >= static_cast<unsigned>(o)) ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  const unsigned long long off = (threadIdx.x > 0) ? part[threadIdx.x - 1] : 0ull;
  for (int k = 0; k < per; ++k) {
    const int n = n0 + k;
    if (n < N) c[n] += off;
  }
  __syncthreads();
  const unsigned long long Q = c[N - 1];
  if (Q == 0ull) {
    if (threadIdx.x == 0) atomicOr(flag, 1);
    return;
  }
  const int slice = (N + gridDim.y - 1) / gridDim.y;
  const int i_hi = min(N, static_cast<int>(blockIdx.y + 1) * slice);
  for (int i = blockIdx.y * slice + threadIdx.x; i < i_hi; i += blockDim.x) {
    double u;
    if (u_given) {
      u = u_given[static_cast<int64_t>(j) * N + i];
    } else {
      const uint4 r = draw(seed, static_cast<uint32_t>(j * N + i), kStreamResample, step);
      u = uniform53(r.x, r.y);
    }
    unsigned long long tau = static_cast<unsigned long long>(floor(__dmul_rn(u, static_cast<double>(Q))));
    if (tau > Q - 1) tau = Q - 1;
    int lo = 0, hi = N - 1;   // first n with c[n] > tau; c[N-1] = Q > tau
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (c[mid] > tau) hi = mid;
      else lo = mid + 1;
    }
    idx[static_cast<int64_t>(j) * N + i] = lo;
  }
}

constexpr int kResidualShift = 12;

// Residual resampling of group j (block (j, slice)): with Q = sum q, particle n gets
// c_n = floor(N q_n / Q) copies, placed first in particle order (positions given by the
// inclusive scan of c), and the R = N - sum c remaining positions i = 0..R-1 take multinomial
// draws on the residuals r_n = (N q_n mod Q) >> 12 by the integer CDF (u_i as in
// resample_kernel). N q_n <= 2^52 and sum r < 2^52: all exact. Every block of the group builds
// the same tables and fills its slice of the N positions. Sets *flag when Q is zero.
__global__ void __launch_bounds__(kResThreads)
resample_residual_kernel(const unsigned long long* __restrict__ qv, int N, const double* __restrict__ u_given,
                         uint64_t seed, uint64_t step, int* __restrict__ idx, int* __restrict__ flag) {
  extern __shared__ unsigned long long rs[];
  unsigned long long* cr = rs;                // [N] inclusive scan of residuals
  unsigned long long* cc = rs + kMaxN;        // [N] inclusive scan of copies
  unsigned long long* part = rs + 2 * kMaxN;  // [threads]
  __shared__ unsigned long long Qs;
  const int j = blockIdx.x;
  const unsigned long long* q = qv + static_cast<int64_t>(j) * N;
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int n0 = threadIdx.x * per;
  // Q
  unsigned long long run = 0;
  for (int k = 0; k < per; ++k)
    if (n0 + k < N) run += q[n0 + k];
  part[threadIdx.x] = run;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x); ++w) t += part[w];
    Qs = t;
  }
  __syncthreads();
  const unsigned long long Q = Qs;
  if (Q == 0ull) {
    if (threadIdx.x == 0) atomicOr(flag, 1);
    return;
  }
  const unsigned long long NN = static_cast<unsigned long long>(N);
  // per-thread runs of copies and residuals, then block scans of both
  unsigned long long rc = 0, rr = 0;
  for (int k = 0; k < per; ++k) {
    const int n = n0 + k;
    if (n < N) {
      const unsigned long long a = NN * q[n];
      rc += a / Q;
      rr += (a % Q) >> kResidualShift;
      cc[n] = rc;
      cr[n] = rr;
    }
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    part[threadIdx.x] = (pass == 0) ? rc : rr;
    __syncthreads();
    for (int o = 1; o < static_cast<int>(blockDim.x); o <<= 1) {
      const unsigned long long v = (threadIdx.x >= static_cast<unsigned>(o)) ? part[threadIdx.x - o] : 0ull;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    const unsigned long long off = (threadIdx.x > 0) ? part[threadIdx.x - 1] : 0ull;
    unsigned long long* c = (pass == 0) ? cc : cr;
    for (int k = 0; k < per; ++k)
      if (n0 + k < N) c[n0 + k] += off;
    __syncthreads();
  }
  const int copies = static_cast<int>(cc[N - 1]);
  const unsigned long long S = cr[N - 1];
  if (copies < N && S == 0ull) {   // only with weights not scaled to a maximum of 1
    if (threadIdx.x == 0) atomicOr(flag, 1);
    return;
  }
  const int slice = (N + gridDim.y - 1) / gridDim.y;
  const int i_hi = min(N, static_cast<int>(blockIdx.y + 1) * slice);
  for (int pos = blockIdx.y * slice + threadIdx.x; pos < i_hi; pos += blockDim.x) {
    const unsigned long long* cdf;
    unsigned long long tau;
    if (pos < copies) {
      cdf = cc;
      tau = static_cast<unsigned long long>(pos);
    } else {
      const int i = pos - copies;
      double u;
      if (u_given) {
        u = u_given[static_cast<int64_t>(j) * N + i];
      } else {
        const uint4 r = draw(seed, static_cast<uint32_t>(j * N + i), kStreamResample, step);
        u = uniform53(r.x, r.y);
      }
      cdf = cr;
      tau = static_cast<unsigned long long>(floor(__dmul_rn(u, static_cast<double>(S))));
      if (tau > S - 1) tau = S - 1;
    }
    int lo = 0, hi = N - 1;   // first n with cdf[n] > tau
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cdf[mid] > tau) hi = mid;
      else lo = mid + 1;
    }
    idx[static_cast<int64_t>(j) * N + pos] = lo;
  }
}

constexpr size_t kResidualSmem = sizeof(unsigned long long) * (2 * kMaxN + kResThreads);

// Launch the scan/search kernel of a resampling scheme on quantised weights q [J*N].
sps_status launch_resample(sps_ctx* ctx, int scheme, const unsigned long long* q, int J, int N, const double* u,
                           uint64_t seed, uint64_t step, int* idx, int* flag) {
  if (scheme == SPS_RESAMPLE_RESIDUAL) {
    SPS_CUDA_TRY(cudaFuncSetAttribute(resample_residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(kResidualSmem)));
    resample_residual_kernel<<<dim3(J, kResBlocks), kResThreads, kResidualSmem, ctx->stream>>>(q, N, u, seed, step,
                                                                                                idx, flag);
  } else if (scheme == SPS_RESAMPLE_MULTINOMIAL) {
    resample_kernel<<<dim3(J, kResBlocks), kResThreads, 0, ctx->stream>>>(q, N, u, seed, step, idx, flag);
  } else {
    return fail(ctx, SPS_ERR_INVALID_ARG, "unknown resampling scheme");
  }
  ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

// dst[p] = src[group(p) * N + idx[p]] for theta rows and the per-particle scalars. A block of
// 256 threads moves ppb = 256 / D whole rows, one thread per element (coalesced writes); the
// first thread of a row also moves ll and lp.
__global__ void gather_kernel(const double* __restrict__ th, const double* __restrict__ ll,
                              const double* __restrict__ lp, const int* __restrict__ idx, int64_t P, int N, int D,
                              double* __restrict__ th_o, double* __restrict__ ll_o, double* __restrict__ lp_o) {
  const int ppb = static_cast<int>(blockDim.x) / D;
  const int pp = static_cast<int>(threadIdx.x) / D;
  const int d = static_cast<int>(threadIdx.x) - pp * D;
  const int64_t p = static_cast<int64_t>(blockIdx.x) * ppb + pp;
  if (pp >= ppb || p >= P) return;
  const int64_t src = (p / N) * N + idx[p];
  th_o[p * D + d] = th[src * D + d];
  if (d == 0) {
    ll_o[p] = ll[src];
    lp_o[p] = lp[src];
  }
}

// ------------------------------------------------------------------------------ M phase


constexpr int kCovSub = 64;        // particles staged per shared-memory pass
constexpr int kCovThreads = 256;
constexpr int kCovMaxEnt = 48;     // moment entries per thread: T + D <= 256 x 48 for D <= 155

// Lower-triangle index e -> (i, j), i >= j, row-major.
__device__ __forceinline__ void tri_ij(int e, int* i, int* j) {
  int r = static_cast<int>((sqrtf(8.0f * static_cast<float>(e) + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > e) --r;
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  *i = r;
  *j = e - r * (r + 1) / 2;
}

// First and second moments of theta about a shift (particle 0): block b sums, over its particle
// range, d = f32(theta_p) - f32(theta_0) and the lower triangle of d d', in FP32 within a
// 64-particle pass and with Kahan compensation across passes, and writes E = T + D FP64
// partials: [0, T) sum d_i d_j, [T, T + D) sum d_i. The covariance is shift-invariant; centring
// on a particle keeps the products at the scale of the spread, not of the location.
// ENT: compile-time bound on the entries of one thread (E <= 256 ENT), so that the per-entry
// state stays in registers.
template <int ENT>
__global__ void __launch_bounds__(kCovThreads)
cov_moments_kernel(const double* __restrict__ th, int64_t P, int D, int64_t per_block,
                   double* __restrict__ partial) {
  extern __shared__ float cs[];   // [kCovSub][D], then the shift [D]
  float* shift = cs + kCovSub * D;
  const int T = D * (D + 1) / 2, E = T + D;
  const int64_t p_lo = blockIdx.x * per_block;
  const int64_t p_hi = min(P, p_lo + per_block);
  for (int d = threadIdx.x; d < D; d += blockDim.x) shift[d] = f64_to_f32(th[d]);
  float acc[ENT], comp[ENT];
  int ei[ENT], ej[ENT];
#pragma unroll
  for (int q = 0; q < ENT; ++q) {
    const int e = threadIdx.x + q * kCovThreads;
    ei[q] = 0;
    ej[q] = -2;   // no entry
    if (e < T) {
      tri_ij(e, &ei[q], &ej[q]);
    } else if (e < E) {
      ei[q] = e - T;
      ej[q] = -1;   // first moment
    }
    acc[q] = 0.f;
    comp[q] = 0.f;
  }
  for (int64_t p0 = p_lo; p0 < p_hi; p0 += kCovSub) {
    const int np = static_cast<int>(p_hi - p0 < kCovSub ? p_hi - p0 : kCovSub);
    __syncthreads();
    for (int q = threadIdx.x; q < np * D; q += blockDim.x) {
      const int pp = q / D, d = q - pp * D;
      cs[pp * D + d] = f64_to_f32(th[(p0 + pp) * D + d]) - shift[d];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ENT; ++q) {
      if (ej[q] == -2) continue;
      float a = 0.f;
      if (ej[q] >= 0) {
        for (int pp = 0; pp < np; ++pp) a = fmaf(cs[pp * D + ei[q]], cs[pp * D + ej[q]], a);
      } else {
        for (int pp = 0; pp < np; ++pp) a += cs[pp * D + ei[q]];
      }
      const float y = a - comp[q];
      const float t = acc[q] + y;
      comp[q] = (t - acc[q]) - y;
      acc[q] = t;
    }
  }
#pragma unroll
  for (int q = 0; q < ENT; ++q) {
    const int e = threadIdx.x + q * kCovThreads;
    if (e < E) partial[static_cast<int64_t>(blockIdx.x) * E + e] = f32_to_f64(acc[q]) - f32_to_f64(comp[q]);
  }
}

// V = (S2 - S1 S1' / P) / (P - 1) from the block partials, one warp per lower-triangle entry
// (lanes take every 32nd block, FP64); writes the full symmetric V and Sigma = scale V.
__global__ void cov_final_kernel(const double* __restrict__ partial, int blocks, int D, int64_t P, double scale_arg,
                                 const double* __restrict__ scale_dev, double* __restrict__ V,
                                 double* __restrict__ Sigma) {
  const double scale = scale_dev ? *scale_dev : scale_arg;   // device-resident h in a captured M phase
  const int T = D * (D + 1) / 2, E = T + D;
  const int e = static_cast<int>((blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= T) return;
  int i, j;
  tri_ij(e, &i, &j);
  double s2 = 0.0, si = 0.0, sj = 0.0;
  for (int b = lane; b < blocks; b += 32) {
    const double* q = partial + static_cast<int64_t>(b) * E;
    s2 += q[e];
    si += q[T + i];
    sj += q[T + j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
    sj += __shfl_xor_sync(0xffffffffu, sj, o);
  }
  if (lane != 0) return;
  const double n = static_cast<double>(P);
  const double v = (s2 - si * sj / n) / (n - 1.0);
  if (V) {
    V[i * D + j] = v;
    V[j * D + i] = v;
  }
  if (Sigma) {
    Sigma[i * D + j] = scale * v;
    Sigma[j * D + i] = scale * v;
  }
}

// Lower Cholesky factor of A [D x D] (FP64, one block, right-looking on the packed lower
// triangle in shared memory). FP64 instructions have about 64 cycles of latency on this GPU (a
// square root about 600, a division about 400), so the critical path is kept short: per column
// one Newton reciprocal square root, the scaled column copied to a separate buffer, and the
// trailing update spread over all threads by triangle entry (about two independent FMAs per
// thread for D = 30). On failure (pivot not positive, or outside (1e-37, 1e37)) sets *flag.
// (A one-warp register variant for D <= 32 ran at 58 us against 35 us at D = 30: masked lanes
// still occupy the FP64 pipe, about 1.5 FMA per clock per SM on this GPU.)
// Writes L in FP64 (full, zero upper part) and the packed lower triangle in FP32.
__device__ __forceinline__ int tri(int i, int k) { return i * (i + 1) / 2 + k; }

// 1/sqrt(a) for a in the float normal range: an FP32 seed refined by two Newton steps in FP64
// (y <- y (3 - a y^2) / 2; the error squares each step, 2^-22 -> 2^-43 -> below 2^-53).
__device__ __forceinline__ double rsqrt_f64(double a) {
  double y = f32_to_f64(rsqrtf(f64_to_f32(a)));
  const double h = 0.5 * a;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

constexpr int kCholThreads = 256;

// One block's factorisation; a: the packed lower triangle in shared memory, col: the scaled
// column, rinv / bad: block-shared scalars.
__device__ __forceinline__ void cholesky_block(const double* __restrict__ A, int D, double* __restrict__ L,
                                               float* __restrict__ L32, int* __restrict__ flag, double* a,
                                               double* col, double& rinv, int& bad) {
  const int T = D * (D + 1) / 2;
  // this thread's entries e = threadIdx.x + q blockDim.x of the packed triangle, as (i << 16) | k
  // computed once (the trailing updates visit them every column)
  constexpr int kQ = (kMaxD * (kMaxD + 1) / 2 + kCholThreads - 1) / kCholThreads;
  int ik[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int e = threadIdx.x + q * kCholThreads;
    ik[q] = 0;
    if (e < T) {
      int i, k;
      tri_ij(e, &i, &k);
      a[e] = A[i * D + k];
      ik[q] = (i << 16) | k;
    }
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < D; ++j) {
    if (threadIdx.x == 0) {
      const double piv = a[tri(j, j)];
      if (!(piv > 1e-37) || !(piv < 1e37)) {
        bad = 1;
      } else {
        const double y = rsqrt_f64(piv);
        a[tri(j, j)] = piv * y;   // sqrt(piv)
        rinv = y;
      }
    }
    __syncthreads();
    if (bad) break;
    const double r = rinv;
    for (int i = j + 1 + threadIdx.x; i < D; i += blockDim.x) {
      const double v = a[tri(i, j)] * r;
      a[tri(i, j)] = v;
      col[i] = v;
    }
    __syncthreads();
    // trailing update a[i][k] -= l_ij l_kj for j < k <= i
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int e = threadIdx.x + q * kCholThreads;
      if (e >= T) break;
      const int i = ik[q] >> 16, k = ik[q] & 0xFFFF;
      if (k > j) a[e] = fma(-col[i], col[k], a[e]);
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicOr(flag, 1);
    return;
  }
  for (int q = threadIdx.x; q < D * D; q += blockDim.x) {
    const int i = q / D, k = q - i * D;
    L[q] = (k <= i) ? a[tri(i, k)] : 0.0;
  }
  for (int e = threadIdx.x; e < T; e += blockDim.x) L32[e] = f64_to_f32(a[e]);
}

__global__ void __launch_bounds__(kCholThreads)
cholesky_kernel(const double* __restrict__ A, int D, double* __restrict__ L,
                float* __restrict__ L32, int* __restrict__ flag) {
  extern __shared__ double a[];   // packed lower triangle, row-major
  __shared__ double col[kMaxD];   // scaled column j
  __shared__ double rinv;
  __shared__ int bad;
  cholesky_block(A, D, L, L32, flag, a, col, rinv, bad);
}

// Several independent factorisations in one launch, one block each (the models of a batched
// run): the same arithmetic as cholesky_kernel per matrix.
struct CholJob {
  const double* A;
  double* L;
  float* L32;
  int* flag;
  int D;
  int pad;
};

__global__ void __launch_bounds__(kCholThreads)
cholesky_batched_kernel(const CholJob* __restrict__ jobs) {
  extern __shared__ double a[];
  __shared__ double col[kMaxD];
  __shared__ double rinv;
  __shared__ int bad;
  const CholJob job = jobs[blockIdx.x];
  cholesky_block(job.A, job.D, job.L, job.L32, job.flag, a, col, rinv, bad);
}

// Particle rows [p0, p0 + np) of a [P x D] FP64 matrix to / from shared memory with row stride
// Dp (odd, so that one row per lane reads without bank conflicts); global accesses coalesced.
__device__ __forceinline__ void stage_rows(const double* __restrict__ src, int64_t p0, int np, int D, int Dp,
                                           double* sm) {
  const double* g = src + p0 * D;
  for (int q = threadIdx.x; q < np * D; q += blockDim.x) {
    const int r = q / D;
    sm[r * Dp + (q - r * D)] = g[q];
  }
}
__device__ __forceinline__ void unstage_rows(double* __restrict__ dst, int64_t p0, int np, int D, int Dp,
                                             const double* sm) {
  double* g = dst + p0 * D;
  for (int q = threadIdx.x; q < np * D; q += blockDim.x) {
    const int r = q / D;
    g[q] = sm[r * Dp + (q - r * D)];
  }
}

constexpr int kPropPart = 64;   // particles per block
constexpr int kPropSub = 4;     // threads per particle: the rows of L z are split among them

// theta' = theta + L z (L packed lower triangle FP32; z FP32 normals from Philox, or given FP64),
// plus the prior log kernel of theta'. The block's theta rows go through shared memory (coalesced
// reads and writes); the four threads of a particle update every fourth row of it (each row's
// dot product in the order j = 0..i), then the first of them evaluates the prior log kernel of
// the new row in the order of prior_log_kernel. Skipped when the factorisation failed.
__global__ void __launch_bounds__(kPropPart * kPropSub)
propose_kernel(const double* __restrict__ th, int64_t P, int D, const float* __restrict__ L32,
               const double* __restrict__ z_given, uint64_t seed, uint64_t step_arg,
               const unsigned long long* __restrict__ step_dev, const double* __restrict__ mu,
               const double* __restrict__ prec, bool full, const int* __restrict__ flag,
               double* __restrict__ th_o, double* __restrict__ lp_o) {
  if (*flag) return;
  const uint64_t step = step_dev ? *step_dev : step_arg;
  extern __shared__ double pd[];
  const int T = D * (D + 1) / 2;
  const int Dp = D | 1;
  double* rows = pd;                                                  // [64][Dp]
  float* Ls = reinterpret_cast<float*>(rows + kPropPart * Dp);        // [T]
  float* zs = Ls + ((T + 3) & ~3);                                    // [D][64]
  float* mus = zs + D * kPropPart;                                    // [D] f32(mu), [D] f32(prec)
  float* prs = mus + D;
  float* ds = prs + D;                                                // [D][64] f32(theta') - f32(mu)
  for (int e = threadIdx.x; e < T; e += blockDim.x) Ls[e] = L32[e];
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    mus[i] = f64_to_f32(mu[i]);
    if (!full) prs[i] = f64_to_f32(prec[i]);
  }
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kPropPart;
  const int np = static_cast<int>(P - p0 < kPropPart ? P - p0 : kPropPart);
  stage_rows(th, p0, np, D, Dp, rows);
  if (z_given) {
    for (int q = threadIdx.x; q < np * D; q += blockDim.x) {
      const int pp = q / D, d = q - pp * D;
      zs[d * kPropPart + pp] = static_cast<float>(z_given[(p0 + pp) * D + d]);
    }
  } else {
    // draw (particle p, word q) as before: counter p * ceil(D / 4) + q
    const int per = (D + 3) / 4;
    for (int q = threadIdx.x; q < np * per; q += blockDim.x) {
      const int pp = q / per, qq = q - pp * per;
      const uint4 r = draw(seed, static_cast<uint32_t>((p0 + pp) * per + qq), kStreamPropose, step);
      const float2 a = normals2(r.x, r.y), b = normals2(r.z, r.w);
      const float v[4] = {a.x, a.y, b.x, b.y};
      for (int u = 0; u < 4; ++u)
        if (4 * qq + u < D) zs[(4 * qq + u) * kPropPart + pp] = v[u];
    }
  }
  __syncthreads();
  const int pp = threadIdx.x / kPropSub, sub = threadIdx.x - pp * kPropSub;
  const bool live = pp < np;
  double* row = rows + pp * Dp;
  if (live)
    for (int i = sub; i < D; i += kPropSub) {
      const float* Li = Ls + i * (i + 1) / 2;
      float dlt = 0.f;
      for (int j = 0; j <= i; ++j) dlt = fmaf(Li[j], zs[j * kPropPart + pp], dlt);
      row[i] = row[i] + f32_to_f64(dlt);
    }
  __syncwarp();   // a particle's four threads are consecutive lanes of one warp
  if (full) {
    // full prior: the particle's threads form r_i = sum_j P32_ij d_j for their rows (j in
    // order) into the normals' slots, then its first thread sum_i d_i r_i in order i: the
    // values and operation order of prior_log_kernel
    if (live)
      for (int j = sub; j < D; j += kPropSub) ds[j * kPropPart + pp] = f64_to_f32(row[j]) - mus[j];
    __syncwarp();
    if (live) {
      const float* p32 = reinterpret_cast<const float*>(prec + static_cast<size_t>(D) * D);
      for (int i = sub; i < D; i += kPropSub) {
        const float* pi = p32 + static_cast<size_t>(i) * D;
        float r = 0.f;
        for (int j = 0; j < D; ++j) r = fmaf(pi[j], ds[j * kPropPart + pp], r);
        zs[i * kPropPart + pp] = r;
      }
    }
    __syncwarp();
  }
  if (live && sub == 0) {
    double lp;
    if (full) {
      float a = 0.f;
      for (int i = 0; i < D; ++i) a = fmaf(ds[i * kPropPart + pp], zs[i * kPropPart + pp], a);
      lp = -0.5 * f32_to_f64(a);
    } else {
      float a = 0.f;   // diagonal prior: the arithmetic of prior_log_kernel
      for (int i = 0; i < D; ++i) {
        const float d = f64_to_f32(row[i]) - mus[i];
        a = fmaf(d * d, prs[i], a);
      }
      lp = -0.5 * f32_to_f64(a);
    }
    lp_o[p0 + pp] = lp;
  }
  __syncthreads();
  unstage_rows(th_o, p0, np, D, Dp, rows);
}

constexpr int kAccThreads = 256;

// log u < la for u in [0, 1), decided as in FP64: la >= 0 always accepts; otherwise an FP32
// logarithm (error below 1e-5 for u >= 1e-30) decides unless it lies within 1e-5 + 1e-6 |la| of
// la, when the FP64 logarithm does.
__device__ __forceinline__ bool log_u_below(double u, double la) {
  if (la >= 0.0) return true;
  if (u >= 1e-30) {
    const double lf = static_cast<double>(logf(static_cast<float>(u)));
    const double margin = 1e-5 + 1e-6 * fabs(la);
    if (lf < la - margin) return true;
    if (lf > la + margin) return false;
  }
  return log(u) < la;
}

// Metropolis accept (Algorithm 2 step 2(c)i): log alpha = ll' - ll + lp' - lp, accept when
// log u < log alpha; the block then copies its accepted rows into the state element by element
// (coalesced). Counts accepts per warp.
__global__ void __launch_bounds__(kAccThreads)
accept_kernel(double* __restrict__ th, double* __restrict__ ll, double* __restrict__ lp,
              const double* __restrict__ th_p, const double* __restrict__ ll_p,
              const double* __restrict__ lp_p, int64_t P, int D, const double* __restrict__ u_given,
              uint64_t seed, uint64_t step_arg, const unsigned long long* __restrict__ step_dev,
              const int* __restrict__ flag, unsigned long long* __restrict__ n_acc, int* __restrict__ nonfinite,
              double* __restrict__ log_alpha_out, int* __restrict__ acc_out) {
  __shared__ unsigned char take[kAccThreads];
  if (*flag) return;
  const uint64_t step = step_dev ? *step_dev : step_arg;
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kAccThreads;
  const int64_t p = p0 + threadIdx.x;
  bool acc = false;
  if (p < P) {
    const double lpp = ll_p[p];
    if (!isfinite(lpp)) atomicOr(nonfinite, 1);
    const double la = (lpp - ll[p]) + (lp_p[p] - lp[p]);
    double u;
    if (u_given) {
      u = u_given[p];
    } else {
      const uint4 r = draw(seed, static_cast<uint32_t>(p), kStreamAccept, step);
      u = uniform53(r.x, r.y);
    }
    acc = log_u_below(u, la);
    if (acc) {
      ll[p] = lpp;
      lp[p] = lp_p[p];
    }
    if (log_alpha_out) log_alpha_out[p] = la;
    if (acc_out) acc_out[p] = acc ? 1 : 0;
  }
  take[threadIdx.x] = acc ? 1 : 0;
  const unsigned ballot = __ballot_sync(0xffffffffu, acc);
  if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(n_acc, static_cast<unsigned long long>(__popc(ballot)));
  __syncthreads();
  const int np = static_cast<int>(P - p0 < kAccThreads ? P - p0 : kAccThreads);
  for (int q = threadIdx.x; q < np * D; q += blockDim.x) {
    const int r = q / D;
    if (take[r]) th[p0 * D + q] = th_p[p0 * D + q];
  }
}

// ------------------------------------------------------------------------------ MALA
// Metropolis-adjusted Langevin M kernel (not in the paper; an exact MH kernel for the same
// posterior). With Sigma = h V = L L' and g the gradient of the log posterior,
//   theta' = theta + L v,  v = (1/2) L' g(theta) + z,   z ~ N(0, I),
// i.e. mean theta + (h/2) V g(theta) and covariance h V. The reverse move has residual
// L^{-1}(theta - theta' - (1/2) L L' g(theta')) = -(v + (1/2) L' g(theta')) =: w, so
//   log alpha = ll' - ll + lp' - lp - |w|^2 / 2 + |z|^2 / 2.

constexpr int kMalaThreads = 64;
// Row stride of the [D][particles] shared-memory arrays: 72, so that the 8 particles x 4 lanes of
// a warp (coordinate j = lane + 4 m) fall on 32 different banks ((8 j + particle) mod 32)
constexpr int kMalaStride = kMalaThreads + 8;

// Gradient of the prior log density, -Prec (theta - mu), component i, in FP32 (the MALA drift
// needs no more: any deterministic drift gives an exact Metropolis-Hastings kernel, and FP64
// arithmetic is scarce on this GPU): from the particle's centred
// coordinates dc[j * kMalaStride] = f32(theta_j) - f32(mu_j) and the FP32 copy of a full
// precision matrix (stored after the FP64 one).
__device__ __forceinline__ float prior_grad_f32(const float* dc, const double* prec, int D, bool full, int i) {
  if (!full) return -(f64_to_f32(prec[i]) * dc[i * kMalaStride]);
  const float* pi = reinterpret_cast<const float*>(prec + static_cast<size_t>(D) * D) + static_cast<size_t>(i) * D;
  float a = 0.f;
  for (int j = 0; j < D; ++j) a = fmaf(pi[j], dc[j * kMalaStride], a);
  return -a;
}

// Four threads per particle (64 particles per block): each takes every fourth row of the
// triangular products and every fourth coordinate of the squared norms |z|^2 and |w|^2 (FP32,
// combined by shuffles); the prior log kernel and the accept decision stay with its first thread.
constexpr int kMalaSub = 4;

// Sum of v over the four lanes of a particle (FP32, the same order in every lane).
__device__ __forceinline__ float quad_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

__global__ void __launch_bounds__(kMalaThreads * kMalaSub)
mala_propose_kernel(const double* __restrict__ th, const double* __restrict__ gll, int64_t P, int D,
                    const float* __restrict__ L32, uint64_t seed, uint64_t step_arg,
                    const unsigned long long* __restrict__ step_dev, const double* __restrict__ mu,
                    const double* __restrict__ prec, bool full, const int* __restrict__ flag,
                    double* __restrict__ th_o, double* __restrict__ lp_o, float* __restrict__ zq_o,
                    double* __restrict__ z2_o, const double* __restrict__ z_given) {
  if (*flag) return;
  const uint64_t step = step_dev ? *step_dev : step_arg;
  extern __shared__ float ms[];
  const int T = D * (D + 1) / 2;
  float* Ls = ms;                                  // [T] packed lower triangle
  float* gs = ms + ((T + 3) & ~3);                 // [D][72] gradient of the log posterior
  float* zs = gs + D * kMalaStride;                // [D][72] normals
  float* vs = zs + D * kMalaStride;                // [D][72] v = (1/2) L' g + z
  for (int e = threadIdx.x; e < T; e += blockDim.x) Ls[e] = L32[e];
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kMalaThreads;
  const int np = static_cast<int>(P - p0 < kMalaThreads ? P - p0 : kMalaThreads);
  const int pp = threadIdx.x / kMalaSub, sub = threadIdx.x - pp * kMalaSub;
  const int64_t p = p0 + pp;
  const bool live = pp < np;
  if (live) {
    // the centred coordinates in vs until v is formed, then the gradient of the log posterior
    const double* t = th + p * D;
    for (int i = sub; i < D; i += kMalaSub) vs[i * kMalaStride + pp] = f64_to_f32(t[i]) - f64_to_f32(mu[i]);
  }
  __syncwarp();
  if (live)
    for (int i = sub; i < D; i += kMalaSub)
      gs[i * kMalaStride + pp] = f64_to_f32(gll[p * D + i]) + prior_grad_f32(vs + pp, prec, D, full, i);
  if (z_given) {
    // given normals (step-level parity), rounded to FP32 like the drawn ones
    for (int q = threadIdx.x; q < np * D; q += blockDim.x) {
      const int qp = q / D, d = q - qp * D;
      zs[d * kMalaStride + qp] = static_cast<float>(z_given[(p0 + qp) * D + d]);
    }
  } else {
    // draw (particle p, word q) as before: counter p * ceil(D / 4) + q
    const int per = (D + 3) / 4;
    for (int q = threadIdx.x; q < np * per; q += blockDim.x) {
      const int qq = q / np, qp = q - qq * np;   // consecutive threads: consecutive particles
      const uint4 r = draw(seed, static_cast<uint32_t>((p0 + qp) * per + qq), kStreamPropose, step);
      const float2 a = normals2(r.x, r.y), b = normals2(r.z, r.w);
      const float v[4] = {a.x, a.y, b.x, b.y};
      for (int u = 0; u < 4; ++u)
        if (4 * qq + u < D) zs[(4 * qq + u) * kMalaStride + qp] = v[u];
    }
  }
  __syncthreads();
  if (live)
    for (int j = sub; j < D; j += kMalaSub) {   // v_j = (1/2) (L' g)_j + z_j
      float a = 0.f;
      for (int i = j; i < D; ++i) a = fmaf(Ls[i * (i + 1) / 2 + j], gs[i * kMalaStride + pp], a);
      vs[j * kMalaStride + pp] = fmaf(0.5f, a, zs[j * kMalaStride + pp]);
    }
  __syncwarp();
  double* o = th_o + p * D;
  if (live) {
    const double* t = th + p * D;
    for (int i = sub; i < D; i += kMalaSub) {
      const float* Li = Ls + i * (i + 1) / 2;
      float dlt = 0.f;
      for (int j = 0; j <= i; ++j) dlt = fmaf(Li[j], vs[j * kMalaStride + pp], dlt);
      o[i] = t[i] + static_cast<double>(dlt);
      zq_o[p * D + i] = vs[i * kMalaStride + pp];
    }
  }
  float zp = 0.f;
  if (live)
    for (int d = sub; d < D; d += kMalaSub) zp = fmaf(zs[d * kMalaStride + pp], zs[d * kMalaStride + pp], zp);
  const float z2 = quad_sum(zp);
  __syncwarp();   // the particle's new row is complete (global writes of its four lanes)
  if (live && sub == 0) {
    z2_o[p] = f32_to_f64(z2);
    lp_o[p] = prior_log_kernel(o, mu, prec, D, full);
  }
}

__global__ void __launch_bounds__(kMalaThreads * kMalaSub)
mala_accept_kernel(double* __restrict__ th, double* __restrict__ ll, double* __restrict__ lp,
                   double* __restrict__ g, const double* __restrict__ th_p, const double* __restrict__ ll_p,
                   const double* __restrict__ lp_p, const double* __restrict__ g_p, const float* __restrict__ zq,
                   const double* __restrict__ z2, const float* __restrict__ L32, int64_t P, int D,
                   const double* __restrict__ mu, const double* __restrict__ prec, bool full, uint64_t seed,
                   uint64_t step_arg, const unsigned long long* __restrict__ step_dev,
                   const int* __restrict__ flag, unsigned long long* __restrict__ n_acc,
                   int* __restrict__ nonfinite, const double* __restrict__ u_given,
                   double* __restrict__ la_out, int* __restrict__ acc_out) {
  if (*flag) return;
  const uint64_t step = step_dev ? *step_dev : step_arg;
  extern __shared__ float ms[];
  const int T = D * (D + 1) / 2;
  float* Ls = ms;
  float* gs = ms + ((T + 3) & ~3);                 // [D][72]
  float* ws = gs + D * kMalaStride;                // [D][72]: centred coordinates of theta', then w
  for (int e = threadIdx.x; e < T; e += blockDim.x) Ls[e] = L32[e];
  const int64_t p0 = static_cast<int64_t>(blockIdx.x) * kMalaThreads;
  const int np = static_cast<int>(P - p0 < kMalaThreads ? P - p0 : kMalaThreads);
  const int pp = threadIdx.x / kMalaSub, sub = threadIdx.x - pp * kMalaSub;
  const int64_t p = p0 + pp;
  const bool live = pp < np;
  if (live) {
    const double* tp = th_p + p * D;
    for (int i = sub; i < D; i += kMalaSub) ws[i * kMalaStride + pp] = f64_to_f32(tp[i]) - f64_to_f32(mu[i]);
  }
  __syncwarp();
  if (live)
    for (int i = sub; i < D; i += kMalaSub)
      gs[i * kMalaStride + pp] = f64_to_f32(g_p[p * D + i]) + prior_grad_f32(ws + pp, prec, D, full, i);
  __syncthreads();
  float wp = 0.f;
  if (live)
    for (int j = sub; j < D; j += kMalaSub) {   // w_j = z_j + (1/2) (L' g')_j
      float b = 0.f;
      for (int i = j; i < D; ++i) b = fmaf(Ls[i * (i + 1) / 2 + j], gs[i * kMalaStride + pp], b);
      const float w = fmaf(0.5f, b, zq[p * D + j]);
      wp = fmaf(w, w, wp);
    }
  const double w2 = f32_to_f64(quad_sum(wp));
  bool acc = false;
  if (live && sub == 0) {
    const double lpp = ll_p[p];
    if (!isfinite(lpp)) atomicOr(nonfinite, 1);
    const double la = (lpp - ll[p]) + (lp_p[p] - lp[p]) - 0.5 * w2 + 0.5 * z2[p];
    double u;
    if (u_given) {
      u = u_given[p];
    } else {
      const uint4 r = draw(seed, static_cast<uint32_t>(p), kStreamAccept, step);
      u = uniform53(r.x, r.y);
    }
    acc = log(u) < la;
    if (la_out) la_out[p] = la;
    if (acc_out) acc_out[p] = acc ? 1 : 0;
    if (acc) {
      ll[p] = lpp;
      lp[p] = lp_p[p];
    }
  }
  // the decision to the particle's four lanes, which copy its row and gradient
  acc = __shfl_sync(0xffffffffu, acc ? 1 : 0, threadIdx.x & ~(kMalaSub - 1) & 31) != 0;
  if (acc)
    for (int d = sub; d < D; d += kMalaSub) {
      th[p * D + d] = th_p[p * D + d];
      g[p * D + d] = g_p[p * D + d];
    }
  const unsigned ballot = __ballot_sync(0xffffffffu, acc && sub == 0);
  if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(n_acc, static_cast<unsigned long long>(__popc(ballot)));
}

// Group sums of monitoring or output functions: functions are theta coordinates f < nth
// (if with_theta), then ll (if with_ll), then the log-odds theta_c' xbar. Per group j and
// function f: sums of (g - ref_f) and (g - ref_f)^2, ref_f the value at particle 0.
__device__ __forceinline__ double fn_value(const double* th, const double* ll, const double* xbar, int64_t p,
                                           int f, int D, int k, bool with_theta, bool with_ll) {
  if (with_theta) {
    if (f < D) return th[p * D + f];
    f -= D;
  }
  if (with_ll) {
    if (f == 0) return ll[p];
    f -= 1;
  }
  // theta_c' xbar: FP32 products and sum (a monitoring function; 1e-7 relative is ample)
  const double* t = th + p * D + f * k;
  float a = 0.f;
  for (int i = 0; i < k; ++i) a = fmaf(f64_to_f32(t[i]), f64_to_f32(xbar[i]), a);
  return f32_to_f64(a);
}

__global__ void group_moments_kernel(const double* __restrict__ th, const double* __restrict__ ll,
                                     const double* __restrict__ xbar, int N, int D, int k, int F, bool with_theta,
                                     bool with_ll, double* __restrict__ sums) {
  __shared__ double sh[33];
  const int j = blockIdx.x, f = blockIdx.y, z = blockIdx.z, S = gridDim.z;
  const int per = (N + S - 1) / S;
  const int n_lo = z * per, n_hi = min(N, n_lo + per);
  const double ref = fn_value(th, ll, xbar, 0, f, D, k, with_theta, with_ll);
  double s1 = 0.0, s2 = 0.0;
  for (int n = n_lo + threadIdx.x; n < n_hi; n += blockDim.x) {
    const double g = fn_value(th, ll, xbar, static_cast<int64_t>(j) * N + n, f, D, k, with_theta, with_ll) - ref;
    s1 += g;
    s2 = fma(g, g, s2);
  }
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    double* o = sums + ((static_cast<int64_t>(j) * F + f) * S + z) * 3;
    o[0] = s1;
    o[1] = s2;
    o[2] = ref;
  }
}

// Monitoring moments after an M step (Algorithm 2 step 2(c)iii): functions f = 0: ll, f = c:
// theta_c' xbar (c = 1..NC), F = NC + 1 <= 4. Block (group j, part z) stages its particles'
// theta rows in shared memory (coalesced), each thread evaluates all F functions of its particle
// and the block writes, per function, the sums of (g - ref_f) and (g - ref_f)^2 with ref_f the
// value at particle 0, in the [J][F][S][3] layout of group_moments_kernel.
constexpr int kMonThreads = 128;

template <int F>
__global__ void __launch_bounds__(kMonThreads)
monitor_moments_kernel(const double* __restrict__ th, const double* __restrict__ ll,
                       const double* __restrict__ xbar, int N, int D, int k, double* __restrict__ sums) {
  extern __shared__ double mrow[];   // [128][Dp]
  __shared__ double sh[33];
  __shared__ float xb[kMaxD];
  const int Dp = D | 1;
  const int j = blockIdx.x, z = blockIdx.y, S = gridDim.y;
  const int per = (N + S - 1) / S;
  const int n_lo = z * per, n_hi = min(N, n_lo + per);
  for (int i = threadIdx.x; i < k; i += blockDim.x) xb[i] = f64_to_f32(xbar[i]);
  __syncthreads();
  auto value = [&](const double* row, double llv, int f) -> double {
    if (f == 0) return llv;
    float a = 0.f;
    const double* t = row + (f - 1) * k;
    for (int i = 0; i < k; ++i) a = fmaf(f64_to_f32(t[i]), xb[i], a);
    return f32_to_f64(a);
  };
  double ref[F];
#pragma unroll
  for (int f = 0; f < F; ++f) ref[f] = value(th, ll[0], f);
  double s1[F], s2[F];
#pragma unroll
  for (int f = 0; f < F; ++f) s1[f] = s2[f] = 0.0;
  for (int n0 = n_lo; n0 < n_hi; n0 += kMonThreads) {
    const int np = min(kMonThreads, n_hi - n0);
    const int64_t p0 = static_cast<int64_t>(j) * N + n0;
    __syncthreads();
    stage_rows(th, p0, np, D, Dp, mrow);
    __syncthreads();
    if (static_cast<int>(threadIdx.x) < np) {
      const double* row = mrow + threadIdx.x * Dp;
      const double llv = ll[p0 + threadIdx.x];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const double g = value(row, llv, f) - ref[f];
        s1[f] += g;
        s2[f] = fma(g, g, s2[f]);
      }
    }
  }
#pragma unroll
  for (int f = 0; f < F; ++f) {
    const double a = block_sum(s1[f], sh);
    const double b = block_sum(s2[f], sh);
    if (threadIdx.x == 0) {
      double* o = sums + ((static_cast<int64_t>(j) * F + f) * S + z) * 3;
      o[0] = a;
      o[1] = b;
      o[2] = ref[f];
    }
  }
}

// Device side of the step-size rule and the stopping rule of an M phase (Algorithm 2 step
// 2(c)ii-iii) for a captured M phase: the group sums of the monitoring functions reduced in the
// order of the host path (reduce_parts, moments_from_sums, read_step, mstep_impl), every
// operation rounded separately as there, so that both paths take identical decisions. Writes
// h, the acceptance rate and the minimum RNE of the step to steplog[r], advances h and the
// Philox step word and sets the loop condition (0 after the stopping rule, r_max steps or an
// error); with sigma_log, also copies the step's Sigma (D x D) to sigma_log[r]. One block; sums:
// J F 3 doubles of dynamic shared memory.
constexpr int kCtlMaxF = 64;

__global__ void __launch_bounds__(128)
mstep_control_kernel(StepCtl* __restrict__ ctl, const unsigned long long* __restrict__ counters,
                     const double* __restrict__ parts, int J, int F, int S, int N, int64_t P, double K,
                     double target, double h_step, double h_min, double h_max, double* __restrict__ steplog,
                     const double* __restrict__ sigma, int D, double* __restrict__ sigma_log,
                     cudaGraphConditionalHandle cond, cudaGraphConditionalHandle cond2, int model_mode,
                     int2* __restrict__ ptiles, int pt_lo, int pt_hi) {
  extern __shared__ double sums[];   // [J][F][3]
  __shared__ double rne[kCtlMaxF];
  if (model_mode && ctl->stop) {   // a stopped model stays stopped (its conditional nodes are off)
    if (threadIdx.x == 0) {
      cudaGraphSetConditional(cond, 0u);
      cudaGraphSetConditional(cond2, 0u);
    }
    return;
  }
  const int r = ctl->r;   // read by every thread before thread 0 advances it
  if (sigma_log)
    for (int e = threadIdx.x; e < D * D; e += blockDim.x)
      sigma_log[static_cast<size_t>(r) * D * D + e] = sigma[e];
  for (int q = threadIdx.x; q < J * F; q += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int z = 0; z < S; ++z) {
      a = __dadd_rn(a, parts[(static_cast<size_t>(q) * S + z) * 3 + 0]);
      b = __dadd_rn(b, parts[(static_cast<size_t>(q) * S + z) * 3 + 1]);
    }
    sums[q * 3 + 0] = a;
    sums[q * 3 + 1] = b;
  }
  __syncthreads();
  const double dN = static_cast<double>(N), dJ = static_cast<double>(J);
  for (int f = threadIdx.x; f < F; f += blockDim.x) {
    double gbar = 0.0, s2 = 0.0;
    for (int j = 0; j < J; ++j) {
      gbar = __dadd_rn(gbar, __ddiv_rn(sums[(j * F + f) * 3 + 0], dN));
      s2 = __dadd_rn(s2, sums[(j * F + f) * 3 + 1]);
    }
    gbar = __ddiv_rn(gbar, dJ);
    double vh = 0.0;
    for (int j = 0; j < J; ++j) {
      const double d = __dsub_rn(__ddiv_rn(sums[(j * F + f) * 3 + 0], dN), gbar);
      vh = __dadd_rn(vh, __dmul_rn(d, d));
    }
    vh = __dmul_rn(vh, __ddiv_rn(dN, __dsub_rn(dJ, 1.0)));
    const double v0 = __dsub_rn(__ddiv_rn(s2, __dmul_rn(dJ, dN)), __dmul_rn(gbar, gbar));
    const double var = (0.0 < v0) ? v0 : 0.0;
    rne[f] = vh > 0.0 ? __ddiv_rn(var, vh) : INFINITY;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int* flags = reinterpret_cast<const int*>(counters + 1);
  const int err = flags[0] ? 1 : (flags[1] ? 2 : 0);
  bool stop;
  if (err) {
    ctl->err = err;
    stop = true;
  } else {
    double rmin = INFINITY;
    for (int f = 0; f < F; ++f) rmin = (rne[f] < rmin) ? rne[f] : rmin;
    const double alpha = __ddiv_rn(static_cast<double>(counters[0]), static_cast<double>(P));
    const double h = ctl->h;
    double hn;
    if (alpha > target) {
      const double a = __dadd_rn(h, h_step);
      hn = (h_max < a) ? h_max : a;
    } else {
      const double a = __dsub_rn(h, h_step);
      hn = (a < h_min) ? h_min : a;
    }
    steplog[3 * r + 0] = h;
    steplog[3 * r + 1] = alpha;
    steplog[3 * r + 2] = rmin;
    ctl->h = hn;
    ctl->step += 1;
    ctl->r = r + 1;
    stop = (rmin >= K) || (r + 1 >= ctl->r_max);
  }
  ctl->stop = stop ? 1 : 0;
  cudaGraphSetConditional(cond, stop ? 0u : 1u);
  if (model_mode) {
    // one model of a batched M phase: cond and cond2 switch its own kernels; once it stops, the
    // batched log-likelihood launch skips its particle tiles (prefix length 0)
    cudaGraphSetConditional(cond2, stop ? 0u : 1u);
    if (stop && ptiles)
      for (int i = pt_lo; i < pt_hi; ++i) ptiles[i].x = 0;
  }
}

// Loop condition of a batched M phase: another lockstep step while any model still moves. ctl[M]
// counts the loop's iterations: past its r_max (the models' step cap, which every model's own
// rule enforces first) the loop ends with err = 3.
__global__ void batch_continue_kernel(StepCtl* __restrict__ ctl, int M, cudaGraphConditionalHandle cond) {
  int any = 0;
  for (int m = 0; m < M; ++m) any |= (ctl[m].stop == 0) ? 1 : 0;
  const int it = ++ctl[M].r;
  if (any && it >= ctl[M].r_max) {
    ctl[M].err = 3;
    any = 0;
  }
  cudaGraphSetConditional(cond, any ? 1u : 0u);
}

}  // namespace

// ------------------------------------------------------------------------------ host helpers

struct Moments {
  std::vector<double> mean, sd, nse, rne;
};

constexpr int kMomParts = 32;  // blocks per group in the monitoring moments (128 particles each at N = 4096)

// Sum the S partial blocks of each (group, function) in a fixed order: [J][F][S][3] -> [J][F][3].
static std::vector<double> reduce_parts(const std::vector<double>& parts, int J, int F, int S) {
  std::vector<double> out(static_cast<size_t>(J) * F * 3, 0.0);
  for (int q = 0; q < J * F; ++q) {
    double a = 0.0, b = 0.0;
    for (int z = 0; z < S; ++z) {
      a += parts[(static_cast<size_t>(q) * S + z) * 3 + 0];
      b += parts[(static_cast<size_t>(q) * S + z) * 3 + 1];
    }
    out[q * 3 + 0] = a;
    out[q * 3 + 1] = b;
    out[q * 3 + 2] = parts[static_cast<size_t>(q) * S * 3 + 2];
  }
  return out;
}

// Eqs. (3), (5), (6), (7) as read (NSE = sqrt(vhat / (J N))), (10) from group sums.
static Moments moments_from_sums(const std::vector<double>& sums, int J, int N, int F) {
  Moments m;
  m.mean.resize(F);
  m.sd.resize(F);
  m.nse.resize(F);
  m.rne.resize(F);
  for (int f = 0; f < F; ++f) {
    const double ref = sums[(0 * F + f) * 3 + 2];
    double gbar = 0.0, s2 = 0.0;
    std::vector<double> gj(J);
    for (int j = 0; j < J; ++j) {
      gj[j] = sums[(j * F + f) * 3 + 0] / N;
      gbar += gj[j];
      s2 += sums[(j * F + f) * 3 + 1];
    }
    gbar /= J;
    double vh = 0.0;
    for (int j = 0; j < J; ++j) vh += (gj[j] - gbar) * (gj[j] - gbar);
    vh *= static_cast<double>(N) / (J - 1.0);
    const double var = std::max(0.0, s2 / (static_cast<double>(J) * N) - gbar * gbar);
    m.mean[f] = ref + gbar;
    m.sd[f] = std::sqrt(var);
    m.nse[f] = std::sqrt(vh / (static_cast<double>(J) * N));
    m.rne[f] = vh > 0.0 ? var / vh : INFINITY;
  }
  return m;
}

static void swapbuf(DevBuf& a, DevBuf& b) {
  std::swap(a.ptr, b.ptr);
  std::swap(a.bytes, b.bytes);
}

static bool prior_full(const sps_ctx* ctx) { return ctx->prior_kind == SPS_PRIOR_FULL; }

static int cov_blocks(int64_t P) { return static_cast<int>(std::min<int64_t>(296, (P + kCovSub - 1) / kCovSub)); }

// V = pooled covariance of theta [P x D] (divisor P - 1) into V and/or Sigma = scale V (device,
// full symmetric); partial: cov_blocks(P) x (T + D) doubles of scratch.
static sps_status launch_cov(sps_ctx* ctx, const double* theta, int64_t P, int D, double scale,
                             const double* scale_dev, double* partial, double* V, double* Sigma) {
  const int T = D * (D + 1) / 2;
  const int blocks = cov_blocks(P);
  const int64_t per = (P + blocks - 1) / blocks;
  const int E = T + D;
  const size_t smem = sizeof(float) * (kCovSub + 1) * D;
  if (E <= 2 * kCovThreads)
    cov_moments_kernel<2><<<blocks, kCovThreads, smem, ctx->stream>>>(theta, P, D, per, partial);
  else if (E <= 8 * kCovThreads)
    cov_moments_kernel<8><<<blocks, kCovThreads, smem, ctx->stream>>>(theta, P, D, per, partial);
  else if (E <= 16 * kCovThreads)
    cov_moments_kernel<16><<<blocks, kCovThreads, smem, ctx->stream>>>(theta, P, D, per, partial);
  else
    cov_moments_kernel<kCovMaxEnt><<<blocks, kCovThreads, smem, ctx->stream>>>(theta, P, D, per, partial);
  ++ctx->launches;
  cov_final_kernel<<<static_cast<unsigned>((T + 7) / 8), 256, 0, ctx->stream>>>(partial, blocks, D, P, scale, scale_dev, V,
                                                                                 Sigma); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

// V (and Sigma = h V unless sigma_in) then its Cholesky factor into st->chol / scratch L32.
// Sigma = h V (or the given Sigma) into st->cov; factor_proposal adds its Cholesky factor.
static sps_status proposal_sigma(sps_ctx* ctx, sps_state* st, const double* d_theta, double h, const double* h_dev,
                                 const double* sigma_host, double* sigma_out) {
  const int D = ctx->D;
  double* d_sigma = st->cov.as<double>();
  if (sigma_host) {
    SPS_CUDA_TRY(cudaMemcpyAsync(d_sigma, sigma_host, sizeof(double) * D * D, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    SPS_TRY(launch_cov(ctx, d_theta, st->P, D, h, h_dev, st->scratch.as<double>(), nullptr, d_sigma));
  }
  if (sigma_out)
    SPS_CUDA_TRY(cudaMemcpyAsync(sigma_out, d_sigma, sizeof(double) * D * D, cudaMemcpyDeviceToHost, ctx->stream));
  return SPS_OK;
}

// The Cholesky job of a state's Sigma (for one batched factorisation of several states).
static CholJob chol_job(sps_ctx* ctx, sps_state* st, int* d_flag) {
  const int D = ctx->D;
  CholJob j;
  j.A = st->cov.as<double>();
  j.L = st->chol.as<double>();
  j.L32 = reinterpret_cast<float*>(st->chol.as<double>() + static_cast<size_t>(D) * D);
  j.flag = d_flag;
  j.D = D;
  j.pad = 0;
  return j;
}

static sps_status factor_proposal(sps_ctx* ctx, sps_state* st, const double* d_theta, double h,
                                  const double* h_dev, const double* sigma_host, double* sigma_out, int* d_flag) {
  const int D = ctx->D;
  const int T = D * (D + 1) / 2;
  double* d_sigma = st->cov.as<double>();
  SPS_TRY(proposal_sigma(ctx, st, d_theta, h, h_dev, sigma_host, sigma_out));
  float* L32 = reinterpret_cast<float*>(st->chol.as<double>() + static_cast<size_t>(D) * D);
  SPS_CUDA_TRY(cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(sizeof(double) * T)));
  cholesky_kernel<<<1, kCholThreads, sizeof(double) * T, ctx->stream>>>(d_sigma, D, st->chol.as<double>(), L32,
                                                                        d_flag); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

static size_t propose_smem(int D) {
  const int T = D * (D + 1) / 2;
  return sizeof(double) * kPropPart * static_cast<size_t>(D | 1) +
         sizeof(float) * (((T + 3) & ~3) + 2 * static_cast<size_t>(D) * kPropPart + 2 * static_cast<size_t>(D));
}

static sps_status launch_propose(sps_ctx* ctx, sps_state* st, const double* d_theta, int64_t P, const double* z,
                                 uint64_t step, const unsigned long long* step_dev, int* d_flag, double* th_o,
                                 double* lp_o) {
  const int D = ctx->D;
  const size_t smem = propose_smem(D);
  SPS_CUDA_TRY(cudaFuncSetAttribute(propose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
  const float* L32 = reinterpret_cast<const float*>(st->chol.as<double>() + static_cast<size_t>(D) * D);
  propose_kernel<<<static_cast<unsigned>((P + kPropPart - 1) / kPropPart), kPropPart * kPropSub, smem, ctx->stream>>>(
      d_theta, P, D, L32, z, st->seed, step, step_dev, ctx->d_prior_mean.as<double>(), ctx->d_prior_prec.as<double>(),
      prior_full(ctx), d_flag, th_o, lp_o); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

// Per-state buffers of the given size (theta etc.), counters and scratch.
static sps_status state_buffers(sps_ctx* ctx, sps_state* st) {
  const int64_t P = st->P;
  const int D = ctx->D;
  const size_t pd = static_cast<size_t>(P) * D * sizeof(double);
  SPS_CUDA_TRY(st->theta.reserve(pd));
  SPS_CUDA_TRY(st->theta_prop.reserve(pd));
  SPS_CUDA_TRY(st->ll.reserve(P * sizeof(double)));
  SPS_CUDA_TRY(st->ll_prop.reserve(P * sizeof(double)));
  SPS_CUDA_TRY(st->lp.reserve(P * sizeof(double)));
  SPS_CUDA_TRY(st->lp_prop.reserve(P * sizeof(double)));
  SPS_CUDA_TRY(st->logw.reserve(P * sizeof(double)));
  SPS_CUDA_TRY(st->logml.reserve(st->J * sizeof(double)));
  SPS_CUDA_TRY(st->idx.reserve(P * sizeof(int)));
  SPS_CUDA_TRY(st->cov.reserve(sizeof(double) * D * D));
  SPS_CUDA_TRY(st->chol.reserve(sizeof(double) * D * D + sizeof(float) * (D * (D + 1) / 2 + 4)));
  const size_t T = static_cast<size_t>(D) * (D + 1) / 2;
  const int F = D + ctx->NC + 1;
  const size_t ess_rows_max = static_cast<size_t>(std::max<int64_t>(1, std::min<int64_t>(1024, (int64_t{1} << 25) / P)));
  SPS_CUDA_TRY(st->scratch.reserve(std::max({sizeof(double) * (T + D) * cov_blocks(P),
                                             sizeof(double) * 3 * static_cast<size_t>(st->J) * F + 64,
                                             sizeof(double) * 2 * static_cast<size_t>(st->J) * kLmeParts,
                                             sizeof(double) * 3 * static_cast<size_t>(st->J) * (1 + ctx->NC) * kMomParts,
                                             sizeof(double) * 3 * kEssParts * ess_rows_max})));
  // counters: [0] accepts (u64), then int flags: [2] chol failure, [3] non-finite, [4] resample
  SPS_CUDA_TRY(st->counters.reserve(64));
  return SPS_OK;
}

}  // namespace sps

using namespace sps;

namespace {

struct Counters {
  unsigned long long accepts;
  int chol_bad, nonfinite, res_bad, pad;
};

sps_status read_counters(sps_ctx* ctx, sps_state* st, Counters* c) {
  SPS_CUDA_TRY(cudaMemcpyAsync(c, st->counters.ptr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

int* flag_ptr(sps_state* st, int which) { return reinterpret_cast<int*>(st->counters.as<char>() + 8) + which; }

sps_status check_state(sps_ctx* ctx, const sps_state* st) {
  if (!ctx || !st || st->ctx != ctx) return fail(ctx, SPS_ERR_INVALID_ARG, "state does not belong to this context");
  return SPS_OK;
}

// Monitoring moments (ll, theta_c' xbar) after an M step: launch the group sums, then read them
// with the step's counters in one synchronisation; min RNE over the set.
void launch_monitoring(sps_ctx* ctx, sps_state* st) {
  const int F = 1 + ctx->NC;
  const size_t smem = sizeof(double) * kMonThreads * (ctx->D | 1);
  const dim3 grid(st->J, kMomParts);
  double* out = st->scratch.as<double>();
  const double* th = st->theta.as<double>();
  const double* ll = st->ll.as<double>();
  const double* xb = ctx->xbar.as<double>();
#define SPS_MON_CASE(FF)                                                                                  \
  if (F == FF) {                                                                                          \
    cudaFuncSetAttribute(monitor_moments_kernel<FF>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                         static_cast<int>(smem));                                                         \
    monitor_moments_kernel<FF><<<grid, kMonThreads, smem, ctx->stream>>>(th, ll, xb, st->N, ctx->D, ctx->k, out); \
  }
  SPS_MON_CASE(2)
  SPS_MON_CASE(3)
  SPS_MON_CASE(4)
#undef SPS_MON_CASE
  if (F > 4)
    group_moments_kernel<<<dim3(st->J, F, kMomParts), 256, 0, ctx->stream>>>(th, ll, xb, st->N, ctx->D, ctx->k, F,
                                                                            false, true, out);
  ++ctx->launches;
}

// An M step's counters and monitoring sums, copied to the state's page-locked host buffer
// (enqueued; readback_result reads them after the stream has synchronised).
sps_status readback_issue(sps_ctx* ctx, sps_state* st) {
  const size_t n_parts = static_cast<size_t>(st->J) * (1 + ctx->NC) * kMomParts * 3;
  const size_t bytes = sizeof(Counters) + n_parts * sizeof(double);
  if (st->pinned_bytes < bytes) {
    if (st->pinned) cudaFreeHost(st->pinned);
    st->pinned = nullptr;
    st->pinned_bytes = 0;
    SPS_CUDA_TRY(cudaMallocHost(&st->pinned, bytes));
    st->pinned_bytes = bytes;
  }
  SPS_CUDA_TRY(cudaGetLastError());
  char* h = static_cast<char*>(st->pinned);
  SPS_CUDA_TRY(cudaMemcpyAsync(h, st->counters.ptr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(h + sizeof(Counters), st->scratch.ptr, n_parts * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
  return SPS_OK;
}

void readback_result(sps_ctx* ctx, const sps_state* st, Counters* c, double* rne_min) {
  const int F = 1 + ctx->NC;
  const char* h = static_cast<const char*>(st->pinned);
  std::memcpy(c, h, sizeof(Counters));
  const double* p = reinterpret_cast<const double*>(h + sizeof(Counters));
  const std::vector<double> parts(p, p + static_cast<size_t>(st->J) * F * kMomParts * 3);
  Moments m = moments_from_sums(reduce_parts(parts, st->J, F, kMomParts), st->J, st->N, F);
  double r = INFINITY;
  for (double v : m.rne) r = std::min(r, v);
  *rne_min = r;
}

// Before an M step: the cached log-likelihood (and, for MALA, its gradient) recomputed with the
// function the proposals are evaluated with, when the C phase or another kernel left it stale.
sps_status mstep_prepare(sps_ctx* ctx, sps_state* st, int kernel) {
  if (kernel != SPS_MKERNEL_RW && kernel != SPS_MKERNEL_MALA)
    return fail(ctx, SPS_ERR_INVALID_ARG, "unknown M kernel");
  const int precision = ctx->opt.precision;
  const int D = ctx->D;
  const bool mala = (kernel == SPS_MKERNEL_MALA);
  const int kind = mala ? 2 : (precision == SPS_PREC_FP32 ? 1 : 0);
  if (mala) {
    SPS_CUDA_TRY(st->grad.reserve(sizeof(double) * st->P * D));
    SPS_CUDA_TRY(st->grad_prop.reserve(sizeof(double) * st->P * D));
    SPS_CUDA_TRY(st->zq.reserve(sizeof(float) * st->P * D));
    SPS_CUDA_TRY(st->z2.reserve(sizeof(double) * st->P));
    if (st->ll_stale || st->ll_kind != kind || !st->grad_valid) {
      SPS_TRY(loglik_grad_dispatch(ctx, st->theta.as<double>(), st->P, st->t, st->ll.as<double>(),
                               st->grad.as<double>()));
      st->ll_stale = false;
      st->ll_kind = kind;
      st->grad_valid = true;
    }
  } else if (st->ll_stale || st->ll_kind != kind) {
    SPS_TRY(loglik_dispatch(ctx, st->theta.as<double>(), st->P, st->t, st->ll.as<double>(), precision));
    st->ll_stale = false;
    st->ll_kind = kind;
  }
  return SPS_OK;
}

// The work of one M step on the stream: counters cleared, Sigma = h V (or the given Sigma) and
// its Cholesky factor, proposals with the prior log kernel, their log-likelihood (and gradient),
// the Metropolis decisions, the monitoring sums. With ctl (a captured M phase) h and the Philox
// step word are read on the device from ctl; otherwise they are h and step.
// Random-walk step, first half: counters cleared, Sigma and its factor, proposals theta' with
// their prior log kernel.
sps_status rw_issue_propose(sps_ctx* ctx, sps_state* st, const double* sigma, double* sigma_used, double h,
                            uint64_t step, StepCtl* ctl) {
  SPS_CUDA_TRY(cudaMemsetAsync(st->counters.ptr, 0, sizeof(Counters), ctx->stream));
  SPS_TRY(factor_proposal(ctx, st, st->theta.as<double>(), h, ctl ? &ctl->h : nullptr, sigma, sigma_used,
                          flag_ptr(st, 0)));
  return launch_propose(ctx, st, st->theta.as<double>(), st->P, nullptr, step, ctl ? &ctl->step : nullptr,
                        flag_ptr(st, 0), st->theta_prop.as<double>(), st->lp_prop.as<double>());
}

// Random-walk step, second half (after ll_prop holds the proposals' log-likelihoods): the
// Metropolis decisions and the monitoring sums.
sps_status rw_issue_accept(sps_ctx* ctx, sps_state* st, uint64_t step, StepCtl* ctl) {
  accept_kernel<<<static_cast<unsigned>((st->P + kAccThreads - 1) / kAccThreads), kAccThreads, 0, ctx->stream>>>(
      st->theta.as<double>(), st->ll.as<double>(), st->lp.as<double>(), st->theta_prop.as<double>(),
      st->ll_prop.as<double>(), st->lp_prop.as<double>(), st->P, ctx->D, nullptr, st->seed, step,
      ctl ? &ctl->step : nullptr, flag_ptr(st, 0), st->counters.as<unsigned long long>(), flag_ptr(st, 1), nullptr,
      nullptr); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  launch_monitoring(ctx, st);
  return SPS_OK;
}

// MALA proposal, the proposals' log-likelihood and gradient, and the Metropolis-Hastings
// decisions, after factor_proposal has left the FP32 factor of Sigma in st->chol. z_given /
// u_given replace the Philox normals / uniforms; la_out / acc_out receive log alpha and the
// decisions (all optional).
static sps_status mala_issue(sps_ctx* ctx, sps_state* st, uint64_t step, const unsigned long long* step_dev,
                             const double* z_given, const double* u_given, double* la_out, int* acc_out) {
  const int D = ctx->D;
  const int T = D * (D + 1) / 2;
  const size_t smem_p = sizeof(float) * (((T + 3) & ~3) + 3 * static_cast<size_t>(D) * kMalaStride);
  const size_t smem_a = sizeof(float) * (((T + 3) & ~3) + 2 * static_cast<size_t>(D) * kMalaStride);
  SPS_CUDA_TRY(cudaFuncSetAttribute(mala_propose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem_p)));
  SPS_CUDA_TRY(cudaFuncSetAttribute(mala_accept_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem_a)));
  const float* L32 = reinterpret_cast<const float*>(st->chol.as<double>() + static_cast<size_t>(D) * D);
  const unsigned blocks = static_cast<unsigned>((st->P + kMalaThreads - 1) / kMalaThreads);
  mala_propose_kernel<<<blocks, kMalaThreads * kMalaSub, smem_p, ctx->stream>>>(
      st->theta.as<double>(), st->grad.as<double>(), st->P, D, L32, st->seed, step, step_dev,
      ctx->d_prior_mean.as<double>(), ctx->d_prior_prec.as<double>(), prior_full(ctx), flag_ptr(st, 0),
      st->theta_prop.as<double>(), st->lp_prop.as<double>(), st->zq.as<float>(), st->z2.as<double>(), z_given);
  ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  SPS_TRY(loglik_grad_dispatch(ctx, st->theta_prop.as<double>(), st->P, st->t, st->ll_prop.as<double>(),
                               st->grad_prop.as<double>()));
  mala_accept_kernel<<<blocks, kMalaThreads * kMalaSub, smem_a, ctx->stream>>>(
      st->theta.as<double>(), st->ll.as<double>(), st->lp.as<double>(), st->grad.as<double>(),
      st->theta_prop.as<double>(), st->ll_prop.as<double>(), st->lp_prop.as<double>(), st->grad_prop.as<double>(),
      st->zq.as<float>(), st->z2.as<double>(), L32, st->P, D, ctx->d_prior_mean.as<double>(),
      ctx->d_prior_prec.as<double>(), prior_full(ctx), st->seed, step, step_dev, flag_ptr(st, 0),
      st->counters.as<unsigned long long>(), flag_ptr(st, 1), u_given, la_out, acc_out);
  ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

sps_status mstep_issue(sps_ctx* ctx, sps_state* st, int kernel, const double* sigma, double* sigma_used, double h,
                       uint64_t step, StepCtl* ctl) {
  const bool mala = (kernel == SPS_MKERNEL_MALA);
  const unsigned long long* step_dev = ctl ? &ctl->step : nullptr;
  if (!mala) {
    SPS_TRY(rw_issue_propose(ctx, st, sigma, sigma_used, h, step, ctl));
    SPS_TRY(loglik_dispatch(ctx, st->theta_prop.as<double>(), st->P, st->t, st->ll_prop.as<double>(),
                            ctx->opt.precision));
    return rw_issue_accept(ctx, st, step, ctl);
  }
  SPS_CUDA_TRY(cudaMemsetAsync(st->counters.ptr, 0, sizeof(Counters), ctx->stream));
  SPS_TRY(factor_proposal(ctx, st, st->theta.as<double>(), h, ctl ? &ctl->h : nullptr, sigma, sigma_used,
                          flag_ptr(st, 0)));
  SPS_TRY(mala_issue(ctx, st, step, step_dev, nullptr, nullptr, nullptr, nullptr));
  launch_monitoring(ctx, st);
  return SPS_OK;
}

sps_status mstep_finish(sps_ctx* ctx, sps_state* st, int kernel, double h, bool adapt, sps_mstep_info* info);
sps_status mstep_rule(sps_ctx* ctx, sps_state* st, int kernel, double h, bool adapt, sps_mstep_info* info);

// One M step, issued and read back (Algorithm 2 step 2(c)): the acceptance rate drives the
// step-size rule unless Sigma is given.
sps_status mstep_impl(sps_ctx* ctx, sps_state* st, int kernel, const double* sigma, double* sigma_used,
                      sps_mstep_info* info) {
  SPS_TRY(mstep_prepare(ctx, st, kernel));
  const double h = st->h;
  const uint64_t step = ++st->step_counter;
  // Sigma is read back after the step's one synchronisation (st->cov still holds it): a copy
  // into pageable host memory issued mid-step would hold the host until the covariance is done
  // and delay the launches of the rest of the step
  SPS_TRY(mstep_issue(ctx, st, kernel, sigma, nullptr, h, step, nullptr));
  if (kernel == SPS_MKERNEL_RW) st->grad_valid = false;
  const sps_status r = mstep_finish(ctx, st, kernel, h, sigma == nullptr, info);
  if (sigma_used) {
    SPS_CUDA_TRY(cudaMemcpyAsync(sigma_used, st->cov.ptr, sizeof(double) * ctx->D * ctx->D, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  return r;
}

// Read an issued M step back and apply the step-size rule (when adapt): errors of the step,
// the acceptance rate and the minimum RNE of the monitoring set.
sps_status mstep_finish(sps_ctx* ctx, sps_state* st, int kernel, double h, bool adapt, sps_mstep_info* info) {
  SPS_TRY(readback_issue(ctx, st));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return mstep_rule(ctx, st, kernel, h, adapt, info);
}

// The step-size rule from a read-back step (after readback_issue and a synchronisation).
sps_status mstep_rule(sps_ctx* ctx, sps_state* st, int kernel, double h, bool adapt, sps_mstep_info* info) {
  Counters c;
  double rmin = 0.0;
  readback_result(ctx, st, &c, &rmin);
  if (c.chol_bad)
    return fail(ctx, SPS_ERR_DEGENERATE, "proposal covariance h V is not positive definite");
  if (c.nonfinite) return fail(ctx, SPS_ERR_NONFINITE, "non-finite log-likelihood of a proposal");
  const double alpha = static_cast<double>(c.accepts) / static_cast<double>(st->P);
  const sps_options& o = ctx->opt;
  double hn = h;
  if (adapt) {
    const double target = (kernel == SPS_MKERNEL_MALA) ? o.mala_target_accept : o.target_accept;
    hn = (alpha > target) ? std::min(h + o.h_step, o.h_max) : std::max(h - o.h_step, o.h_min);
    st->h = hn;
  }
  if (info) {
    info->h = h;
    info->accept_rate = alpha;
    info->rne_min = rmin;
    info->h_next = hn;
  }
  return SPS_OK;
}

// The rest of an adaptive M phase, after its first (eager) step, as one graph launch: a
// conditional WHILE node whose body is one M step (mstep_issue with h and the Philox step word
// on the device) and mstep_control_kernel, captured when the key changes (each cycle's t, a swap
// of the particle buffers, a reallocation) and replayed otherwise. The host synchronises once
// per phase. Returns with *fallback set (and nothing run) when the graph cannot be built; then
// the caller continues step by step.
sps_status mphase_graph(sps_ctx* ctx, sps_state* st, int kernel, double K, int r_done, int* r_end,
                        sps_schedule* rec, int64_t rec_step0, sps_mstep_info* info, bool* fallback) {
  *fallback = false;
  const sps_options& o = ctx->opt;
  // a fallback leaves its reason in the context's last-error string (the call still succeeds)
  auto give_up = [&](const char* what, cudaError_t e) {
    ctx->last_error = std::string("M-phase graph not used: ") + what + (e != cudaSuccess ? std::string(": ") +
                      cudaGetErrorString(e) : std::string());
    cudaGetLastError();
    *fallback = true;
    return SPS_OK;
  };
  const int F = 1 + ctx->NC;
  if (F > kCtlMaxF || o.r_max <= r_done) return give_up("shape", cudaSuccess);
  // the control kernel's group sums in dynamic shared memory (plus its static RNE array):
  // settled before any capture, so that no launch inside a capture can be invalid
  const size_t ctl_smem = sizeof(double) * 3 * static_cast<size_t>(st->J) * F;
  if (ctl_smem + sizeof(double) * kCtlMaxF > 200 * 1024) return give_up("groups", cudaSuccess);
  {
    const cudaError_t ea = cudaFuncSetAttribute(mstep_control_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(ctl_smem));
    if (ea != cudaSuccess) return give_up("control kernel shared memory", ea);
  }
  SPS_CUDA_TRY(st->ctl.reserve(sizeof(StepCtl)));
  SPS_CUDA_TRY(st->steplog.reserve(sizeof(double) * 3 * static_cast<size_t>(o.r_max)));
  const bool want_sigma = rec && rec->sigma;
  const size_t DD = static_cast<size_t>(ctx->D) * ctx->D;
  if (want_sigma) SPS_CUDA_TRY(st->sigmalog.reserve(sizeof(double) * DD * o.r_max));
  sps_state::MKey key;
  key.t = st->t;
  key.kernel = kernel;
  key.precision = o.precision;
  key.gen = buffer_generation();
  key.sig = want_sigma ? 1 : 0;
  const void* bufs[8] = {st->theta.ptr, st->theta_prop.ptr, st->ll.ptr, st->ll_prop.ptr,
                         st->lp.ptr,    st->lp_prop.ptr,    st->grad.ptr, st->grad_prop.ptr};
  for (int i = 0; i < 8; ++i) key.bufs[i] = bufs[i];
  StepCtl* d_ctl = st->ctl.as<StepCtl>();
  if (!st->mgraph || !(st->mkey == key)) {
    if (st->mgraph) {
      cudaGraphExecDestroy(st->mgraph);
      st->mgraph = nullptr;
    }
    if (!ctx->cap_stream) {
      const cudaError_t ec = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
      if (ec != cudaSuccess) {
        ctx->cap_stream = nullptr;
        return give_up("capture stream", ec);
      }
    }
    cudaGraph_t g = nullptr;
    SPS_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle cond;
    cudaGraphNodeParams np{};
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = cond;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    // the step is recorded on the private stream (nothing runs during capture); the graph is
    // launched on the context's stream
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(ctx->cap_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return give_up("conditional node", e);
    }
    const int64_t launches0 = ctx->launches;
    const cudaStream_t user_stream = ctx->stream;
    ctx->stream = ctx->cap_stream;
    ctx->capturing = true;
    sps_status is = mstep_issue(ctx, st, kernel, nullptr, nullptr, 0.0, 0, d_ctl);
    if (is == SPS_OK) {
      const double target = (kernel == SPS_MKERNEL_MALA) ? o.mala_target_accept : o.target_accept;
      {
        mstep_control_kernel<<<1, 128, ctl_smem, ctx->stream>>>(d_ctl, st->counters.as<unsigned long long>(),
                                                            st->scratch.as<double>(), st->J, F, kMomParts, st->N,
                                                            st->P, K, target, o.h_step, o.h_min, o.h_max,
                                                            st->steplog.as<double>(), st->cov.as<double>(), ctx->D,
                                                            want_sigma ? st->sigmalog.as<double>() : nullptr, cond,
                                                            cond, 0, nullptr, 0, 0);
        ++ctx->launches;
        if (cudaGetLastError() != cudaSuccess) is = SPS_ERR_CUDA;
      }
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(ctx->cap_stream, &captured);
    ctx->capturing = false;
    ctx->stream = user_stream;
    const int64_t per_step = ctx->launches - launches0;
    ctx->launches = launches0;
    if (is != SPS_OK || e != cudaSuccess || buffer_generation() != key.gen) {
      // nothing of the capture ran; continue step by step
      cudaGraphDestroy(g);
      const std::string why = is != SPS_OK ? "capture: " + ctx->last_error
                              : e != cudaSuccess ? std::string("end capture") : std::string("reallocation");
      return give_up(why.c_str(), e);
    }
    e = cudaGraphInstantiate(&st->mgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      st->mgraph = nullptr;
      return give_up("instantiate", e);
    }
    st->mkey = key;
    st->mgraph_launches = per_step;
  }
  StepCtl c{st->h, static_cast<unsigned long long>(st->step_counter + 1), r_done, o.r_max, 0, 0};
  SPS_CUDA_TRY(cudaMemcpyAsync(d_ctl, &c, sizeof c, cudaMemcpyHostToDevice, ctx->stream));
  SPS_CUDA_TRY(cudaGraphLaunch(st->mgraph, ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(&c, d_ctl, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const int ran = c.r - r_done + (c.err ? 1 : 0);
  ctx->launches += static_cast<int64_t>(ran) * st->mgraph_launches;
  st->graph_steps += ran;
  st->step_counter = c.step - 1 + (c.err ? 1 : 0);
  if (kernel == SPS_MKERNEL_RW) st->grad_valid = false;
  if (c.err == 1) return fail(ctx, SPS_ERR_DEGENERATE, "proposal covariance h V is not positive definite");
  if (c.err == 2) return fail(ctx, SPS_ERR_NONFINITE, "non-finite log-likelihood of a proposal");
  std::vector<double> lg(3 * static_cast<size_t>(c.r - r_done));
  if (!lg.empty()) {
    SPS_CUDA_TRY(cudaMemcpy(lg.data(), st->steplog.as<double>() + 3 * static_cast<size_t>(r_done),
                            sizeof(double) * lg.size(), cudaMemcpyDeviceToHost));
  }
  if (want_sigma && c.r > r_done && rec_step0 + r_done < rec->cap_steps) {
    const int64_t n_copy = std::min<int64_t>(c.r - r_done, rec->cap_steps - (rec_step0 + r_done));
    SPS_CUDA_TRY(cudaMemcpy(rec->sigma + (rec_step0 + r_done) * DD, st->sigmalog.as<double>() + r_done * DD,
                            sizeof(double) * DD * n_copy, cudaMemcpyDeviceToHost));
  }
  for (int r = r_done; r < c.r; ++r) {
    const double* q = lg.data() + 3 * static_cast<size_t>(r - r_done);
    const int64_t rs = rec_step0 + r;
    if (rec && rs < rec->cap_steps) {
      if (rec->h) rec->h[rs] = q[0];
      if (rec->accept) rec->accept[rs] = q[1];
    }
    if (info && r + 1 == c.r) {
      info->h = q[0];
      info->accept_rate = q[1];
      info->rne_min = q[2];
      info->h_next = c.h;
    }
  }
  st->h = c.h;
  *r_end = c.r;
  return SPS_OK;
}

// The rest of a lockstep M phase of a batched run, after its first step (or, with prepare, the
// whole phase: first the cached log-likelihoods, and for MALA the gradients, at the phase's t),
// as one graph launch: a conditional WHILE node whose body holds, per model still moving, conditional IF nodes around
// the model's own kernels (proposal, decisions, monitoring sums and mstep_control_kernel, which
// switches the model's IF nodes off once its stopping rule is met), between them the one batched
// fused-kernel evaluation of the proposals (split-precision random walk; the tiles of stopped
// models are skipped), and batch_continue_kernel, which ends the loop when every model has
// stopped. The models' IF nodes have no mutual dependencies, so their kernels run concurrently.
// The graph is captured for each phase (t and the particle buffers change between phases) and
// launched once; the host synchronises once. The models are the phase's (models[i] with
// moving[i] after the first step, batched[i] if evaluated by the batched launch); steps[i] is
// the model's step count, updated. *fallback: the graph could not be built and nothing ran.
sps_status batched_mphase_graph(sps_ctx* ctx, const std::vector<sps_ctx*>& cs, const std::vector<sps_state*>& ss,
                                const std::vector<char>& moving, const std::vector<char>& batched, int kernel,
                                bool prepare, std::vector<int>& steps, DevBuf& ctl_buf, bool* fallback) {
  *fallback = false;
  const sps_options& o = ctx->opt;
  auto give_up = [&](const char* what, cudaError_t e) {
    ctx->last_error = std::string("batched M-phase graph not used: ") + what +
                      (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string());
    cudaGetLastError();
    *fallback = true;
    return SPS_OK;
  };
  const int Mp = static_cast<int>(cs.size());
  const int F = 1 + ctx->NC;
  const int J = ss[0]->J;
  if (F > kCtlMaxF) return give_up("shape", cudaSuccess);
  const size_t ctl_smem = sizeof(double) * 3 * static_cast<size_t>(J) * F;
  if (ctl_smem + sizeof(double) * kCtlMaxF > 200 * 1024) return give_up("groups", cudaSuccess);
  {
    const cudaError_t ea = cudaFuncSetAttribute(mstep_control_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(ctl_smem));
    if (ea != cudaSuccess) return give_up("control kernel shared memory", ea);
  }
  SPS_CUDA_TRY(ctl_buf.reserve(sizeof(StepCtl) * static_cast<size_t>(Mp + 1)));
  for (sps_state* st : ss) SPS_CUDA_TRY(st->steplog.reserve(sizeof(double) * 3 * static_cast<size_t>(o.r_max)));
  if (!ctx->cap_stream) {
    const cudaError_t ec = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (ec != cudaSuccess) {
      ctx->cap_stream = nullptr;
      return give_up("capture stream", ec);
    }
  }
  // the batched evaluation of the proposals, prepared (tables in device memory) before the capture
  std::vector<int> bpos(Mp, -1);
  std::vector<int2> tiles;
  int2* ptab = nullptr;
  {
    std::vector<int32_t> bk;
    std::vector<int64_t> bP, bt;
    std::vector<const double*> bth;
    std::vector<double*> bll;
    std::vector<char> bskip;
    for (int i = 0; i < Mp; ++i) {
      if (!batched[i]) continue;
      bpos[i] = static_cast<int>(bk.size());
      bk.push_back(cs[i]->k);
      bP.push_back(ss[i]->P);
      bt.push_back(ss[i]->t);
      bth.push_back(ss[i]->theta_prop.as<double>());
      bll.push_back(ss[i]->ll_prop.as<double>());
      bskip.push_back(moving[i] ? 0 : 1);
    }
    if (!bk.empty()) {
      SPS_TRY(loglik_split_batched_prepare(ctx, 0, static_cast<int>(bk.size()), bk.data(), bP.data(), bt.data(),
                                           bth.data(), bll.data(), bskip.data(), &tiles, &ptab));
      if (prepare) {
        // the cached log-likelihoods at the phase's t, by the same batched launch (plan slot 1)
        for (size_t q = 0; q < bk.size(); ++q) bskip[q] = 0;
        std::vector<const double*> cth;
        std::vector<double*> cll;
        for (int i = 0; i < Mp; ++i)
          if (batched[i]) {
            cth.push_back(ss[i]->theta.as<double>());
            cll.push_back(ss[i]->ll.as<double>());
          }
        SPS_TRY(loglik_split_batched_prepare(ctx, 1, static_cast<int>(bk.size()), bk.data(), bP.data(), bt.data(),
                                             cth.data(), cll.data(), bskip.data(), nullptr, nullptr));
      }
    }
  }
  // with prepare, the models outside the batched launch (MALA, FP32) refresh their cached
  // log-likelihoods (and gradients) at the phase's t eagerly, on the stream ahead of the graph:
  // their launchers size buffers and caches by t, which must happen outside the capture
  if (prepare)
    for (int i = 0; i < Mp; ++i)
      if (!batched[i]) {
        const sps_status e = mstep_prepare(cs[i], ss[i], kernel);
        if (e != SPS_OK) {
          ctx->last_error = std::string("model context: ") + cs[i]->last_error;
          return e;
        }
      }
  StepCtl* d_ctl = ctl_buf.as<StepCtl>();
  // the models' control blocks, then the loop's iteration count (bounded by the step cap)
  std::vector<StepCtl> hc(static_cast<size_t>(Mp + 1));
  for (int i = 0; i < Mp; ++i)
    hc[i] = StepCtl{ss[i]->h, static_cast<unsigned long long>(ss[i]->step_counter + 1), steps[i], o.r_max,
                    moving[i] ? 0 : 1, 0};
  hc[Mp] = StepCtl{0.0, 0ull, 0, o.r_max + 1, 0, 0};
  const uint64_t gen = buffer_generation();
  const double target = (kernel == SPS_MKERNEL_MALA) ? o.mala_target_accept : o.target_accept;

  cudaGraph_t g = nullptr;
  SPS_CUDA_TRY(cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { if (g) cudaGraphDestroy(g); }
  } guard{g};
  std::string cap_error;
  // with prepare: the phase's first evaluations as child graphs of g, before the loop
  std::vector<cudaGraphNode_t> pre;
  int64_t prep_launches = 0;
  cudaError_t e = cudaSuccess;
  if (prepare) {
    auto child = [&](sps_ctx* c, const std::function<sps_status()>& issue) -> cudaError_t {
      cudaError_t ee = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
      if (ee != cudaSuccess) return ee;
      const cudaStream_t user = c->stream;
      c->stream = ctx->cap_stream;
      c->capturing = true;
      const int64_t l0 = c->launches;
      const sps_status is = issue();
      prep_launches += c->launches - l0;
      c->launches = l0;
      c->capturing = false;
      c->stream = user;
      cudaGraph_t sub = nullptr;
      ee = cudaStreamEndCapture(ctx->cap_stream, &sub);
      if (is != SPS_OK) {
        cap_error = c->last_error;
        ee = cudaErrorUnknown;
      }
      cudaGraphNode_t nd;
      if (ee == cudaSuccess) ee = cudaGraphAddChildGraphNode(&nd, g, nullptr, 0, sub);
      if (sub) cudaGraphDestroy(sub);
      if (ee == cudaSuccess) pre.push_back(nd);
      return ee;
    };
    if (!tiles.empty()) e = child(ctx, [&]() { return loglik_split_batched_launch(ctx, 1); });
    if (e != cudaSuccess) {
      const std::string why = !cap_error.empty() ? "capture: " + cap_error : std::string("prepare nodes");
      return give_up(why.c_str(), e);
    }
  }
  cudaGraphConditionalHandle wh;
  e = cudaGraphConditionalHandleCreate(&wh, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams wp{};
  cudaGraphNode_t wnode;
  if (e == cudaSuccess) {
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = wh;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, g, pre.empty() ? nullptr : pre.data(), nullptr, pre.size(), &wp);
  }
  if (e != cudaSuccess) return give_up("conditional node", e);
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  // an IF node in the loop body (after deps) whose body graph receives what issue() launches on
  // the context c, recorded on the capture stream
  auto add_if = [&](cudaGraphConditionalHandle* h, const std::vector<cudaGraphNode_t>& deps, sps_ctx* c,
                    const std::function<sps_status()>& issue, cudaGraphNode_t* node) -> cudaError_t {
    cudaError_t ee = cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault);
    if (ee != cudaSuccess) return ee;
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = *h;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    ee = cudaGraphAddNode(node, body, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &ip);
    if (ee != cudaSuccess) return ee;
    ee = cudaStreamBeginCaptureToGraph(ctx->cap_stream, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeRelaxed);
    if (ee != cudaSuccess) return ee;
    const cudaStream_t user = c->stream;
    c->stream = ctx->cap_stream;
    c->capturing = true;
    const sps_status is = issue();
    c->capturing = false;
    c->stream = user;
    cudaGraph_t out = nullptr;
    ee = cudaStreamEndCapture(ctx->cap_stream, &out);
    if (is != SPS_OK) {
      cap_error = c->last_error;
      return cudaErrorUnknown;
    }
    return ee;
  };
  std::vector<cudaGraphConditionalHandle> hA(Mp), hB(Mp);
  std::vector<cudaGraphNode_t> nA(Mp), nB(Mp), last;
  std::vector<int64_t> chain_launches(Mp, 0);
  for (int i = 0; i < Mp && e == cudaSuccess; ++i) {
    if (!moving[i]) continue;
    sps_ctx* c = cs[i];
    sps_state* st = ss[i];
    StepCtl* ctl = d_ctl + i;
    const double K = (st->t >= c->n) ? o.rne_final : o.rne_cycle;
    const int2 tr = (bpos[i] >= 0) ? tiles[bpos[i]] : make_int2(0, 0);
    auto control = [&, c, st, ctl, K, tr, i]() -> sps_status {
      mstep_control_kernel<<<1, 128, ctl_smem, c->stream>>>(ctl, st->counters.as<unsigned long long>(),
                                                           st->scratch.as<double>(), st->J, F, kMomParts, st->N,
                                                           st->P, K, target, o.h_step, o.h_min, o.h_max,
                                                           st->steplog.as<double>(), st->cov.as<double>(), c->D,
                                                           nullptr, hA[i], batched[i] ? hB[i] : hA[i], 1,
                                                           batched[i] ? ptab : nullptr, tr.x, tr.y);
      ++c->launches;
      SPS_CUDA_TRY(cudaGetLastError());
      return SPS_OK;
    };
    const int64_t l0 = c->launches;
    if (batched[i]) {
      // the handle of the second IF node exists before the control kernel that sets it is captured
      e = cudaGraphConditionalHandleCreate(&hB[i], g, 1, cudaGraphCondAssignDefault);
      if (e == cudaSuccess)
        e = add_if(&hA[i], {}, c, [&, c, st, ctl]() { return rw_issue_propose(c, st, nullptr, nullptr, 0.0, 0, ctl); },
                   &nA[i]);
    } else {
      e = add_if(&hA[i], {}, c, [&, c, st, ctl, control]() {
            SPS_TRY(mstep_issue(c, st, kernel, nullptr, nullptr, 0.0, 0, ctl));
            return control();
          }, &nA[i]);
      last.push_back(nA[i]);
    }
    chain_launches[i] = c->launches - l0;
    c->launches = l0;
  }
  int64_t eval_launches = 0;
  if (e == cudaSuccess && !tiles.empty()) {
    // the batched evaluation after every batched model's proposal, as a child graph
    std::vector<cudaGraphNode_t> deps;
    for (int i = 0; i < Mp; ++i)
      if (moving[i] && batched[i]) deps.push_back(nA[i]);
    e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      const cudaStream_t user = ctx->stream;
      ctx->stream = ctx->cap_stream;
      ctx->capturing = true;
      const int64_t l0 = ctx->launches;
      const sps_status is = loglik_split_batched_launch(ctx, 0);
      eval_launches = ctx->launches - l0;
      ctx->launches = l0;
      ctx->capturing = false;
      ctx->stream = user;
      cudaGraph_t ge = nullptr;
      e = cudaStreamEndCapture(ctx->cap_stream, &ge);
      if (is != SPS_OK) {
        cap_error = ctx->last_error;
        e = cudaErrorUnknown;
      }
      cudaGraphNode_t en;
      if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&en, body, deps.data(), deps.size(), ge);
      if (ge) cudaGraphDestroy(ge);
      for (int i = 0; i < Mp && e == cudaSuccess; ++i) {
        if (!moving[i] || !batched[i]) continue;
        sps_ctx* c = cs[i];
        sps_state* st = ss[i];
        StepCtl* ctl = d_ctl + i;
        const double K = (st->t >= c->n) ? o.rne_final : o.rne_cycle;
        const int2 tr = tiles[bpos[i]];
        const int64_t l0c = c->launches;
        // hB[i] already exists: create the IF node with it directly
        cudaGraphNodeParams ip{};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = hB[i];
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        e = cudaGraphAddNode(&nB[i], body, &en, nullptr, 1, &ip);
        if (e == cudaSuccess)
          e = cudaStreamBeginCaptureToGraph(ctx->cap_stream, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                            cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) break;
        const cudaStream_t user_c = c->stream;
        c->stream = ctx->cap_stream;
        c->capturing = true;
        sps_status is2 = rw_issue_accept(c, st, 0, ctl);
        if (is2 == SPS_OK) {
          mstep_control_kernel<<<1, 128, ctl_smem, c->stream>>>(ctl, st->counters.as<unsigned long long>(),
                                                               st->scratch.as<double>(), st->J, F, kMomParts, st->N,
                                                               st->P, K, target, o.h_step, o.h_min, o.h_max,
                                                               st->steplog.as<double>(), st->cov.as<double>(), c->D,
                                                               nullptr, hA[i], hB[i], 1, ptab, tr.x, tr.y);
          ++c->launches;
          if (cudaGetLastError() != cudaSuccess) is2 = SPS_ERR_CUDA;
        }
        c->capturing = false;
        c->stream = user_c;
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(ctx->cap_stream, &out);
        if (is2 != SPS_OK) {
          cap_error = c->last_error;
          e = cudaErrorUnknown;
        }
        chain_launches[i] += c->launches - l0c;
        c->launches = l0c;
        last.push_back(nB[i]);
      }
    }
  }
  if (e == cudaSuccess) {
    // another step while any model moves
    int Mi = Mp;
    void* args[] = {&d_ctl, &Mi, &wh};
    cudaKernelNodeParams kp{};
    kp.func = reinterpret_cast<void*>(batch_continue_kernel);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    cudaGraphNode_t cn;
    e = cudaGraphAddKernelNode(&cn, body, last.data(), last.size(), &kp);
  }
  if (e != cudaSuccess || buffer_generation() != gen) {
    const std::string why = !cap_error.empty() ? "capture: " + cap_error
                            : e != cudaSuccess ? std::string("graph construction") : std::string("reallocation");
    return give_up(why.c_str(), e);
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) return give_up("instantiate", e);
  struct ExecGuard {
    cudaGraphExec_t x;
    ~ExecGuard() { if (x) cudaGraphExecDestroy(x); }
  } xguard{exec};
  SPS_CUDA_TRY(cudaMemcpyAsync(d_ctl, hc.data(), sizeof(StepCtl) * hc.size(), cudaMemcpyHostToDevice, ctx->stream));
  SPS_CUDA_TRY(cudaGraphLaunch(exec, ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(hc.data(), d_ctl, sizeof(StepCtl) * hc.size(), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (hc[Mp].err) return fail(ctx, SPS_ERR_STATE, "batched M-phase graph: step cap passed without every model stopping");
  int iters = 0;
  for (int i = 0; i < Mp; ++i) {
    if (!moving[i]) continue;
    const StepCtl& c = hc[i];
    sps_state* st = ss[i];
    const int ran = c.r - steps[i] + (c.err ? 1 : 0);
    iters = std::max(iters, ran);
    cs[i]->launches += static_cast<int64_t>(ran) * chain_launches[i];
    st->graph_steps += ran;
    st->step_counter = c.step - 1 + (c.err ? 1 : 0);
    if (kernel == SPS_MKERNEL_RW) st->grad_valid = false;
    if (c.err == 1) return fail(ctx, SPS_ERR_DEGENERATE, "model context: proposal covariance h V is not positive definite");
    if (c.err == 2) return fail(ctx, SPS_ERR_NONFINITE, "model context: non-finite log-likelihood of a proposal");
    st->h = c.h;
    steps[i] = c.r;
  }
  ctx->launches += static_cast<int64_t>(iters) * (eval_launches + 1) + prep_launches;
  if (prepare)
    for (int i = 0; i < Mp; ++i)
      if (batched[i]) {
        ss[i]->ll_stale = false;
        ss[i]->ll_kind = 0;
      }
  return SPS_OK;
}

// C phase (Algorithm 1 step 2(a)): running log weights over blocks of observations (doubling
// from the configured block), the ESS of every observation of a block read back at once, stop at
// the first s with ESS / P below the threshold (or at t_target / n); then the per-group log
// marginal-likelihood increments and the cached log-likelihood at the new t. One synchronisation
// per block, plus one to return the increments when lme_out is given.
// C-phase block rows: at most 1024 and 2^25 running weights.
static int64_t cphase_max_rows(int64_t P) { return std::max<int64_t>(1, std::min<int64_t>(1024, (int64_t{1} << 25) / P)); }
static int64_t cphase_first_block(const sps_ctx* ctx, int64_t max_rows) {
  return std::max<int64_t>(1, std::min<int64_t>(ctx->opt.cphase_block > 0 ? ctx->opt.cphase_block : 64, max_rows));
}

// The C phase's buffers: block rows of running weights, the running state, the rows' ESS (plus
// one slot that keeps the ESS at the stop row of a known-target C phase), group maxima.
static sps_status cphase_reserve(sps_ctx* ctx, sps_state* st, bool lpl) {
  const int64_t P = st->P, max_rows = cphase_max_rows(P);
  SPS_CUDA_TRY(st->lwbuf.reserve(sizeof(float2) * max_rows * P));
  SPS_CUDA_TRY(st->lwstate.reserve(sizeof(float2) * P));
  const int64_t ess_slot = std::max<int64_t>(max_rows, st->J);
  SPS_CUDA_TRY(st->ess_buf.reserve(sizeof(double) * (ess_slot + 1)));
  SPS_CUDA_TRY(st->gmax.reserve(sizeof(double) * st->J));
  if (lpl) SPS_CUDA_TRY(st->lpl_dev.reserve(sizeof(double) * max_rows * st->J));
  return SPS_OK;
}

// After the stop row: the log marginal likelihood increment per group (added to the state's
// log ML), the group maxima, and the cached log-likelihood advanced by the log weights.
static sps_status cphase_tail(sps_ctx* ctx, sps_state* st) {
  group_lme_part_kernel<<<dim3(st->J, kLmeParts), 256, 0, ctx->stream>>>(st->logw.as<double>(), st->N,
                                                                         st->scratch.as<double>()); ++ctx->launches;
  group_lme_merge_kernel<<<(st->J + 63) / 64, 64, 0, ctx->stream>>>(st->scratch.as<double>(), st->J, kLmeParts, st->N,
                                                                    st->ess_buf.as<double>(), st->logml.as<double>(),
                                                                    st->gmax.as<double>()); ++ctx->launches;
  add_kernel<<<static_cast<unsigned>((st->P + 255) / 256), 256, 0, ctx->stream>>>(st->ll.as<double>(),
                                                                                   st->logw.as<double>(), st->P);
  ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

sps_status cphase_impl(sps_ctx* ctx, sps_state* st, int64_t t_target, int64_t* t_new, double* ess_out,
                       double* lme_out, double* lpl_out) {
  const int64_t n = ctx->n, P = st->P;
  if (st->t >= n) return fail(ctx, SPS_ERR_STATE, "C phase: no observations left");
  if (t_target > 0 && (t_target <= st->t || t_target > n)) return fail(ctx, SPS_ERR_INVALID_ARG, "C phase: bad t_target");
  const int64_t max_rows = cphase_max_rows(P);
  int64_t block = cphase_first_block(ctx, max_rows);
  SPS_TRY(cphase_reserve(ctx, st, lpl_out != nullptr));
  const int64_t ess_slot = std::max<int64_t>(max_rows, st->J);
  SPS_CUDA_TRY(cudaMemsetAsync(st->lwstate.ptr, 0, sizeof(float2) * P, ctx->stream));
  float2* rows = st->lwbuf.as<float2>();
  int64_t s = st->t;
  std::vector<double> ess(max_rows);
  std::vector<double> lme_rows, lme_prev(st->J, 0.0);   // log mean of the weights before s
  int64_t found = -1;
  double ess_found = 0.0;
  // With a target and no log predictive likelihoods the stop row is known: blocks end at the
  // target, no ESS is read back inside the loop and the call synchronises at most once, at the end.
  const bool known = (t_target > 0) && !lpl_out;
  while (s < n) {
    const int64_t b = known ? std::min<int64_t>(block, t_target - s) : std::min<int64_t>(block, n - s);
    SPS_TRY(cphase_increments(ctx, st->theta.as<double>(), P, s, s + b, st->lwstate.as<float2>(), rows));
    ess_part_kernel<float2><<<dim3(static_cast<unsigned>(b), kEssParts), 512, 0, ctx->stream>>>(
        rows, P, st->scratch.as<double>(), nullptr); ++ctx->launches;
    ess_merge_kernel<<<static_cast<unsigned>((b + 63) / 64), 64, 0, ctx->stream>>>(
        st->scratch.as<double>(), static_cast<int>(b), kEssParts, st->ess_buf.as<double>(), nullptr); ++ctx->launches;
    if (lpl_out) {
      row_group_lme_kernel<<<dim3(static_cast<unsigned>(b), st->J), 256, 0, ctx->stream>>>(
          rows, P, st->N, st->lpl_dev.as<double>()); ++ctx->launches;
      lme_rows.resize(static_cast<size_t>(b) * st->J);
      SPS_CUDA_TRY(cudaMemcpyAsync(lme_rows.data(), st->lpl_dev.ptr, sizeof(double) * b * st->J,
                                   cudaMemcpyDeviceToHost, ctx->stream));
    }
    SPS_CUDA_TRY(cudaGetLastError());
    if (known) {
      if (s + b == t_target) {
        if (ess_out) SPS_CUDA_TRY(cudaMemcpyAsync(st->ess_buf.as<double>() + ess_slot, st->ess_buf.as<double>() + (b - 1),
                                                  sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        found = b - 1;
        lw_to_f64_kernel<<<static_cast<unsigned>((P + 255) / 256), 256, 0, ctx->stream>>>(rows + found * P, P,
                                                                                         st->logw.as<double>()); ++ctx->launches;
        SPS_CUDA_TRY(cudaGetLastError());
        s = t_target;
        break;
      }
      SPS_CUDA_TRY(cudaMemcpyAsync(st->lwstate.ptr, rows + (b - 1) * P, sizeof(float2) * P, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
      s += b;
      block = std::min<int64_t>(block * 2, max_rows);
      continue;
    }
    SPS_CUDA_TRY(cudaMemcpyAsync(ess.data(), st->ess_buf.ptr, sizeof(double) * b, cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int64_t j = 0; j < b; ++j) {
      const int64_t sj = s + j + 1;
      const bool stop = (t_target > 0) ? (sj == t_target)
                                       : (ess[j] / static_cast<double>(P) < ctx->opt.ess_fraction || sj == n);
      if (lpl_out) {
        // log predictive likelihood of observation sj per group (row j of this block)
        double* o = lpl_out + (sj - 1 - st->t) * st->J;
        for (int g = 0; g < st->J; ++g) {
          const double cur = lme_rows[static_cast<size_t>(j) * st->J + g];
          o[g] = cur - lme_prev[g];
          lme_prev[g] = cur;
        }
      }
      if (stop) {
        found = j;
        ess_found = ess[j];
        break;
      }
    }
    if (found >= 0) {
      lw_to_f64_kernel<<<static_cast<unsigned>((P + 255) / 256), 256, 0, ctx->stream>>>(rows + found * P, P,
                                                                                       st->logw.as<double>()); ++ctx->launches;
      SPS_CUDA_TRY(cudaGetLastError());
      s = s + found + 1;
      break;
    }
    SPS_CUDA_TRY(cudaMemcpyAsync(st->lwstate.ptr, rows + (b - 1) * P, sizeof(float2) * P, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    s += b;
    block = std::min<int64_t>(block * 2, max_rows);
  }
  // log marginal likelihood increment per group, group maxima, cached log-likelihood at the new t
  SPS_TRY(cphase_tail(ctx, st));
  if (known && ess_out) {
    SPS_CUDA_TRY(cudaMemcpyAsync(&ess_found, st->ess_buf.as<double>() + ess_slot, sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    if (!lme_out) SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  if (lme_out) {
    SPS_CUDA_TRY(cudaMemcpyAsync(lme_out, st->ess_buf.ptr, sizeof(double) * st->J, cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  st->t = s;
  st->have_weights = true;
  st->ll_stale = true;
  if (t_new) *t_new = s;
  if (ess_out) *ess_out = ess_found;
  return SPS_OK;
}

// S phase (Algorithm 1 step 2(b)): quantised weights, per-group integer-CDF draws, gather.
// The C-phase row buffer holds the quantised weights (uint64 [P]) here.
// The S phase's kernels (Philox step word `step` unless uniforms d_u are given): counters cleared,
// quantised weights, per-group draws, the gathered particles into the proposal buffers.
static sps_status sphase_issue(sps_ctx* ctx, sps_state* st, const double* d_u, uint64_t step) {
  SPS_CUDA_TRY(cudaMemsetAsync(st->counters.ptr, 0, sizeof(Counters), ctx->stream));
  unsigned long long* q = st->lwbuf.as<unsigned long long>();
  resample_q_kernel<<<static_cast<unsigned>((st->P + 255) / 256), 256, 0, ctx->stream>>>(
      st->logw.as<double>(), 0, st->N, st->P, st->gmax.as<double>(), q); ++ctx->launches;
  SPS_TRY(launch_resample(ctx, ctx->opt.resampling, q, st->J, st->N, d_u, st->seed, step, st->idx.as<int>(),
                          flag_ptr(st, 2)));
  gather_kernel<<<static_cast<unsigned>((st->P + 256 / ctx->D - 1) / (256 / ctx->D)), 256, 0, ctx->stream>>>(
      st->theta.as<double>(), st->ll.as<double>(), st->lp.as<double>(), st->idx.as<int>(), st->P, st->N, ctx->D,
      st->theta_prop.as<double>(), st->ll_prop.as<double>(), st->lp_prop.as<double>()); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

// After the S phase's kernels ran: the gathered particles become the state's.
static void sphase_commit(sps_state* st) {
  swapbuf(st->theta, st->theta_prop);
  swapbuf(st->ll, st->ll_prop);
  swapbuf(st->lp, st->lp_prop);
  st->have_weights = false;
  st->grad_valid = false;   // gradients are not gathered
}

sps_status sphase_impl(sps_ctx* ctx, sps_state* st, const double* d_u, int* d_idx_out, int* h_idx_out = nullptr) {
  if (!st->have_weights) return fail(ctx, SPS_ERR_STATE, "S phase before a C phase");
  SPS_CUDA_TRY(st->lwbuf.reserve(sizeof(unsigned long long) * st->P));
  const uint64_t step = ++st->cycle_counter;
  SPS_TRY(sphase_issue(ctx, st, d_u, step));
  if (d_idx_out)
    SPS_CUDA_TRY(cudaMemcpyAsync(d_idx_out, st->idx.ptr, sizeof(int) * st->P, cudaMemcpyDeviceToDevice, ctx->stream));
  if (h_idx_out)   // completes with the counters' synchronisation below
    SPS_CUDA_TRY(cudaMemcpyAsync(h_idx_out, st->idx.ptr, sizeof(int) * st->P, cudaMemcpyDeviceToHost, ctx->stream));
  Counters c;
  SPS_TRY(read_counters(ctx, st, &c));
  if (c.res_bad) return fail(ctx, SPS_ERR_DEGENERATE, "all resampling weights of a group vanished");
  sphase_commit(st);
  return SPS_OK;
}

// The C and S phases of several models (a cycle of a batched run, Algorithm 1 steps 2(a)-(b)) as
// one graph launch: per model the running weights cleared, then a conditional WHILE node whose
// body holds, per model, a conditional IF node around one C-phase block (running weights of the
// block's observations, their ESS, cphase_scan_kernel, which applies the stopping rule and
// picks the next block, and cphase_advance_kernel), then per model the C phase's tail (log ML
// increments, cached log-likelihood) and the S phase's kernels. The same kernels and decisions
// as cphase_impl and sphase_impl, without their host round trips; the models' branches run
// concurrently. Captured for each cycle (the Philox step words and buffers change); the host
// synchronises once. *fallback: the graph could not be built and nothing ran.
sps_status batched_cs_graph(sps_ctx* ctx, const std::vector<sps_ctx*>& cs, const std::vector<sps_state*>& ss,
                            DevBuf& cc_buf, bool* fallback) {
  *fallback = false;
  auto give_up = [&](const char* what, cudaError_t e) {
    ctx->last_error = std::string("batched C/S-phase graph not used: ") + what +
                      (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string());
    cudaGetLastError();
    *fallback = true;
    return SPS_OK;
  };
  const int Mp = static_cast<int>(cs.size());
  for (int i = 0; i < Mp; ++i) {
    if (ss[i]->t >= cs[i]->n) return fail(ctx, SPS_ERR_STATE, "C phase: no observations left");
    SPS_TRY(cphase_reserve(cs[i], ss[i], false));
    SPS_CUDA_TRY(ss[i]->lwbuf.reserve(sizeof(unsigned long long) * ss[i]->P));
  }
  SPS_CUDA_TRY(cc_buf.reserve(sizeof(CphaseCtl) * static_cast<size_t>(Mp + 1)));
  if (!ctx->cap_stream) {
    const cudaError_t ec = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (ec != cudaSuccess) {
      ctx->cap_stream = nullptr;
      return give_up("capture stream", ec);
    }
  }
  CphaseCtl* d_cc = cc_buf.as<CphaseCtl>();
  std::vector<CphaseCtl> hc(static_cast<size_t>(Mp + 1));
  int64_t iter_cap = 64;
  for (int i = 0; i < Mp; ++i) {
    const int64_t n = cs[i]->n, P = ss[i]->P, t = ss[i]->t;
    const int64_t mr = cphase_max_rows(P), b0 = cphase_first_block(cs[i], mr);
    CphaseCtl& c = hc[i];
    c = CphaseCtl{};
    c.range[0] = t;
    c.range[1] = t + std::min<int64_t>(b0, n - t);
    c.block = b0;
    c.max_rows = mr;
    c.n = n;
    c.P = P;
    c.frac = cs[i]->opt.ess_fraction;
    iter_cap = std::max<int64_t>(iter_cap, (n - t) / b0 + 64);   // every block takes at least b0 rows
  }
  hc[Mp] = CphaseCtl{};
  hc[Mp].max_rows = iter_cap;
  const uint64_t gen = buffer_generation();

  cudaGraph_t g = nullptr;
  SPS_CUDA_TRY(cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { if (g) cudaGraphDestroy(g); }
  } guard{g};
  std::string cap_error;
  // what issue() launches on the context c, recorded on the capture stream into `into`
  auto record = [&](cudaGraph_t into, sps_ctx* c, const std::function<sps_status()>& issue) -> cudaError_t {
    cudaError_t ee = cudaStreamBeginCaptureToGraph(ctx->cap_stream, into, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeRelaxed);
    if (ee != cudaSuccess) return ee;
    const cudaStream_t user = c->stream;
    c->stream = ctx->cap_stream;
    c->capturing = true;
    const sps_status is = issue();
    c->capturing = false;
    c->stream = user;
    cudaGraph_t out = nullptr;
    ee = cudaStreamEndCapture(ctx->cap_stream, &out);
    if (is != SPS_OK) {
      cap_error = c->last_error;
      return cudaErrorUnknown;
    }
    return ee;
  };
  // the same as a child graph node of g after deps
  auto child = [&](const std::vector<cudaGraphNode_t>& deps, sps_ctx* c, const std::function<sps_status()>& issue,
                   cudaGraphNode_t* node) -> cudaError_t {
    cudaGraph_t sub = nullptr;
    cudaError_t ee = cudaGraphCreate(&sub, 0);
    if (ee != cudaSuccess) return ee;
    ee = record(sub, c, issue);
    if (ee == cudaSuccess)
      ee = cudaGraphAddChildGraphNode(node, g, deps.empty() ? nullptr : deps.data(), deps.size(), sub);
    cudaGraphDestroy(sub);
    return ee;
  };
  cudaError_t e = cudaSuccess;
  std::vector<cudaGraphNode_t> init(Mp);
  for (int i = 0; i < Mp && e == cudaSuccess; ++i) {
    sps_ctx* c = cs[i];
    sps_state* st = ss[i];
    e = child({}, c, [c, st]() {
          sps_ctx* ctx = c;   // the model's context takes any error
          SPS_CUDA_TRY(cudaMemsetAsync(st->lwstate.ptr, 0, sizeof(float2) * st->P, ctx->stream));
          return SPS_OK;
        }, &init[i]);
  }
  cudaGraphConditionalHandle wh;
  cudaGraphNodeParams wp{};
  cudaGraphNode_t wnode;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&wh, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = wh;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, g, init.data(), nullptr, init.size(), &wp);
  }
  std::vector<cudaGraphNode_t> ifs(Mp);
  std::vector<int64_t> block_launches(Mp, 0), tail_launches(Mp, 0);
  if (e == cudaSuccess) {
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    for (int i = 0; i < Mp && e == cudaSuccess; ++i) {
      sps_ctx* c = cs[i];
      sps_state* st = ss[i];
      CphaseCtl* cc = d_cc + i;
      const int64_t mr = hc[i].max_rows;
      cudaGraphConditionalHandle hi;
      e = cudaGraphConditionalHandleCreate(&hi, g, 1, cudaGraphCondAssignDefault);
      if (e != cudaSuccess) break;
      cudaGraphNodeParams ip{};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = hi;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      e = cudaGraphAddNode(&ifs[i], body, nullptr, nullptr, 0, &ip);
      if (e != cudaSuccess) break;
      const int64_t l0 = c->launches;
      e = record(ip.conditional.phGraph_out[0], c, [c, st, cc, mr, hi]() {
        sps_ctx* ctx = c;   // the model's context takes any error
        const int64_t P = st->P;
        float2* rows = st->lwbuf.as<float2>();
        SPS_TRY(cphase_increments(c, st->theta.as<double>(), P, 0, 0, st->lwstate.as<float2>(), rows, cc->range));
        ess_part_kernel<float2><<<dim3(static_cast<unsigned>(mr), kEssParts), 512, 0, c->stream>>>(
            rows, P, st->scratch.as<double>(), cc->range); ++c->launches;
        ess_merge_kernel<<<static_cast<unsigned>((mr + 63) / 64), 64, 0, c->stream>>>(
            st->scratch.as<double>(), static_cast<int>(mr), kEssParts, st->ess_buf.as<double>(), cc->range);
        ++c->launches;
        cphase_scan_kernel<<<1, 1, 0, c->stream>>>(cc, st->ess_buf.as<double>(), hi); ++c->launches;
        cphase_advance_kernel<<<static_cast<unsigned>((P + 255) / 256), 256, 0, c->stream>>>(
            cc, rows, P, st->lwstate.as<float2>(), st->logw.as<double>()); ++c->launches;
        SPS_CUDA_TRY(cudaGetLastError());
        return SPS_OK;
      });
      block_launches[i] = c->launches - l0;
      c->launches = l0;
    }
    if (e == cudaSuccess) {
      int Mi = Mp;
      void* args[] = {&d_cc, &Mi, &wh};
      cudaKernelNodeParams kp{};
      kp.func = reinterpret_cast<void*>(cphase_continue_kernel);
      kp.gridDim = dim3(1);
      kp.blockDim = dim3(1);
      kp.sharedMemBytes = 0;
      kp.kernelParams = args;
      cudaGraphNode_t cn;
      e = cudaGraphAddKernelNode(&cn, body, ifs.data(), ifs.size(), &kp);
    }
  }
  for (int i = 0; i < Mp && e == cudaSuccess; ++i) {
    sps_ctx* c = cs[i];
    sps_state* st = ss[i];
    const uint64_t step = st->cycle_counter + 1;
    cudaGraphNode_t tn;
    const int64_t l0 = c->launches;
    e = child({wnode}, c, [c, st, step]() {
          SPS_TRY(cphase_tail(c, st));
          return sphase_issue(c, st, nullptr, step);
        }, &tn);
    tail_launches[i] = c->launches - l0;
    c->launches = l0;
  }
  if (e != cudaSuccess || buffer_generation() != gen) {
    const std::string why = !cap_error.empty() ? "capture: " + cap_error
                            : e != cudaSuccess ? std::string("graph construction") : std::string("reallocation");
    return give_up(why.c_str(), e);
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) return give_up("instantiate", e);
  struct ExecGuard {
    cudaGraphExec_t x;
    ~ExecGuard() { if (x) cudaGraphExecDestroy(x); }
  } xguard{exec};
  SPS_CUDA_TRY(cudaMemcpyAsync(d_cc, hc.data(), sizeof(CphaseCtl) * hc.size(), cudaMemcpyHostToDevice, ctx->stream));
  SPS_CUDA_TRY(cudaGraphLaunch(exec, ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(hc.data(), d_cc, sizeof(CphaseCtl) * hc.size(), cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<Counters> cnt(static_cast<size_t>(Mp));
  for (int i = 0; i < Mp; ++i)
    SPS_CUDA_TRY(cudaMemcpyAsync(&cnt[i], ss[i]->counters.ptr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (hc[Mp].err) return fail(ctx, SPS_ERR_STATE, "batched C-phase graph: block loop passed its bound");
  for (int i = 0; i < Mp; ++i) {
    sps_ctx* c = cs[i];
    sps_state* st = ss[i];
    c->launches += hc[i].blocks * block_launches[i] + tail_launches[i];
    st->t = hc[i].t_new;
    st->ll_stale = true;
    st->cycle_counter += 1;
    if (cnt[i].res_bad) return fail(ctx, SPS_ERR_DEGENERATE, "model context: all resampling weights of a group vanished");
    sphase_commit(st);
  }
  ctx->launches += hc[Mp].row;   // the loop's condition kernel
  return SPS_OK;
}

sps_status mphase_impl(sps_ctx* ctx, sps_state* st, int kernel, int fixed_steps, const double* sigmas,
                       sps_schedule* rec, int64_t rec_step0, int* steps, double* last_acc, double* last_rne) {
  const double K = (st->t >= ctx->n) ? ctx->opt.rne_final : ctx->opt.rne_cycle;
  const int D = ctx->D;
  int r = 0;
  sps_mstep_info info{};
  bool use_graph = ctx->opt.graphs && fixed_steps <= 0 && !sigmas;
  while (true) {
    const int64_t rs = rec_step0 + r;
    double* sig_out = nullptr;
    if (rec && rec->sigma && rs < rec->cap_steps) sig_out = rec->sigma + rs * D * D;
    const double* sig_in = sigmas ? sigmas + static_cast<int64_t>(r) * D * D : nullptr;
    SPS_TRY(mstep_impl(ctx, st, kernel, sig_in, sig_out, &info));
    if (rec && rs < rec->cap_steps) {
      if (rec->h) rec->h[rs] = info.h;
      if (rec->accept) rec->accept[rs] = info.accept_rate;
    }
    ++r;
    if (fixed_steps > 0) {
      if (r >= fixed_steps) break;
    } else if (info.rne_min >= K || r >= ctx->opt.r_max) {
      break;
    }
    if (use_graph) {
      bool fallback = false;
      int r_end = r;
      SPS_TRY(mphase_graph(ctx, st, kernel, K, r, &r_end, rec, rec_step0, &info, &fallback));
      if (!fallback) {
        r = r_end;
        break;
      }
      use_graph = false;
    }
  }
  if (steps) *steps = r;
  if (last_acc) *last_acc = info.accept_rate;
  if (last_rne) *last_rne = info.rne_min;
  return SPS_OK;
}

// Outputs of a finished run (Eqs. 3, 5-7, 10 and the log ML): moments of theta and of the
// log-odds theta_c' xbar (Eq. 15) from the final particles, and the per-group log ML.
sps_status finish_run(sps_ctx* ctx, sps_state* st, int32_t L, int64_t total_steps, sps_result* out) {
  const int D = ctx->D;
  // outputs: moments of theta and of the log-odds theta_c' xbar (Eq. 15), and the log ML
  const int F = D + ctx->NC;
  SPS_CUDA_TRY(st->scratch.reserve(sizeof(double) * 3 * static_cast<size_t>(st->J) * F + 64));
  group_moments_kernel<<<dim3(st->J, F, 1), 256, 0, ctx->stream>>>(st->theta.as<double>(), st->ll.as<double>(),
                                                          ctx->xbar.as<double>(), st->N, D, ctx->k, F, true, false,
                                                          st->scratch.as<double>()); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  std::vector<double> sums(static_cast<size_t>(st->J) * F * 3), lml(st->J);
  SPS_CUDA_TRY(cudaMemcpyAsync(sums.data(), st->scratch.ptr, sums.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(lml.data(), st->logml.ptr, sizeof(double) * st->J, cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  Moments m = moments_from_sums(sums, st->J, st->N, F);
  for (int f = 0; f < F; ++f) {
    out->mean[f] = m.mean[f];
    out->sd[f] = m.sd[f];
    out->nse[f] = m.nse[f];
    out->rne[f] = m.rne[f];
  }
  double mean = 0.0, mx = -INFINITY;
  for (int j = 0; j < st->J; ++j) {
    out->log_ml_group[j] = lml[j];
    mean += lml[j];
    mx = std::max(mx, lml[j]);
  }
  mean /= st->J;
  double var = 0.0, se = 0.0;
  for (int j = 0; j < st->J; ++j) {
    var += (lml[j] - mean) * (lml[j] - mean);
    se += std::exp(lml[j] - mx);
  }
  out->log_ml = mean;
  out->log_ml_nse = std::sqrt(var / (st->J - 1.0)) / std::sqrt(static_cast<double>(st->J));
  out->log_ml_pooled = mx + std::log(se / st->J);
  out->n_cycles = L;
  out->m_steps = total_steps;
  out->graph_steps = st->graph_steps;
  return SPS_OK;
}

}  // namespace

extern "C" {

sps_status sps_state_create(sps_ctx* ctx, int32_t J, int32_t N, uint64_t seed, sps_state** out) {
  if (!out) return SPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (J < 2 || N < 2 || N > kMaxN) return fail(ctx, SPS_ERR_INVALID_ARG, "need 2 <= J and 2 <= N <= 4096");
  if (ctx->D > kMaxD) return fail(ctx, SPS_ERR_UNSUPPORTED, "the simulator supports at most 155 parameters");
  sps_state* st = new sps_state();
  st->ctx = ctx;
  st->J = J;
  st->N = N;
  st->P = static_cast<int64_t>(J) * N;
  st->seed = seed;
  st->h = ctx->opt.h_init;
  sps_status s = state_buffers(ctx, st);
  if (s != SPS_OK) {
    delete st;
    return s;
  }
  const int D = ctx->D;
  DevBuf z;
  if (z.reserve(static_cast<size_t>(st->P) * D * sizeof(double)) != cudaSuccess) {
    delete st;
    return fail(ctx, SPS_ERR_OOM, "state: out of device memory");
  }
  (void)cudaGetLastError();   // clear a stale error of an earlier, unrelated runtime call
  prior_init_kernel<<<static_cast<unsigned>((st->P + 127) / 128), 128, 0, ctx->stream>>>(
      seed, st->P, D, ctx->d_prior_mean.as<double>(), ctx->d_prior_chol.as<double>(), ctx->d_prior_prec.as<double>(),
      prior_full(ctx), st->theta.as<double>(), st->lp.as<double>(), z.as<double>()); ++ctx->launches;
  cudaMemsetAsync(st->ll.ptr, 0, sizeof(double) * st->P, ctx->stream);
  cudaMemsetAsync(st->logw.ptr, 0, sizeof(double) * st->P, ctx->stream);
  cudaMemsetAsync(st->logml.ptr, 0, sizeof(double) * J, ctx->stream);
  const cudaError_t e_launch = cudaGetLastError();
  const cudaError_t e_sync = cudaStreamSynchronize(ctx->stream);
  if (e_launch != cudaSuccess || e_sync != cudaSuccess) {
    delete st;
    return fail(ctx, SPS_ERR_CUDA, std::string("state: prior draw failed: launch ") + cudaGetErrorString(e_launch) +
                                       ", sync " + cudaGetErrorString(e_sync));
  }
  *out = st;
  return SPS_OK;
}

void sps_state_destroy(sps_state* st) {
  if (!st) return;
  if (st->ctx) cudaStreamSynchronize(st->ctx->stream);
  if (st->mgraph) cudaGraphExecDestroy(st->mgraph);
  if (st->pinned) cudaFreeHost(st->pinned);
  delete st;
}

sps_status sps_state_get(sps_ctx* ctx, const sps_state* st, double* theta, double* ll, double* logw, int64_t* t,
                         double* h) {
  SPS_TRY(check_state(ctx, st));
  if (theta)
    SPS_CUDA_TRY(cudaMemcpyAsync(theta, st->theta.ptr, sizeof(double) * st->P * ctx->D, cudaMemcpyDeviceToHost,
                                 ctx->stream));
  if (ll) SPS_CUDA_TRY(cudaMemcpyAsync(ll, st->ll.ptr, sizeof(double) * st->P, cudaMemcpyDeviceToHost, ctx->stream));
  if (logw)
    SPS_CUDA_TRY(cudaMemcpyAsync(logw, st->logw.ptr, sizeof(double) * st->P, cudaMemcpyDeviceToHost, ctx->stream));
  if (theta || ll || logw) SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));   // t and h are host-side
  if (t) *t = st->t;
  if (h) *h = st->h;
  return SPS_OK;
}

sps_status sps_state_result(sps_ctx* ctx, sps_state* st, sps_result* out) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  SPS_TRY(check_state(ctx, st));
  if (!out || !out->mean || !out->sd || !out->nse || !out->rne || !out->log_ml_group)
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_state_result: result arrays missing");
  return finish_run(ctx, st, static_cast<int32_t>(st->cycle_counter), static_cast<int64_t>(st->step_counter), out);
}

sps_status sps_state_set(sps_ctx* ctx, sps_state* st, const double* theta, const double* ll, int64_t t) {
  SPS_TRY(check_state(ctx, st));
  if (!theta || t < 0 || t > ctx->n) return fail(ctx, SPS_ERR_INVALID_ARG, "state_set: bad arguments");
  SPS_CUDA_TRY(cudaMemcpyAsync(st->theta.ptr, theta, sizeof(double) * st->P * ctx->D, cudaMemcpyHostToDevice,
                               ctx->stream));
  prior_lp_kernel<<<static_cast<unsigned>((st->P + 255) / 256), 256, 0, ctx->stream>>>(
      st->theta.as<double>(), st->P, ctx->D, ctx->d_prior_mean.as<double>(), ctx->d_prior_prec.as<double>(),
      prior_full(ctx), st->lp.as<double>()); ++ctx->launches;
  st->t = t;
  if (ll) {
    SPS_CUDA_TRY(cudaMemcpyAsync(st->ll.ptr, ll, sizeof(double) * st->P, cudaMemcpyHostToDevice, ctx->stream));
    st->ll_stale = false;
    st->ll_kind = (ctx->opt.precision == SPS_PREC_FP32) ? 1 : 0;   // taken as the RW kernel's values
  } else {
    st->ll_stale = true;
  }
  st->have_weights = false;
  st->grad_valid = false;
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

sps_status sps_cphase(sps_ctx* ctx, sps_state* st, int64_t t_target, int64_t* t_new, double* ess,
                      double* logml_inc, double* log_pred) {
  SPS_TRY(check_state(ctx, st));
  return cphase_impl(ctx, st, t_target, t_new, ess, logml_inc, log_pred);
}

sps_status sps_sphase(sps_ctx* ctx, sps_state* st, const double* uniforms, int32_t* idx_out, int32_t mem) {
  SPS_TRY(check_state(ctx, st));
  if (mem == SPS_MEM_DEVICE) return sphase_impl(ctx, st, uniforms, idx_out);
  // host indices are copied from the state's own index buffer (no staging allocation per call)
  DevBuf du;
  if (uniforms) {
    SPS_CUDA_TRY(du.reserve(sizeof(double) * st->P));
    SPS_CUDA_TRY(cudaMemcpyAsync(du.ptr, uniforms, sizeof(double) * st->P, cudaMemcpyHostToDevice, ctx->stream));
  }
  return sphase_impl(ctx, st, uniforms ? du.as<double>() : nullptr, nullptr, idx_out);
}

sps_status sps_mstep(sps_ctx* ctx, sps_state* st, int32_t kernel, const double* sigma, double* sigma_used,
                     sps_mstep_info* info) {
  SPS_TRY(check_state(ctx, st));
  if (st->t <= 0) return fail(ctx, SPS_ERR_STATE, "M step before any observation was added");
  return mstep_impl(ctx, st, kernel, sigma, sigma_used, info);
}

sps_status sps_mphase(sps_ctx* ctx, sps_state* st, int32_t kernel, int32_t fixed_steps, int32_t* steps,
                      double* accept_rate, double* rne_min) {
  SPS_TRY(check_state(ctx, st));
  if (st->t <= 0) return fail(ctx, SPS_ERR_STATE, "M phase before any observation was added");
  return mphase_impl(ctx, st, kernel, fixed_steps, nullptr, nullptr, 0, steps, accept_rate, rne_min);
}

sps_status sps_run(sps_ctx* ctx, int32_t groups, int32_t particles_per_group, const sps_schedule* schedule,
                   sps_schedule* record, sps_result* out) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!out || !out->mean || !out->sd || !out->nse || !out->rne || !out->log_ml_group)
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_run: result arrays missing");
  const auto t0 = std::chrono::steady_clock::now();
  sps_state* st = nullptr;
  SPS_TRY(sps_state_create(ctx, groups, particles_per_group, ctx->opt.seed, &st));
  struct Guard {
    sps_state* s;
    ~Guard() { sps_state_destroy(s); }
  } guard{st};
  const int D = ctx->D;
  const bool replay = schedule && schedule->n_cycles > 0;
  int32_t L = 0;
  int64_t total_steps = 0;
  const bool want_lpl = out->log_pred || out->log_pred_nse;
  std::vector<double> lpl(want_lpl ? static_cast<size_t>(ctx->n) * groups : 0);
  while (st->t < ctx->n) {
    if (replay && L >= schedule->n_cycles) return fail(ctx, SPS_ERR_INVALID_ARG, "schedule ends before T");
    const int64_t target = replay ? schedule->t[L] : 0;
    int64_t tn = 0;
    const int64_t t_before = st->t;
    SPS_TRY(cphase_impl(ctx, st, target, &tn, nullptr, nullptr,
                        want_lpl ? lpl.data() + t_before * groups : nullptr));
    SPS_TRY(sphase_impl(ctx, st, nullptr, nullptr));
    int steps = 0;
    double acc = 0.0, rne = 0.0;
    if (replay) {
      const int R = schedule->R[L];
      if (!schedule->sigma) return fail(ctx, SPS_ERR_INVALID_ARG, "replayed schedule has no Sigma matrices");
      int64_t before = 0;
      for (int q = 0; q < L; ++q) before += schedule->R[q];
      SPS_TRY(mphase_impl(ctx, st, ctx->opt.mkernel, R, schedule->sigma + before * D * D, record, total_steps,
                          &steps, &acc, &rne));
    } else {
      SPS_TRY(mphase_impl(ctx, st, ctx->opt.mkernel, 0, nullptr, record, total_steps, &steps, &acc, &rne));
    }
    if (record) {
      if (L >= record->cap_cycles) return fail(ctx, SPS_ERR_INVALID_ARG, "schedule record: too many cycles");
      record->t[L] = tn;
      record->R[L] = steps;
      if (total_steps + steps > record->cap_steps)
        return fail(ctx, SPS_ERR_INVALID_ARG, "schedule record: too many M steps");
    }
    total_steps += steps;
    ++L;
  }
  if (record) record->n_cycles = L;
  SPS_TRY(finish_run(ctx, st, L, total_steps, out));
  if (want_lpl)
    for (int64_t q = 0; q < ctx->n; ++q) {
      const double* row = lpl.data() + q * groups;
      double m = 0.0;
      for (int j = 0; j < groups; ++j) m += row[j];
      m /= groups;
      double v = 0.0;
      for (int j = 0; j < groups; ++j) v += (row[j] - m) * (row[j] - m);
      if (out->log_pred) out->log_pred[q] = m;
      if (out->log_pred_nse) out->log_pred_nse[q] = std::sqrt(v / (groups - 1.0)) / std::sqrt(static_cast<double>(groups));
    }
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SPS_OK;
}

sps_status sps_run_batched(sps_ctx* ctx, int32_t M, const int32_t* k_models, double g, int32_t groups,
                           int32_t particles_per_group, sps_result* out) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (M < 1 || M > 1024 || !k_models || !out) return fail(ctx, SPS_ERR_INVALID_ARG, "sps_run_batched: bad arguments");
  for (int m = 0; m < M; ++m) {
    if (k_models[m] < 1 || k_models[m] > ctx->k)
      return fail(ctx, SPS_ERR_INVALID_ARG, "sps_run_batched: model covariate count out of range");
    const sps_result& o = out[m];
    if (!o.mean || !o.sd || !o.nse || !o.rne || !o.log_ml_group)
      return fail(ctx, SPS_ERR_INVALID_ARG, "sps_run_batched: result arrays missing");
  }
  const bool mala = (ctx->opt.mkernel == SPS_MKERNEL_MALA);
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = ctx->n;
  const int k = ctx->k, NC = ctx->NC, D = ctx->D;
  // the data on the host once, to build each model's context
  std::vector<double> X(static_cast<size_t>(n) * k);
  std::vector<int32_t> y(static_cast<size_t>(n));
  SPS_CUDA_TRY(cudaMemcpyAsync(X.data(), ctx->Xd.ptr, sizeof(double) * X.size(), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(y.data(), ctx->y.ptr, sizeof(int32_t) * y.size(), cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  struct Model {
    sps_ctx* c = nullptr;
    sps_state* st = nullptr;
    int32_t L = 0;
    int64_t steps = 0;
  };
  struct Models {
    std::vector<Model> v;
    ~Models() {
      for (Model& m : v) {
        sps_state_destroy(m.st);
        sps_destroy(m.c);
      }
    }
  } models;
  models.v.resize(M);
  // the sub-context's last error becomes the caller's
  auto pass = [&](sps_ctx* c, sps_status st) {
    ctx->last_error = std::string("model context: ") + c->last_error;
    return st;
  };
  for (int m = 0; m < M; ++m) {
    const int km = k_models[m], Dm = km * NC;
    std::vector<double> Xm(static_cast<size_t>(n) * km);
    for (int64_t s = 0; s < n; ++s)
      for (int i = 0; i < km; ++i) Xm[s * km + i] = X[s * k + i];
    // prior of the model's coordinates (theta_c, i < k_m): the marginal of the context's prior
    std::vector<int> idx;
    for (int c = 0; c < NC; ++c)
      for (int i = 0; i < km; ++i) idx.push_back(c * k + i);
    std::vector<double> mu(Dm), cov;
    for (int a = 0; a < Dm; ++a) mu[a] = ctx->prior_mean[idx[a]];
    sps_prior pr{};
    if (ctx->prior_kind == SPS_PRIOR_FULL) {
      cov.resize(static_cast<size_t>(Dm) * Dm);
      for (int a = 0; a < Dm; ++a)
        for (int b = 0; b < Dm; ++b) cov[a * Dm + b] = ctx->prior_cov[static_cast<size_t>(idx[a]) * D + idx[b]];
      pr.kind = SPS_PRIOR_FULL;
    } else {
      cov.resize(Dm);
      for (int a = 0; a < Dm; ++a) cov[a] = std::sqrt(ctx->prior_cov[static_cast<size_t>(idx[a]) * D + idx[a]]);
      pr.kind = SPS_PRIOR_DIAG;
    }
    pr.mean = mu.data();
    pr.cov_or_sd = cov.data();
    sps_options o = ctx->opt;
    o.graphs = 0;
    const sps_status si = sps_init(&models.v[m].c, Xm.data(), n, km, y.data(), ctx->C, &pr, &o);
    if (si != SPS_OK) {
      if (models.v[m].c) return pass(models.v[m].c, si);
      return fail(ctx, si, "sps_run_batched: model context");
    }
    sps_ctx* c = models.v[m].c;
    c->stream = ctx->stream;
    if (g > 0.0) {
      // the paper's g-prior of this model's covariates
      std::vector<double> gm(Dm), gc(static_cast<size_t>(Dm) * Dm);
      sps_status e = sps_gprior(c, g, gm.data(), gc.data());
      sps_prior pg{};
      pg.kind = SPS_PRIOR_FULL;
      pg.mean = gm.data();
      pg.cov_or_sd = gc.data();
      if (e == SPS_OK) e = sps_set_prior(c, &pg);
      if (e != SPS_OK) return pass(c, e);
    }
    const uint64_t seed = ctx->opt.seed + 0x9E3779B97F4A7C15ull * static_cast<uint64_t>(m + 1);
    const sps_status ss = sps_state_create(c, groups, particles_per_group, seed, &models.v[m].st);
    if (ss != SPS_OK) return pass(c, ss);
  }
  const bool split = (ctx->opt.precision == SPS_PREC_SPLIT);
  // Which function evaluates a model's log-likelihoods (both sides of every Metropolis ratio use
  // the same one): in split precision the batched fused-kernel launch, in which each model's
  // tiles use the model's own encoding of its covariates (c5, 24 models of 16 384 particles:
  // 1.09 / 3.44 / 27.5 ms per batched launch against 1.16 / 3.86 / 28.5 ms for 24 own launches at
  // t = 10^3 / 10^4 / 10^5); FP32 precision: the model's own FP32 launch.
  std::vector<char> in_batch(M, 0);
  std::vector<int32_t> bk;
  std::vector<int64_t> bP, bt;
  std::vector<const double*> bth;
  std::vector<double*> bll;
  std::vector<char> bskip;
  // the log-likelihoods of the listed models' particles (or proposals); with moving, only of the
  // models moving[m] marks: the batched launch keeps every listed model and skips the tiles of
  // the others, so that its work decomposition, and with it the rounding of every model's
  // sums, stays that of the phase's first step (and of the captured phase)
  auto evaluate = [&](const std::vector<int>& list, bool proposals, const std::vector<char>* moving) -> sps_status {
    bk.clear(); bP.clear(); bt.clear(); bth.clear(); bll.clear(); bskip.clear();
    for (int m : list) {
      sps_state* st = models.v[m].st;
      const double* th = proposals ? st->theta_prop.as<double>() : st->theta.as<double>();
      double* ll = proposals ? st->ll_prop.as<double>() : st->ll.as<double>();
      const bool mv = !moving || (*moving)[m];
      if (in_batch[m]) {
        bk.push_back(k_models[m]);
        bP.push_back(st->P);
        bt.push_back(st->t);
        bth.push_back(th);
        bll.push_back(ll);
        bskip.push_back(mv ? 0 : 1);
      } else if (mv) {
        sps_ctx* c = models.v[m].c;
        const sps_status e = loglik_dispatch(c, th, st->P, st->t, ll, ctx->opt.precision);
        if (e != SPS_OK) return pass(c, e);
      }
    }
    if (bk.empty()) return SPS_OK;
    return loglik_split_batched(ctx, static_cast<int>(bk.size()), bk.data(), bP.data(), bt.data(), bth.data(),
                                bll.data(), bskip.data());
  };
  const sps_options& o = ctx->opt;
  DevBuf jobs_dev, ctl_buf, cc_buf;
  SPS_CUDA_TRY(jobs_dev.reserve(sizeof(CholJob) * static_cast<size_t>(M)));
  bool use_graph = o.graphs != 0, use_cs_graph = o.graphs != 0, warm = false;
  while (true) {
    std::vector<int> active;
    for (int m = 0; m < M; ++m)
      if (models.v[m].st->t < n) active.push_back(m);
    if (active.empty()) break;
    // C and S phases per model (Algorithm 1 steps 2(a), 2(b)): with graphs, all models' phases in
    // one graph launch; else one model after the other from the host
    bool cs_done = false;
    if (use_cs_graph) {
      std::vector<sps_ctx*> pc;
      std::vector<sps_state*> ps;
      for (int m : active) {
        pc.push_back(models.v[m].c);
        ps.push_back(models.v[m].st);
      }
      bool fallback = false;
      SPS_TRY(batched_cs_graph(ctx, pc, ps, cc_buf, &fallback));
      cs_done = !fallback;
      if (fallback) use_cs_graph = false;
    }
    for (int m : active) {
      Model& md = models.v[m];
      if (!cs_done) {
        int64_t tn = 0;
        sps_status e = cphase_impl(md.c, md.st, 0, &tn, nullptr, nullptr, nullptr);
        if (e == SPS_OK) e = sphase_impl(md.c, md.st, nullptr, nullptr);
        if (e != SPS_OK) return pass(md.c, e);
      }
      ++md.L;
    }
    // M phases in lockstep (Algorithm 2 step 2(c)): every step of the models still moving is
    // one batched evaluation of their proposals; a model leaves when its RNE criterion or the
    // step cap is met. With graphs, after the first cycle (which sizes every buffer) the whole
    // phase is one graph launch; else its first step runs from the host and the rest as a graph.
    std::vector<int> run = active, r(M, 0);
    for (int m : active) in_batch[m] = split && !mala;
    if (use_graph && warm) {
      std::vector<sps_ctx*> pc;
      std::vector<sps_state*> ps;
      std::vector<char> pm, pb;
      std::vector<int> pr;
      for (int m : active) {
        pc.push_back(models.v[m].c);
        ps.push_back(models.v[m].st);
        pm.push_back(1);
        pb.push_back(in_batch[m]);
        pr.push_back(0);
      }
      bool fallback = false;
      SPS_TRY(batched_mphase_graph(ctx, pc, ps, pm, pb, ctx->opt.mkernel, true, pr, ctl_buf, &fallback));
      if (!fallback) {
        for (size_t i = 0; i < active.size(); ++i) r[active[i]] = pr[i];
        run.clear();
      } else {
        use_graph = false;
      }
    }
    warm = true;
    if (run.empty()) {
      // the phase ran in the graph
    } else if (mala) {
      // MALA: each model's log-likelihood and gradient come from its own gradient launch (the
      // cached values at the start of the phase included)
      for (int m : active) {
        const sps_status e = mstep_prepare(models.v[m].c, models.v[m].st, SPS_MKERNEL_MALA);
        if (e != SPS_OK) return pass(models.v[m].c, e);
      }
    } else {
      SPS_TRY(evaluate(active, false, nullptr));   // cached log-likelihoods with the proposals' function
      for (int m : active) {
        models.v[m].st->ll_stale = false;
        models.v[m].st->ll_kind = split ? 0 : 1;
      }
    }
    std::vector<char> moving(M, 0);
    for (int m : run) moving[m] = 1;
    std::vector<double> hs(M);
    std::vector<uint64_t> steps(M);
    std::vector<CholJob> jobs;
    jobs.reserve(M);
    while (!run.empty()) {
      // every model's Sigma = h V, their Cholesky factors in one launch (one block each), then
      // the proposals: the operations of rw_issue_propose, with the factorisations batched
      jobs.clear();
      size_t tmax = 1;
      for (int m : run) {
        Model& md = models.v[m];
        hs[m] = md.st->h;
        steps[m] = ++md.st->step_counter;
        SPS_CUDA_TRY(cudaMemsetAsync(md.st->counters.ptr, 0, sizeof(Counters), ctx->stream));
        const sps_status e = proposal_sigma(md.c, md.st, md.st->theta.as<double>(), hs[m], nullptr, nullptr, nullptr);
        if (e != SPS_OK) return pass(md.c, e);
        jobs.push_back(chol_job(md.c, md.st, flag_ptr(md.st, 0)));
        const size_t Dm = static_cast<size_t>(md.c->D);
        tmax = std::max(tmax, Dm * (Dm + 1) / 2);
      }
      SPS_CUDA_TRY(cudaMemcpyAsync(jobs_dev.ptr, jobs.data(), sizeof(CholJob) * jobs.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
      SPS_CUDA_TRY(cudaFuncSetAttribute(cholesky_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(sizeof(double) * tmax)));
      cholesky_batched_kernel<<<static_cast<unsigned>(jobs.size()), kCholThreads, sizeof(double) * tmax,
                                ctx->stream>>>(jobs_dev.as<CholJob>()); ++ctx->launches;
      SPS_CUDA_TRY(cudaGetLastError());
      if (mala) {
        // proposals with the drift, their log-likelihoods and gradients, the decisions
        for (int m : run) {
          Model& md = models.v[m];
          sps_status e = mala_issue(md.c, md.st, steps[m], nullptr, nullptr, nullptr, nullptr, nullptr);
          if (e == SPS_OK) {
            launch_monitoring(md.c, md.st);
            e = readback_issue(md.c, md.st);
          }
          if (e != SPS_OK) return pass(md.c, e);
        }
      } else {
        for (int m : run) {
          Model& md = models.v[m];
          const sps_status e = launch_propose(md.c, md.st, md.st->theta.as<double>(), md.st->P, nullptr, steps[m],
                                              nullptr, flag_ptr(md.st, 0), md.st->theta_prop.as<double>(),
                                              md.st->lp_prop.as<double>());
          if (e != SPS_OK) return pass(md.c, e);
        }
        SPS_TRY(evaluate(active, true, &moving));
        // every model's decisions and read-back enqueued, then one synchronisation
        for (int m : run) {
          Model& md = models.v[m];
          sps_status e = rw_issue_accept(md.c, md.st, steps[m], nullptr);
          if (e == SPS_OK) e = readback_issue(md.c, md.st);
          if (e != SPS_OK) return pass(md.c, e);
        }
      }
      SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      std::vector<int> next;
      for (int m : run) {
        Model& md = models.v[m];
        sps_mstep_info info{};
        const sps_status e = mstep_rule(md.c, md.st, ctx->opt.mkernel, hs[m], true, &info);
        if (e != SPS_OK) return pass(md.c, e);
        if (!mala) md.st->grad_valid = false;
        ++r[m];
        const double K = (md.st->t >= n) ? o.rne_final : o.rne_cycle;
        if (!(info.rne_min >= K || r[m] >= o.r_max)) next.push_back(m);
        else moving[m] = 0;
      }
      run.swap(next);
      if (use_graph && !run.empty()) {
        // the rest of the phase as one graph launch
        std::vector<sps_ctx*> pc;
        std::vector<sps_state*> ps;
        std::vector<char> pm, pb;
        std::vector<int> pr;
        for (int m : active) {
          pc.push_back(models.v[m].c);
          ps.push_back(models.v[m].st);
          pm.push_back(moving[m]);
          pb.push_back(in_batch[m] && !mala);
          pr.push_back(r[m]);
        }
        bool fallback = false;
        SPS_TRY(batched_mphase_graph(ctx, pc, ps, pm, pb, ctx->opt.mkernel, false, pr, ctl_buf, &fallback));
        if (!fallback) {
          for (size_t i = 0; i < active.size(); ++i) r[active[i]] = pr[i];
          run.clear();
        } else {
          use_graph = false;
        }
      }
    }
    for (int m : active) models.v[m].steps += r[m];
  }
  for (int m = 0; m < M; ++m) {
    Model& md = models.v[m];
    const sps_status e = finish_run(md.c, md.st, md.L, md.steps, &out[m]);
    if (e != SPS_OK) return pass(md.c, e);
    out[m].seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return SPS_OK;
}

// ------------------------------------------------------------------------------ building blocks

sps_status sps_resample(sps_ctx* ctx, const double* w, const double* u, int32_t J, int32_t N, int32_t scheme,
                        int32_t* idx, int32_t mem) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!w || !u || !idx || J < 1 || N < 1 || N > kMaxN) return fail(ctx, SPS_ERR_INVALID_ARG, "sps_resample: bad arguments");
  const size_t P = static_cast<size_t>(J) * N;
  DevBuf dw, du, di, df;
  SPS_CUDA_TRY(df.reserve(sizeof(int)));
  SPS_CUDA_TRY(cudaMemsetAsync(df.ptr, 0, sizeof(int), ctx->stream));
  const double* pw = w;
  const double* pu = u;
  int* pi = idx;
  if (mem == SPS_MEM_HOST) {
    SPS_CUDA_TRY(dw.reserve(P * sizeof(double)));
    SPS_CUDA_TRY(du.reserve(P * sizeof(double)));
    SPS_CUDA_TRY(di.reserve(P * sizeof(int)));
    SPS_CUDA_TRY(cudaMemcpyAsync(dw.ptr, w, P * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    SPS_CUDA_TRY(cudaMemcpyAsync(du.ptr, u, P * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    pw = dw.as<double>();
    pu = du.as<double>();
    pi = di.as<int>();
  }
  DevBuf dq;
  SPS_CUDA_TRY(dq.reserve(P * sizeof(unsigned long long)));
  resample_q_kernel<<<static_cast<unsigned>((P + 255) / 256), 256, 0, ctx->stream>>>(
      pw, 1, N, static_cast<int64_t>(P), nullptr, dq.as<unsigned long long>()); ++ctx->launches;
  SPS_TRY(launch_resample(ctx, scheme, dq.as<unsigned long long>(), J, N, pu, 0, 0, pi, df.as<int>()));
  if (mem == SPS_MEM_HOST) {
    int bad = 0;
    SPS_CUDA_TRY(cudaMemcpyAsync(idx, di.ptr, P * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA_TRY(cudaMemcpyAsync(&bad, df.ptr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (bad) return fail(ctx, SPS_ERR_DEGENERATE, "all weights of a group quantise to zero");
  } else {
    SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));   // the flag buffer is local to this call
  }
  return SPS_OK;
}

sps_status sps_philox(sps_ctx* ctx, uint32_t key0, uint32_t key1, uint32_t ctr0, uint32_t ctr1, uint32_t ctr2,
                      uint32_t ctr3, int64_t count, uint32_t* out, int32_t mem) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!out || count < 1) return fail(ctx, SPS_ERR_INVALID_ARG, "sps_philox: bad arguments");
  DevBuf d;
  uint4* po = reinterpret_cast<uint4*>(out);
  if (mem == SPS_MEM_HOST) {
    SPS_CUDA_TRY(d.reserve(static_cast<size_t>(count) * 16));
    po = d.as<uint4>();
  }
  philox_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, ctx->stream>>>(
      key0, key1, make_uint4(ctr0, ctr1, ctr2, ctr3), count, po); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  if (mem == SPS_MEM_HOST) {
    SPS_CUDA_TRY(cudaMemcpyAsync(out, d.ptr, static_cast<size_t>(count) * 16, cudaMemcpyDeviceToHost, ctx->stream));
    SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  }
  return SPS_OK;
}

sps_status sps_ess(sps_ctx* ctx, const double* logw, int64_t P, int32_t J, double* ess, double* lme, int32_t mem) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!logw || P < 1 || J < 1 || P % J != 0) return fail(ctx, SPS_ERR_INVALID_ARG, "sps_ess: bad arguments");
  DevBuf dl, de, dm;
  const double* pl = logw;
  if (mem == SPS_MEM_HOST) {
    SPS_CUDA_TRY(dl.reserve(P * sizeof(double)));
    SPS_CUDA_TRY(cudaMemcpyAsync(dl.ptr, logw, P * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    pl = dl.as<double>();
  }
  SPS_CUDA_TRY(de.reserve(sizeof(double)));
  SPS_CUDA_TRY(dm.reserve(sizeof(double) * J));
  double* pe = (mem == SPS_MEM_DEVICE && ess) ? ess : de.as<double>();
  double* pm = (mem == SPS_MEM_DEVICE && lme) ? lme : dm.as<double>();
  DevBuf dparts;
  SPS_CUDA_TRY(dparts.reserve(sizeof(double) * std::max<size_t>(3 * kEssParts, 2 * static_cast<size_t>(J) * kLmeParts)));
  ess_part_kernel<double><<<dim3(1, kEssParts), 512, 0, ctx->stream>>>(pl, P, dparts.as<double>(), nullptr);
  ++ctx->launches;
  ess_merge_kernel<<<1, 64, 0, ctx->stream>>>(dparts.as<double>(), 1, kEssParts, pe, nullptr); ++ctx->launches;
  group_lme_part_kernel<<<dim3(J, kLmeParts), 256, 0, ctx->stream>>>(pl, static_cast<int>(P / J),
                                                                     dparts.as<double>()); ++ctx->launches;
  group_lme_merge_kernel<<<(J + 63) / 64, 64, 0, ctx->stream>>>(dparts.as<double>(), J, kLmeParts,
                                                                static_cast<int>(P / J), pm, nullptr,
                                                                nullptr); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  if (mem == SPS_MEM_HOST) {
    if (ess) SPS_CUDA_TRY(cudaMemcpyAsync(ess, pe, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (lme) SPS_CUDA_TRY(cudaMemcpyAsync(lme, pm, sizeof(double) * J, cudaMemcpyDeviceToHost, ctx->stream));
  }
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

sps_status sps_particle_cov(sps_ctx* ctx, const double* theta, int64_t P, double* V, int32_t mem) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!theta || !V || P < 2) return fail(ctx, SPS_ERR_INVALID_ARG, "sps_particle_cov: bad arguments");
  const int D = ctx->D;
  if (D > 155) return fail(ctx, SPS_ERR_UNSUPPORTED, "sps_particle_cov: at most 155 parameters");
  const int T = D * (D + 1) / 2;
  const int blocks = cov_blocks(P);
  DevBuf dt, dv, dpart;
  const double* pt = theta;
  if (mem == SPS_MEM_HOST) {
    SPS_CUDA_TRY(dt.reserve(sizeof(double) * P * D));
    SPS_CUDA_TRY(cudaMemcpyAsync(dt.ptr, theta, sizeof(double) * P * D, cudaMemcpyHostToDevice, ctx->stream));
    pt = dt.as<double>();
  }
  SPS_CUDA_TRY(dv.reserve(sizeof(double) * D * D));
  SPS_CUDA_TRY(dpart.reserve(sizeof(double) * (T + D) * blocks));
  double* pv = (mem == SPS_MEM_DEVICE) ? V : dv.as<double>();
  SPS_TRY(launch_cov(ctx, pt, P, D, 1.0, nullptr, dpart.as<double>(), pv, nullptr));
  if (mem == SPS_MEM_HOST)
    SPS_CUDA_TRY(cudaMemcpyAsync(V, pv, sizeof(double) * D * D, cudaMemcpyDeviceToHost, ctx->stream));
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return SPS_OK;
}

sps_status sps_rw_step_given(sps_ctx* ctx, double* theta, double* ll, int64_t P, int64_t t, const double* sigma,
                             const double* z, const double* u, int32_t precision, double* log_alpha,
                             int32_t* accepted, int32_t mem) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!theta || !ll || !sigma || !z || !u || P < 1 || t < 0 || t > ctx->n)
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_rw_step_given: bad arguments");
  const int D = ctx->D;
  if (D > kMaxD) return fail(ctx, SPS_ERR_UNSUPPORTED, "at most 155 parameters");
  // a temporary state holds the buffers; its particles are the caller's
  sps_state tmp;
  tmp.ctx = ctx;
  tmp.J = 1;
  tmp.N = 2;
  tmp.P = P;
  SPS_TRY(state_buffers(ctx, &tmp));
  DevBuf dz, du, dla, dacc;
  const size_t pd = sizeof(double) * P * D;
  const double* pz = z;
  const double* pu = u;
  double* pla = log_alpha;
  int* pacc = accepted;
  if (mem == SPS_MEM_HOST) {
    SPS_CUDA_TRY(cudaMemcpyAsync(tmp.theta.ptr, theta, pd, cudaMemcpyHostToDevice, ctx->stream));
    SPS_CUDA_TRY(cudaMemcpyAsync(tmp.ll.ptr, ll, sizeof(double) * P, cudaMemcpyHostToDevice, ctx->stream));
    SPS_CUDA_TRY(dz.reserve(pd));
    SPS_CUDA_TRY(du.reserve(sizeof(double) * P));
    SPS_CUDA_TRY(dla.reserve(sizeof(double) * P));
    SPS_CUDA_TRY(dacc.reserve(sizeof(int) * P));
    SPS_CUDA_TRY(cudaMemcpyAsync(dz.ptr, z, pd, cudaMemcpyHostToDevice, ctx->stream));
    SPS_CUDA_TRY(cudaMemcpyAsync(du.ptr, u, sizeof(double) * P, cudaMemcpyHostToDevice, ctx->stream));
    pz = dz.as<double>();
    pu = du.as<double>();
    pla = dla.as<double>();
    pacc = dacc.as<int>();
  } else {
    SPS_CUDA_TRY(cudaMemcpyAsync(tmp.theta.ptr, theta, pd, cudaMemcpyDeviceToDevice, ctx->stream));
    SPS_CUDA_TRY(cudaMemcpyAsync(tmp.ll.ptr, ll, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  SPS_CUDA_TRY(cudaMemsetAsync(tmp.counters.ptr, 0, sizeof(Counters), ctx->stream));
  prior_lp_kernel<<<static_cast<unsigned>((P + 255) / 256), 256, 0, ctx->stream>>>(
      tmp.theta.as<double>(), P, D, ctx->d_prior_mean.as<double>(), ctx->d_prior_prec.as<double>(), prior_full(ctx),
      tmp.lp.as<double>()); ++ctx->launches;
  SPS_TRY(factor_proposal(ctx, &tmp, tmp.theta.as<double>(), 1.0, nullptr, sigma, nullptr, flag_ptr(&tmp, 0)));
  SPS_TRY(launch_propose(ctx, &tmp, tmp.theta.as<double>(), P, pz, 0, nullptr, flag_ptr(&tmp, 0),
                         tmp.theta_prop.as<double>(), tmp.lp_prop.as<double>()));
  SPS_TRY(loglik_dispatch(ctx, tmp.theta_prop.as<double>(), P, t, tmp.ll_prop.as<double>(), precision));
  accept_kernel<<<static_cast<unsigned>((P + kAccThreads - 1) / kAccThreads), kAccThreads, 0, ctx->stream>>>(
      tmp.theta.as<double>(), tmp.ll.as<double>(), tmp.lp.as<double>(), tmp.theta_prop.as<double>(),
      tmp.ll_prop.as<double>(), tmp.lp_prop.as<double>(), P, D, pu, 0, 0, nullptr, flag_ptr(&tmp, 0),
      tmp.counters.as<unsigned long long>(), flag_ptr(&tmp, 1), pla, pacc); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  Counters c;
  SPS_TRY(read_counters(ctx, &tmp, &c));
  if (c.chol_bad) return fail(ctx, SPS_ERR_DEGENERATE, "sigma is not positive definite");
  const cudaMemcpyKind k = (mem == SPS_MEM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  SPS_CUDA_TRY(cudaMemcpyAsync(theta, tmp.theta.ptr, pd, k, ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(ll, tmp.ll.ptr, sizeof(double) * P, k, ctx->stream));
  if (mem == SPS_MEM_HOST) {
    if (log_alpha) SPS_CUDA_TRY(cudaMemcpyAsync(log_alpha, pla, sizeof(double) * P, k, ctx->stream));
    if (accepted) SPS_CUDA_TRY(cudaMemcpyAsync(accepted, pacc, sizeof(int) * P, k, ctx->stream));
  }
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (c.nonfinite) return fail(ctx, SPS_ERR_NONFINITE, "non-finite log-likelihood of a proposal");
  return SPS_OK;
}

sps_status sps_mala_step_given(sps_ctx* ctx, double* theta, double* ll, int64_t P, int64_t t, const double* sigma,
                               const double* z, const double* u, double* log_alpha, int32_t* accepted,
                               int32_t mem) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!theta || !ll || !sigma || !z || !u || P < 1 || t < 1 || t > ctx->n)
    return fail(ctx, SPS_ERR_INVALID_ARG, "sps_mala_step_given: bad arguments");
  const int D = ctx->D;
  if (D > kMaxD) return fail(ctx, SPS_ERR_UNSUPPORTED, "at most 155 parameters");
  // a temporary state holds the buffers; its particles are the caller's
  sps_state tmp;
  tmp.ctx = ctx;
  tmp.J = 1;
  tmp.N = 2;
  tmp.P = P;
  tmp.t = t;
  SPS_TRY(state_buffers(ctx, &tmp));
  const size_t pd = sizeof(double) * P * D;
  SPS_CUDA_TRY(tmp.grad.reserve(pd));
  SPS_CUDA_TRY(tmp.grad_prop.reserve(pd));
  SPS_CUDA_TRY(tmp.zq.reserve(sizeof(float) * P * D));
  SPS_CUDA_TRY(tmp.z2.reserve(sizeof(double) * P));
  DevBuf dz, du, dla, dacc;
  const double* pz = z;
  const double* pu = u;
  double* pla = log_alpha;
  int* pacc = accepted;
  const cudaMemcpyKind kin = (mem == SPS_MEM_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  SPS_CUDA_TRY(cudaMemcpyAsync(tmp.theta.ptr, theta, pd, kin, ctx->stream));
  if (mem == SPS_MEM_HOST) {
    SPS_CUDA_TRY(dz.reserve(pd));
    SPS_CUDA_TRY(du.reserve(sizeof(double) * P));
    SPS_CUDA_TRY(dla.reserve(sizeof(double) * P));
    SPS_CUDA_TRY(dacc.reserve(sizeof(int) * P));
    SPS_CUDA_TRY(cudaMemcpyAsync(dz.ptr, z, pd, cudaMemcpyHostToDevice, ctx->stream));
    SPS_CUDA_TRY(cudaMemcpyAsync(du.ptr, u, sizeof(double) * P, cudaMemcpyHostToDevice, ctx->stream));
    pz = dz.as<double>();
    pu = du.as<double>();
    pla = dla.as<double>();
    pacc = dacc.as<int>();
  }
  SPS_CUDA_TRY(cudaMemsetAsync(tmp.counters.ptr, 0, sizeof(Counters), ctx->stream));
  prior_lp_kernel<<<static_cast<unsigned>((P + 255) / 256), 256, 0, ctx->stream>>>(
      tmp.theta.as<double>(), P, D, ctx->d_prior_mean.as<double>(), ctx->d_prior_prec.as<double>(), prior_full(ctx),
      tmp.lp.as<double>()); ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  // the log-likelihood and its gradient at theta, from the function that evaluates the proposals
  SPS_TRY(loglik_grad_dispatch(ctx, tmp.theta.as<double>(), P, t, tmp.ll.as<double>(), tmp.grad.as<double>()));
  SPS_TRY(factor_proposal(ctx, &tmp, tmp.theta.as<double>(), 1.0, nullptr, sigma, nullptr, flag_ptr(&tmp, 0)));
  SPS_TRY(mala_issue(ctx, &tmp, 0, nullptr, pz, pu, pla, pacc));
  Counters c;
  SPS_TRY(read_counters(ctx, &tmp, &c));
  if (c.chol_bad) return fail(ctx, SPS_ERR_DEGENERATE, "sigma is not positive definite");
  const cudaMemcpyKind k = (mem == SPS_MEM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  SPS_CUDA_TRY(cudaMemcpyAsync(theta, tmp.theta.ptr, pd, k, ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(ll, tmp.ll.ptr, sizeof(double) * P, k, ctx->stream));
  if (mem == SPS_MEM_HOST) {
    if (log_alpha) SPS_CUDA_TRY(cudaMemcpyAsync(log_alpha, pla, sizeof(double) * P, k, ctx->stream));
    if (accepted) SPS_CUDA_TRY(cudaMemcpyAsync(accepted, pacc, sizeof(int) * P, k, ctx->stream));
  }
  SPS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (c.nonfinite) return fail(ctx, SPS_ERR_NONFINITE, "non-finite log-likelihood of a proposal");
  return SPS_OK;
}

}  // extern "C"
