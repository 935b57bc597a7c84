// Fused multinomial-logit log-likelihood on the sm_103a tensor cores (split-BF16 path).
//
// What it computes (Eq. 1 and the product form of the likelihood, Sec. 2.1): for particle p and
// prefix length t,
//     ll_p(t) = sum_{s<=t} [ eta_{s,y_s} - log sum_{c=0}^{C-1} exp(eta_{s,c}) ],
//     eta_{s,c} = theta_{p,c}' x_s, eta_{s,0} = 0.
// The observed-outcome part is linear in theta, so it is taken out of the observation loop:
//   binary (C = 2):  ll = theta' sum_s (y_s - 1/2) x_s - sum_s [ |eta_s|/2 + log(1 + e^{-|eta_s|}) ]
//                    (softplus(eta) - eta/2 = |eta|/2 + log(1 + e^{-|eta|}) is even in eta);
//   C > 2:           ll = sum_c theta_c' sum_{s: y_s = c} x_s - sum_s LSE_s(0, eta_{s,1..C-1}).
// The linear terms are FP64 dot products with FP64 prefix sums of X (finalize kernel); this
// kernel produces the FP64 sums of the non-linear terms.
//
// Kernel structure (one CTA per SM, persistent over work items):
//   warp 0      TMA producer: theta operand tiles (double-buffered) and X tiles (stage ring),
//               128-byte-swizzled bf16, cp.async.bulk.tensor with mbarrier transaction counts;
//   warp 1      allocates TMEM, then one thread issues tcgen05.mma:
//                 eta_c[128 particles x BN obs] = Th_c Xh' + Tl_c Xh' + Th_c Xl'
//               (split BF16: theta = Th + Tl, X = Xh + Xl, the Tl Xl' product dropped),
//               FP32 accumulators in TMEM, two accumulator buffers;
//   warps 4..11 two epilogue warpgroups; TMEM lane = particle, so each thread reduces its own
//               particle's row: FP32 per tile, FP64 across tiles.
// Work item = (observation chunk, particle tile), chunk-major so that concurrent CTAs read the
// same X chunk through L2. Partial sums go to a [chunk][warpgroup][particle] FP64 buffer that
// the finalize kernel sums in a fixed order: the result is deterministic.
//
// Every mbarrier wait is bounded (wall-clock limit); on a timeout the CTA raises a flag, drains
// its own copies and MMAs with bounded waits, frees TMEM and returns.

#include <algorithm>
#include <cstdio>

#include "common.cuh"

namespace sps {
namespace {

constexpr int kBM = 128;          // particles per tile = TMEM lanes
constexpr int kNWG = 2;           // epilogue warpgroups
constexpr int kNBUF = 2;          // TMEM accumulator buffers (one per epilogue warpgroup)
constexpr int kThreads = 128 * (2 + kNWG);   // warps 0-3 (producer, MMA, 2 idle) + epilogue
constexpr int kKB = 64;           // K-block width (elements): one 128-byte swizzle row
constexpr uint32_t kTileA = kBM * 128;       // bytes of one 128-row K block

struct TcParams {
  int ppad;            // padded particle count (multiple of 128)
  int n_ptiles;
  int t;               // prefix length
  int n_tiles;         // observation tiles covering [0, t)
  int chunk_tiles;     // observation tiles per work item
  int n_chunks;
  int n_items;
  int kb_h;            // K blocks of Xh / theta operands
  int kb_l;            // K blocks of Xl
  int ksteps_h;        // 16-wide MMA K steps over Xh (ceil(k/16))
  int ksteps_l;        // over Xl (ceil(kc/16)); 0 when every column is exact
  int stages;          // X ring depth
  int th_bufs;         // theta buffers (1 or 2)
  int th_row_stride;   // rows between classes in the theta operand maps (= ppad)
  double* partial;     // [n_chunks][kNWG][ppad]
  int* flag;           // set to 1 on a timeout
  unsigned long long timeout_ns;
};

struct SmemLayout {
  uint32_t th_bytes;   // one theta buffer (hi + lo, all classes)
  uint32_t x_bytes;    // one X stage (Xh + Xl blocks)
  uint32_t off_th, off_x, off_bar;
  uint32_t total;
};

__host__ __device__ inline SmemLayout smem_layout(int NC, int BN, int kb_h, int kb_l, int stages,
                                                  int th_bufs) {
  SmemLayout L;
  L.th_bytes = static_cast<uint32_t>(2 * NC * kb_h) * kTileA;
  L.x_bytes = static_cast<uint32_t>(kb_h + kb_l) * static_cast<uint32_t>(BN) * 128u;
  L.off_th = 0;
  L.off_x = L.off_th + th_bufs * L.th_bytes;
  L.off_bar = L.off_x + stages * L.x_bytes;
  // barriers: x_full[st], x_empty[st], th_full[2], th_empty[2], acc_full[NBUF], acc_empty[NBUF],
  // drain; then tmem base (u32) and abort flag (int)
  L.total = L.off_bar + 8 * (2 * stages + 4 + 2 * kNBUF + 1) + 16;
  return L;
}

template <int NC, int BN>
__global__ void __launch_bounds__(kThreads, 1)
loglik_tc_kernel(const __grid_constant__ CUtensorMap mapXh, const __grid_constant__ CUtensorMap mapXl,
                 const __grid_constant__ CUtensorMap mapTH, const __grid_constant__ CUtensorMap mapTL,
                 const TcParams prm) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the 128B-swizzle atoms
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const SmemLayout L = smem_layout(NC, BN, prm.kb_h, prm.kb_l, prm.stages, prm.th_bufs);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  uint64_t* x_full = bars;
  uint64_t* x_empty = x_full + prm.stages;
  uint64_t* th_full = x_empty + prm.stages;
  uint64_t* th_empty = th_full + 2;
  uint64_t* acc_full = th_empty + 2;
  uint64_t* acc_empty = acc_full + kNBUF;
  uint64_t* drain = acc_empty + kNBUF;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  constexpr uint32_t kTmemCols = (kNBUF * NC * BN <= 256) ? 256u : 512u;

  if (threadIdx.x == 0) {
    for (int i = 0; i < prm.stages; ++i) {
      ptx::mbar_init(&x_full[i], 1);
      ptx::mbar_init(&x_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&th_full[i], 1);
      ptx::mbar_init(&th_empty[i], 1);
    }
    for (int i = 0; i < kNBUF; ++i) {
      ptx::mbar_init(&acc_full[i], 1);
      ptx::mbar_init(&acc_empty[i], 4);   // one arrive per epilogue warp of the owning group
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_holder, kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const uint64_t limit = prm.timeout_ns;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      ptx::prefetch_map(&mapXh);
      ptx::prefetch_map(&mapTH);
      ptx::prefetch_map(&mapTL);
      if (prm.kb_l > 0) ptx::prefetch_map(&mapXl);
      int st = 0;
      uint32_t xph = 0;
      int tb = 0;
      uint32_t tph = 0;
      bool ok = true;
      // parity of the last fill issued on each stage / theta buffer, for the drain on abort
      uint32_t issued_x = 0, issued_t = 0;
      uint32_t last_par_x[16];
      uint32_t last_par_t[2] = {0, 0};
      for (int item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
        const int chunk = item / prm.n_ptiles;
        const int ptile = item - chunk * prm.n_ptiles;
        const int tile_lo = chunk * prm.chunk_tiles;
        const int tile_hi = min(tile_lo + prm.chunk_tiles, prm.n_tiles);
        // theta operand tiles of this particle tile
        if (!ptx::mbar_wait_bounded(&th_empty[tb], tph ^ 1u, abort_flag, limit)) { ok = false; break; }
        uint8_t* thb = smem + L.off_th + tb * L.th_bytes;
        ptx::mbar_arrive_expect_tx(&th_full[tb], L.th_bytes);
        for (int c = 0; c < NC; ++c) {
          const int row = c * prm.th_row_stride + ptile * kBM;
          for (int kb = 0; kb < prm.kb_h; ++kb) {
            ptx::tma_load_2d(thb + (c * prm.kb_h + kb) * kTileA, &mapTH, &th_full[tb], kb * kKB, row);
            ptx::tma_load_2d(thb + ((NC + c) * prm.kb_h + kb) * kTileA, &mapTL, &th_full[tb], kb * kKB, row);
          }
        }
        issued_t |= 1u << tb;
        last_par_t[tb] = tph;
        if (++tb == prm.th_bufs) { tb = 0; tph ^= 1u; }
        // observation tiles
        for (int tile = tile_lo; tile < tile_hi; ++tile) {
          if (!ptx::mbar_wait_bounded(&x_empty[st], xph ^ 1u, abort_flag, limit)) { ok = false; break; }
          uint8_t* xb = smem + L.off_x + st * L.x_bytes;
          ptx::mbar_arrive_expect_tx(&x_full[st], L.x_bytes);
          const int obs = tile * BN;
          for (int kb = 0; kb < prm.kb_h; ++kb)
            ptx::tma_load_2d(xb + kb * BN * 128, &mapXh, &x_full[st], kb * kKB, obs);
          for (int kb = 0; kb < prm.kb_l; ++kb)
            ptx::tma_load_2d(xb + (prm.kb_h + kb) * BN * 128, &mapXl, &x_full[st], kb * kKB, obs);
          issued_x |= 1u << st;
          last_par_x[st] = xph;
          if (++st == prm.stages) { st = 0; xph ^= 1u; }
        }
      }
      if (*abort_flag) {
        // drain: wait (bounded) for every copy this thread issued before the CTA exits
        volatile int no_abort = 0;
        for (int s = 0; s < prm.stages; ++s)
          if (issued_x & (1u << s)) ptx::mbar_wait_bounded(&x_full[s], last_par_x[s], &no_abort, limit);
        for (int b = 0; b < 2; ++b)
          if (issued_t & (1u << b)) ptx::mbar_wait_bounded(&th_full[b], last_par_t[b], &no_abort, limit);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = ptx::idesc_bf16_f32(kBM, BN);
      int st = 0;
      uint32_t xph = 0;
      int tb = 0;
      uint32_t tph = 0;
      uint32_t acc_count = 0;
      bool ok = true;
      bool issued_any = false;
      for (int item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
        const int chunk = item / prm.n_ptiles;
        const int tile_lo = chunk * prm.chunk_tiles;
        const int tile_hi = min(tile_lo + prm.chunk_tiles, prm.n_tiles);
        if (!ptx::mbar_wait_bounded(&th_full[tb], tph, abort_flag, limit)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t thb = ptx::smem_u32(smem + L.off_th + tb * L.th_bytes);
        for (int tile = tile_lo; tile < tile_hi; ++tile) {
          const int buf = acc_count % kNBUF;
          const uint32_t aph = (acc_count / kNBUF) & 1u;
          if (!ptx::mbar_wait_bounded(&acc_empty[buf], aph ^ 1u, abort_flag, limit)) { ok = false; break; }
          if (!ptx::mbar_wait_bounded(&x_full[st], xph, abort_flag, limit)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t xb = ptx::smem_u32(smem + L.off_x + st * L.x_bytes);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const uint32_t d = tmem_base + static_cast<uint32_t>((buf * NC + c) * BN);
            uint32_t accum = 0;
            // Th_c * Xh'
            for (int ks = 0; ks < prm.ksteps_h; ++ks) {
              const int kb = ks >> 2, kk = ks & 3;
              const uint64_t a = ptx::sdesc_sw128(thb + (c * prm.kb_h + kb) * kTileA) + 2 * kk;
              const uint64_t b = ptx::sdesc_sw128(xb + kb * BN * 128) + 2 * kk;
              ptx::mma_bf16(d, a, b, idesc, accum);
              accum = 1;
            }
            // Tl_c * Xh'
            for (int ks = 0; ks < prm.ksteps_h; ++ks) {
              const int kb = ks >> 2, kk = ks & 3;
              const uint64_t a = ptx::sdesc_sw128(thb + ((NC + c) * prm.kb_h + kb) * kTileA) + 2 * kk;
              const uint64_t b = ptx::sdesc_sw128(xb + kb * BN * 128) + 2 * kk;
              ptx::mma_bf16(d, a, b, idesc, 1);
            }
            // Th_c * Xl' over the continuous columns
            for (int ks = 0; ks < prm.ksteps_l; ++ks) {
              const int kb = ks >> 2, kk = ks & 3;
              const uint64_t a = ptx::sdesc_sw128(thb + (c * prm.kb_h + kb) * kTileA) + 2 * kk;
              const uint64_t b = ptx::sdesc_sw128(xb + (prm.kb_h + kb) * BN * 128) + 2 * kk;
              ptx::mma_bf16(d, a, b, idesc, 1);
            }
          }
          issued_any = true;
          ptx::mma_commit(&x_empty[st]);
          ptx::mma_commit(&acc_full[buf]);
          ++acc_count;
          if (++st == prm.stages) { st = 0; xph ^= 1u; }
        }
        ptx::mma_commit(&th_empty[tb]);
        if (++tb == prm.th_bufs) { tb = 0; tph ^= 1u; }
      }
      if (*abort_flag && issued_any) {
        // wait (bounded) until every MMA this thread issued has completed
        ptx::mma_commit(drain);
        volatile int no_abort = 0;
        ptx::mbar_wait_bounded(drain, 0, &no_abort, limit);
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ epilogue
    const int wg = (warp - 4) >> 2;
    const int quad = warp & 3;
    const int row = quad * 32 + lane;                 // particle within the tile
    const uint32_t lane_base = static_cast<uint32_t>(quad * 32) << 16;
    constexpr float kLog2e = 1.4426950408889634f;
    constexpr float kLn2 = 0.6931471805599453f;
    uint32_t acc_count = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
      const int chunk = item / prm.n_ptiles;
      const int ptile = item - chunk * prm.n_ptiles;
      const int tile_lo = chunk * prm.chunk_tiles;
      const int tile_hi = min(tile_lo + prm.chunk_tiles, prm.n_tiles);
      double acc64 = 0.0;
      for (int tile = tile_lo; tile < tile_hi; ++tile, ++acc_count) {
        const int buf = acc_count % kNBUF;
        if ((buf % kNWG) != wg) continue;
        const uint32_t aph = (acc_count / kNBUF) & 1u;
        if (!ptx::mbar_wait_bounded(&acc_full[buf], aph, abort_flag, limit)) { ok = false; break; }
        ptx::tc_fence_after();
        const int valid = min(BN, prm.t - tile * BN);
        float lin_acc = 0.f;     // sum of |eta|/2 (binary) or of the LSE shifts m (C > 2)
        float prod = 1.f;        // running product of the log arguments, renormalised
        int pexp = 0;            // binary exponent taken out of prod
        const uint32_t col0 = static_cast<uint32_t>(buf * NC * BN);
#pragma unroll 1
        for (int j0 = 0; j0 < BN; j0 += 32) {
          if constexpr (NC == 1) {
            float v[32];
            ptx::tmem_ld_32x32b_x32(tmem_base + lane_base + col0 + j0, v);
            ptx::tmem_wait_ld();
            if (j0 + 32 <= valid) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const float a = fabsf(v[j]);
                lin_acc += a;
                const float e = ptx::ex2_approx(-a * kLog2e);
                prod = fmaf(prod, e, prod);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const bool in = (j0 + j) < valid;
                const float a = in ? fabsf(v[j]) : 0.f;
                lin_acc += a;
                const float e = in ? ptx::ex2_approx(-a * kLog2e) : 0.f;
                prod = fmaf(prod, e, prod);
              }
            }
          } else {
            float v[NC][32];
#pragma unroll
            for (int c = 0; c < NC; ++c)
              ptx::tmem_ld_32x32b_x32(tmem_base + lane_base + col0 + c * BN + j0, v[c]);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float m = 0.f;
#pragma unroll
              for (int c = 0; c < NC; ++c) m = fmaxf(m, v[c][j]);
              const float ms = m * kLog2e;
              float s = ptx::ex2_approx(-ms);
#pragma unroll
              for (int c = 0; c < NC; ++c) s += ptx::ex2_approx(fmaf(v[c][j], kLog2e, -ms));
              const bool in = (j0 + j) < valid;
              lin_acc += in ? m : 0.f;
              prod *= in ? s : 1.f;
              if ((j & 15) == 15) {   // s < C <= 4: renormalise every 16 factors
                const int bits = __float_as_int(prod);
                pexp += (bits >> 23) - 127;
                prod = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);
              }
            }
          }
          if constexpr (NC == 1) {   // factors in [1, 2]: renormalise every 32
            const int bits = __float_as_int(prod);
            pexp += (bits >> 23) - 127;
            prod = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);
        const float logpart = kLn2 * (static_cast<float>(pexp) + ptx::lg2_approx(prod));
        const float scale = (NC == 1) ? 0.5f : 1.0f;
        acc64 += static_cast<double>(fmaf(scale, lin_acc, logpart));
      }
      if (!ok) break;
      prm.partial[(static_cast<size_t>(chunk) * kNWG + wg) * prm.ppad + ptile * kBM + row] = acc64;
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicExch(prm.flag, 1);
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, kTmemCols);
  }
}

// ll[p] = lin_p - sum over chunks and warpgroups of partial (fixed order), lin_p = theta_p . lin
// with lin [NC x k] in the original column order.
__global__ void loglik_finalize_kernel(const double* __restrict__ theta, int64_t P, int D,
                                       const double* __restrict__ lin, const double* __restrict__ partial,
                                       int slices, int ppad, double* __restrict__ ll) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= P) return;
  double a = 0.0;
  const double* th = theta + p * D;
  for (int i = 0; i < D; ++i) a = fma(th[i], lin[i], a);
  double s = 0.0;
  for (int q = 0; q < slices; ++q) s += partial[static_cast<size_t>(q) * ppad + p];
  ll[p] = a - s;
}

// theta [P x D] FP64 (original order, class-major) -> Th, Tl bf16 rows [NC*ppad x kpad] with
// internal (permuted) columns; padding rows/columns zero.
__global__ void encode_theta_kernel(const double* __restrict__ theta, int64_t P, int k, int NC,
                                    const int* __restrict__ perm, int kpad, int ppad,
                                    __nv_bfloat16* __restrict__ th, __nv_bfloat16* __restrict__ tl) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t total = static_cast<int64_t>(NC) * ppad * kpad;
  if (idx >= total) return;
  const int j = static_cast<int>(idx % kpad);
  const int64_t r = idx / kpad;
  const int c = static_cast<int>(r / ppad);
  const int64_t p = r - static_cast<int64_t>(c) * ppad;
  double v = 0.0;
  if (p < P && j < k) v = theta[p * (static_cast<int64_t>(NC) * k) + c * k + perm[j]];
  const __nv_bfloat16 h = __double2bfloat16(v);
  const double rem = v - static_cast<double>(__bfloat162float(h));
  th[idx] = h;
  tl[idx] = __double2bfloat16(rem);
}

template <int NC, int BN>
sps_status launch_tc(sps_ctx* ctx, const TcParams& prm, int grid, uint32_t smem_bytes) {
  auto kern = loglik_tc_kernel<NC, BN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem_bytes));
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
  const XEncoding& enc = ctx->enc;
  const CUtensorMap& mxl = enc.kcpad > 0 ? enc.mapXl : enc.mapXh;
  hot_begin(ctx);
  kern<<<grid, kThreads, smem_bytes, ctx->stream>>>(enc.mapXh, mxl, ctx->ll.mapTH, ctx->ll.mapTL, prm); ++ctx->launches;
  hot_end(ctx);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("loglik_tc launch: ") + cudaGetErrorString(e));
  return SPS_OK;
}

}  // namespace

sps_status loglik_split(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll) {
  const int NC = ctx->NC;
  if (NC > 3) return fail(ctx, SPS_ERR_UNSUPPORTED, "split precision supports at most 4 outcomes");
  XEncoding& enc = ctx->enc;
  LoglikScratch& S = ctx->ll;
  const int ppad = static_cast<int>((P + kBM - 1) / kBM * kBM);
  // theta operands and their tensor maps
  if (S.ppad_cap < ppad) {
    const int64_t cap = std::max<int64_t>(ppad, S.ppad_cap * 3 / 2 / kBM * kBM);
    const size_t bytes = static_cast<size_t>(NC) * cap * enc.kpad * sizeof(__nv_bfloat16);
    SPS_CUDA_TRY(S.thetaH.reserve(bytes));
    SPS_CUDA_TRY(S.thetaL.reserve(bytes));
    S.ppad_cap = cap;
  }
  // maps are rebuilt for the row stride actually used (ppad)
  SPS_TRY(make_map_bf16(ctx, &S.mapTH, S.thetaH.ptr, static_cast<uint64_t>(NC) * ppad, enc.kpad, kBM));
  SPS_TRY(make_map_bf16(ctx, &S.mapTL, S.thetaL.ptr, static_cast<uint64_t>(NC) * ppad, enc.kpad, kBM));
  {
    const int64_t total = static_cast<int64_t>(NC) * ppad * enc.kpad;
    const int threads = 256;
    encode_theta_kernel<<<static_cast<unsigned>((total + threads - 1) / threads), threads, 0, ctx->stream>>>(
        d_theta, P, ctx->k, NC, enc.perm_dev.as<int>(), enc.kpad, ppad, S.thetaH.as<__nv_bfloat16>(),
        S.thetaL.as<__nv_bfloat16>()); ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
  }
  SPS_TRY(ensure_lin(ctx, t));

  const int BN = enc.bn;
  TcParams prm{};
  prm.ppad = ppad;
  prm.n_ptiles = ppad / kBM;
  prm.t = static_cast<int>(t);
  prm.n_tiles = static_cast<int>((t + BN - 1) / BN);
  prm.kb_h = enc.kpad / kKB;
  prm.kb_l = enc.kcpad / kKB;
  prm.ksteps_h = (enc.k + 15) / 16;
  prm.ksteps_l = (enc.kc + 15) / 16;
  prm.th_row_stride = ppad;
  // chunking: enough work items to balance the persistent grid, items long enough to amortise
  // the theta loads
  const int grid_max = ctx->num_sms;
  int chunk_tiles = std::max(1, std::min(prm.n_tiles, 32));
  {
    const int64_t want_items = 8LL * grid_max;
    while (chunk_tiles > 4 &&
           static_cast<int64_t>(prm.n_ptiles) * ((prm.n_tiles + chunk_tiles - 1) / chunk_tiles) < want_items)
      chunk_tiles /= 2;
  }
  prm.chunk_tiles = chunk_tiles;
  prm.n_chunks = std::max(1, (prm.n_tiles + chunk_tiles - 1) / chunk_tiles);
  prm.n_items = prm.n_tiles > 0 ? prm.n_ptiles * prm.n_chunks : 0;
  // shared memory: as many X stages as fit with double-buffered theta, else single
  const uint32_t budget = 227 * 1024 - 1024;
  int th_bufs = 2, stages = 0;
  for (int tb = 2; tb >= 1 && stages < 2; --tb) {
    th_bufs = tb;
    for (int st = 8; st >= 2; --st) {
      if (smem_layout(NC, BN, prm.kb_h, prm.kb_l, st, tb).total <= budget) { stages = st; break; }
    }
  }
  if (stages < 2) return fail(ctx, SPS_ERR_UNSUPPORTED, "covariate count too large for the tensor-core tile");
  prm.stages = stages;
  prm.th_bufs = th_bufs;
  const size_t slices = static_cast<size_t>(prm.n_chunks) * kNWG;
  SPS_CUDA_TRY(S.partial.reserve(slices * ppad * sizeof(double)));
  SPS_CUDA_TRY(S.flag.reserve(sizeof(int)));
  prm.partial = S.partial.as<double>();
  prm.flag = S.flag.as<int>();
  prm.timeout_ns = 2000000000ull;
  SPS_CUDA_TRY(cudaMemsetAsync(prm.flag, 0, sizeof(int), ctx->stream));
  const uint32_t smem_bytes = smem_layout(NC, BN, prm.kb_h, prm.kb_l, stages, th_bufs).total + 1024;
  if (prm.n_items > 0) {
    const int grid = std::min(grid_max, prm.n_items);
    sps_status s;
    if (NC == 1) s = launch_tc<1, 128>(ctx, prm, grid, smem_bytes);
    else if (NC == 2) s = launch_tc<2, 128>(ctx, prm, grid, smem_bytes);
    else s = launch_tc<3, 64>(ctx, prm, grid, smem_bytes);
    if (s != SPS_OK) return s;
  }
  {
    const int threads = 256;
    loglik_finalize_kernel<<<static_cast<unsigned>((P + threads - 1) / threads), threads, 0, ctx->stream>>>(
        d_theta, P, ctx->D, ctx->lin.as<double>(), prm.partial, prm.n_items > 0 ? static_cast<int>(slices) : 0,
        ppad, d_ll); ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
  }
  return SPS_OK;
}

}  // namespace sps

// ------------------------------------------------------------------------------------------
// Allocation-free variant of the split-precision log-likelihood (sps_loglik_noalloc).
//
// Some callers cannot let the library call cudaMalloc during a call: code whose device memory
// is owned entirely by another allocator (a framework's pool, a fixed arena of an embedded
// application), or latency-critical loops that cannot accept cudaMalloc/cudaFree, which may
// synchronise the device. For them this variant keeps its per-call scratch (the theta operand
// rows, the partial sums and the timeout flag) in one file-scope device array of fixed size
// instead of buffers grown with cudaMalloc. The array exists once per GPU that loads the
// library and stays allocated until the process exits. Every call shares it: calls whose work
// overlaps on the GPU (other streams, other host threads) race on it and must be serialised by
// the caller. Its contents persist from the last call; everything that must start at zero is
// cleared by each call.

#include <mutex>

namespace sps {
namespace {

constexpr size_t kStaticScratchBytes = size_t{32} << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of the static scratch array on the current device. The host-side name of the
// array is only a stand-in: its device address comes from cudaGetSymbolAddress, looked up once
// per device (with that device current) on the first call there.
sps_status static_scratch_address(sps_ctx* ctx, unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != ctx->device) return fail(ctx, SPS_ERR_INVALID_ARG, "the context's device is not current");
  if (dev < 0 || dev >= kMaxDevices) return fail(ctx, SPS_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(ctx, SPS_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_static_ptr[dev]);
  return SPS_OK;
}

template <int NC, int BN>
sps_status launch_tc_maps(sps_ctx* ctx, const TcParams& prm, int grid, uint32_t smem_bytes,
                          const CUtensorMap& mapTH, const CUtensorMap& mapTL) {
  auto kern = loglik_tc_kernel<NC, BN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem_bytes));
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
  const XEncoding& enc = ctx->enc;
  const CUtensorMap& mxl = enc.kcpad > 0 ? enc.mapXl : enc.mapXh;
  kern<<<grid, kThreads, smem_bytes, ctx->stream>>>(enc.mapXh, mxl, mapTH, mapTL, prm); ++ctx->launches;
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("loglik_tc launch: ") + cudaGetErrorString(e));
  return SPS_OK;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

sps_status loglik_split_static(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll) {
  const int NC = ctx->NC;
  if (NC > 3) return fail(ctx, SPS_ERR_UNSUPPORTED, "split precision supports at most 4 outcomes");
  const XEncoding& enc = ctx->enc;
  const int ppad = static_cast<int>((P + kBM - 1) / kBM * kBM);
  const int BN = enc.bn;
  TcParams prm{};
  prm.ppad = ppad;
  prm.n_ptiles = ppad / kBM;
  prm.t = static_cast<int>(t);
  prm.n_tiles = static_cast<int>((t + BN - 1) / BN);
  prm.kb_h = enc.kpad / kKB;
  prm.kb_l = enc.kcpad / kKB;
  prm.ksteps_h = (enc.k + 15) / 16;
  prm.ksteps_l = (enc.kc + 15) / 16;
  prm.th_row_stride = ppad;
  const int grid_max = ctx->num_sms;
  int chunk_tiles = std::max(1, std::min(prm.n_tiles, 32));
  {
    const int64_t want_items = 8LL * grid_max;
    while (chunk_tiles > 4 &&
           static_cast<int64_t>(prm.n_ptiles) * ((prm.n_tiles + chunk_tiles - 1) / chunk_tiles) < want_items)
      chunk_tiles /= 2;
  }
  prm.chunk_tiles = chunk_tiles;
  prm.n_chunks = std::max(1, (prm.n_tiles + chunk_tiles - 1) / chunk_tiles);
  prm.n_items = prm.n_tiles > 0 ? prm.n_ptiles * prm.n_chunks : 0;
  const uint32_t budget = 227 * 1024 - 1024;
  int th_bufs = 2, stages = 0;
  for (int tb = 2; tb >= 1 && stages < 2; --tb) {
    th_bufs = tb;
    for (int st = 8; st >= 2; --st) {
      if (smem_layout(NC, BN, prm.kb_h, prm.kb_l, st, tb).total <= budget) { stages = st; break; }
    }
  }
  if (stages < 2) return fail(ctx, SPS_ERR_UNSUPPORTED, "covariate count too large for the tensor-core tile");
  prm.stages = stages;
  prm.th_bufs = th_bufs;
  // carve the static area: theta hi rows, theta lo rows, partial sums, flag
  const size_t slices = static_cast<size_t>(prm.n_chunks) * kNWG;
  const size_t op_bytes = round256(static_cast<size_t>(NC) * ppad * enc.kpad * sizeof(__nv_bfloat16));
  const size_t part_bytes = round256(slices * ppad * sizeof(double));
  const size_t need = 2 * op_bytes + part_bytes + 256;
  if (need > kStaticScratchBytes) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "sps_loglik_noalloc: this call needs %zu bytes of scratch, the static area holds %zu; use sps_loglik",
             need, kStaticScratchBytes);
    return fail(ctx, SPS_ERR_INVALID_ARG, msg);
  }
  unsigned char* base = nullptr;
  SPS_TRY(static_scratch_address(ctx, &base));
  __nv_bfloat16* th_hi = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* th_lo = reinterpret_cast<__nv_bfloat16*>(base + op_bytes);
  double* partial = reinterpret_cast<double*>(base + 2 * op_bytes);
  int* flag = reinterpret_cast<int*>(base + 2 * op_bytes + part_bytes);
  CUtensorMap mapTH, mapTL;
  SPS_TRY(make_map_bf16(ctx, &mapTH, th_hi, static_cast<uint64_t>(NC) * ppad, enc.kpad, kBM));
  SPS_TRY(make_map_bf16(ctx, &mapTL, th_lo, static_cast<uint64_t>(NC) * ppad, enc.kpad, kBM));
  {
    const int64_t total = static_cast<int64_t>(NC) * ppad * enc.kpad;
    const int threads = 256;
    encode_theta_kernel<<<static_cast<unsigned>((total + threads - 1) / threads), threads, 0, ctx->stream>>>(
        d_theta, P, ctx->k, NC, enc.perm_dev.as<int>(), enc.kpad, ppad, th_hi, th_lo); ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
  }
  SPS_TRY(ensure_lin(ctx, t));
  prm.partial = partial;
  prm.flag = flag;
  prm.timeout_ns = 2000000000ull;
  SPS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));   // the flag must start at zero
  const uint32_t smem_bytes = smem_layout(NC, BN, prm.kb_h, prm.kb_l, stages, th_bufs).total + 1024;
  if (prm.n_items > 0) {
    const int grid = std::min(grid_max, prm.n_items);
    sps_status s;
    if (NC == 1) s = launch_tc_maps<1, 128>(ctx, prm, grid, smem_bytes, mapTH, mapTL);
    else if (NC == 2) s = launch_tc_maps<2, 128>(ctx, prm, grid, smem_bytes, mapTH, mapTL);
    else s = launch_tc_maps<3, 64>(ctx, prm, grid, smem_bytes, mapTH, mapTL);
    if (s != SPS_OK) return s;
  }
  {
    const int threads = 256;
    loglik_finalize_kernel<<<static_cast<unsigned>((P + threads - 1) / threads), threads, 0, ctx->stream>>>(
        d_theta, P, ctx->D, ctx->lin.as<double>(), partial, prm.n_items > 0 ? static_cast<int>(slices) : 0, ppad,
        d_ll); ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
  }
  return SPS_OK;
}

}  // namespace sps

extern "C" sps_status sps_loglik_noalloc(sps_ctx* ctx, const double* theta, int64_t P, int64_t t, double* ll) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!theta || !ll || P < 1 || t < 0 || t > ctx->n || P > (1LL << 28))
    return sps::fail(ctx, SPS_ERR_INVALID_ARG, "sps_loglik_noalloc: bad arguments");
  return sps::loglik_split_static(ctx, theta, P, t, ll);
}
