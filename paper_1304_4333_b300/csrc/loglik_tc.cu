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
// kernel produces the FP64 sums of the non-linear terms. Theta enters the tensor cores scaled by
// log2(e), so the accumulators hold u = eta log2(e) and each exponential is one ex2. Logarithms
// are taken once per tile, of running products of the (1 + 2^{-|u|}) factors (binary: four
// chains, at most 32 factors in [1, 2] each, no rescaling needed; packed FP32x2 adds and FMAs)
// or of the shifted sums of exponentials (C > 2: four chains whose binary exponents are moved to
// an integer as they grow).
//
// Operands (128-byte-swizzled BF16, K blocks of 64 elements): an X row holds [Xh | Xl] with
// Xh = bf16(x) over k16 columns and Xl = bf16(x - Xh) over the kc16 continuous columns; a theta
// row holds [Th | Tl] of theta log2(e) over k16 columns. Per tile and class the MMA warp issues
//     u_c[128 particles x BN obs] = Th_c Xh' + Tl_c Xh' + Th_c Xl'
// (the Tl Xl' product, relative size 2^-16, is dropped).
//
// Kernel structure (one CTA per SM, persistent over work items):
//   warp 0      TMA producer: theta tiles (double-buffered when they fit) and X tiles (stage
//               ring), cp.async.bulk.tensor with mbarrier transaction counts;
//   warp 1      allocates TMEM, then one thread issues tcgen05.mma into the TMEM accumulators;
//   warps 2..   epilogue groups of four warps; warp w reads TMEM lane quadrant w % 4, so a
//               group covers the 128 lanes (lane = particle). C = 2: four groups, two per
//               accumulator, each taking half of its columns; C > 2: two groups, each owning
//               whole accumulators; a group visits only the tiles of its accumulator. Each
//               thread reduces its own particle's row: FP32 within a tile, FP32 with Kahan
//               compensation across the tiles of a work item, FP64 across work items.
// Work item = (observation chunk, group of CL particle tiles), chunk-major so that concurrent
// CTAs read the same X chunk through L2. With CL = 2 the two CTAs of a cluster form a tensor-core
// pair: the even CTA issues cta_group::2 MMAs of 256 particles (each CTA's 128 particles in its
// own shared and tensor memory) x BN observations, each CTA loading and holding only BN / 2 rows
// of every X tile. Per observation processed, a CTA then receives half the X bytes of a single
// CTA, and the pipeline holds twice the MMA time per stage. Every TMA copy completes on a barrier
// of its own CTA; the odd CTA's MMA warp relays each of its landed X stages and theta buffers to
// the even CTA as the second arrive on the even CTA's full barrier of the same index, so that the
// MMA thread waits once per stage (each wait of the MMA-issuing thread is a shared-memory access
// that queues behind the MMAs' own operand reads and stalls the tensor pipe). The MMA completions
// arrive on both CTAs' barriers, and both CTAs' epilogue warps release accumulators on the even
// CTA's barrier. (On a timeout the even CTA's producer drains its copies through those two-arrive
// barriers: if the relay stopped first, that wait runs to its limit, far beyond any copy's
// latency, before the CTA leaves.)
// Partial sums go to a [chunk][group][particle] FP64 buffer that the finalize kernel sums in a
// fixed order: the result is deterministic.
//
// Every mbarrier wait is bounded (wall-clock limit); on a timeout the CTA raises a flag, drains
// its own copies and MMAs with bounded waits, frees TMEM and returns (a stalled peer makes the
// other CTA of its pair time out as well; both meet at the cluster barriers before and after the
// pair's TMEM is freed). Warps
// reconverge before every .sync.aligned tcgen05 instruction, and the producer waits for every
// stage it filled to be released before the CTA exits, so no asynchronous arrive is still in
// flight at exit.

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace sps {
namespace {

constexpr int kBM = 128;                        // particles per tile = TMEM lanes
// TMEM accumulators of NC x BN columns: as many as the 512 columns hold, at most four.
__host__ __device__ constexpr int nbuf_for(int NC, int BN) {
  return (512 / (NC * BN)) >= 4 ? 4 : 512 / (NC * BN);
}
// Epilogue groups of four warps (warp w reads TMEM lane quadrant w % 4): four, each owning one
// accumulator or a share of one's columns (C > 2 reads 16 columns of each class at a time, so
// that four groups fit the registers; four outcomes, k = 50: 6.42 -> 6.23 ms per launch against
// two groups of 32-column reads).
__host__ __device__ constexpr int nwg_for(int) { return 4; }
__host__ __device__ constexpr int threads_for(int NC) { return 32 * (2 + 4 * nwg_for(NC)); }
constexpr int kKB = 64;                         // K-block width (elements): one 128-byte swizzle row
constexpr uint32_t kTileA = kBM * 128;          // bytes of one 128-row K block

struct TcParams {
  int ppad;            // padded particle count (multiple of 128 x cluster size)
  int n_ptiles;
  int n_pgroups;       // n_ptiles / cluster size
  int t;               // prefix length
  int n_tiles;         // observation tiles covering [0, t)
  int chunk_tiles;     // observation tiles per work item
  int n_chunks;
  int n_items;
  int kbx;             // K blocks of an X row
  int kbt;             // K blocks of a theta row
  int k16;             // element offset of the low parts in both rows
  int ksh;             // 16-wide MMA K steps over Xh (k16 / 16)
  int ksl;             // over Xl (kc16 / 16); 0 when every column is exact
  int stages;          // X ring depth
  int th_bufs;         // theta buffers (1 or 2)
  int th_row_stride;   // rows between classes in the theta operand map (= ppad)
  double* partial;     // [n_chunks][nwg][ppad]
  int* flag;           // set to 1 on a timeout
  unsigned long long timeout_ns;
  int stall;           // diagnostics: non-zero makes the TMA producer issue no copy
  // batched models: per particle tile {prefix length, model slot}, or null; per model slot its X
  // tensor map (the model's own encoding of its first k_m covariates), K blocks and MMA slices
  const int2* ptile_info;
  const BatchModel* bmodels;
};

// Observation tiles [tile_lo, result) of a work item: its chunk cut at the prefix length of its
// particle tile (an empty range when the chunk starts beyond it).
template <int BN, bool BATCH>
__device__ __forceinline__ int item_tile_hi(const TcParams& prm, int tile_lo, int ptile) {
  if constexpr (BATCH)
    return max(tile_lo, min(tile_lo + prm.chunk_tiles, (prm.ptile_info[ptile].x + BN - 1) / BN));
  else
    return min(tile_lo + prm.chunk_tiles, prm.n_tiles);
}

struct SmemLayout {
  uint32_t th_bytes;   // one theta buffer (all classes)
  uint32_t x_bytes;    // one X stage (this CTA's rows of a tile)
  uint32_t off_th, off_x, off_bar;
  uint32_t total;
};

// CL = 2: a CTA pair; each CTA holds BN / 2 rows of every X tile.
__host__ __device__ inline SmemLayout smem_layout(int NC, int BN, int CL, int kbx, int kbt, int stages,
                                                  int th_bufs) {
  SmemLayout L;
  L.th_bytes = static_cast<uint32_t>(NC * kbt) * kTileA;
  L.x_bytes = static_cast<uint32_t>(kbx) * static_cast<uint32_t>(BN / CL) * 128u;
  L.off_th = 0;
  L.off_x = L.off_th + th_bufs * L.th_bytes;
  L.off_bar = L.off_x + stages * L.x_bytes;
  // barriers: x_full[st], x_empty[st], th_full[2], th_empty[2], acc_full[NBUF], acc_empty[NBUF],
  // drain; then tmem base (u32) and abort flag (int)
  L.total = L.off_bar + 8 * (2 * stages + 4 + 2 * nbuf_for(NC, BN) + 1) + 16;
  return L;
}

constexpr uint32_t kSmemBudget = 227 * 1024 - 1024;

// Pipeline depth for a tile shape: double-buffered theta (no bubble when a CTA moves to its
// next particle tile) if at least 4 X stages still fit, else single-buffered theta with as many
// stages as fit (c3: 8 stages single-buffered 8.5 ms, 2 stages double-buffered 16.0 ms); false
// when fewer than 2 stages fit.
bool pick_stages(int NC, int BN, int CL, int kbx, int kbt, int* stages, int* th_bufs) {
  for (int tb = 2; tb >= 1; --tb) {
    int st = 0;
    for (int s = 8; s >= 2; --s)
      if (smem_layout(NC, BN, CL, kbx, kbt, s, tb).total <= kSmemBudget) { st = s; break; }
    if (st >= 4 || (tb == 1 && st >= 2)) {
      *stages = st;
      *th_bufs = tb;
      return true;
    }
  }
  return false;
}

// Offset, in the 16-byte units of a descriptor's start address, of the 16-element K slice
// starting at element `e` of an operand tile made of 64-element K blocks of `rows` rows each:
// the descriptor of the slice is the tile's descriptor plus this offset (shared-memory addresses
// stay below 2^18, so the start-address field does not overflow).
__device__ __forceinline__ uint64_t kslice_off(int rows, int e) {
  return static_cast<uint64_t>((e >> 6) * rows * 8 + ((e & 63) >> 3));
}

// BATCH: particle tiles of several nested models; a separate instance so that the single-model
// issue loop stays minimal.
// CL = 1: one CTA per work item (cta_group::1 MMAs of 128 particles x BN observations).
// CL = 2: a CTA pair per work item. The even CTA issues cta_group::2 MMAs of 256 particles
// (128 in each CTA's shared memory and tensor memory) x BN observations, each CTA holding BN / 2
// rows of every X tile; each CTA's TMA copies complete on its own barriers, and the odd CTA's
// MMA warp relays each completed stage and theta buffer to the even CTA with a remote arrive on
// the even CTA's full barrier of that stage (which counts two arrives), so that the MMA thread
// waits once per stage.
// The MMA completions arrive on both CTAs' barriers (commit multicast), and both CTAs' epilogue
// warps release an accumulator on the even CTA's barrier.
template <int NC, int BN, int CL, bool BATCH>
__global__ void __launch_bounds__(threads_for(NC), 1)
loglik_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapT,
                 const TcParams prm) {
  static_assert(CL == 1 || CL == 2, "one CTA or a CTA pair");
  constexpr int HR = BN / CL;                     // X rows of a tile held by this CTA
  constexpr uint16_t kPair = 3u;                  // both CTAs of the pair
  constexpr int NBUF = nbuf_for(NC, BN);
  constexpr int NWG = nwg_for(NC);
  static_assert(NWG % NBUF == 0 || NBUF % NWG == 0, "groups and accumulators");
  // Groups own whole accumulators, or GPB groups share one by columns. (Sharing every tile among
  // all groups shortens the turnaround but makes all warps convoy on each tile: slower.)
  constexpr int GPB = (NWG >= NBUF) ? NWG / NBUF : 1;   // groups per accumulator
  constexpr int COLS = BN / GPB;                  // columns of a tile per group
  static_assert(NBUF * NC * BN <= 512, "TMEM has 512 columns");
  constexpr uint32_t kTmemCols = (NBUF * NC * BN <= 256) ? 256u : 512u;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the 128B-swizzle atoms
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const SmemLayout L = smem_layout(NC, BN, CL, prm.kbx, prm.kbt, prm.stages, prm.th_bufs);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  uint64_t* x_full = bars;                        // even CTA of a pair: also the odd CTA's relay
  uint64_t* x_empty = x_full + prm.stages;
  uint64_t* th_full = x_empty + prm.stages;        // even CTA of a pair: also the odd CTA's relay
  uint64_t* th_empty = th_full + 2;
  uint64_t* acc_full = th_empty + 2;
  uint64_t* acc_empty = acc_full + NBUF;
  uint64_t* drain = acc_empty + NBUF;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int rank = (CL > 1) ? static_cast<int>(ptx::cluster_ctarank()) : 0;
  const int cluster_id = blockIdx.x / CL;
  const int n_clusters = gridDim.x / CL;

  if (threadIdx.x == 0) {
    // the even CTA of a pair counts its own producer's arrive and the odd CTA's relay on its full
    // barriers, so that one wait covers the stage (or theta buffer) in both CTAs
    const uint32_t fulls = (CL > 1 && rank == 0) ? 2u : 1u;
    for (int i = 0; i < prm.stages; ++i) {
      ptx::mbar_init(&x_full[i], fulls);
      ptx::mbar_init(&x_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&th_full[i], fulls);
      ptx::mbar_init(&th_empty[i], 1);
    }
    for (int i = 0; i < NBUF; ++i) {
      ptx::mbar_init(&acc_full[i], 1);
      ptx::mbar_init(&acc_empty[i], 4 * GPB * CL);   // one arrive per warp of the owning groups
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (CL > 1) {
      ptx::tmem_alloc_pair(tmem_holder, kTmemCols);
      ptx::tmem_relinquish_pair();
    } else {
      ptx::tmem_alloc(tmem_holder, kTmemCols);
      ptx::tmem_relinquish();
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  // the peer's arrives and MMA completions target this CTA's barriers: both must be initialised
  if constexpr (CL > 1) ptx::cluster_sync();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const uint64_t limit = prm.timeout_ns;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      ptx::prefetch_map(&mapX);
      ptx::prefetch_map(&mapT);
      int st = 0;
      uint32_t xph = 0;
      int tb = 0;
      uint32_t tph = 0;
      bool ok = (prm.stall == 0);   // diagnostics: a stalled producer issues no copy at all
      // bit s: stage / theta buffer s was filled; parity of its last fill
      uint32_t issued_x = 0, issued_t = 0, par_x = 0, par_t = 0;
      for (int item = cluster_id; ok && item < prm.n_items; item += n_clusters) {
        const int chunk = item / prm.n_pgroups;
        const int ptile = (item - chunk * prm.n_pgroups) * CL + rank;
        const int tile_lo = chunk * prm.chunk_tiles;
        const int tile_hi = item_tile_hi<BN, BATCH>(prm, tile_lo, ptile);
        if (BATCH && tile_hi == tile_lo) continue;   // nothing of this item lies inside its prefix
        // the X tiles of this item: the launch's map, or (batched models) the item's model's own
        const CUtensorMap* mx = &mapX;
        int kbx = prm.kbx;
        if constexpr (BATCH) {
          const BatchModel* bm = prm.bmodels + prm.ptile_info[ptile].y;
          mx = &bm->mapX;
          kbx = bm->kbx;
        }
        if (!ptx::mbar_wait_bounded(&th_empty[tb], tph ^ 1u, abort_flag, limit)) { ok = false; break; }
        uint8_t* thb = smem + L.off_th + tb * L.th_bytes;
        ptx::mbar_arrive_expect_tx(&th_full[tb], L.th_bytes);
        for (int c = 0; c < NC; ++c) {
          const int row = c * prm.th_row_stride + ptile * kBM;
          for (int kb = 0; kb < prm.kbt; ++kb)
            ptx::tma_load_2d(thb + (c * prm.kbt + kb) * kTileA, &mapT, &th_full[tb], kb * kKB, row);
        }
        issued_t |= 1u << tb;
        par_t = (par_t & ~(1u << tb)) | (tph << tb);
        if (++tb == prm.th_bufs) { tb = 0; tph ^= 1u; }
        const uint32_t x_bytes = static_cast<uint32_t>(kbx) * HR * 128u;   // this CTA's rows of a tile
        for (int tile = tile_lo; tile < tile_hi; ++tile) {
          if (!ptx::mbar_wait_bounded(&x_empty[st], xph ^ 1u, abort_flag, limit)) { ok = false; break; }
          uint8_t* xb = smem + L.off_x + st * L.x_bytes;
          ptx::mbar_arrive_expect_tx(&x_full[st], x_bytes);
          const int obs = tile * BN + rank * HR;
          for (int kb = 0; kb < kbx; ++kb)
            ptx::tma_load_2d(xb + kb * HR * 128, mx, &x_full[st], kb * kKB, obs);
          issued_x |= 1u << st;
          par_x = (par_x & ~(1u << st)) | (xph << st);
          if (++st == prm.stages) { st = 0; xph ^= 1u; }
        }
      }
      if (*abort_flag) {
        // drain: wait (bounded) for every copy this thread issued before the CTA exits
        volatile int no_abort = 0;
        for (int s = 0; s < prm.stages; ++s)
          if (issued_x & (1u << s)) ptx::mbar_wait_bounded(&x_full[s], (par_x >> s) & 1u, &no_abort, limit);
        for (int b = 0; b < 2; ++b)
          if (issued_t & (1u << b)) ptx::mbar_wait_bounded(&th_full[b], (par_t >> b) & 1u, &no_abort, limit);
      } else {
        // tail: stages are released by asynchronous tcgen05.commit arrives; wait until every
        // stage and theta buffer filled here has been released
        for (int s = 0; s < prm.stages; ++s)
          if (issued_x & (1u << s)) ptx::mbar_wait_bounded(&x_empty[s], (par_x >> s) & 1u, abort_flag, limit);
        for (int b = 0; b < 2; ++b)
          if (issued_t & (1u << b)) ptx::mbar_wait_bounded(&th_empty[b], (par_t >> b) & 1u, abort_flag, limit);
      }
    }
  } else if (warp == 1 && CL > 1 && rank != 0) {
    // ------------------------------------------------------------------ relay (odd CTA of a pair)
    // each landed theta buffer and X stage of this CTA is announced by an arrive on the even
    // CTA's th_full / x_full barrier of the same index, in the order the MMA thread consumes them
    if (lane == 0) {
      const uint32_t r_th_peer = ptx::cluster_addr(th_full, 0);
      const uint32_t r_x_peer = ptx::cluster_addr(x_full, 0);
      int st = 0, tb = 0;
      uint32_t xph = 0, tph = 0;
      bool ok = true;
      for (int item = cluster_id; ok && item < prm.n_items; item += n_clusters) {
        const int chunk = item / prm.n_pgroups;
        const int ptile = (item - chunk * prm.n_pgroups) * CL + rank;
        const int tile_lo = chunk * prm.chunk_tiles;
        const int tile_hi = item_tile_hi<BN, BATCH>(prm, tile_lo, ptile);
        if (BATCH && tile_hi == tile_lo) continue;
        if (!ptx::mbar_wait_bounded_cluster(&th_full[tb], tph, abort_flag, limit)) { ok = false; break; }
        ptx::mbar_arrive_remote(r_th_peer + 8u * static_cast<uint32_t>(tb));
        if (++tb == prm.th_bufs) { tb = 0; tph ^= 1u; }
        for (int tile = tile_lo; tile < tile_hi; ++tile) {
          if (!ptx::mbar_wait_bounded_cluster(&x_full[st], xph, abort_flag, limit)) { ok = false; break; }
          ptx::mbar_arrive_remote(r_x_peer + 8u * static_cast<uint32_t>(st));
          if (++st == prm.stages) { st = 0; xph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    // The whole warp runs the loop, so that the descriptors and counters are warp-uniform values;
    // lane 0 issues the MMAs and commits. (Measured against one thread running it: 4.8 % less
    // time per c4 launch, 4 % per c2 launch.)
    {
      const uint32_t issue = (lane == 0) ? 1u : 0u;
      const uint32_t idesc = ptx::idesc_bf16_f32(kBM * CL, BN);
      int st = 0;
      uint32_t xph = 0;
      int tb = 0;
      uint32_t tph = 0;
      uint32_t acc_count = 0;
      bool ok = true;
      bool issued_any = false;
      for (int item = cluster_id; ok && item < prm.n_items; item += n_clusters) {
        const int chunk = item / prm.n_pgroups;
        const int ptile = (item - chunk * prm.n_pgroups) * CL + rank;
        const int tile_lo = chunk * prm.chunk_tiles;
        const int tile_hi = item_tile_hi<BN, BATCH>(prm, tile_lo, ptile);
        if (BATCH && tile_hi == tile_lo) continue;
        // the MMA slices of this item's rows: the launch's, or (batched models) those of the
        // item's model's own encoding
        int ksh = prm.ksh, ksl = prm.ksl, k16 = prm.k16;
        if constexpr (BATCH) {
          const BatchModel* bm = prm.bmodels + prm.ptile_info[ptile].y;
          ksh = bm->ksh;
          ksl = bm->ksl;
          k16 = bm->k16;
        }
        if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded_cluster(&th_full[tb], tph, abort_flag, limit))) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t thb = ptx::smem_u32(smem + L.off_th + tb * L.th_bytes);
        for (int tile = tile_lo; tile < tile_hi; ++tile) {
          const int buf = acc_count % NBUF;
          const uint32_t aph = (acc_count / NBUF) & 1u;
          if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded_cluster(&acc_empty[buf], aph ^ 1u, abort_flag, limit))) {
            ok = false;
            break;
          }
          if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded_cluster(&x_full[st], xph, abort_flag, limit))) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint64_t dx = ptx::sdesc_sw128(ptx::smem_u32(smem + L.off_x + st * L.x_bytes));
          // the NC classes accumulate into independent TMEM accumulators: issuing each K slice
          // for all classes before the next keeps NC dependent MMA chains in flight
          uint32_t d[NC];
          uint64_t dt[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            d[c] = tmem_base + static_cast<uint32_t>((buf * NC + c) * BN);
            dt[c] = ptx::sdesc_sw128(thb + static_cast<uint32_t>(c * prm.kbt) * kTileA);
          }
          auto mma = [&](int c, uint64_t ka, uint64_t kb, uint32_t acc) {
            if constexpr (CL > 1) ptx::mma_bf16_pair_if(issue, d[c], dt[c] + ka, dx + kb, idesc, acc);
            else ptx::mma_bf16_if(issue, d[c], dt[c] + ka, dx + kb, idesc, acc);
          };
          for (int i = 0; i < ksh; ++i) {   // Th_c Xh'
            const uint64_t ka = kslice_off(kBM, 16 * i), kb = kslice_off(HR, 16 * i);
#pragma unroll
            for (int c = 0; c < NC; ++c) mma(c, ka, kb, i > 0);
          }
          for (int i = 0; i < ksh; ++i) {   // Tl_c Xh'
            const uint64_t ka = kslice_off(kBM, k16 + 16 * i), kb = kslice_off(HR, 16 * i);
#pragma unroll
            for (int c = 0; c < NC; ++c) mma(c, ka, kb, 1);
          }
          for (int i = 0; i < ksl; ++i) {   // Th_c Xl' over the continuous columns
            const uint64_t ka = kslice_off(kBM, 16 * i), kb = kslice_off(HR, k16 + 16 * i);
#pragma unroll
            for (int c = 0; c < NC; ++c) mma(c, ka, kb, 1);
          }
          issued_any = true;
          if constexpr (CL > 1) {
            ptx::mma_commit_pair_if(issue, &x_empty[st], kPair);
            ptx::mma_commit_pair_if(issue, &acc_full[buf], kPair);
          } else {
            ptx::mma_commit_if(issue, &x_empty[st]);
            ptx::mma_commit_if(issue, &acc_full[buf]);
          }
          ++acc_count;
          if (++st == prm.stages) { st = 0; xph ^= 1u; }
        }
        if constexpr (CL > 1) ptx::mma_commit_pair_if(issue, &th_empty[tb], kPair);
        else ptx::mma_commit_if(issue, &th_empty[tb]);
        if (++tb == prm.th_bufs) { tb = 0; tph ^= 1u; }
      }
      if (*abort_flag && issued_any) {
        if constexpr (CL > 1) ptx::mma_commit_pair_if(issue, drain, 1u);
        else ptx::mma_commit_if(issue, drain);
        volatile int no_abort = 0;
        ptx::mbar_wait_bounded(drain, 0, &no_abort, limit);
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int wg = (warp - 2) >> 2;
    // With at least as many groups as accumulators, GPB groups share accumulator wg / GPB by
    // columns and take every NBUF-th tile; otherwise group wg owns the accumulators b with
    // b % NWG == wg and takes every NWG-th tile.
    constexpr int STEP = (NWG >= NBUF) ? NBUF : NWG;
    const int own = (NWG >= NBUF) ? wg / GPB : wg;     // tiles with acc_count % STEP == own
    const int col0 = (NWG >= NBUF) ? (wg % GPB) * COLS : 0;   // first column of this group
    const int quad = warp & 3;
    const int row = quad * 32 + lane;                 // particle within the tile
    const uint32_t lane_base = static_cast<uint32_t>(quad * 32) << 16;
    // the accumulator release goes to the MMA-issuing CTA (this CTA when alone)
    const uint32_t r_acc_empty = (CL > 1) ? ptx::cluster_addr(acc_empty, 0) : 0u;
    constexpr float kLn2 = 0.6931471805599453f;
    constexpr int NCH = COLS / 32;                    // 32-column chunks per group and tile
    uint32_t acc_base = 0;                            // accumulator uses before this item
    bool ok = true;
    for (int item = cluster_id; ok && item < prm.n_items; item += n_clusters) {
      const int chunk = item / prm.n_pgroups;
      const int ptile = (item - chunk * prm.n_pgroups) * CL + rank;
      const int tile_lo = chunk * prm.chunk_tiles;
      const int tile_hi = item_tile_hi<BN, BATCH>(prm, tile_lo, ptile);
      int t_item = prm.t;
      if constexpr (BATCH) t_item = prm.ptile_info[ptile].x;
      // FP32 sum of this item's tiles with Kahan compensation (converted to FP64 once per item)
      float ksum = 0.f, kcomp = 0.f;
      const int first = tile_lo + static_cast<int>((static_cast<uint32_t>(own) + STEP - acc_base % STEP) % STEP);
      for (int tile = first; tile < tile_hi; tile += STEP) {
        const uint32_t acc_count = acc_base + static_cast<uint32_t>(tile - tile_lo);
        const int buf = static_cast<int>(acc_count % NBUF);
        const uint32_t aph = (acc_count / NBUF) & 1u;
        // every lane waits; the vote reconverges the warp before the .sync.aligned TMEM loads
        ok = __all_sync(0xffffffffu, ptx::mbar_wait_bounded(&acc_full[buf], aph, abort_flag, limit));
        if (!ok) break;
        ptx::tc_fence_after();
        const int valid = t_item - tile * BN - col0;   // columns of this group inside [0, t)
        const bool whole = valid >= COLS;
        const uint32_t tbase = tmem_base + lane_base + static_cast<uint32_t>(buf * NC * BN + col0);
        auto release = [&]() {
          // this group's columns are in registers: release its share of the accumulator
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if constexpr (CL > 1) ptx::mbar_arrive_remote(r_acc_empty + 8u * static_cast<uint32_t>(buf));
            else ptx::mbar_arrive(&acc_empty[buf]);
          }
        };
        float tile_val;                               // this tile's non-linear sum in log2 units
        if constexpr (NC == 1) {
          // four chains as two packed pairs (one FP32x2 add and one FP32x2 FMA per two terms):
          // sums of |u| and products of the factors 1 + 2^-|u| in [1, 2]
          float2 la = make_float2(0.f, 0.f), lb = make_float2(0.f, 0.f);
          float2 pa = make_float2(1.f, 1.f), pb = make_float2(1.f, 1.f);
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) {
            float v[32];
            ptx::tmem_ld_32x32b_x32(tbase + ch * 32, v);
            ptx::tmem_wait_ld();
            if (ch == NCH - 1) release();
            if (whole) {
#pragma unroll
              for (int j = 0; j < 32; j += 4) {
                const float a0 = fabsf(v[j]), a1 = fabsf(v[j + 1]), a2 = fabsf(v[j + 2]), a3 = fabsf(v[j + 3]);
                la = __fadd2_rn(la, make_float2(a0, a1));
                lb = __fadd2_rn(lb, make_float2(a2, a3));
                pa = __ffma2_rn(pa, make_float2(ptx::ex2_approx(-a0), ptx::ex2_approx(-a1)), pa);
                pb = __ffma2_rn(pb, make_float2(ptx::ex2_approx(-a2), ptx::ex2_approx(-a3)), pb);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 32; j += 4) {
                float a[4], e[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const bool in = (ch * 32 + j + q) < valid;
                  a[q] = in ? fabsf(v[j + q]) : 0.f;
                  e[q] = in ? ptx::ex2_approx(-a[q]) : 0.f;
                }
                la = __fadd2_rn(la, make_float2(a[0], a[1]));
                lb = __fadd2_rn(lb, make_float2(a[2], a[3]));
                pa = __ffma2_rn(pa, make_float2(e[0], e[1]), pa);
                pb = __ffma2_rn(pb, make_float2(e[2], e[3]), pb);
              }
            }
          }
          // at most COLS / 4 <= 32 factors in [1, 2] per chain, so each pair's product is at
          // most 2^64: no overflow within a tile
          static_assert(COLS <= 128, "product chains must not overflow");
          const float lsum = (la.x + la.y) + (lb.x + lb.y);
          tile_val = fmaf(0.5f, lsum, ptx::lg2_approx(pa.x * pa.y) + ptx::lg2_approx(pb.x * pb.y));
        } else {
          // four chains: sums of the shifts m and products of the sums 1 + sum_c 2^u_c (or, for
          // a chunk where that overflows, of the shifted sums, < NC + 1 <= 4 each), binary
          // exponents moved to an integer after every 16-column read
          float la[4] = {0.f, 0.f, 0.f, 0.f};
          float pr[4] = {1.f, 1.f, 1.f, 1.f};
          int pexp = 0;
          auto renorm = [&]() {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int bits = __float_as_int(pr[q]);
              pexp += (bits >> 23) - 127;
              pr[q] = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);
            }
          };
          constexpr int NCH16 = COLS / 16;
#pragma unroll 1
          for (int ch = 0; ch < NCH16; ++ch) {
            float v[NC][16];
#pragma unroll
            for (int c = 0; c < NC; ++c) ptx::tmem_ld_32x32b_x16(tbase + c * BN + ch * 16, v[c]);
            ptx::tmem_wait_ld();
            if (ch == NCH16 - 1) release();
            const int j0 = ch * 16;
            const int lim = whole ? 16 : valid - j0;   // columns of this chunk inside [0, t)
            // direct form: sx = 1 + sum_c 2^u_c, no shift, while no factor or product overflows
            // (|u| below about 30 for every particle near the posterior); the product chains
            // start each chunk in [1, 2), so an overflow shows as an infinite chain
            float pf[4] = {pr[0], pr[1], pr[2], pr[3]};
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float sx = 1.f;
#pragma unroll
              for (int c = 0; c < NC; ++c) sx += ptx::ex2_approx(v[c][j]);
              pf[j & 3] *= (j < lim) ? sx : 1.f;
            }
            if ((pf[0] + pf[1]) + (pf[2] + pf[3]) < INFINITY) {
#pragma unroll
              for (int q = 0; q < 4; ++q) pr[q] = pf[q];
            } else {
              // shifted form, log2 sum_c 2^u_c = m + log2 sum_c 2^(u_c - m), m = max(0, u_c)
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                float m = 0.f;
#pragma unroll
                for (int c = 0; c < NC; ++c) m = fmaxf(m, v[c][j]);
                float sx = ptx::ex2_approx(-m);
#pragma unroll
                for (int c = 0; c < NC; ++c) sx += ptx::ex2_approx(v[c][j] - m);
                const bool in = j < lim;
                la[j & 3] += in ? m : 0.f;
                pr[j & 3] *= in ? sx : 1.f;
              }
            }
            renorm();
          }
          const float pm = (pr[0] * pr[1]) * (pr[2] * pr[3]);   // product of four mantissas < 16
          const float lsum = (la[0] + la[1]) + (la[2] + la[3]);
          tile_val = (lsum + static_cast<float>(pexp)) + ptx::lg2_approx(pm);
        }
        const float y = kLn2 * tile_val - kcomp;
        const float tsum = ksum + y;
        kcomp = (tsum - ksum) - y;
        ksum = tsum;
      }
      if (!ok) break;
      acc_base += static_cast<uint32_t>(tile_hi - tile_lo);
      prm.partial[(static_cast<size_t>(chunk) * NWG + wg) * prm.ppad + ptile * kBM + row] =
          static_cast<double>(ksum) - static_cast<double>(kcomp);
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicExch(prm.flag, 1);
  // a pair's MMAs write both CTAs' tensor memory and read both CTAs' shared memory: neither CTA
  // frees its tensor memory before the even CTA's MMA thread has seen them all complete
  if constexpr (CL > 1) ptx::cluster_sync();
  if (warp == 1) {
    __syncwarp();   // lane 0 ran the MMA role alone: reconverge before the aligned dealloc
    ptx::tc_fence_after();
    if constexpr (CL > 1) ptx::tmem_dealloc_pair(tmem_base, kTmemCols);
    else ptx::tmem_dealloc(tmem_base, kTmemCols);
  }
  // no CTA leaves while its peer may still arrive on its barriers or read its shared memory
  if constexpr (CL > 1) ptx::cluster_sync();
}

// ll[p] = lin_p - sum over chunks and groups of partial (fixed order), lin_p = theta_p . lin
// with lin [NC x k] in the original column order (FP64, four interleaved partial sums each).
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads)
loglik_finalize_kernel(const double* __restrict__ theta, int64_t P, int D,
                       const double* __restrict__ lin, const double* __restrict__ partial,
                       int slices, int ppad, double* __restrict__ ll, const int* __restrict__ poison) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= P) return;
  if (poison && *poison) {
    // the fused kernel gave up on a bounded wait: its partial sums are incomplete
    ll[p] = __longlong_as_double(0x7FF8000000000000LL);
    return;
  }
  const double* th = theta + p * D;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int i = 0;
  for (; i + 4 <= D; i += 4) {
    a0 = fma(th[i], lin[i], a0);
    a1 = fma(th[i + 1], lin[i + 1], a1);
    a2 = fma(th[i + 2], lin[i + 2], a2);
    a3 = fma(th[i + 3], lin[i + 3], a3);
  }
  for (; i < D; ++i) a0 = fma(th[i], lin[i], a0);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  const double* q = partial + p;
  int j = 0;
  for (; j + 4 <= slices; j += 4) {
    s0 += q[static_cast<size_t>(j) * ppad];
    s1 += q[static_cast<size_t>(j + 1) * ppad];
    s2 += q[static_cast<size_t>(j + 2) * ppad];
    s3 += q[static_cast<size_t>(j + 3) * ppad];
  }
  for (; j < slices; ++j) s0 += q[static_cast<size_t>(j) * ppad];
  ll[p] = ((a0 + a1) + (a2 + a3)) - ((s0 + s1) + (s2 + s3));
}

// ---- batched models: M nested models, model m using the first k_m covariates, its particles in
// its own block of operand rows (row_off_m, padded to the CTAs of a work item) laid out as the
// model's own encoding (its continuous columns first, low parts at k16_m), zeros beyond.
// Model table rows (int64): [row_off, P, k, theta address, particle_off, t, ll address, address
// of the model's column permutation, k16_m].
constexpr int kTab = 9;

__device__ __forceinline__ int model_of_row(const int64_t* __restrict__ tab, int M, int64_t q) {
  int m = 0;
  while (m + 1 < M && tab[(m + 1) * kTab + 0] <= q) ++m;
  return m;
}
__device__ __forceinline__ int model_of_particle(const int64_t* __restrict__ tab, int M, int64_t g) {
  int m = 0;
  while (m + 1 < M && tab[(m + 1) * kTab + 4] <= g) ++m;
  return m;
}

__global__ void encode_theta_batched_kernel(const int64_t* __restrict__ tab, int M, int NC, int kt,
                                            int64_t PP, __nv_bfloat16* __restrict__ out) {
  const int64_t r = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= NC * PP) return;
  const int c = static_cast<int>(r / PP);
  const int64_t q = r - c * PP;
  const int m = model_of_row(tab, M, q);
  const int64_t p = q - tab[m * kTab + 0];
  const int64_t Pm = tab[m * kTab + 1];
  const int km = static_cast<int>(tab[m * kTab + 2]);
  const double* src = reinterpret_cast<const double*>(tab[m * kTab + 3]) + p * (static_cast<int64_t>(NC) * km) + c * km;
  const int* perm = reinterpret_cast<const int*>(tab[m * kTab + 7]);
  const int k16 = static_cast<int>(tab[m * kTab + 8]);
  __nv_bfloat16* rowp = out + r * kt;
  for (int j = lane; j < k16; j += 32) {
    float v = 0.f;
    if (p < Pm && j < km) v = f64_to_f32(src[perm[j]]) * 1.44269504f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    rowp[j] = h;
    rowp[k16 + j] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
  for (int jj = 2 * k16 + lane; jj < kt; jj += 32) rowp[jj] = __float2bfloat16_rn(0.f);
}

// A model's own operand rows of X[:, :km] (row stride k of the context's FP64 X): [Xh | Xl | 0]
// over its internal columns (its continuous columns first), as the context's encoding of X.
__global__ void encode_x_model_kernel(const double* __restrict__ X, int64_t n, int k, int km,
                                      const int* __restrict__ perm, int k16, int kc, int kx,
                                      __nv_bfloat16* __restrict__ Xp) {
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= n * kx) return;
  const int64_t s = idx / kx;
  const int e = static_cast<int>(idx - s * kx);
  double v = 0.0;
  if (e < k16) {
    if (e < km) v = static_cast<double>(__bfloat162float(__double2bfloat16(X[s * k + perm[e]])));
  } else if (e - k16 < kc) {
    const double x = X[s * k + perm[e - k16]];
    v = x - static_cast<double>(__bfloat162float(__double2bfloat16(x)));
  }
  Xp[idx] = __double2bfloat16(v);
}

// lin[m][c*k + i] = prefix[t_m / 128] + the tail rows [128 (t_m / 128), t_m), one warp per entry.
__global__ void lin_tail_batched_kernel(const double* __restrict__ prefix, const double* __restrict__ X,
                                        const int* __restrict__ y, int k, int NC, const int64_t* __restrict__ tab,
                                        int M, double* __restrict__ lin) {
  const int64_t w = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= static_cast<int64_t>(M) * NC * k) return;
  const int m = static_cast<int>(w / (NC * k));
  const int idx = static_cast<int>(w - static_cast<int64_t>(m) * NC * k);
  const int c = idx / k, i = idx - c * k;
  const int64_t t = tab[m * kTab + 5];
  const int64_t tile = t / 128;
  double a = 0.0;
  for (int64_t s = tile * 128 + lane; s < t; s += 32) {
    const int ys = y[s];
    const double wgt = (NC == 1) ? (ys == 1 ? 0.5 : -0.5) : (ys == c + 1 ? 1.0 : 0.0);
    a = fma(wgt, X[s * k + i], a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) lin[w] = prefix[tile * NC * k + idx] + a;
}

__global__ void finalize_batched_kernel(const int64_t* __restrict__ tab, int M, int NC, int k, int64_t Ptot,
                                        const double* __restrict__ lin, const double* __restrict__ partial,
                                        int slices, int64_t PP) {
  const int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (g >= Ptot) return;
  const int m = model_of_particle(tab, M, g);
  const int64_t p = g - tab[m * kTab + 4];
  const int km = static_cast<int>(tab[m * kTab + 2]);
  const double* th = reinterpret_cast<const double*>(tab[m * kTab + 3]) + p * (static_cast<int64_t>(NC) * km);
  const double* lm = lin + static_cast<int64_t>(m) * NC * k;
  double a0 = 0.0, a1 = 0.0;
  for (int c = 0; c < NC; ++c)
    for (int i = 0; i < km; ++i) {
      if (i & 1) a1 = fma(th[c * km + i], lm[c * k + i], a1);
      else a0 = fma(th[c * km + i], lm[c * k + i], a0);
    }
  const double* q = partial + tab[m * kTab + 0] + p;
  double s0 = 0.0, s1 = 0.0;
  for (int j = 0; j < slices; ++j) {
    if (j & 1) s1 += q[static_cast<size_t>(j) * PP];
    else s0 += q[static_cast<size_t>(j) * PP];
  }
  reinterpret_cast<double*>(tab[m * kTab + 6])[p] = (a0 + a1) - (s0 + s1);
}

// ============================================================== log-likelihood and gradient
// The gradient of Eq. 1, G_c = sum_{s<=t} (1[y_s = c] - p_{s,c}) x_s (the paper prints none), as
// a second tensor-core contraction. Write q_{s,c} = p_{s,c} - 1/2 for C = 2 (the linear part of
// the C = 2 log-likelihood uses y - 1/2) and q_{s,c} = p_{s,c} for C > 2; then G_c = lin_c(t) -
// sum_s q_{s,c} x_s with lin the same prefix sums as the log-likelihood. Per tile of 128
// particles x BN observations the forward MMAs give u = eta log2 e in TMEM (as in
// loglik_tc_kernel); the epilogue forms the log-likelihood terms and q, writes q as BF16 hi + lo
// tiles into shared memory (K-major, 128-byte swizzle: the A operand of the second MMA), and the
// MMA thread accumulates D_c[particle, j] += sum_obs q x_j with the X tile already in shared
// memory as the B operand read MN-major (N = the covariate columns [Xh | Xl], K = observations).
// D stays in TMEM across the tiles of a work item (gch chains per class, by K slice) and is
// written once per item as FP32 partials.
// producer, MMA issuer and the epilogue groups of four warps: four groups with two forward
// accumulators, one with one (C - 1 = 3; a smaller block leaves its warps more registers)
__host__ __device__ constexpr int grad_groups(int NC) { return NC == 3 ? 1 : 4; }
__host__ __device__ constexpr int grad_threads(int NC) { return 32 * (2 + 4 * grad_groups(NC)); }
// Forward accumulators and the TMEM column where the gradient accumulators start, per shape:
// two accumulators of NC x BN columns (C - 1 <= 2) or one (C - 1 = 3, 32-observation tiles).
__host__ __device__ constexpr int grad_nbuf(int NC) { return NC == 3 ? 1 : 2; }
__host__ __device__ constexpr int grad_bn(int NC) { return NC == 1 ? 128 : (NC == 2 ? 64 : 32); }
__host__ __device__ constexpr uint32_t grad_goff(int NC) {
  return static_cast<uint32_t>(grad_nbuf(NC) * NC * grad_bn(NC));
}

struct GradParams {
  int t, ppad, n_ptiles, n_tiles, chunk_tiles, n_chunks, n_items;
  int kbx, kbt, k16, ksh, ksl, th_row_stride;
  int stages, th_bufs, nq;   // X stages, theta buffers, q buffers
  int ng;                    // gradient columns per class: k16 + kc16 ([Xh | Xl] of a row)
  int gch;                   // accumulator chains per class (K slices alternate between them)
  double* partial;           // [n_chunks][groups][ppad] log-likelihood partial sums
  float* gpartial;           // [n_chunks][ppad][NC ng] gradient partial sums
  int* flag;
  unsigned long long timeout_ns;
};

struct GradLayout {
  uint32_t x_bytes, th_bytes, q_bytes;
  uint32_t off_x, off_th, off_q, off_bar, total;
};

// X stages first, so that the operand reads of the second MMA stay inside the allocation
__host__ __device__ inline GradLayout grad_layout(int NC, int BN, int kbx, int kbt, int stages, int th_bufs,
                                                  int nq) {
  GradLayout L;
  L.x_bytes = static_cast<uint32_t>(kbx) * static_cast<uint32_t>(BN) * 128u;
  L.th_bytes = static_cast<uint32_t>(NC * kbt) * kTileA;
  L.q_bytes = static_cast<uint32_t>(NC * 2 * ((BN + 63) / 64)) * kTileA;   // [class][hi, lo][K block]
  L.off_x = 0;
  L.off_th = L.off_x + stages * L.x_bytes;
  L.off_q = L.off_th + th_bufs * L.th_bytes;
  L.off_bar = L.off_q + nq * L.q_bytes;
  // x_full[st], x_empty[st], th_full[2], th_empty[2], acc_full[2], acc_empty[2], q_full[2],
  // q_empty[2], g_full, g_empty, drain; then tmem base and abort flag
  L.total = L.off_bar + 8 * (2 * stages + 12 + 3) + 16;
  return L;
}

// Descriptor of an MN-major operand tile written by TMA with 128-byte swizzle: 64-element rows
// of 128 bytes along N, consecutive K rows 128 bytes apart in 1024-byte 8-row atoms (stride
// byte offset), the next 64 N elements lbo bytes further (leading byte offset).
__device__ __forceinline__ uint64_t sdesc_sw128_mn(uint32_t saddr, uint32_t lbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>(1024u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(2u) << 61;
  return d;
}

// 32 lanes x 16 consecutive 32-bit columns from 16 registers: thread i writes lane (base + i).
__device__ __forceinline__ void tmem_st_32x32b_x16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// bf16(a) in the low and bf16(b) in the high 16 bits (round to nearest even), one instruction
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// QT: q tiles in tensor memory (TMEM columns 384-511: hi then lo, two bf16 per column, one
// buffer; the gradient MMAs read A from TMEM) instead of shared memory. C = 2 only.
constexpr uint32_t kQtHi = 384, kQtLo = 448;

// TT: theta also in TMEM (columns 320-383, one copy per theta buffer, copied from its shared-memory
// tile by tcgen05.cp at the start of each work item): the forward MMAs then read only X from
// shared memory. An N = 128 MMA with both operands in shared memory reads 8 KB per 64 clocks, the
// whole shared-memory bandwidth of the SM, and the MMA thread's barrier waits queue behind those
// reads while the tensor pipe drains; with theta in TMEM the forward MMAs read half as much.
constexpr uint32_t kTt = 320;

template <int NC, int BN, bool QT, bool TT = false>
__global__ void __launch_bounds__(grad_threads(NC), 1)
grad_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapT,
               const GradParams prm) {
  static_assert(!QT || (NC == 1 && BN == 128), "q in TMEM: 64 columns each for hi and lo");
  static_assert(!TT || QT, "theta in TMEM only beside q in TMEM");
  static_assert(BN == grad_bn(NC), "tile rows of the shape");
  constexpr int NBUF = grad_nbuf(NC);
  constexpr uint32_t GOFF = grad_goff(NC);
  constexpr int QKB = (BN + 63) / 64;             // 64-observation swizzle blocks of a q tile (a
                                                  // 32-observation tile uses half of each row)
  // with two accumulators two groups share each, half of a tile's columns each; with one, a
  // single group takes whole tiles and the others idle
  constexpr int GPW = (NBUF == 2) ? 2 : 1;        // working groups per accumulator
  constexpr int COLS = BN / GPW;
  // TMEM loads of W columns per class: 32 for C = 2, 8 for C > 2 (two or three classes of 32
  // values each left the epilogue short of registers: C = 3, k = 74, 16 384 particles at 10^5
  // observations 5.30 -> 4.83 ms per launch with 16 columns, 4.70 ms with 8, which leaves no
  // spill at 96 registers a thread; C = 4 (c3) 22.28 -> 20.21 ms with 16 columns, 19.93 with 8)
  constexpr int W = (NC == 1) ? 32 : 8;
  constexpr int NCH = COLS / W;
  static_assert(COLS % 32 == 0, "32-column TMEM loads");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const GradLayout L = grad_layout(NC, BN, prm.kbx, prm.kbt, prm.stages, prm.th_bufs, QT ? 0 : prm.nq);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  uint64_t* x_full = bars;
  uint64_t* x_empty = x_full + prm.stages;
  uint64_t* th_full = x_empty + prm.stages;
  uint64_t* th_empty = th_full + 2;
  uint64_t* acc_full = th_empty + 2;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* q_full = acc_empty + 2;
  uint64_t* q_empty = q_full + 2;
  uint64_t* g_full = q_empty + 2;
  uint64_t* g_empty = g_full + 1;
  uint64_t* drain = g_empty + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < prm.stages; ++i) {
      ptx::mbar_init(&x_full[i], 1);
      ptx::mbar_init(&x_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(&th_full[i], 1);
      ptx::mbar_init(&th_empty[i], 1);
      ptx::mbar_init(&acc_full[i], 1);
      ptx::mbar_init(&acc_empty[i], 4 * GPW);   // the warps of the owning groups
      // q in TMEM: the two halves of a tile's q (the two groups of its accumulator, 64
      // observations each) are handed over separately, q_full[h] / q_empty[h]
      ptx::mbar_init(&q_full[i], QT ? 4 : 4 * GPW);
      ptx::mbar_init(&q_empty[i], 1);
    }
    ptx::mbar_init(g_full, 1);
    ptx::mbar_init(g_empty, 4);            // the four warps of group 0
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_holder, 512);
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
      ptx::prefetch_map(&mapX);
      ptx::prefetch_map(&mapT);
      int st = 0, tb = 0;
      uint32_t xph = 0, tph = 0;
      bool ok = true;
      uint32_t issued_x = 0, issued_t = 0, par_x = 0, par_t = 0;
      for (int item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
        const int chunk = item / prm.n_ptiles;
        const int ptile = item - chunk * prm.n_ptiles;
        const int tile_lo = chunk * prm.chunk_tiles;
        const int tile_hi = min(tile_lo + prm.chunk_tiles, prm.n_tiles);
        if (!ptx::mbar_wait_bounded(&th_empty[tb], tph ^ 1u, abort_flag, limit)) { ok = false; break; }
        uint8_t* thb = smem + L.off_th + tb * L.th_bytes;
        ptx::mbar_arrive_expect_tx(&th_full[tb], L.th_bytes);
        for (int c = 0; c < NC; ++c) {
          const int row = c * prm.th_row_stride + ptile * kBM;
          for (int kb = 0; kb < prm.kbt; ++kb)
            ptx::tma_load_2d(thb + (c * prm.kbt + kb) * kTileA, &mapT, &th_full[tb], kb * kKB, row);
        }
        issued_t |= 1u << tb;
        par_t = (par_t & ~(1u << tb)) | (tph << tb);
        if (++tb == prm.th_bufs) { tb = 0; tph ^= 1u; }
        for (int tile = tile_lo; tile < tile_hi; ++tile) {
          if (!ptx::mbar_wait_bounded(&x_empty[st], xph ^ 1u, abort_flag, limit)) { ok = false; break; }
          uint8_t* xb = smem + L.off_x + st * L.x_bytes;
          ptx::mbar_arrive_expect_tx(&x_full[st], L.x_bytes);
          for (int kb = 0; kb < prm.kbx; ++kb)
            ptx::tma_load_2d(xb + kb * BN * 128, &mapX, &x_full[st], kb * kKB, tile * BN);
          issued_x |= 1u << st;
          par_x = (par_x & ~(1u << st)) | (xph << st);
          if (++st == prm.stages) { st = 0; xph ^= 1u; }
        }
      }
      volatile int no_abort = 0;
      if (*abort_flag) {
        for (int s = 0; s < prm.stages; ++s)
          if (issued_x & (1u << s)) ptx::mbar_wait_bounded(&x_full[s], (par_x >> s) & 1u, &no_abort, limit);
        for (int b = 0; b < 2; ++b)
          if (issued_t & (1u << b)) ptx::mbar_wait_bounded(&th_full[b], (par_t >> b) & 1u, &no_abort, limit);
      } else {
        for (int s = 0; s < prm.stages; ++s)
          if (issued_x & (1u << s)) ptx::mbar_wait_bounded(&x_empty[s], (par_x >> s) & 1u, abort_flag, limit);
        for (int b = 0; b < 2; ++b)
          if (issued_t & (1u << b)) ptx::mbar_wait_bounded(&th_empty[b], (par_t >> b) & 1u, abort_flag, limit);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    // one thread runs the loop (the warp-wide form of the log-likelihood kernel measured 7 % slower
    // here)
    if (lane == 0) {
      const uint32_t issue = 1u;
      const uint32_t idesc_f = ptx::idesc_bf16_f32(kBM, BN);
      const uint32_t idesc_g = ptx::idesc_bf16_f32(kBM, prm.ng) | (1u << 16);   // B MN-major
      const uint32_t lbo = static_cast<uint32_t>(BN) * 128u;
      int st = 0, tb = 0;
      uint32_t xph = 0, tph = 0, acc_count = 0, item_count = 0;
      bool ok = true, issued_any = false;
      for (int item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
        const int chunk = item / prm.n_ptiles;
        const int tile_lo = chunk * prm.chunk_tiles;
        const int tile_hi = min(tile_lo + prm.chunk_tiles, prm.n_tiles);
        if (!ptx::mbar_wait_bounded(&th_full[tb], tph, abort_flag, limit)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t thb = ptx::smem_u32(smem + L.off_th + tb * L.th_bytes);
        uint64_t dt[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) dt[c] = ptx::sdesc_sw128(thb + static_cast<uint32_t>(c * prm.kbt) * kTileA);
        // TMEM copy of this item's theta rows (buffer tb): 16 K elements (8 columns) per copy. The
        // copy and the MMAs that read it are executed in issue order; the buffer is overwritten
        // only after the producer refilled shared-memory buffer tb, i.e. after every MMA of the
        // item that last used it completed (th_empty)
        const uint32_t tt = tmem_base + kTt + static_cast<uint32_t>(tb * prm.kbt * 32);
        if constexpr (TT) {
          for (int e = 0; e < prm.kbt * kKB; e += 16)
            ptx::tmem_cp_128x256b_if(issue, tt + static_cast<uint32_t>(e >> 1), dt[0] + kslice_off(kBM, e));
        }
        bool first_grad = true;
        int pend_st = -1;
        uint32_t pend_count = 0;
        // the gradient MMAs of tile `count` (X stage `xs`), then release the stage and q buffer
        auto gradient = [&](int xs, uint32_t count) -> bool {
          if constexpr (QT) {
            // per half: wait for that group's q, issue its four K slices, release that half, so
            // that the next tile's group of this half may write its q while the other half's
            // MMAs still run (c2: 1.136 -> 1.121 ms per launch)
            static_assert(!QT || GPW == 2, "q halves: two groups per accumulator");
            const uint32_t qph = count & 1u;
            const uint32_t xs_addr = ptx::smem_u32(smem + L.off_x + xs * L.x_bytes);
            for (int h = 0; h < 2; ++h) {
              if (!ptx::mbar_wait_bounded(&q_full[h], qph, abort_flag, limit)) return false;
              if (h == 0 && first_grad &&
                  !ptx::mbar_wait_bounded(g_empty, (item_count & 1u) ^ 1u, abort_flag, limit))
                return false;
              ptx::tc_fence_after();
              for (int s = h * (BN / 32); s < (h + 1) * (BN / 32); ++s) {
                const int ch = s % prm.gch;
                const uint64_t bx = sdesc_sw128_mn(xs_addr + static_cast<uint32_t>(s) * 2048u, lbo);
                const uint32_t acc = (first_grad && s < prm.gch) ? 0u : 1u;
                const uint32_t dg = tmem_base + GOFF + static_cast<uint32_t>(ch * prm.ng);
                const uint32_t s8 = static_cast<uint32_t>(s) * 8u;   // 16 observations = 8 columns
                ptx::mma_bf16_ts_if(issue, dg, tmem_base + kQtHi + s8, bx, idesc_g, acc);
                ptx::mma_bf16_ts_if(issue, dg, tmem_base + kQtLo + s8, bx, idesc_g, 1u);
              }
              ptx::mma_commit_if(issue, &q_empty[h]);
            }
            first_grad = false;
            ptx::mma_commit_if(issue, &x_empty[xs]);
            return true;
          }
          const int qb = static_cast<int>(count % static_cast<uint32_t>(prm.nq));
          const uint32_t qph = (count / static_cast<uint32_t>(prm.nq)) & 1u;
          if (!ptx::mbar_wait_bounded(&q_full[qb], qph, abort_flag, limit)) return false;
          if (first_grad && !ptx::mbar_wait_bounded(g_empty, (item_count & 1u) ^ 1u, abort_flag, limit))
            return false;
          ptx::tc_fence_after();
          const uint32_t xs_addr = ptx::smem_u32(smem + L.off_x + xs * L.x_bytes);
          const uint32_t qbase = ptx::smem_u32(smem + L.off_q + qb * L.q_bytes);
          for (int s = 0; s < BN / 16; ++s) {
            const int ch = s % prm.gch;
            const uint64_t bx = sdesc_sw128_mn(xs_addr + static_cast<uint32_t>(s) * 2048u, lbo);
            const uint64_t ka = kslice_off(kBM, 16 * s);
            const uint32_t acc = (first_grad && s < prm.gch) ? 0u : 1u;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              const uint32_t dg = tmem_base + GOFF + static_cast<uint32_t>((c * prm.gch + ch) * prm.ng);
              if constexpr (QT) {
                const uint32_t s8 = static_cast<uint32_t>(s) * 8u;   // 16 observations = 8 columns
                ptx::mma_bf16_ts_if(issue, dg, tmem_base + kQtHi + s8, bx, idesc_g, acc);
                ptx::mma_bf16_ts_if(issue, dg, tmem_base + kQtLo + s8, bx, idesc_g, 1u);
              } else {
                const uint64_t ah = ptx::sdesc_sw128(qbase + static_cast<uint32_t>((c * 2 + 0) * QKB) * kTileA);
                const uint64_t al = ptx::sdesc_sw128(qbase + static_cast<uint32_t>((c * 2 + 1) * QKB) * kTileA);
                ptx::mma_bf16_if(issue, dg, ah + ka, bx, idesc_g, acc);
                ptx::mma_bf16_if(issue, dg, al + ka, bx, idesc_g, 1u);
              }
            }
          }
          first_grad = false;
          ptx::mma_commit_if(issue, &x_empty[xs]);
          ptx::mma_commit_if(issue, &q_empty[qb]);
          return true;
        };
        for (int tile = tile_lo; tile < tile_hi; ++tile) {
          const int buf = static_cast<int>(acc_count % NBUF);
          const uint32_t aph = (acc_count / NBUF) & 1u;
          if (!ptx::mbar_wait_bounded(&acc_empty[buf], aph ^ 1u, abort_flag, limit)) {
            ok = false;
            break;
          }
          if (!ptx::mbar_wait_bounded(&x_full[st], xph, abort_flag, limit)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint64_t dx = ptx::sdesc_sw128(ptx::smem_u32(smem + L.off_x + st * L.x_bytes));
          uint32_t d[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) d[c] = tmem_base + static_cast<uint32_t>((buf * NC + c) * BN);
          if constexpr (TT) {
            for (int i = 0; i < prm.ksh; ++i)   // Th Xh'
              ptx::mma_bf16_ts_if(issue, d[0], tt + static_cast<uint32_t>(8 * i), dx + kslice_off(BN, 16 * i), idesc_f, i > 0);
            for (int i = 0; i < prm.ksh; ++i)   // Tl Xh'
              ptx::mma_bf16_ts_if(issue, d[0], tt + static_cast<uint32_t>((prm.k16 >> 1) + 8 * i), dx + kslice_off(BN, 16 * i),
                             idesc_f, 1);
            for (int i = 0; i < prm.ksl; ++i)   // Th Xl'
              ptx::mma_bf16_ts_if(issue, d[0], tt + static_cast<uint32_t>(8 * i), dx + kslice_off(BN, prm.k16 + 16 * i), idesc_f,
                             1);
          } else {
          for (int i = 0; i < prm.ksh; ++i) {   // Th_c Xh'
            const uint64_t ka = kslice_off(kBM, 16 * i), kb = kslice_off(BN, 16 * i);
#pragma unroll
            for (int c = 0; c < NC; ++c) ptx::mma_bf16_if(issue, d[c], dt[c] + ka, dx + kb, idesc_f, i > 0);
          }
          for (int i = 0; i < prm.ksh; ++i) {   // Tl_c Xh'
            const uint64_t ka = kslice_off(kBM, prm.k16 + 16 * i), kb = kslice_off(BN, 16 * i);
#pragma unroll
            for (int c = 0; c < NC; ++c) ptx::mma_bf16_if(issue, d[c], dt[c] + ka, dx + kb, idesc_f, 1);
          }
          for (int i = 0; i < prm.ksl; ++i) {   // Th_c Xl'
            const uint64_t ka = kslice_off(kBM, 16 * i), kb = kslice_off(BN, prm.k16 + 16 * i);
#pragma unroll
            for (int c = 0; c < NC; ++c) ptx::mma_bf16_if(issue, d[c], dt[c] + ka, dx + kb, idesc_f, 1);
          }
          }
          issued_any = true;
          ptx::mma_commit_if(issue, &acc_full[buf]);
          // the previous tile's q is being (or has been) written: its gradient MMAs go next, so
          // this tile's forward MMAs overlap that tile's epilogue
          if (pend_st >= 0 && !gradient(pend_st, pend_count)) { ok = false; break; }
          pend_st = st;
          pend_count = acc_count;
          ++acc_count;
          if (++st == prm.stages) { st = 0; xph ^= 1u; }
        }
        if (ok && pend_st >= 0 && !gradient(pend_st, pend_count)) ok = false;
        if (!ok) break;
        ptx::mma_commit_if(issue, g_full);
        ptx::mma_commit_if(issue, &th_empty[tb]);
        ++item_count;
        if (++tb == prm.th_bufs) { tb = 0; tph ^= 1u; }
      }
      if (*abort_flag && issued_any) {
        ptx::mma_commit_if(issue, drain);
        volatile int no_abort = 0;
        ptx::mbar_wait_bounded(drain, 0, &no_abort, limit);
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int wg = (warp - 2) >> 2;                   // group
    const bool working = wg < NBUF * GPW;             // idle groups only write zero partials
    const int own = wg / GPW;                         // its tiles: acc_count % NBUF == own
    const int col0 = (wg % GPW) * COLS;               // its share of each tile's columns
    const int quad = warp & 3;
    const int row = quad * 32 + lane;                 // particle within the tile
    const uint32_t lane_base = static_cast<uint32_t>(quad * 32) << 16;
    constexpr float kLn2 = 0.6931471805599453f;
    uint32_t acc_base = 0, item_count = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
      const int chunk = item / prm.n_ptiles;
      const int ptile = item - chunk * prm.n_ptiles;
      const int tile_lo = chunk * prm.chunk_tiles;
      const int tile_hi = min(tile_lo + prm.chunk_tiles, prm.n_tiles);
      float ksum = 0.f, kcomp = 0.f;
      const int first = working ? tile_lo + static_cast<int>((static_cast<uint32_t>(own) + NBUF - acc_base % NBUF) % NBUF)
                                : tile_hi;
      for (int tile = first; tile < tile_hi; tile += NBUF) {
        const uint32_t acc_count = acc_base + static_cast<uint32_t>(tile - tile_lo);
        const int buf = static_cast<int>(acc_count % NBUF);
        const uint32_t aph = (acc_count / NBUF) & 1u;
        const int qb = static_cast<int>(acc_count % static_cast<uint32_t>(prm.nq));
        const uint32_t qph = (acc_count / static_cast<uint32_t>(prm.nq)) & 1u;
        ok = __all_sync(0xffffffffu, ptx::mbar_wait_bounded(&acc_full[buf], aph, abort_flag, limit) &&
                                         (QT || ptx::mbar_wait_bounded(&q_empty[qb], qph ^ 1u, abort_flag, limit)));
        if (!ok) break;
        ptx::tc_fence_after();
        const int valid = prm.t - tile * BN - col0;   // columns of this group inside [0, t)
        const uint32_t tbase = tmem_base + lane_base + static_cast<uint32_t>(buf * NC * BN + col0);
        const uint32_t qrow = ptx::smem_u32(smem + L.off_q + qb * L.q_bytes) + static_cast<uint32_t>(row) * 128u;
        float la[4] = {0.f, 0.f, 0.f, 0.f};
        float pr[4] = {1.f, 1.f, 1.f, 1.f};
        int pexp = 0;
#pragma unroll 1
        for (int ch = 0; ch < NCH; ++ch) {
          float v[NC][W];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if constexpr (W == 32) ptx::tmem_ld_32x32b_x32(tbase + c * BN + ch * W, v[c]);
            else if constexpr (W == 16) ptx::tmem_ld_32x32b_x16(tbase + c * BN + ch * W, v[c]);
            else ptx::tmem_ld_32x32b_x8(tbase + c * BN + ch * W, v[c]);
          }
          ptx::tmem_wait_ld();
          if (ch == NCH - 1) {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&acc_empty[buf]);
          }
          // per column: the log-likelihood factor and q (overwrites v with q)
          if (NC == 1 && (ch * W + W) <= valid) {
            // whole chunk: no masks
#pragma unroll
            for (int j = 0; j < W; ++j) {
              const float u = v[0][j];
              const float a = fabsf(u);
              const float e = ptx::ex2_approx(-a);
              const float r = __fdividef(1.f, 1.f + e);
              la[j & 3] += a;
              pr[j & 3] *= 1.f + e;
              // sigmoid(eta) - 1/2 = sign(u) (1/2 - e / (1 + e))
              v[0][j] = copysignf(fmaf(-e, r, 0.5f), u);
            }
          } else
#pragma unroll
          for (int j = 0; j < W; ++j) {
            const bool in = (ch * W + j) < valid;
            if constexpr (NC == 1) {
              const float u = v[0][j];
              const float a = fabsf(u);
              const float e = ptx::ex2_approx(-a);
              const float r = __fdividef(1.f, 1.f + e);
              la[j & 3] += in ? a : 0.f;
              pr[j & 3] *= in ? 1.f + e : 1.f;
              v[0][j] = in ? ((u >= 0.f) ? r : e * r) - 0.5f : 0.f;
            } else {
              float m = 0.f;
#pragma unroll
              for (int c = 0; c < NC; ++c) m = fmaxf(m, v[c][j]);
              float ec[NC];
              float sx = ptx::ex2_approx(-m);
#pragma unroll
              for (int c = 0; c < NC; ++c) {
                ec[c] = ptx::ex2_approx(v[c][j] - m);
                sx += ec[c];
              }
              const float r = __fdividef(1.f, sx);
              la[j & 3] += in ? m : 0.f;
              pr[j & 3] *= in ? sx : 1.f;
#pragma unroll
              for (int c = 0; c < NC; ++c) v[c][j] = in ? ec[c] * r : 0.f;
            }
          }
          if (((ch + 1) * W) % 128 == 0) {   // every 128 terms, as with 32-column chunks
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const int bits = __float_as_int(pr[qq]);
              pexp += (bits >> 23) - 127;
              pr[qq] = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);
            }
          }
          if constexpr (QT) {
            // q as BF16 hi + lo pairs into TMEM: observation pair (2w, 2w + 1) of the tile in
            // column w of the hi and lo blocks; the previous tile's gradient MMAs must be done
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int h = 0; h < 16; ++h) {
              const float q0 = v[0][2 * h], q1 = v[0][2 * h + 1];
              hw[h] = pack_bf16x2(q0, q1);
              const float h0 = __uint_as_float(hw[h] << 16), h1 = __uint_as_float(hw[h] & 0xFFFF0000u);
              lw[h] = pack_bf16x2(q0 - h0, q1 - h1);
            }
            if (ch == 0) {
              ok = __all_sync(0xffffffffu, ptx::mbar_wait_bounded(&q_empty[wg % GPW], qph ^ 1u, abort_flag, limit));
              if (!ok) break;
              ptx::tc_fence_after();
            }
            const uint32_t wcol = static_cast<uint32_t>((col0 + ch * W) >> 1);
            tmem_st_32x32b_x16(tmem_base + lane_base + kQtHi + wcol, hw);
            tmem_st_32x32b_x16(tmem_base + lane_base + kQtLo + wcol, lw);
          } else {
          // q as BF16 hi + lo into the swizzled tile: 8 observations (16 bytes) per store
#pragma unroll
          for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int g8 = 0; g8 < W / 8; ++g8) {
              const int col = col0 + ch * W + g8 * 8;    // observation within the tile
              const uint32_t kb = static_cast<uint32_t>(col >> 6);
              const uint32_t chunk16 = static_cast<uint32_t>((col & 63) >> 3) ^ static_cast<uint32_t>(row & 7);
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                // one packed conversion for the two high parts, one for the two low parts
                const float q0 = v[c][g8 * 8 + 2 * h], q1 = v[c][g8 * 8 + 2 * h + 1];
                hw[h] = pack_bf16x2(q0, q1);
                const float h0 = __uint_as_float(hw[h] << 16), h1 = __uint_as_float(hw[h] & 0xFFFF0000u);
                lw[h] = pack_bf16x2(q0 - h0, q1 - h1);
              }
              const uint32_t base_h = qrow + (static_cast<uint32_t>(c * 2 + 0) * QKB + kb) * kTileA + chunk16 * 16u;
              const uint32_t base_l = qrow + (static_cast<uint32_t>(c * 2 + 1) * QKB + kb) * kTileA + chunk16 * 16u;
              st_shared_v4(base_h, hw[0], hw[1], hw[2], hw[3]);
              st_shared_v4(base_l, lw[0], lw[1], lw[2], lw[3]);
            }
        }
          }
        if (!ok) break;
        // q visible to the tensor cores, then the MMA thread may take it
        if constexpr (QT) {
          tmem_wait_st();
          ptx::tc_fence_before();
        } else {
          fence_proxy_async_smem();
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&q_full[QT ? wg % GPW : qb]);
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const int bits = __float_as_int(pr[qq]);
          pexp += (bits >> 23) - 127;
          pr[qq] = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);
        }
        float tile_val;
        if constexpr (NC == 1) {
          // sum over terms of |u|/2 + log2(1 + 2^-|u|): the even part of softplus
          const float lsum = (la[0] + la[1]) + (la[2] + la[3]);
          tile_val = fmaf(0.5f, lsum, static_cast<float>(pexp) + ptx::lg2_approx((pr[0] * pr[1]) * (pr[2] * pr[3])));
        } else {
          const float lsum = (la[0] + la[1]) + (la[2] + la[3]);
          tile_val = (lsum + static_cast<float>(pexp)) + ptx::lg2_approx((pr[0] * pr[1]) * (pr[2] * pr[3]));
        }
        const float y = kLn2 * tile_val - kcomp;
        const float tsum = ksum + y;
        kcomp = (tsum - ksum) - y;
        ksum = tsum;
      }
      if (!ok) break;
      acc_base += static_cast<uint32_t>(tile_hi - tile_lo);
      prm.partial[(static_cast<size_t>(chunk) * grad_groups(NC) + wg) * prm.ppad + ptile * kBM + row] =
          static_cast<double>(ksum) - static_cast<double>(kcomp);
      if (wg == 0) {
        // the item's gradient sums: TMEM -> FP32 partials, chains added
        ok = __all_sync(0xffffffffu, ptx::mbar_wait_bounded(g_full, item_count & 1u, abort_flag, limit));
        if (!ok) break;
        ptx::tc_fence_after();
        float* gout = prm.gpartial + (static_cast<size_t>(chunk) * prm.ppad + ptile * kBM + row) *
                                         static_cast<size_t>(NC * prm.ng);
        for (int c = 0; c < NC; ++c)
          for (int j0 = 0; j0 < prm.ng; j0 += 32) {
            float g[32];
            ptx::tmem_ld_32x32b_x32(tmem_base + lane_base + GOFF + static_cast<uint32_t>(c * prm.gch * prm.ng + j0), g);
            ptx::tmem_wait_ld();
            for (int ch = 1; ch < prm.gch; ++ch) {
              float h[32];
              ptx::tmem_ld_32x32b_x32(
                  tmem_base + lane_base + GOFF + static_cast<uint32_t>((c * prm.gch + ch) * prm.ng + j0), h);
              ptx::tmem_wait_ld();
#pragma unroll
              for (int q = 0; q < 32; ++q) g[q] += h[q];
            }
            const int nj = min(32, prm.ng - j0);
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (q < nj) gout[c * prm.ng + j0 + q] = g[q];
          }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(g_empty);
      }
      ++item_count;
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicExch(prm.flag, 1);
  if (warp == 1) {
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, 512);
  }
}

// grad[p][c k + i] = lin_c[i] - sum over chunks of D_c[internal column of i] (+ its low-part
// column when i is continuous); FP64 in a fixed order. One thread per gradient entry.
__global__ void grad_tc_finalize_kernel(const float* __restrict__ gpartial, int n_chunks, int64_t P, int ppad,
                                        int NC, int k, int ng, int k16, int kc, const int* __restrict__ invperm,
                                        const double* __restrict__ lin, double* __restrict__ grad) {
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int D = NC * k;
  if (e >= P * D) return;
  const int64_t p = e / D;
  const int ci = static_cast<int>(e - p * D);
  const int c = ci / k, i = ci - c * k;
  const int j = invperm[i];
  double s = 0.0;
  for (int q = 0; q < n_chunks; ++q) {
    const float* g = gpartial + (static_cast<size_t>(q) * ppad + p) * static_cast<size_t>(NC * ng) + c * ng;
    double v = static_cast<double>(g[j]);
    if (j < kc) v += static_cast<double>(g[k16 + j]);
    s += v;
  }
  grad[e] = lin[ci] - s;
}

sps_status launch_finalize(sps_ctx* ctx, const double* theta, int64_t P, const double* partial, int slices,
                           int ppad, double* ll, const int* poison = nullptr) {
  loglik_finalize_kernel<<<static_cast<unsigned>((P + kFinThreads - 1) / kFinThreads), kFinThreads, 0,
                           ctx->stream>>>(theta, P, ctx->D, ctx->lin.as<double>(), partial, slices, ppad, ll,
                                          poison);
  ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

// theta [P x D] FP64 (original order, class-major) -> operand rows [NC*ppad x kt] bf16 holding
// [hi(theta log2 e) | lo(theta log2 e)] over the internal (permuted) columns; padding zero.
// FP32 arithmetic: v = f32(theta) log2(e) carries 23 bits, of which hi + lo keep 16. One warp
// per operand row (rows = NC * ppad < 2^31), lanes over its columns.
__global__ void encode_theta_kernel(const double* __restrict__ theta, int64_t P, int k, int NC,
                                    const int* __restrict__ perm, int k16, int kt, int ppad,
                                    __nv_bfloat16* __restrict__ out) {
  const int r = static_cast<int>((blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= NC * ppad) return;
  const int c = r / ppad;
  const int p = r - c * ppad;
  const double* src = theta + static_cast<int64_t>(p) * (NC * k) + c * k;
  __nv_bfloat16* rowp = out + static_cast<int64_t>(r) * kt;
  for (int j = lane; j < k16; j += 32) {
    float v = 0.f;
    if (p < P && j < k) v = f64_to_f32(src[perm[j]]) * 1.44269504f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    rowp[j] = h;
    rowp[k16 + j] = __float2bfloat16_rn(v - __bfloat162float(h));   // v - h is exact
  }
  for (int jj = 2 * k16 + lane; jj < kt; jj += 32) rowp[jj] = __float2bfloat16_rn(0.f);
}

cudaLaunchConfig_t launch_config(int grid, int NC, uint32_t smem_bytes, cudaStream_t stream, int CL,
                                 cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(static_cast<unsigned>(threads_for(NC)));
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(CL);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Launch (launch = true) or query the co-resident clusters of one instance (launch = false).
template <int NC, int BN, int CL, bool BATCH>
sps_status run_tc(sps_ctx* ctx, const TcParams* prm, int grid, uint32_t smem_bytes, const CUtensorMap* mapT,
                  bool timed, int* max_clusters) {
  auto kern = loglik_tc_kernel<NC, BN, CL, BATCH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem_bytes));
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
  cudaLaunchAttribute attr[1];
  if (!prm) {
    cudaLaunchConfig_t cfg = launch_config(CL * ctx->num_sms, NC, smem_bytes, ctx->stream, CL, attr);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    *max_clusters = n;
    return SPS_OK;
  }
  cudaLaunchConfig_t cfg = launch_config(grid, NC, smem_bytes, ctx->stream, CL, attr);
  if (timed) hot_begin(ctx);
  e = cudaLaunchKernelEx(&cfg, kern, ctx->enc.mapX, *mapT, *prm); ++ctx->launches;
  if (timed) hot_end(ctx);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("loglik_tc launch: ") + cudaGetErrorString(e));
  return SPS_OK;
}

template <int NC, int BN>
sps_status run_cl(sps_ctx* ctx, int CL, const TcParams* prm, int grid, uint32_t smem_bytes, const CUtensorMap* mapT,
                  bool timed, int* max_clusters) {
  if (prm && prm->ptile_info)
    return CL == 2 ? run_tc<NC, BN, 2, true>(ctx, prm, grid, smem_bytes, mapT, timed, max_clusters)
                   : run_tc<NC, BN, 1, true>(ctx, prm, grid, smem_bytes, mapT, timed, max_clusters);
  return CL == 2 ? run_tc<NC, BN, 2, false>(ctx, prm, grid, smem_bytes, mapT, timed, max_clusters)
                 : run_tc<NC, BN, 1, false>(ctx, prm, grid, smem_bytes, mapT, timed, max_clusters);
}

sps_status run_any(sps_ctx* ctx, int CL, const TcParams* prm, int grid, uint32_t smem_bytes, const CUtensorMap* mapT,
                   bool timed, int* max_clusters) {
  const int NC = ctx->NC, BN = ctx->enc.bn;
  if (NC == 1 && BN == 256) return run_cl<1, 256>(ctx, CL, prm, grid, smem_bytes, mapT, timed, max_clusters);
  if (NC == 1 && BN == 128) return run_cl<1, 128>(ctx, CL, prm, grid, smem_bytes, mapT, timed, max_clusters);
  if (NC == 2 && BN == 128) return run_cl<2, 128>(ctx, CL, prm, grid, smem_bytes, mapT, timed, max_clusters);
  if (NC == 2 && BN == 64) return run_cl<2, 64>(ctx, CL, prm, grid, smem_bytes, mapT, timed, max_clusters);
  if (NC == 3 && BN == 128) return run_cl<3, 128>(ctx, CL, prm, grid, smem_bytes, mapT, timed, max_clusters);
  if (NC == 3 && BN == 64) return run_cl<3, 64>(ctx, CL, prm, grid, smem_bytes, mapT, timed, max_clusters);
  if (NC == 3 && BN == 32) return run_cl<3, 32>(ctx, CL, prm, grid, smem_bytes, mapT, timed, max_clusters);
  return fail(ctx, SPS_ERR_UNSUPPORTED, "no tensor-core tile for this shape");
}

// Persistent grid of one call: CL CTAs per cluster, at most the co-resident clusters, at most
// one cluster per work item.
int grid_for(const sps_ctx* ctx, const TcParams& prm) {
  const int CL = ctx->enc.cl;
  const int cap = (CL > 1) ? ctx->enc.max_clusters : ctx->num_sms;
  return CL * std::max(1, std::min(cap, prm.n_items));
}

// Tiles of the busiest of g_max clusters (g_max or fewer when there are fewer items) that take
// the work items (chunk-major: item = chunk * gp + particle group, chunks of ct tiles, the last
// one shorter) round robin, counting each item's start (its theta tile, its partial sums) as two
// tiles.
static int64_t busiest_cluster_tiles(int n_tiles, int ct, int64_t gp, int64_t g_max) {
  constexpr int kItemCost = 2;
  const int nch = (n_tiles + ct - 1) / ct;
  const int64_t items = gp * nch;
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>(g_max, items));
  int64_t worst = 0;
  for (int64_t c = 0; c < g; ++c) {
    int64_t load = 0;
    for (int q = 0; q < nch; ++q) {
      const int64_t a = q * gp, b = (q + 1) * gp;   // the items of chunk q: [a, b)
      if (b - 1 < c) continue;
      const int64_t j0 = (a > c) ? (a - c + g - 1) / g : 0;   // c + j g in [a, b)
      const int64_t j1 = (b - 1 - c) / g;
      if (j1 < j0) continue;
      const int tiles = std::min(ct, n_tiles - q * ct);
      load += (j1 - j0 + 1) * (tiles + kItemCost);
    }
    worst = std::max(worst, load);
  }
  return worst;
}

// Work decomposition and pipeline depth of one call; false when the tile does not fit.
bool plan_call(const sps_ctx* ctx, int64_t P, int64_t t, TcParams* prm, uint32_t* smem_bytes) {
  const XEncoding& enc = ctx->enc;
  const int NC = ctx->NC, BN = enc.bn;
  const int prow = kBM * enc.cl;                  // particle rows of one work item
  const int ppad = static_cast<int>((P + prow - 1) / prow * prow);
  *prm = TcParams{};
  prm->ppad = ppad;
  prm->n_ptiles = ppad / kBM;
  prm->n_pgroups = prm->n_ptiles / enc.cl;
  prm->t = static_cast<int>(t);
  prm->n_tiles = static_cast<int>((t + BN - 1) / BN);
  prm->kbx = enc.kx / kKB;
  prm->kbt = enc.kt / kKB;
  prm->k16 = enc.k16;
  prm->ksh = enc.k16 / 16;
  prm->ksl = enc.kc16 / 16;
  prm->th_row_stride = ppad;
  // chunking: enough work items to balance the persistent grid, items long enough to amortise
  // the theta loads
  const int grid_max = (enc.cl > 1) ? enc.max_clusters : ctx->num_sms;   // concurrent work items
  // autotuned, else 16384: each work item writes its particles' partial sums once (at 10^6
  // observations and 65 536 particles, 4096-observation items wrote 514 MB of partial sums per
  // launch, more than the 384 MB of X) and reloads its theta tile once
  const int chunk_obs = enc.chunk_obs > 0 ? enc.chunk_obs : 16384;
  int chunk_tiles = std::max(1, std::min(prm->n_tiles, chunk_obs / BN));
  const int64_t want_items = 8LL * grid_max;
  while (chunk_tiles > 2 &&
         static_cast<int64_t>(prm->n_pgroups) * ((prm->n_tiles + chunk_tiles - 1) / chunk_tiles) < want_items)
    chunk_tiles /= 2;
  // the persistent clusters take work items round robin: where equal chunks (as many, or up to
  // three more) leave the busiest cluster at least 2 % less work than this length, take them (a
  // short last chunk, or one item more for some clusters, decides the launch's tail; c3: 4.47 ->
  // 4.29 ms per launch; c2 and c4 keep their lengths)
  if (prm->n_tiles > 0) {
    const int nch0 = (prm->n_tiles + chunk_tiles - 1) / chunk_tiles;
    const int64_t base = busiest_cluster_tiles(prm->n_tiles, chunk_tiles, prm->n_pgroups, grid_max);
    int64_t best = base;
    int best_ct = chunk_tiles;
    for (int nch = nch0; nch <= nch0 + 3 && nch <= prm->n_tiles; ++nch) {
      const int ct = (prm->n_tiles + nch - 1) / nch;
      const int64_t w = busiest_cluster_tiles(prm->n_tiles, ct, prm->n_pgroups, grid_max);
      if (w < best && 50 * w <= 49 * base) {
        best = w;
        best_ct = ct;
      }
    }
    chunk_tiles = best_ct;
  }
  prm->chunk_tiles = chunk_tiles;
  prm->n_chunks = std::max(1, (prm->n_tiles + chunk_tiles - 1) / chunk_tiles);
  prm->n_items = prm->n_tiles > 0 ? prm->n_pgroups * prm->n_chunks : 0;
  int stages = 0, th_bufs = 0;
  if (!pick_stages(NC, BN, enc.cl, prm->kbx, prm->kbt, &stages, &th_bufs)) return false;
  prm->stages = stages;
  prm->th_bufs = th_bufs;
  prm->timeout_ns = ctx->debug_timeout_ns ? ctx->debug_timeout_ns : 2000000000ull;
  prm->stall = ctx->debug_stall;
  *smem_bytes = smem_layout(NC, BN, enc.cl, prm->kbx, prm->kbt, stages, th_bufs).total + 1024;
  return true;
}

}  // namespace

double tc_waves(const sps_ctx* ctx, int64_t P, int64_t t) {
  TcParams prm;
  uint32_t smem = 0;
  if (ctx->enc.bn == 0 || !plan_call(ctx, P, t, &prm, &smem)) return 0.0;
  const int conc = (ctx->enc.cl > 1) ? ctx->enc.max_clusters : ctx->num_sms;
  return static_cast<double>(prm.n_items) / std::max(1, conc);
}

// Observation rows per tensor-core tile for one CTA (CL = 1) or a CTA pair (CL = 2, each CTA
// holding half of every X tile): the widest tile for the outcome count that keeps at least
// three X stages in shared memory (0 when none fits).
int tc_tile_rows(int NC, int kx, int kt, int CL) {
  // C = 4: one 384-column accumulator of 128-observation tiles (its epilogue groups share each
  // tile by columns) before two of 64 (c3: 6.12 -> 4.40 ms per launch; N = 128 MMAs run at
  // about 102 clocks against 119 for N = 64); 32-observation tiles for wide rows
  const int cands[3][3] = {{256, 128, 0}, {128, 64, 0}, {128, 64, 32}};
  if (NC < 1 || NC > 3) return 0;
  int last = 0;
  for (int q = 0; q < 3 && cands[NC - 1][q] > 0; ++q) {
    const int BN = cands[NC - 1][q];
    int st = 0, tb = 0;
    if (pick_stages(NC, BN, CL, kx / kKB, kt / kKB, &st, &tb) && st >= 3) return BN;
    last = BN;
  }
  int st = 0, tb = 0;
  return pick_stages(NC, last, CL, kx / kKB, kt / kKB, &st, &tb) ? last : 0;
}

// One launch shape of the fused kernel: tile rows, cluster size (with its co-resident
// clusters) and work-item length, and the X tensor map for it.
static sps_status tc_set_shape(sps_ctx* ctx, int bn, int cl, int max_clusters, int chunk_obs) {
  XEncoding& enc = ctx->enc;
  enc.bn = bn;
  enc.cl = cl;
  enc.max_clusters = max_clusters;
  enc.chunk_obs = chunk_obs;
  return make_map_bf16(ctx, &enc.mapX, enc.Xp.ptr, static_cast<uint64_t>(ctx->n), enc.kx,
                       static_cast<uint32_t>(bn / cl));
}

sps_status tc_autotune(sps_ctx* ctx, int64_t P, int64_t t, sps_tune_result* out) {
  XEncoding& enc = ctx->enc;
  const int NC = ctx->NC;
  if (NC > 3 || enc.bn == 0) return fail(ctx, SPS_ERR_UNSUPPORTED, "autotune: no tensor-core tile for this shape");
  const int bn0 = enc.bn, cl0 = enc.cl, mc0 = enc.max_clusters, ch0 = enc.chunk_obs;
  DevBuf th, ll;
  SPS_CUDA_TRY(th.reserve(sizeof(double) * static_cast<size_t>(P) * ctx->D));
  SPS_CUDA_TRY(ll.reserve(sizeof(double) * static_cast<size_t>(P)));
  SPS_CUDA_TRY(cudaMemsetAsync(th.ptr, 0, sizeof(double) * static_cast<size_t>(P) * ctx->D, ctx->stream));
  cudaEvent_t e0, e1;
  SPS_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, SPS_ERR_CUDA, "autotune: event");
  }
  const bool timing = ctx->timing;
  ctx->timing = false;
  // time one shape: 1 untimed and 3 timed launches; +inf when it cannot run
  auto time_shape = [&](int bn, int cl, int mc, int chunk) -> double {
    if (tc_set_shape(ctx, bn, cl, mc, chunk) != SPS_OK) return INFINITY;
    if (loglik_split(ctx, th.as<double>(), P, t, ll.as<double>()) != SPS_OK) return INFINITY;
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 3; ++r)
      if (loglik_split(ctx, th.as<double>(), P, t, ll.as<double>()) != SPS_OK) return INFINITY;
    cudaEventRecord(e1, ctx->stream);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return INFINITY;
    return ms / 3.0;
  };
  const double ms_default = time_shape(bn0, cl0, mc0, ch0);
  double best = ms_default;
  int bb = bn0, bc = cl0, bm = mc0, bk = ch0, tried = 1;
  const int cands[3][2] = {{256, 128}, {128, 64}, {128, 64}};
  const char* env = getenv("SPS_TC_CLUSTER");
  const bool allow_cl2 = !(env && env[0] == '1' && env[1] == 0);
  for (int q = 0; q < 2; ++q) {
    const int bn = cands[NC - 1][q];
    for (int cl = 1; cl <= 2; ++cl) {
      int stages = 0, th_bufs = 0;
      if (!pick_stages(NC, bn, cl, enc.kx / kKB, enc.kt / kKB, &stages, &th_bufs)) continue;
      const uint32_t smem_bytes = smem_layout(NC, bn, cl, enc.kx / kKB, enc.kt / kKB, stages, th_bufs).total + 1024;
      int mc = 0;
      if (cl == 2) {
        if (!allow_cl2) continue;
        enc.bn = bn;
        if (run_any(ctx, 2, nullptr, 0, smem_bytes, nullptr, false, &mc) != SPS_OK || mc < 1) continue;
      }
      for (int chunk = 512; chunk <= 65536; chunk *= 2) {
        if (chunk < bn) continue;
        const double ms = time_shape(bn, cl, mc, chunk);
        ++tried;
        if (ms < best) {
          best = ms;
          bb = bn;
          bc = cl;
          bm = mc;
          bk = chunk;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->timing = timing;
  cudaGetLastError();
  ctx->last_error.clear();
  SPS_TRY(tc_set_shape(ctx, bb, bc, bm, bk));
  if (out) {
    out->tile_rows = bb;
    out->cluster = bc;
    out->chunk_obs = bk > 0 ? bk : 16384;   // 0: the default of plan_call
    out->n_candidates = tried;
    out->ms = best;
    out->ms_default = ms_default;
  }
  if (!std::isfinite(best)) return fail(ctx, SPS_ERR_CUDA, "autotune: no candidate ran");
  return SPS_OK;
}

sps_status tc_configure_cluster(sps_ctx* ctx) {
  XEncoding& enc = ctx->enc;
  const int NC = ctx->NC;
  enc.cl = 1;
  enc.max_clusters = 0;
  enc.bn = (NC <= 3) ? tc_tile_rows(NC, enc.kx, enc.kt, 1) : 0;
  if (enc.bn == 0) return SPS_OK;
  const char* env = getenv("SPS_TC_CLUSTER");
  if (env && env[0] == '1' && env[1] == 0) return SPS_OK;
  const bool force_pairs = env && env[0] == '2' && env[1] == 0;
  // CTA pairs where a tile's MMAs take longer than its epilogue (tensor-bound shapes: the pair
  // halves the X bytes each CTA receives per MMA clock and doubles the MMA time a stage covers),
  // and where two CTAs of the pair's shape can be co-scheduled. An epilogue-bound shape stays on
  // single CTAs: there the pair's cross-CTA accumulator release only lengthens the turnaround
  // (binary logit k = 30: 0.32 ms per launch in pairs against 0.24 ms).
  const int bn1 = enc.bn, bn2 = tc_tile_rows(NC, enc.kx, enc.kt, 2);
  {
    const double slices = 2.0 * (enc.k16 / 16) + enc.kc16 / 16;   // K = 16 MMAs per class and tile
    const double mma_clk = slices * NC * std::max(54.0, bn1 / 2.0);    // M = 128 MMA issue cost
    const double epi_clk = 128.0 * bn1 * (NC == 1 ? 1 : NC + 1) / 30.0; // ex2 per tile at 30 / clk
    // C > 2: the two-group epilogue is latency-bound whatever the MMA does (four outcomes,
    // k = 50: 6.65 ms per launch in pairs against 6.42 ms on single CTAs)
    if (!force_pairs && (NC > 1 || mma_clk <= epi_clk)) return SPS_OK;
  }
  int stages = 0, th_bufs = 0;
  if (bn2 == 0 || !pick_stages(NC, bn2, 2, enc.kx / kKB, enc.kt / kKB, &stages, &th_bufs)) return SPS_OK;
  const uint32_t smem_bytes = smem_layout(NC, bn2, 2, enc.kx / kKB, enc.kt / kKB, stages, th_bufs).total + 1024;
  int n = 0;
  enc.bn = bn2;
  const sps_status s = run_any(ctx, 2, nullptr, 0, smem_bytes, nullptr, false, &n);
  enc.bn = bn1;
  SPS_TRY(s);
  if (n >= 1) {
    enc.bn = bn2;
    enc.cl = 2;
    enc.max_clusters = n;
  }
  return SPS_OK;
}

sps_status loglik_split(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll) {
  const int NC = ctx->NC;
  if (NC > 3 || ctx->enc.bn == 0) return fail(ctx, SPS_ERR_UNSUPPORTED, "split precision: unsupported shape");
  XEncoding& enc = ctx->enc;
  LoglikScratch& S = ctx->ll;
  TcParams prm;
  uint32_t smem_bytes = 0;
  if (!plan_call(ctx, P, t, &prm, &smem_bytes))
    return fail(ctx, SPS_ERR_UNSUPPORTED, "covariate count too large for the tensor-core tile");
  const int ppad = prm.ppad;
  if (S.ppad_cap < ppad) {
    const int64_t cap = std::max<int64_t>(ppad, S.ppad_cap * 3 / 2 / kBM * kBM);
    SPS_CUDA_TRY(S.thetaP.reserve(static_cast<size_t>(NC) * cap * enc.kt * sizeof(__nv_bfloat16)));
    S.ppad_cap = cap;
  }
  SPS_TRY(make_map_bf16(ctx, &S.mapT, S.thetaP.ptr, static_cast<uint64_t>(NC) * ppad, enc.kt, kBM));
  {
    const int64_t rows = static_cast<int64_t>(NC) * ppad;   // one warp per row, 8 rows per block
    encode_theta_kernel<<<static_cast<unsigned>((rows + 7) / 8), 256, 0, ctx->stream>>>(
        d_theta, P, ctx->k, NC, enc.perm_dev.as<int>(), enc.k16, enc.kt, ppad, S.thetaP.as<__nv_bfloat16>());
    ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
  }
  SPS_TRY(ensure_lin(ctx, t));
  const size_t slices = static_cast<size_t>(prm.n_chunks) * nwg_for(NC);
  SPS_CUDA_TRY(S.partial.reserve(slices * ppad * sizeof(double)));
  SPS_CUDA_TRY(S.flag.reserve(sizeof(int)));
  prm.partial = S.partial.as<double>();
  prm.flag = S.flag.as<int>();
  SPS_CUDA_TRY(cudaMemsetAsync(prm.flag, 0, sizeof(int), ctx->stream));
  if (prm.n_items > 0)
    SPS_TRY(run_any(ctx, enc.cl, &prm, grid_for(ctx, prm), smem_bytes, &S.mapT, true, nullptr));
  return launch_finalize(ctx, d_theta, P, prm.partial, prm.n_items > 0 ? static_cast<int>(slices) : 0, ppad, d_ll);
}

// Shape of a gradient call, or false when the tensor-core form does not fit (C - 1 > 2, or the
// gradient accumulators or the pipeline do not fit TMEM / shared memory).
static bool grad_shape(const sps_ctx* ctx, int* BN, int* ng, int* gch, int* stages, int* th_bufs, int* nq,
                       uint32_t* smem_bytes, bool* qt) {
  const XEncoding& enc = ctx->enc;
  const int NC = ctx->NC;
  if (NC < 1 || NC > 3 || enc.bn == 0) return false;
  *BN = grad_bn(NC);
  *ng = enc.k16 + enc.kc16;
  if (*ng > 256) return false;
  const int off = static_cast<int>(grad_goff(NC));
  // q in TMEM (C = 2) when the gradient accumulators end by column 384
  *qt = (NC == 1) && off + *ng <= static_cast<int>(kQtHi);
  if (*qt) {
    *gch = (off + 2 * *ng <= static_cast<int>(kQtHi)) ? 2 : 1;
  } else {
    // the 32-column TMEM reads of the last accumulator run 16 columns past it when ng is an odd
    // multiple of 16 (C = 3, k = 74 with alternating columns: ng = 128 fills the 512 columns)
    const int over = (*ng % 32) ? 32 - *ng % 32 : 0;
    *gch = (off + NC * 2 * *ng + over <= 512) ? 2 : 1;
    if (off + NC * *gch * *ng + over > 512) return false;
  }
  const int kbx = enc.kx / kKB, kbt = enc.kt / kKB;
  for (int q = 2; q >= 1; --q)
    for (int tb = 2; tb >= 1; --tb)
      for (int st = 6; st >= 3; --st) {
        const int q_smem = *qt ? 0 : q;
        if (grad_layout(NC, *BN, kbx, kbt, st, tb, q_smem).total + 1024 <= kSmemBudget + 1024) {
          *stages = st;
          *th_bufs = tb;
          *nq = *qt ? 1 : q;
          *smem_bytes = grad_layout(NC, *BN, kbx, kbt, st, tb, q_smem).total + 1024;
          return true;
        }
      }
  return false;
}

template <int NC, int BN, bool QT, bool TT = false>
static sps_status run_grad(sps_ctx* ctx, const GradParams& prm, int grid, uint32_t smem_bytes) {
  auto kern = grad_tc_kernel<NC, BN, QT, TT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_bytes));
  if (e == cudaSuccess) {
    kern<<<grid, grad_threads(NC), smem_bytes, ctx->stream>>>(ctx->ll.mapXg, ctx->ll.mapT, prm);
    ++ctx->launches;
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(ctx, SPS_ERR_CUDA, std::string("grad_tc launch: ") + cudaGetErrorString(e));
  return SPS_OK;
}

sps_status loglik_grad_tc(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll, double* d_grad) {
  const int NC = ctx->NC, k = ctx->k;
  XEncoding& enc = ctx->enc;
  LoglikScratch& S = ctx->ll;
  int BN = 0, ng = 0, gch = 0, stages = 0, th_bufs = 0, nq = 0;
  uint32_t smem_bytes = 0;
  bool qt = false;
  if (!grad_shape(ctx, &BN, &ng, &gch, &stages, &th_bufs, &nq, &smem_bytes, &qt))
    return fail(ctx, SPS_ERR_UNSUPPORTED, "tensor-core gradient: unsupported shape");
  if (t < 1) return fail(ctx, SPS_ERR_UNSUPPORTED, "tensor-core gradient: empty prefix");
  GradParams prm{};
  const int ppad = static_cast<int>((P + kBM - 1) / kBM * kBM);
  prm.t = static_cast<int>(t);
  prm.ppad = ppad;
  prm.n_ptiles = ppad / kBM;
  prm.n_tiles = static_cast<int>((t + BN - 1) / BN);
  // as few observation chunks as keep four work items per SM: fewer gradient partials to
  // write and sum (each item writes its particles' gradient once)
  const int64_t want_chunks = std::max<int64_t>(1, (4LL * ctx->num_sms + prm.n_ptiles - 1) / prm.n_ptiles);
  int chunk_tiles = static_cast<int>(std::max<int64_t>(1, (prm.n_tiles + want_chunks - 1) / want_chunks));
  {
    // the persistent CTAs take the items round robin: where up to eight more chunks leave the
    // busiest CTA at least 2 % less work, take them (a last wave that fills few SMs decides the
    // launch; 16 384 particles at 10^5 observations, C = 3, k = 74: 5 -> 8 chunks, 4.3 -> 6.9
    // waves, 5.53 -> 5.29 ms per launch; c2 and c3 keep their chunks)
    const int nch0 = (prm.n_tiles + chunk_tiles - 1) / chunk_tiles;
    const int64_t base = busiest_cluster_tiles(prm.n_tiles, chunk_tiles, prm.n_ptiles, ctx->num_sms);
    int64_t best = base;
    int best_ct = chunk_tiles;
    for (int nch = nch0 + 1; nch <= nch0 + 8 && nch <= prm.n_tiles; ++nch) {
      const int ct = (prm.n_tiles + nch - 1) / nch;
      const int64_t w = busiest_cluster_tiles(prm.n_tiles, ct, prm.n_ptiles, ctx->num_sms);
      if (w < best && 50 * w <= 49 * base) {
        best = w;
        best_ct = ct;
      }
    }
    chunk_tiles = best_ct;
  }
  prm.chunk_tiles = chunk_tiles;
  prm.n_chunks = (prm.n_tiles + chunk_tiles - 1) / chunk_tiles;
  prm.n_items = prm.n_ptiles * prm.n_chunks;
  prm.kbx = enc.kx / kKB;
  prm.kbt = enc.kt / kKB;
  prm.k16 = enc.k16;
  prm.ksh = enc.k16 / 16;
  prm.ksl = enc.kc16 / 16;
  prm.th_row_stride = ppad;
  prm.stages = stages;
  prm.th_bufs = th_bufs;
  prm.nq = nq;
  prm.ng = ng;
  prm.gch = gch;
  prm.timeout_ns = 2000000000ull;
  // operands: theta rows as for the log-likelihood, X tiles of BN rows, inverse permutation
  if (S.ppad_cap < ppad) {
    const int64_t cap = std::max<int64_t>(ppad, S.ppad_cap * 3 / 2 / kBM * kBM);
    SPS_CUDA_TRY(S.thetaP.reserve(static_cast<size_t>(NC) * cap * enc.kt * sizeof(__nv_bfloat16)));
    S.ppad_cap = cap;
  }
  SPS_TRY(make_map_bf16(ctx, &S.mapT, S.thetaP.ptr, static_cast<uint64_t>(NC) * ppad, enc.kt, kBM));
  if (S.mapXg_rows != BN) {
    SPS_TRY(make_map_bf16(ctx, &S.mapXg, enc.Xp.ptr, static_cast<uint64_t>(ctx->n), enc.kx, static_cast<uint32_t>(BN)));
    S.mapXg_rows = BN;
  }
  if (enc.invperm_dev.bytes < sizeof(int) * static_cast<size_t>(k)) {
    std::vector<int> inv(k);
    for (int j = 0; j < k; ++j) inv[enc.perm[j]] = j;
    SPS_CUDA_TRY(enc.invperm_dev.reserve(sizeof(int) * k));
    SPS_CUDA_TRY(cudaMemcpy(enc.invperm_dev.ptr, inv.data(), sizeof(int) * k, cudaMemcpyHostToDevice));
  }
  {
    const int64_t rows = static_cast<int64_t>(NC) * ppad;
    encode_theta_kernel<<<static_cast<unsigned>((rows + 7) / 8), 256, 0, ctx->stream>>>(
        d_theta, P, k, NC, enc.perm_dev.as<int>(), enc.k16, enc.kt, ppad, S.thetaP.as<__nv_bfloat16>());
    ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
  }
  SPS_TRY(ensure_lin(ctx, t));
  SPS_CUDA_TRY(S.partial.reserve(sizeof(double) * static_cast<size_t>(prm.n_chunks) * grad_groups(NC) * ppad));
  SPS_CUDA_TRY(S.gpartial.reserve(sizeof(float) * static_cast<size_t>(prm.n_chunks) * ppad * NC * ng));
  SPS_CUDA_TRY(S.flag.reserve(sizeof(int)));
  prm.partial = S.partial.as<double>();
  prm.gpartial = S.gpartial.as<float>();
  prm.flag = S.flag.as<int>();
  SPS_CUDA_TRY(cudaMemsetAsync(prm.flag, 0, sizeof(int), ctx->stream));
  const int grid = std::max(1, std::min(ctx->num_sms, prm.n_items));
  hot_begin(ctx);
  sps_status st;
  // theta in TMEM beside q when the gradient accumulators (one chain) end by column 320 and the
  // theta copies fit columns 320-383
  const bool tt = qt && ng <= 64 && th_bufs * (enc.kt / 2) <= 64;
  if (tt) prm.gch = 1;
  if (NC == 1 && tt) st = run_grad<1, 128, true, true>(ctx, prm, grid, smem_bytes);
  else if (NC == 1 && qt) st = run_grad<1, 128, true>(ctx, prm, grid, smem_bytes);
  else if (NC == 1) st = run_grad<1, 128, false>(ctx, prm, grid, smem_bytes);
  else if (NC == 2) st = run_grad<2, 64, false>(ctx, prm, grid, smem_bytes);
  else st = run_grad<3, 32, false>(ctx, prm, grid, smem_bytes);
  hot_end(ctx);
  SPS_TRY(st);
  SPS_TRY(launch_finalize(ctx, d_theta, P, prm.partial, prm.n_chunks * grad_groups(NC), ppad, d_ll));
  const int64_t entries = P * ctx->D;
  grad_tc_finalize_kernel<<<static_cast<unsigned>((entries + 255) / 256), 256, 0, ctx->stream>>>(
      prm.gpartial, prm.n_chunks, P, ppad, NC, k, ng, enc.k16, enc.kc, enc.invperm_dev.as<int>(),
      ctx->lin.as<double>(), d_grad);
  ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

sps_status loglik_grad_dispatch(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll,
                                double* d_grad) {
  int BN, ng, gch, stages, tb, nq;
  uint32_t smem;
  bool qt;
  if (ctx->opt.precision == SPS_PREC_SPLIT && t >= 1 && grad_shape(ctx, &BN, &ng, &gch, &stages, &tb, &nq, &smem, &qt))
    return loglik_grad_tc(ctx, d_theta, P, t, d_ll, d_grad);
  return loglik_grad_fp32(ctx, d_theta, P, t, d_ll, d_grad);
}

// The encoding of X[:, :km] for batched calls: the model's continuous columns (in original order,
// as the context found them) first, then its exact ones; built once per k_m and kept.
static sps_status model_encoding(sps_ctx* ctx, int km, ModelEncoding** out) {
  auto it = ctx->model_enc.find(km);
  if (it != ctx->model_enc.end()) {
    *out = it->second.get();
    return SPS_OK;
  }
  const XEncoding& enc = ctx->enc;
  std::unique_ptr<ModelEncoding> me(new ModelEncoding());
  std::vector<int> perm;
  for (int j = 0; j < enc.kc; ++j)
    if (enc.perm[j] < km) perm.push_back(enc.perm[j]);
  me->kc = static_cast<int>(perm.size());
  for (int j = enc.kc; j < ctx->k; ++j)
    if (enc.perm[j] < km) perm.push_back(enc.perm[j]);
  me->k = km;
  me->k16 = (km + 15) / 16 * 16;
  me->kc16 = (me->kc + 15) / 16 * 16;
  me->kx = (me->k16 + me->kc16 + 63) / 64 * 64;
  SPS_CUDA_TRY(me->perm_dev.reserve(sizeof(int) * km));
  SPS_CUDA_TRY(cudaMemcpy(me->perm_dev.ptr, perm.data(), sizeof(int) * km, cudaMemcpyHostToDevice));
  SPS_CUDA_TRY(me->Xp.reserve(static_cast<size_t>(ctx->n) * me->kx * sizeof(__nv_bfloat16)));
  const int64_t tot = ctx->n * me->kx;
  encode_x_model_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, ctx->stream>>>(
      ctx->Xd.as<double>(), ctx->n, ctx->k, km, me->perm_dev.as<int>(), me->k16, me->kc, me->kx,
      me->Xp.as<__nv_bfloat16>());
  ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  *out = me.get();
  ctx->model_enc[km] = std::move(me);
  return SPS_OK;
}

struct SplitBatchedPlan {
  TcParams prm;
  uint32_t smem_bytes = 0;
  int M = 0;
  int64_t PP = 0, Ptot = 0;
  size_t slices = 0;
  DevBuf tab;     // int64 [M x kTab] model table of this launch
  DevBuf ptile;   // int2 [n_ptiles] prefix length and model slot of each particle tile
};

sps_status loglik_split_batched_prepare(sps_ctx* ctx, int plan_slot, int M, const int32_t* km, const int64_t* Pm,
                                        const int64_t* tm, const double* const* d_theta, double* const* d_ll,
                                        const char* skip, std::vector<int2>* tiles, int2** ptile_table) {
  const int NC = ctx->NC;
  if (NC > 3 || ctx->enc.bn == 0) return fail(ctx, SPS_ERR_UNSUPPORTED, "split precision: unsupported shape");
  XEncoding& enc = ctx->enc;
  LoglikScratch& S = ctx->ll;
  const int64_t prow = static_cast<int64_t>(kBM) * enc.cl;
  std::vector<int64_t> tab(static_cast<size_t>(M) * kTab);
  int64_t PP = 0, Ptot = 0, tmax = 0;
  for (int m = 0; m < M; ++m) {
    tab[m * kTab + 0] = PP;
    tab[m * kTab + 1] = Pm[m];
    tab[m * kTab + 2] = km[m];
    tab[m * kTab + 3] = static_cast<int64_t>(reinterpret_cast<uintptr_t>(d_theta[m]));
    tab[m * kTab + 4] = Ptot;
    tab[m * kTab + 5] = tm[m];
    tab[m * kTab + 6] = static_cast<int64_t>(reinterpret_cast<uintptr_t>(d_ll[m]));
    PP += (Pm[m] + prow - 1) / prow * prow;
    Ptot += Pm[m];
    tmax = std::max<int64_t>(tmax, tm[m]);
  }
  if (PP > (int64_t{1} << 28)) return fail(ctx, SPS_ERR_INVALID_ARG, "batched log-likelihood: too many particles");
  // the work decomposition of one call over PP operand rows and the longest prefix (skipped
  // models included, so that it does not depend on which models are skipped); each particle
  // tile then stops at its own model's prefix
  if (plan_slot < 0 || plan_slot > 1) return fail(ctx, SPS_ERR_INVALID_ARG, "batched log-likelihood: plan slot");
  if (!S.bplan[plan_slot]) S.bplan[plan_slot] = std::make_shared<SplitBatchedPlan>();
  SplitBatchedPlan* plan = S.bplan[plan_slot].get();
  TcParams& prm = plan->prm;
  if (!plan_call(ctx, PP, tmax, &prm, &plan->smem_bytes))
    return fail(ctx, SPS_ERR_UNSUPPORTED, "covariate count too large for the tensor-core tile");
  if (prm.ppad != PP) return fail(ctx, SPS_ERR_INVALID_ARG, "batched log-likelihood: internal padding mismatch");
  // each model's own encoding of its first k_m covariates (built on first use and kept): its tiles
  // load only its own X bytes and issue only its own MMA slices
  std::vector<BatchModel> bms(static_cast<size_t>(M));
  for (int m = 0; m < M; ++m) {
    ModelEncoding* me = nullptr;
    SPS_TRY(model_encoding(ctx, km[m], &me));
    SPS_TRY(make_map_bf16(ctx, &bms[m].mapX, me->Xp.ptr, static_cast<uint64_t>(ctx->n), me->kx,
                          static_cast<uint32_t>(enc.bn / enc.cl)));
    bms[m].kbx = me->kx / kKB;
    bms[m].k16 = me->k16;
    bms[m].ksh = me->k16 / 16;
    bms[m].ksl = me->kc16 / 16;
    tab[m * kTab + 7] = static_cast<int64_t>(reinterpret_cast<uintptr_t>(me->perm_dev.ptr));
    tab[m * kTab + 8] = me->k16;
  }
  // per particle tile: its model's prefix length (0 for a skipped model: no work item of the
  // tile has an observation) and slot
  std::vector<int2> ptile_info(static_cast<size_t>(prm.n_ptiles));
  if (tiles) tiles->assign(static_cast<size_t>(M), make_int2(0, 0));
  for (int m = 0; m < M; ++m) {
    const int64_t r0 = tab[m * kTab + 0] / kBM;
    const int64_t r1 = r0 + (Pm[m] + prow - 1) / prow * prow / kBM;
    const int tl = (skip && skip[m]) ? 0 : static_cast<int>(tm[m]);
    for (int64_t r = r0; r < r1; ++r) ptile_info[r] = make_int2(tl, m);
    if (tiles) (*tiles)[m] = make_int2(static_cast<int>(r0), static_cast<int>(r1));
  }
  SPS_CUDA_TRY(S.batch_models.reserve(sizeof(BatchModel) * bms.size()));
  SPS_CUDA_TRY(cudaMemcpyAsync(S.batch_models.ptr, bms.data(), sizeof(BatchModel) * bms.size(),
                               cudaMemcpyHostToDevice, ctx->stream));
  SPS_CUDA_TRY(plan->tab.reserve(sizeof(int64_t) * tab.size()));
  SPS_CUDA_TRY(plan->ptile.reserve(sizeof(int2) * ptile_info.size()));
  SPS_CUDA_TRY(S.batch_lin.reserve(sizeof(double) * M * NC * ctx->k));
  SPS_CUDA_TRY(cudaMemcpyAsync(plan->tab.ptr, tab.data(), sizeof(int64_t) * tab.size(), cudaMemcpyHostToDevice,
                               ctx->stream));
  SPS_CUDA_TRY(cudaMemcpyAsync(plan->ptile.ptr, ptile_info.data(), sizeof(int2) * ptile_info.size(),
                               cudaMemcpyHostToDevice, ctx->stream));
  if (S.ppad_cap < PP) {
    const int64_t cap = std::max<int64_t>(PP, S.ppad_cap * 3 / 2 / kBM * kBM);
    SPS_CUDA_TRY(S.thetaP.reserve(static_cast<size_t>(NC) * cap * enc.kt * sizeof(__nv_bfloat16)));
    S.ppad_cap = cap;
  }
  SPS_TRY(make_map_bf16(ctx, &S.mapT, S.thetaP.ptr, static_cast<uint64_t>(NC) * PP, enc.kt, kBM));
  plan->slices = static_cast<size_t>(prm.n_chunks) * nwg_for(NC);
  SPS_CUDA_TRY(S.partial.reserve(plan->slices * PP * sizeof(double)));
  SPS_CUDA_TRY(S.flag.reserve(sizeof(int)));
  prm.partial = S.partial.as<double>();
  prm.flag = S.flag.as<int>();
  prm.ptile_info = plan->ptile.as<int2>();
  prm.bmodels = S.batch_models.as<BatchModel>();
  plan->M = M;
  plan->PP = PP;
  plan->Ptot = Ptot;
  if (ptile_table) *ptile_table = plan->ptile.as<int2>();
  return SPS_OK;
}

sps_status loglik_split_batched_launch(sps_ctx* ctx, int plan_slot) {
  LoglikScratch& S = ctx->ll;
  if (plan_slot < 0 || plan_slot > 1 || !S.bplan[plan_slot])
    return fail(ctx, SPS_ERR_STATE, "batched log-likelihood: no prepared launch");
  SplitBatchedPlan& pl = *S.bplan[plan_slot];
  XEncoding& enc = ctx->enc;
  const int NC = ctx->NC, M = pl.M;
  TcParams prm = pl.prm;
  const int64_t* dtab = pl.tab.as<int64_t>();
  {
    const int64_t rows = static_cast<int64_t>(NC) * pl.PP;
    encode_theta_batched_kernel<<<static_cast<unsigned>((rows + 7) / 8), 256, 0, ctx->stream>>>(
        dtab, M, NC, enc.kt, pl.PP, S.thetaP.as<__nv_bfloat16>());
    ++ctx->launches;
    const int64_t warps = static_cast<int64_t>(M) * NC * ctx->k;
    lin_tail_batched_kernel<<<static_cast<unsigned>((warps + 3) / 4), 128, 0, ctx->stream>>>(
        ctx->lin_prefix.as<double>(), ctx->Xd.as<double>(), ctx->y.as<int>(), ctx->k, NC, dtab, M,
        S.batch_lin.as<double>());
    ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
  }
  SPS_CUDA_TRY(cudaMemsetAsync(prm.flag, 0, sizeof(int), ctx->stream));
  if (prm.n_items > 0)
    SPS_TRY(run_any(ctx, enc.cl, &prm, grid_for(ctx, prm), pl.smem_bytes, &S.mapT, true, nullptr));
  finalize_batched_kernel<<<static_cast<unsigned>((pl.Ptot + 255) / 256), 256, 0, ctx->stream>>>(
      dtab, M, NC, ctx->k, pl.Ptot, S.batch_lin.as<double>(), prm.partial,
      prm.n_items > 0 ? static_cast<int>(pl.slices) : 0, pl.PP);
  ++ctx->launches;
  SPS_CUDA_TRY(cudaGetLastError());
  return SPS_OK;
}

sps_status loglik_split_batched(sps_ctx* ctx, int M, const int32_t* km, const int64_t* Pm, const int64_t* tm,
                                const double* const* d_theta, double* const* d_ll, const char* skip) {
  SPS_TRY(loglik_split_batched_prepare(ctx, 0, M, km, Pm, tm, d_theta, d_ll, skip, nullptr, nullptr));
  return loglik_split_batched_launch(ctx, 0);
}

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

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

sps_status loglik_split_static(sps_ctx* ctx, const double* d_theta, int64_t P, int64_t t, double* d_ll) {
  const int NC = ctx->NC;
  if (NC > 3 || ctx->enc.bn == 0) return fail(ctx, SPS_ERR_UNSUPPORTED, "split precision: unsupported shape");
  const XEncoding& enc = ctx->enc;
  TcParams prm;
  uint32_t smem_bytes = 0;
  if (!plan_call(ctx, P, t, &prm, &smem_bytes))
    return fail(ctx, SPS_ERR_UNSUPPORTED, "covariate count too large for the tensor-core tile");
  const int ppad = prm.ppad;
  // carve the static area: theta operand rows, partial sums, flag
  const size_t slices = static_cast<size_t>(prm.n_chunks) * nwg_for(NC);
  const size_t op_bytes = round256(static_cast<size_t>(NC) * ppad * enc.kt * sizeof(__nv_bfloat16));
  const size_t part_bytes = round256(slices * ppad * sizeof(double));
  const size_t need = op_bytes + part_bytes + 256;
  if (need > kStaticScratchBytes) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "sps_loglik_noalloc: this call needs %zu bytes of scratch, the static area holds %zu; use sps_loglik",
             need, kStaticScratchBytes);
    return fail(ctx, SPS_ERR_INVALID_ARG, msg);
  }
  unsigned char* base = nullptr;
  SPS_TRY(static_scratch_address(ctx, &base));
  __nv_bfloat16* ops = reinterpret_cast<__nv_bfloat16*>(base);
  double* partial = reinterpret_cast<double*>(base + op_bytes);
  int* flag = reinterpret_cast<int*>(base + op_bytes + part_bytes);
  CUtensorMap mapT;
  SPS_TRY(make_map_bf16(ctx, &mapT, ops, static_cast<uint64_t>(NC) * ppad, enc.kt, kBM));
  {
    const int64_t rows = static_cast<int64_t>(NC) * ppad;   // one warp per row, 8 rows per block
    encode_theta_kernel<<<static_cast<unsigned>((rows + 7) / 8), 256, 0, ctx->stream>>>(
        d_theta, P, ctx->k, NC, enc.perm_dev.as<int>(), enc.k16, enc.kt, ppad, ops);
    ++ctx->launches;
    SPS_CUDA_TRY(cudaGetLastError());
  }
  SPS_TRY(ensure_lin(ctx, t));
  prm.partial = partial;
  prm.flag = flag;
  SPS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));   // the flag must start at zero
  if (prm.n_items > 0)
    SPS_TRY(run_any(ctx, enc.cl, &prm, grid_for(ctx, prm), smem_bytes, &mapT, false, nullptr));
  // a timeout leaves NaN in every ll (this call returns before the kernel runs, so the flag cannot
  // be read back here)
  return launch_finalize(ctx, d_theta, P, partial, prm.n_items > 0 ? static_cast<int>(slices) : 0, ppad, d_ll,
                         flag);
}

}  // namespace sps

extern "C" sps_status sps_loglik_noalloc(sps_ctx* ctx, const double* theta, int64_t P, int64_t t, double* ll) {
  if (!ctx) return SPS_ERR_INVALID_ARG;
  if (!theta || !ll || P < 1 || t < 0 || t > ctx->n || P > (1LL << 28))
    return sps::fail(ctx, SPS_ERR_INVALID_ARG, "sps_loglik_noalloc: bad arguments");
  return sps::loglik_split_static(ctx, theta, P, t, ll);
}
