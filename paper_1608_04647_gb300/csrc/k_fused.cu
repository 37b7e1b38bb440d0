// Single-pass form of the two streaming contractions of the EM iteration
// (k <= 64, T <= 1024, BF16 store, tensor cores).
//
// The M-step needs A_i = X^_i E[S]^T and its Gram A_i^T A_i
// (eq:srm_mapping_update); the next E-step needs W_i^T X^_i
// (eq:srm_mean_distributed), and with W_i = A_i M_i, M_i = (A_i^T A_i)^-1/2,
// that is M_i (A_i^T X^_i), where only the k x k M_i waits for the Gram.  So
// one pass over X^ can produce A_i, its Gram and P_i = A_i^T X^_i: for each
// 128-voxel tile,
//   phase 1: A_tile = X^_tile E[S]^T      M = 128 voxels x N = 64 x K = t
//   phase 2: P[t][f] += sum_v X^_tile[v][t] A_tile[v][f]
//                                         M = 128 t x N = 64 x K = 128 voxels
//            G += A_tile^T A_tile          (Gram, as in the two-pass M-pass)
// Phase 2 needs the whole A_tile, so it re-reads the tile's X^ chunks one
// tile later; at that distance they are still in L2 (the pass reads X^ from
// HBM once instead of twice).
//
// P for a 512-wide T-block takes 256 TMEM columns (4 blocks of 128 t x 64),
// the phase-1 accumulators 2 x 64 and the Gram 64.  For T > 512 a cluster of
// C = 2 CTAs shares each tile: CTA r streams t in [512 r, 512 r + 512), so
// phase 1 gives it a partial A over its half of T.  The halves are summed
// through distributed shared memory: CTA r completes rows [64 r, 64 r + 64)
// (the other CTA's partial arrives by st.async), writes them as BF16 into its
// own operand tile and copies them into the other CTA's (cp.async.bulk), so
// that both hold the whole A_tile for phase 2.  Each CTA accumulates the Gram
// over its own 64 rows.  P and Gram partials go to fixed slots per
// (cluster, subject segment, CTA) and are summed in a fixed order by the
// E-step reduction and the polar-factor kernel: results are reproducible.
//
// Warp roles (256 threads): warp 0 TMA loads of the first-read ring, warp 6
// those of the second-read ring, warp 1 TMEM owner and phase-1 MMA issue,
// warp 7 phase-2 MMA issue, warps 2-5 epilogue.  The two rings split the four
// 32 KB stages (s_h and 4 - s_h), or for T <= 512 eight or nine 16 KB slots,
// so the HBM stream of phase 1 never waits behind the L2 re-reads and MMAs
// of phase 2.  With s_h = 4 the original
// schedule runs instead: one ring, warp 0 loading and warp 1 issuing the
// phases of consecutive tiles in turn (warps 6 and 7 idle).  Every wait is bounded; a CTA that gives up
// raises the status word and stops issuing work.
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "srm_internal.cuh"
#include "tc_ptx.cuh"

namespace srm {

using namespace tc;

namespace {

constexpr int FT = 256;               // threads per CTA
constexpr int F_TB = 512;             // t per CTA (one T-block)
constexpr uint32_t F_BOX = 16384;     // 64 t x 128 voxel rows (BF16)
constexpr uint32_t F_STAGE = 32768;   // two boxes: 128 t x 128 rows
constexpr uint32_t F_ECH = 8192;      // one 64-t chunk of E[S] (64 feature rows)
constexpr uint32_t F_GOP = 16384;     // A_tile, 128 voxel rows x 64 features (BF16)
constexpr uint32_t F_EXCH = 16384;    // 64 rows x 64 FP32 partials
constexpr int F_RESERVE = 10;         // SMs left to the Sigma_s chain that runs beside the pass
constexpr int F_PF = 0;               // L2 prefetch distance (tiles)
// L2 eviction hints (bits of the kernel's `hints`): phase-1 loads evict last,
// phase-2 loads (the tile's last use) evict first, A_i stores evict first
constexpr int F_HINT_KEEP = 1, F_HINT_DROP = 2, F_HINT_STORE = 4;
constexpr int F_HINTS = 0;
// Default ring split (the tuner replaces it): two rings of 2 stages each.
constexpr int F_SH = 2;

struct SegF {
  int64_t tile_begin, tile_end;  // 128-row tiles (global)
  int subject;
  int pslot;  // first of C P slots ([512][64] FP32 each), CTA r uses pslot + r
  int gslot;  // first of C Gram slots ([64][64] FP32 each)
  int pad;
};

// Four 32 KB stages in both forms.
template <int C>
constexpr int f_stages() {
  return 4;
}
// Two A_tile buffers in both forms.  With C = 2 the other CTA's FP32 partial
// rows (64 rows x 64 features, 16 KB) land in the A_tile buffer that their
// sum will fill, so no separate exchange buffer is needed.
template <int C>
constexpr int f_gops() {
  return 2;
}
// The fine-slot form (one CTA per tile, two rings): the 160 KB of stages and
// A_tile buffers are cut into ten 16 KB units, nine slots and one A_tile
// buffer or eight and two.  A first-read slot holds one 64-t box of the tile
// (128 voxel rows); a second-read slot holds 128 t of 64 voxel rows (two
// 64 x 64 boxes), half the K of one P block.  The rings can then split the
// stage memory unevenly: the L2 re-reads wait about as long as the HBM
// reads, and with one A_tile buffer they can hold 80 KB beside the HBM
// ring's 64 KB.  The MMAs of every accumulator are those of the 32 KB form,
// in the same order, so both forms give bitwise equal results.
constexpr uint32_t F_HBOX = 8192;  // 64 t x 64 voxel rows (BF16)
constexpr int F_UNITS = 10;        // 16 KB units of the fine form
template <int C, bool FINE>
constexpr int f_smax() {  // most stages or slots (barrier arrays)
  return FINE ? F_UNITS - 1 : f_stages<C>();
}
template <int C, bool FINE>
constexpr size_t f_smem_bytes() {
  return FINE ? 1024 + (size_t)F_UNITS * F_BOX + 8 * F_ECH + 384
              : 1024 + (size_t)f_stages<C>() * F_STAGE + f_gops<C>() * F_GOP + 8 * F_ECH + 320;
}
static_assert(f_smem_bytes<1, false>() <= 232448 && f_smem_bytes<2, false>() <= 232448 &&
                  f_smem_bytes<1, true>() <= 232448,
              "fused pass shared memory");

__device__ __forceinline__ bool warp_wait_f(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  bool ok = mbar_wait(bar, parity, abort, status, ST_TIMEOUT);
  return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ bool warp_wait_cl(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  bool ok = mbar_wait_cluster(bar, parity, abort, status, ST_TIMEOUT);
  return __all_sync(0xffffffffu, ok);
}
// Waits of up to a tile's duration: lane 0 polls with a short back-off.
__device__ __forceinline__ bool warp_wait_soon(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_patient(bar, parity, abort, status, ST_TIMEOUT, 256);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  return ok && mbar_try_wait(bar, parity);
}
__device__ __forceinline__ bool warp_wait_long(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_patient(bar, parity, abort, status, ST_TIMEOUT, 2048);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  return ok && mbar_try_wait(bar, parity);
}

template <int C, bool FINE>
__global__ void __launch_bounds__(FT, 1)
    fpass_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapE,
                 const __grid_constant__ CUtensorMap mapAs, const __grid_constant__ CUtensorMap mapXp,
                 const __grid_constant__ CUtensorMap mapX64, const SegF* __restrict__ segs,
                 const int* __restrict__ seg_off, int T, int s_h, int lead, int pf_dist, int hints, int ng,
                 float* __restrict__ ppart, float* __restrict__ gpart, int* status) {
  static_assert(!FINE || C == 1, "the fine-slot form runs one CTA per tile");
  constexpr int SMAX = f_smax<C, FINE>();
  constexpr uint32_t SLOT = FINE ? F_BOX : F_STAGE;
  constexpr int NG_C = f_gops<C>(), SN_C = f_stages<C>();
  // stages (slots) and A_tile buffers; the fine form takes ng buffers of its ten units
  const int NG = FINE ? ng : NG_C;
  const int S_N = FINE ? F_UNITS - ng : SN_C;
  constexpr uint32_t IDESC_KM = idesc_bf16(128, 64, false, false);  // phase 1: both K-major
  constexpr uint32_t IDESC_MN = idesc_bf16(128, 64, true, true);    // phase 2 and Gram: both MN-major
  constexpr uint32_t TMEM_COLS = 512;
  constexpr uint32_t T_GRAM = 128;  // TMEM columns: [0,128) phase 1 x2, [128,192) Gram, [256,512) P
  constexpr uint32_t T_P = 256;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // the A_tile buffers and the 16 KB after them are consecutive: the Gram
  // MMA reads M = 128 "features" from a tile and the 16 KB that follow it;
  // rows 64..127 of its accumulator are never read.
  uint8_t* gop = smem + S_N * SLOT;
  uint8_t* eres = gop + NG * F_GOP;                        // E[S] chunks of this CTA's T-block
  uint64_t* full = reinterpret_cast<uint64_t*>(eres + 8 * F_ECH);
  uint64_t* empty = full + SMAX;
  uint64_t* acc_full = empty + SMAX;   // [2] phase-1 accumulators
  uint64_t* acc_empty = acc_full + 2;  // [2]
  uint64_t* gop_full = acc_empty + 2;  // [2] A_tile complete in this CTA's copy
  uint64_t* gop_free = gop_full + 2;   // [2] phase 2 of every CTA of the cluster is done with it
  uint64_t* p_full = gop_free + 2;
  uint64_t* p_empty = p_full + 1;
  uint64_t* gram_full = p_empty + 1;
  uint64_t* gram_empty = gram_full + 1;
  uint64_t* exch_full = gram_empty + 1;  // the other CTA's partial rows have arrived (in the A_tile buffer)
  uint64_t* exch_free = exch_full + 1;   // the other CTA has read the partial rows this CTA sent
  uint64_t* e_full = exch_free + 1;
  uint64_t* done = e_full + 1;          // [2] every MMA of the phase-1 / phase-2 issuer has completed
  uint64_t* epi_bar = done + 2;
  uint64_t* own_bar = epi_bar + 1;
  uint64_t* tdone = own_bar + 1;  // [4] phase 2 of tile n done (slot n % 4; two rings only)
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(tdone + 4);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_s + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = C == 2 ? cluster_ctarank() : 0u;
  const uint32_t peer = rank ^ 1u;
  const int pair = blockIdx.x / C;
  const int g0 = seg_off[pair], g1 = seg_off[pair + 1];
  const int t0 = F_TB * (int)rank;
  const int nk2 = min(4, (min(T, t0 + F_TB) - t0 + 127) / 128);  // 128-t stages per tile and phase
  // s_h = S_N: the shared-ring schedule (warps 6 and 7 idle); otherwise two
  // rings (always in the fine form)
  const bool shared = !FINE && s_h >= S_N;
  // loads per tile and ring: 128-t stages, or 16 KB slots in the fine form
  const int nld = FINE ? 2 * nk2 : nk2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S_N; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
      mbar_init(&gop_full[b], 1);
      mbar_init(&gop_free[b], C);
    }
    mbar_init(p_full, 1);
    mbar_init(p_empty, 4);
    mbar_init(gram_full, 1);
    mbar_init(gram_empty, 4);
    mbar_init(exch_full, 1);
    mbar_init(exch_free, 1);
    mbar_init(e_full, 1);
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    for (int q = 0; q < 4; ++q) mbar_init(&tdone[q], 1);
    mbar_init(epi_bar, 4);
    mbar_init(own_bar, 2);
    *abort_s = 0;
    fence_mbar_init();
  }
  if (threadIdx.x == 32) {
    tma_prefetch(&mapX);
    tma_prefetch(&mapE);
    tma_prefetch(&mapAs);
    tma_prefetch(&mapXp);
  }
  if (warp == 1) {
    tmem_alloc(tmem_s, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (C == 2) cluster_sync_all();  // the other CTA's barriers exist before anything arrives on them
  const uint32_t tmem = *tmem_s;

  if (shared && warp == 0) {
    // shared-ring schedule: one producer interleaves the first read of tile n
    // and the second read of tile n - 1 in one ring of all S_N stages
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int issued[SMAX] = {};
      uint32_t iss_ph[SMAX] = {};
      bool ok = true;
      if (g0 < g1) {
        mbar_arrive_expect_tx(e_full, (uint32_t)(2 * nk2) * F_ECH);
        for (int c2 = 0; c2 < 2 * nk2; ++c2) tma_load_2d(eres + c2 * F_ECH, &mapE, t0 + 64 * c2, 0, e_full);
      }
      // the tile's nk2 stages (the same loads serve phase 1 and, one tile
      // later, phase 2)
      const uint64_t pol_first = (hints & F_HINT_KEEP) ? l2_evict_last() : l2_evict_normal();
      const uint64_t pol_again = (hints & F_HINT_DROP) ? l2_evict_first() : l2_evict_normal();
      auto load_tile = [&](int64_t tile, bool again) -> bool {
        const uint64_t pol = again ? pol_again : pol_first;
        for (int j = 0; j < nk2; ++j) {
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_s, status, ST_TIMEOUT)) return false;
          uint8_t* st = smem + s * F_STAGE;
          mbar_arrive_expect_tx(&full[s], F_STAGE);
          tma_load_2d_hint(st, &mapX, t0 + 128 * j, (int)(tile * 128), &full[s], pol);
          tma_load_2d_hint(st + F_BOX, &mapX, t0 + 128 * j + 64, (int)(tile * 128), &full[s], pol);
          issued[s] = 1;
          iss_ph[s] = ph;
          if (++s == S_N) {
            s = 0;
            ph ^= 1u;
          }
        }
        return true;
      };
      // L2 prefetch of the tiles pf_dist ahead in this CTA's list (phase-1
      // loads come from HBM; the stages alone hold too few bytes in flight)
      int pg = g0;
      int64_t ptile = g0 < g1 ? segs[g0].tile_begin : 0;
      const int nwide = (nk2 + 1) / 2;  // 256-t boxes per tile
      auto pf_issue = [&]() {
        if (pg >= g1) return;
        for (int w = 0; w < nwide; ++w) tma_prefetch_l2_2d(&mapXp, t0 + 256 * w, (int)(ptile * 128));
        if (++ptile >= segs[pg].tile_end && ++pg < g1) ptile = segs[pg].tile_begin;
      };
      for (int q = 0; q < pf_dist; ++q) pf_issue();
      int64_t prev = -1;
      for (int g = g0; g < g1 && ok; ++g)
        for (int64_t tile = segs[g].tile_begin; tile < segs[g].tile_end && ok; ++tile) {
          if (pf_dist > 0) pf_issue();
          ok = load_tile(tile, false) && (prev < 0 || load_tile(prev, true));
          prev = tile;
        }
      if (ok && prev >= 0) ok = load_tile(prev, true);
      if (!ok) {
        for (int q = 0; q < S_N; ++q)
          if (issued[q])
            mbar_drain(&full[q], iss_ph[q], 128);
        if (g0 < g1)
          mbar_drain(e_full, 0, 128);
      }
    }
  } else if (shared && warp == 1) {
    // shared-ring schedule: one issuer interleaves phase 1 of tile n and
    // phase 2 of tile n - 1
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t ae_ph[2] = {0, 0}, gf_ph[2] = {0, 0}, pe_ph = 0, ge_ph = 0;
      bool ok = true;
      if (g0 < g1 && !mbar_wait(e_full, 0, abort_s, status, ST_TIMEOUT)) ok = false;
      // phase 1 of tile n: A_tile partial over this CTA's t range
      auto p1 = [&](int64_t n) -> bool {
        const int b = (int)(n & 1);
        if (!mbar_wait(&acc_empty[b], ae_ph[b] ^ 1u, abort_s, status, ST_TIMEOUT)) return false;
        ae_ph[b] ^= 1u;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)b * 64u;
        for (int j = 0; j < nk2; ++j) {
          if (!mbar_wait(&full[s], ph, abort_s, status, ST_TIMEOUT)) return false;
          tc_fence_after();
          const uint32_t xs = smem_u32(smem + s * F_STAGE);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t xb = xs + h * F_BOX;
            const uint32_t eb = smem_u32(eres + (2 * j + h) * F_ECH);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(dacc, sdesc_sw128(xb + 32 * kk, 16, 1024), sdesc_sw128(eb + 32 * kk, 16, 1024), IDESC_KM,
                       (j | h | kk) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
          if (++s == S_N) {
            s = 0;
            ph ^= 1u;
          }
        }
        mma_commit(&acc_full[b]);
        return true;
      };
      // phase 2 of tile n: Gram over this CTA's rows, then P over its t range
      auto p2 = [&](int64_t n, bool first, bool last) -> bool {
        const int b = (int)(n % NG);
        if (!mbar_wait_cluster(&gop_full[b], gf_ph[b], abort_s, status, ST_TIMEOUT)) return false;
        gf_ph[b] ^= 1u;
        if (first) {
          if (!mbar_wait(p_empty, pe_ph ^ 1u, abort_s, status, ST_TIMEOUT)) return false;
          pe_ph ^= 1u;
          if (!mbar_wait(gram_empty, ge_ph ^ 1u, abort_s, status, ST_TIMEOUT)) return false;
          ge_ph ^= 1u;
        }
        tc_fence_after();
        const uint32_t ga = smem_u32(gop + b * F_GOP);
        constexpr int JG = 8 / C;  // 16-row K steps of the Gram per CTA
#pragma unroll
        for (int j = 0; j < JG; ++j) {
          const uint64_t d = sdesc_sw128(ga + (uint32_t)(rank * JG + j) * 2048u, F_GOP, 1024);
          mma_bf16(tmem + T_GRAM, d, d, IDESC_MN, (first && j == 0) ? 0u : 1u);
        }
        for (int m = 0; m < nk2; ++m) {
          if (!mbar_wait(&full[s], ph, abort_s, status, ST_TIMEOUT)) return false;
          tc_fence_after();
          const uint32_t xs = smem_u32(smem + s * F_STAGE);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            mma_bf16(tmem + T_P + (uint32_t)m * 64u, sdesc_sw128(xs + j * 2048, F_BOX, 1024),
                     sdesc_sw128(ga + j * 2048, F_GOP, 1024), IDESC_MN, (first && j == 0) ? 0u : 1u);
          mma_commit(&empty[s]);
          if (++s == S_N) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (C == 2)
          mma_commit_mc(&gop_free[b], (uint16_t)0x3);
        else
          mma_commit(&gop_free[b]);
        if (last) {
          mma_commit(p_full);
          mma_commit(gram_full);
        }
        return true;
      };
      int64_t n = 0;
      bool pv = false, pfirst = false, plast = false;
      for (int g = g0; g < g1 && ok; ++g) {
        const SegF sg = segs[g];
        for (int64_t tile = sg.tile_begin; tile < sg.tile_end; ++tile, ++n) {
          if (!p1(n) || (pv && !p2(n - 1, pfirst, plast))) {
            ok = false;
            break;
          }
          pv = true;
          pfirst = tile == sg.tile_begin;
          plast = tile == sg.tile_end - 1;
        }
      }
      if (ok && pv) ok = p2(n - 1, pfirst, plast);
      // everything issued must have completed before TMEM is freed
      mma_commit(&done[0]);
      mbar_drain(&done[0], 0, 64);
    }
  } else if (shared && (warp == 6 || warp == 7)) {
    // idle in the shared-ring schedule
  } else if (warp == 0 || warp == 6) {
    // TMA producers.  Warp 0 fills the first-read ring (stages [0, s_h):
    // each tile's chunks for phase 1, from HBM); warp 6 fills the
    // second-read ring (stages [s_h, S_N): the same chunks again for phase 2,
    // normally from L2).  The rings are independent, so the HBM stream never
    // waits behind phase 2.
    if (lane == 0) {
      const bool first = warp == 0;
      const int nst = first ? s_h : S_N - s_h;
      const int sbase = first ? 0 : s_h;
      int s = 0;
      uint32_t ph = 0;
      int issued[SMAX];
      uint32_t iss_ph[SMAX];
      for (int q = 0; q < S_N; ++q) {
        issued[q] = 0;
        iss_ph[q] = 0;
      }
      bool ok = true;
      if (first && g0 < g1) {
        mbar_arrive_expect_tx(e_full, (uint32_t)(2 * nk2) * F_ECH);
        for (int c2 = 0; c2 < 2 * nk2; ++c2) tma_load_2d(eres + c2 * F_ECH, &mapE, t0 + 64 * c2, 0, e_full);
      }
      // L2 policies: a tile's first read keeps its lines for the second, which
      // is their last use in the pass
      const uint64_t pol = first ? ((hints & F_HINT_KEEP) ? l2_evict_last() : l2_evict_normal())
                                 : ((hints & F_HINT_DROP) ? l2_evict_first() : l2_evict_normal());
      // L2 prefetch of the tiles pf_dist ahead in this CTA's list (first ring only)
      int pg = g0;
      int64_t ptile = g0 < g1 ? segs[g0].tile_begin : 0;
      const int nwide = (nk2 + 1) / 2;  // 256-t boxes per tile
      auto pf_issue = [&]() {
        if (pg >= g1) return;
        for (int w = 0; w < nwide; ++w) tma_prefetch_l2_2d(&mapXp, t0 + 256 * w, (int)(ptile * 128));
        if (++ptile >= segs[pg].tile_end && ++pg < g1) ptile = segs[pg].tile_begin;
      };
      if (first)
        for (int q = 0; q < pf_dist; ++q) pf_issue();
      int64_t tn = 0;  // tile counter
      for (int g = g0; g < g1 && ok; ++g)
        for (int64_t tile = segs[g].tile_begin; tile < segs[g].tile_end && ok; ++tile, ++tn) {
          if (first && pf_dist > 0) pf_issue();
          // the first read of tile n waits for phase 2 of tile n - lead: the
          // second read then comes soon enough to find the lines in L2
          if (first && lead > 0 && tn >= lead) {
            const int64_t m = tn - lead;
            if (!mbar_wait(&tdone[m & 3], (uint32_t)((m >> 2) & 1), abort_s, status, ST_TIMEOUT)) {
              ok = false;
              break;
            }
          }
          for (int j = 0; j < nld; ++j) {
            const int si = sbase + s;
            if (!mbar_wait(&empty[si], ph ^ 1u, abort_s, status, ST_TIMEOUT)) {
              ok = false;
              break;
            }
            uint8_t* st = smem + si * SLOT;
            mbar_arrive_expect_tx(&full[si], SLOT);
            if (FINE && first) {
              // 64-t box j of the tile
              tma_load_2d_hint(st, &mapX, t0 + 64 * j, (int)(tile * 128), &full[si], pol);
            } else if (FINE) {
              // P block j / 2 (128 t), voxel rows [64 (j % 2), 64 (j % 2) + 64) of the tile
              const int tt = t0 + 128 * (j >> 1), rr = (int)(tile * 128) + 64 * (j & 1);
              tma_load_2d_hint(st, &mapX64, tt, rr, &full[si], pol);
              tma_load_2d_hint(st + F_HBOX, &mapX64, tt + 64, rr, &full[si], pol);
            } else {
              tma_load_2d_hint(st, &mapX, t0 + 128 * j, (int)(tile * 128), &full[si], pol);
              tma_load_2d_hint(st + F_BOX, &mapX, t0 + 128 * j + 64, (int)(tile * 128), &full[si], pol);
            }
            issued[si] = 1;
            iss_ph[si] = ph;
            if (++s == nst) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
      if (!ok) {
        for (int q = sbase; q < sbase + nst; ++q)
          if (issued[q])
            mbar_drain(&full[q], iss_ph[q], 128);
        if (first && g0 < g1)
          mbar_drain(e_full, 0, 128);
      }
    }
  } else if (warp == 1) {
    // phase-1 MMA issue: A_tile partial over this CTA's t range, into one of
    // two accumulators
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t ae_ph[2] = {0, 0};
      bool ok = true;
      if (g0 < g1 && !mbar_wait(e_full, 0, abort_s, status, ST_TIMEOUT)) ok = false;
      int64_t n = 0;
      for (int g = g0; g < g1 && ok; ++g)
        for (int64_t tile = segs[g].tile_begin; tile < segs[g].tile_end && ok; ++tile, ++n) {
          const int b = (int)(n & 1);
          if (!mbar_wait(&acc_empty[b], ae_ph[b] ^ 1u, abort_s, status, ST_TIMEOUT)) {
            ok = false;
            break;
          }
          ae_ph[b] ^= 1u;
          tc_fence_after();
          const uint32_t dacc = tmem + (uint32_t)b * 64u;
          for (int j = 0; j < nld; ++j) {
            if (!mbar_wait(&full[s], ph, abort_s, status, ST_TIMEOUT)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t xs = smem_u32(smem + s * SLOT);
            if (FINE) {
              // one 64-t box against E[S] chunk j
              const uint32_t eb = smem_u32(eres + j * F_ECH);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_bf16(dacc, sdesc_sw128(xs + 32 * kk, 16, 1024), sdesc_sw128(eb + 32 * kk, 16, 1024), IDESC_KM,
                         (j | kk) ? 1u : 0u);
            } else {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const uint32_t xb = xs + h * F_BOX;
                const uint32_t eb = smem_u32(eres + (2 * j + h) * F_ECH);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_bf16(dacc, sdesc_sw128(xb + 32 * kk, 16, 1024), sdesc_sw128(eb + 32 * kk, 16, 1024),
                           IDESC_KM, (j | h | kk) ? 1u : 0u);
              }
            }
            mma_commit(&empty[s]);
            if (++s == s_h) {
              s = 0;
              ph ^= 1u;
            }
          }
          if (ok) mma_commit(&acc_full[b]);
        }
      // everything this thread issued completes before TMEM is freed
      mma_commit(&done[0]);
      mbar_drain(&done[0], 0, 64);
    }
  } else if (warp == 7) {
    // phase-2 MMA issue, one tile behind: Gram over this CTA's rows, then P
    // over its t range, from the second-read ring
    if (lane == 0) {
      const int nst = S_N - s_h;
      int s = 0;
      uint32_t ph = 0;
      uint32_t gf_ph[2] = {0, 0}, pe_ph = 0, ge_ph = 0;
      bool ok = true;
      int64_t n = 0;
      for (int g = g0; g < g1 && ok; ++g) {
        const SegF sg = segs[g];
        for (int64_t tile = sg.tile_begin; tile < sg.tile_end && ok; ++tile, ++n) {
          const bool first = tile == sg.tile_begin, last = tile == sg.tile_end - 1;
          const int b = (int)(n % NG);
          if (!mbar_wait_cluster(&gop_full[b], gf_ph[b], abort_s, status, ST_TIMEOUT)) {
            ok = false;
            break;
          }
          gf_ph[b] ^= 1u;
          if (first) {
            if (!mbar_wait(p_empty, pe_ph ^ 1u, abort_s, status, ST_TIMEOUT) ||
                !mbar_wait(gram_empty, ge_ph ^ 1u, abort_s, status, ST_TIMEOUT)) {
              ok = false;
              break;
            }
            pe_ph ^= 1u;
            ge_ph ^= 1u;
          }
          tc_fence_after();
          const uint32_t ga = smem_u32(gop + b * F_GOP);
          constexpr int JG = 8 / C;  // 16-row K steps of the Gram per CTA
#pragma unroll
          for (int j = 0; j < JG; ++j) {
            const uint64_t d = sdesc_sw128(ga + (uint32_t)(rank * JG + j) * 2048u, F_GOP, 1024);
            mma_bf16(tmem + T_GRAM, d, d, IDESC_MN, (first && j == 0) ? 0u : 1u);
          }
          for (int m = 0; m < nld; ++m) {
            const int si = s_h + s;
            if (!mbar_wait(&full[si], ph, abort_s, status, ST_TIMEOUT)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t xs = smem_u32(smem + si * SLOT);
            if (FINE) {
              // P block m / 2 over voxel rows [64 h, 64 h + 64): four 16-row K steps
              const int h = m & 1;
              const uint32_t dp = tmem + T_P + (uint32_t)(m >> 1) * 64u;
#pragma unroll
              for (int j = 0; j < 4; ++j)
                mma_bf16(dp, sdesc_sw128(xs + j * 2048, F_HBOX, 1024),
                         sdesc_sw128(ga + (uint32_t)(4 * h + j) * 2048u, F_GOP, 1024), IDESC_MN,
                         (first && h == 0 && j == 0) ? 0u : 1u);
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                mma_bf16(tmem + T_P + (uint32_t)m * 64u, sdesc_sw128(xs + j * 2048, F_BOX, 1024),
                         sdesc_sw128(ga + j * 2048, F_GOP, 1024), IDESC_MN, (first && j == 0) ? 0u : 1u);
            }
            mma_commit(&empty[si]);
            if (++s == nst) {
              s = 0;
              ph ^= 1u;
            }
          }
          if (!ok) break;
          if (C == 2)
            mma_commit_mc(&gop_free[b], (uint16_t)0x3);
          else
            mma_commit(&gop_free[b]);
          mma_commit(&tdone[n & 3]);
          if (last) {
            mma_commit(p_full);
            mma_commit(gram_full);
          }
        }
      }
      mma_commit(&done[1]);
      mbar_drain(&done[1], 0, 64);
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter of this warp
    const int row = q * 32 + lane;
    const bool owner = C == 1 || (uint32_t)(row >> 6) == rank;
    const bool leader = C == 1 ? threadIdx.x == 64 : (owner && lane == 0 && (q & 1) == 0);
    uint32_t af_ph[2] = {0, 0}, gfr_ph[2] = {0, 0}, pf_ph = 0, gfl_ph = 0, ef_ph = 0, ex_ph = 0, eb_ph = 0,
             ob_ph = 0, cp_ph = 0;
    bool used[2] = {false, false};  // A_tile buffers used (final wait for their release)
    bool ok = true;
    auto epi_sync = [&]() -> bool {  // the four epilogue warps
      __syncwarp();
      if (lane == 0) mbar_arrive(epi_bar);
      const bool r = warp_wait_f(epi_bar, eb_ph, abort_s, status);
      eb_ph ^= 1u;
      return r;
    };
    auto own_sync = [&]() -> bool {  // the two warps owning this CTA's rows (C == 2)
      __syncwarp();
      if (lane == 0) mbar_arrive(own_bar);
      const bool r = warp_wait_f(own_bar, ob_ph, abort_s, status);
      ob_ph ^= 1u;
      return r;
    };
    // A_i is not read again in the pass: its lines go first
    const uint64_t pol_store = (hints & F_HINT_STORE) ? l2_evict_first() : l2_evict_normal();
    uint32_t peer_gop = 0, peer_exch_full = 0, peer_exch_free = 0;
    if (C == 2) {
      peer_gop = mapa_shared(smem_u32(gop), peer);
      peer_exch_full = mapa_shared(smem_u32(exch_full), peer);
      peer_exch_free = mapa_shared(smem_u32(exch_free), peer);
    }

    // phase-1 result of tile n -> BF16 operand tile(s), A_i rows to HBM
    auto tile_epi = [&](int64_t n, int64_t tile) -> bool {
      const int a = (int)(n & 1);   // phase-1 accumulator
      const int b = (int)(n % NG);  // A_tile buffer
      if (!warp_wait_soon(&acc_full[a], af_ph[a], abort_s, status)) return false;
      af_ph[a] ^= 1u;
      tc_fence_after();
      float v[64];
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)a * 64u, v);
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)a * 64u + 32u, v + 32);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[a]);
      uint8_t* gb = gop + b * F_GOP;
      if (C == 2 && !owner) {
        // partial row for the CTA that completes it, into that CTA's A_tile
        // buffer b: free once phase 2 of tile n - NG is done in both CTAs
        // (gop_free is signalled to both), and once the other CTA has read
        // the partials of the previous tile (exch_full counts one tile's
        // bytes at a time)
        if (!warp_wait_cl(&gop_free[b], gfr_ph[b] ^ 1u, abort_s, status)) return false;
        gfr_ph[b] ^= 1u;
        if (!warp_wait_cl(exch_free, ef_ph ^ 1u, abort_s, status)) return false;
        ef_ph ^= 1u;
        const int prow = row - 64 * (int)peer;
        const uint32_t dst = peer_gop + (uint32_t)b * F_GOP;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const uint32_t off = (uint32_t)prow * 256u + (uint32_t)((u ^ (prow & 15)) * 16);
          st_async_v4(dst + off, __float_as_uint(v[4 * u]), __float_as_uint(v[4 * u + 1]),
                      __float_as_uint(v[4 * u + 2]), __float_as_uint(v[4 * u + 3]), peer_exch_full);
        }
        return true;
      }
      if (!warp_wait_cl(&gop_free[b], gfr_ph[b] ^ 1u, abort_s, status)) return false;
      gfr_ph[b] ^= 1u;
      used[b] = true;
      if (leader) bulk_wait_read0();  // the A_i store of this buffer's previous tile has read it
      if (C == 2) {
        if (leader) mbar_arrive_expect_tx(exch_full, F_EXCH);
        if (!warp_wait_cl(exch_full, ex_ph, abort_s, status)) return false;
        ex_ph ^= 1u;
        const int orow = row - 64 * (int)rank;
        const float4* src = reinterpret_cast<const float4*>(gb + orow * 256);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float4 w = src[u ^ (orow & 15)];
          v[4 * u] += w.x;
          v[4 * u + 1] += w.y;
          v[4 * u + 2] += w.z;
          v[4 * u + 3] += w.w;
        }
        if (!own_sync()) return false;  // every owner row has read the partials
        if (leader) mbar_arrive_remote(peer_exch_free);
      } else {
        if (!epi_sync()) return false;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * u], v[8 * u + 1]);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * u + 2], v[8 * u + 3]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * u + 4], v[8 * u + 5]);
        __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * u + 6], v[8 * u + 7]);
        const uint4 pk = make_uint4(*reinterpret_cast<uint32_t*>(&h0), *reinterpret_cast<uint32_t*>(&h1),
                                    *reinterpret_cast<uint32_t*>(&h2), *reinterpret_cast<uint32_t*>(&h3));
        *reinterpret_cast<uint4*>(gb + row * 128 + ((u ^ (row & 7)) * 16)) = pk;
      }
      fence_proxy_async_smem();
      if (C == 2 ? !own_sync() : !epi_sync()) return false;
      if (C == 2) {
        // the other CTA has read the partials this CTA sent into its buffer b
        // before this CTA's rows land there
        if (!warp_wait_cl(exch_free, cp_ph, abort_s, status)) return false;
        cp_ph ^= 1u;
      }
      if (leader) {
        if (C == 2) {
          const uint32_t o = rank * 64u * 128u;
          // this CTA's rows now; the other CTA's rows by its copy
          mbar_arrive_expect_tx(&gop_full[b], 64u * 128u);
          bulk_copy_to_cta(mapa_shared(smem_u32(gb + o), peer), gb + o, 64u * 128u,
                           mapa_shared(smem_u32(&gop_full[b]), peer));
          tma_store_2d_hint(&mapAs, 0, (int)(tile * 128 + 64 * (int64_t)rank), gb + o, pol_store);
        } else {
          mbar_arrive(&gop_full[b]);
          tma_store_2d_hint(&mapAs, 0, (int)(tile * 128), gb, pol_store);
        }
        bulk_commit();
      }
      return true;
    };
    // P and Gram of a finished subject segment -> its slots
    auto flush = [&](const SegF& sg) -> bool {
      if (!warp_wait_long(p_full, pf_ph, abort_s, status)) return false;
      pf_ph ^= 1u;
      tc_fence_after();
      float* slot = ppart + (int64_t)(sg.pslot + (int)rank) * F_TB * 64;
      for (int m = 0; m < nk2; ++m) {
        float* dst = slot + (int64_t)(m * 128 + row) * 64;
#pragma unroll
        for (int cc = 0; cc < 64; cc += 32) {
          float r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + T_P + (uint32_t)(m * 64 + cc), r);
          float4* d4 = reinterpret_cast<float4*>(dst + cc);
#pragma unroll
          for (int u = 0; u < 8; ++u) d4[u] = make_float4(r[4 * u], r[4 * u + 1], r[4 * u + 2], r[4 * u + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(p_empty);
      if (!warp_wait_f(gram_full, gfl_ph, abort_s, status)) return false;
      gfl_ph ^= 1u;
      tc_fence_after();
      if (q < 2) {
        float* gp = gpart + (int64_t)(sg.gslot + (int)rank) * 64 * 64 + (int64_t)row * 64;
#pragma unroll
        for (int cc = 0; cc < 64; cc += 32) {
          float r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + T_GRAM + (uint32_t)cc, r);
          float4* d4 = reinterpret_cast<float4*>(gp + cc);
#pragma unroll
          for (int u = 0; u < 8; ++u) d4[u] = make_float4(r[4 * u], r[4 * u + 1], r[4 * u + 2], r[4 * u + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(gram_empty);
      return true;
    };

    int64_t n = 0;
    bool pv = false, plast = false;
    SegF psg{};
    for (int g = g0; g < g1 && ok; ++g) {
      const SegF sg = segs[g];
      for (int64_t tile = sg.tile_begin; tile < sg.tile_end; ++tile, ++n) {
        // the previous tile's segment is flushed after this tile's phase-1
        // epilogue (the MMA issues phase 2 of tile n-1 after phase 1 of n)
        if (!tile_epi(n, tile) || (pv && plast && !flush(psg))) {
          ok = false;
          break;
        }
        pv = true;
        plast = tile == sg.tile_end - 1;
        psg = sg;
      }
    }
    if (ok && pv) ok = flush(psg);
    if (ok) {
      // every arrival the other CTA makes on this CTA's barriers has landed
      // before the cluster exits
      if (owner) {
        for (int b = 0; b < NG && ok; ++b)
          if (used[b]) ok = warp_wait_cl(&gop_free[b], gfr_ph[b] ^ 1u, abort_s, status);
      } else if (n > 0) {
        ok = warp_wait_cl(exch_free, ef_ph ^ 1u, abort_s, status);
      }
    }
    if (leader) bulk_wait0();  // the A_i stores have landed
  }
  tc_fence_before();
  __syncthreads();
  if (C == 2) cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
            cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D BF16 tensor map with the 128-byte swizzle; inner = contiguous extent.
bool bf16_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes, uint32_t box_in,
              uint32_t box_out, bool swizzle = true) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_in, box_out};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct FState {
  CUtensorMap mapX, mapE, mapAs, mapXp, mapX64;
  SegF* d_seg = nullptr;
  int* d_seg_off = nullptr;
  int C = 1, clusters = 0;
  int pf = F_PF;  // L2 prefetch distance (tiles)
  int hints = F_HINTS;
  int s_h = F_SH;  // stages of the first-read ring (the second-read ring has the rest)
  int lead = 0;    // tiles the first read may run ahead of phase 2 (0: no limit; two rings only)
  int slots = 0;   // 0: four 32 KB stages; 8 or 9: 16 KB slots (and 2 or 1 A_tile buffers)
  // Gram slots of the two forms; the context points at the active form's
  float* f_gpart = nullptr;
  int* f_gslot_off = nullptr;
  int f_ngslots = 0;
  int64_t f_gel = 0;
  float* m_gpart = nullptr;
  int* m_gslot_off = nullptr;
  int m_ngslots = 0;
  int64_t m_gel = 0;
};

template <typename T>
srm_status upload_vec(T** d, const std::vector<T>& h, const char* what) {
  if (cudaMalloc(reinterpret_cast<void**>(d), std::max<size_t>(1, h.size()) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMalloc failed for ") + what);
    return SRM_ERR_NOMEM;
  }
  if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error(std::string("cudaMemcpy failed for ") + what);
    return SRM_ERR_CUDA;
  }
  return SRM_OK;
}

}  // namespace

bool fused_supported(const Ctx* c) { return c->batched && c->kld == 64 && c->T <= 2 * F_TB; }

namespace {

// Persistent clusters that fit beside `reserve` idle SMs.
int fused_clusters(Ctx* c, int C, int reserve) {
  int clusters = std::max(1, (c->num_sms - reserve) / C);
  if (C == 2) {
    // at most as many clusters as can be resident at once (persistent CTAs)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(FT);
    cfg.dynamicSmemBytes = f_smem_bytes<2, false>();
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int mc = 0;
    if (cudaOccupancyMaxActiveClusters(&mc, fpass_kernel<2, false>, &cfg) == cudaSuccess && mc > 0)
      clusters = std::min(clusters, mc);
    cudaGetLastError();
  }
  return clusters;
}

// Schedule, partial slots and reduction tables of the pass for `clusters`
// clusters (replacing any earlier ones).
srm_status fused_build(Ctx* c, int clusters) {
  auto* f = static_cast<FState*>(c->fs);
  const int C = f->C, N = c->N;
  // the context points at the two-pass Gram slots while these are rebuilt
  // (and stays so if the rebuild fails)
  const bool was_on = c->fused;
  if (was_on) fused_select(c, false);
  c->p_from_f = false;  // the pass's partials are gone: the next E-step streams X^ again
  void* old[] = {f->d_seg, f->d_seg_off, c->f_ppart, c->f_chunk_src, c->f_chunk_src_off, f->f_gpart, f->f_gslot_off};
  for (void* q : old)
    if (q) cudaFree(q);
  f->d_seg = nullptr;
  f->d_seg_off = nullptr;
  c->f_ppart = nullptr;
  c->f_chunk_src = nullptr;
  c->f_chunk_src_off = nullptr;
  f->f_gpart = nullptr;
  f->f_gslot_off = nullptr;
  f->clusters = clusters;
  // 128-row tiles split evenly over the clusters, segments at subject boundaries
  const int64_t NTl = c->Vpad_tot / 128;
  std::vector<SegF> seg;
  std::vector<int> seg_off(clusters + 1, 0);
  for (int q = 0; q < clusters; ++q) {
    const int64_t a = NTl * q / clusters, e = NTl * (q + 1) / clusters;
    int64_t t = a;
    while (t < e) {
      const int64_t rowi = t * 128;
      const int i = (int)(std::upper_bound(c->off.begin(), c->off.begin() + N + 1, rowi) - c->off.begin()) - 1;
      const int64_t tend = std::min<int64_t>(e, c->off[i + 1] / 128);
      seg.push_back({t, tend, i, (int)seg.size() * C, 0, 0});
      t = tend;
    }
    seg_off[q + 1] = (int)seg.size();
  }
  // Gram slots contiguous per subject (segment order, then CTA rank)
  std::vector<int> gslot_off(N + 1, 0);
  for (const SegF& g : seg) gslot_off[g.subject + 1] += C;
  for (int i = 0; i < N; ++i) gslot_off[i + 1] += gslot_off[i];
  {
    std::vector<int> fill(gslot_off.begin(), gslot_off.end() - 1);
    for (SegF& g : seg) {
      g.gslot = fill[g.subject];
      fill[g.subject] += C;
    }
  }
  // E-step reduction sources: slot (segment, rank) holds t-chunks 8 rank .. 8 rank + 7
  std::vector<std::vector<int64_t>> lists((size_t)N * c->nchunk);
  for (const SegF& g : seg)
    for (int r = 0; r < C; ++r)
      for (int cl = 0; cl < F_TB / TCH; ++cl) {
        const int ch = r * (F_TB / TCH) + cl;
        if (ch >= c->nchunk) break;
        lists[(size_t)g.subject * c->nchunk + ch].push_back((int64_t)(g.pslot + r) * F_TB * 64 + (int64_t)cl * TCH * 64);
      }
  std::vector<ChunkSrc> src;
  std::vector<int> src_off(lists.size() + 1);
  for (size_t j = 0; j < lists.size(); ++j) {
    src_off[j] = (int)src.size();
    for (int64_t o : lists[j]) src.push_back({o});
  }
  src_off[lists.size()] = (int)src.size();

  srm_status st;
  if ((st = upload_vec(&f->d_seg, seg, "single-pass schedule")) != SRM_OK) return st;
  if ((st = upload_vec(&f->d_seg_off, seg_off, "single-pass schedule offsets")) != SRM_OK) return st;
  if ((st = upload_vec(&c->f_chunk_src, src, "single-pass chunk table")) != SRM_OK) return st;
  if ((st = upload_vec(&c->f_chunk_src_off, src_off, "single-pass chunk table offsets")) != SRM_OK) return st;
  if ((st = upload_vec(&f->f_gslot_off, gslot_off, "single-pass Gram slot table")) != SRM_OK) return st;
  const int64_t pel = (int64_t)seg.size() * C * F_TB * 64;
  const int64_t gel = (int64_t)seg.size() * C * 64 * 64;
  if (cudaMalloc(&c->f_ppart, sizeof(float) * std::max<int64_t>(1, pel)) != cudaSuccess ||
      cudaMalloc(&f->f_gpart, sizeof(float) * std::max<int64_t>(1, gel)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed for single-pass partial slots");
    return SRM_ERR_NOMEM;
  }
  f->f_ngslots = (int)seg.size() * C;
  f->f_gel = gel;
  // the polar-factor and eigen kernels read the Gram slots through the context
  if (was_on) fused_select(c, true);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "single-pass setup");
  return SRM_OK;
}

}  // namespace

srm_status fused_setup(Ctx* c) {
  if (!fused_supported(c)) {
    set_error("single-pass form: needs the batched BF16 form, k <= 64 and T <= 1024");
    return SRM_ERR_UNSUPPORTED;
  }
  auto* f = new FState();
  c->fs = f;
  const int C = c->T > F_TB ? 2 : 1;
  f->C = C;
  if (C == 2) {
    cudaFuncSetAttribute(fpass_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)f_smem_bytes<2, false>());
  } else {
    cudaFuncSetAttribute(fpass_kernel<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)f_smem_bytes<1, false>());
    cudaFuncSetAttribute(fpass_kernel<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)f_smem_bytes<1, true>());
  }
  f->s_h = F_SH;
  bool ok = bf16_map(&f->mapX, c->Xh, c->T, c->Vpad_tot, (uint64_t)c->ldT * 2, 64, 128) &&
            bf16_map(&f->mapE, c->ESb, c->T, 64, (uint64_t)c->ldT * 2, 64, 64) &&
            bf16_map(&f->mapAs, c->A, 64, c->Vpad_tot, 64 * 2, 64, 128 / C) &&
            // L2 prefetch only (never lands in shared memory): 256 t x 128 rows per box
            bf16_map(&f->mapXp, c->Xh, c->T, c->Vpad_tot, (uint64_t)c->ldT * 2, 256, 128, false) &&
            // second-read slots of the fine form: 64 t x 64 rows per box
            bf16_map(&f->mapX64, c->Xh, c->T, c->Vpad_tot, (uint64_t)c->ldT * 2, 64, 64);
  if (!ok) {
    set_error("cuTensorMapEncodeTiled failed for the single-pass form");
    return SRM_ERR_CUDA;
  }
  // the two-pass form's Gram slots, which fused_select swaps back in
  f->m_gpart = c->Gpart;
  f->m_gslot_off = c->gslot_off;
  f->m_ngslots = c->n_gslots;
  f->m_gel = c->Gpart_elems;
  // the pass's partials summed per (subject, chunk), and the table that
  // gives the E-step reduction one source per (subject, chunk) among them
  {
    const int64_t nb = (int64_t)c->N * c->nchunk;
    std::vector<ChunkSrc> src((size_t)nb);
    std::vector<int> off((size_t)nb + 1);
    for (int64_t j = 0; j < nb; ++j) {
      src[(size_t)j].off = j * TCH * 64;
      off[(size_t)j] = (int)j;
    }
    off[(size_t)nb] = (int)nb;
    srm_status st;
    if ((st = upload_vec(&c->psum_src, src, "slot-sum table")) != SRM_OK) return st;
    if ((st = upload_vec(&c->psum_src_off, off, "slot-sum table offsets")) != SRM_OK) return st;
    if (cudaMalloc(&c->psum, sizeof(float) * (size_t)nb * TCH * 64) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc failed for the single pass's slot sums");
      return SRM_ERR_NOMEM;
    }
  }
  return fused_build(c, fused_clusters(c, C, F_RESERVE));
}

int fused_get_reserve(const Ctx* c) {
  const auto* f = static_cast<const FState*>(c->fs);
  return f ? c->num_sms - f->clusters * f->C : F_RESERVE;
}

srm_status fused_set_reserve(Ctx* c, int reserve) {
  auto* f = static_cast<FState*>(c->fs);
  if (!f) return SRM_OK;
  if (reserve < 0 || reserve > c->num_sms - f->C) {
    set_error("plan: the single-pass reserve must leave at least one cluster to the pass");
    return SRM_ERR_ARG;
  }
  const int clusters = fused_clusters(c, f->C, reserve);
  if (clusters == f->clusters && c->f_ppart) return SRM_OK;
  return fused_build(c, clusters);
}

void fused_select(Ctx* c, bool on) {
  auto* f = static_cast<FState*>(c->fs);
  if (!f) return;
  c->Gpart = on ? f->f_gpart : f->m_gpart;
  c->gslot_off = on ? f->f_gslot_off : f->m_gslot_off;
  c->n_gslots = on ? f->f_ngslots : f->m_ngslots;
  c->Gpart_elems = on ? f->f_gel : f->m_gel;
  c->fused = on;
}

int fused_get_pf(const Ctx* c) { return c->fs ? static_cast<const FState*>(c->fs)->pf : F_PF; }
int fused_get_hints(const Ctx* c) { return c->fs ? static_cast<const FState*>(c->fs)->hints : F_HINTS; }
int fused_get_first_stages(const Ctx* c) { return c->fs ? static_cast<const FState*>(c->fs)->s_h : F_SH; }
int fused_get_lead(const Ctx* c) { return c->fs ? static_cast<const FState*>(c->fs)->lead : 0; }
int fused_get_slots(const Ctx* c) { return c->fs ? static_cast<const FState*>(c->fs)->slots : 0; }
bool fused_fine_supported(const Ctx* c) { return fused_supported(c) && c->T <= F_TB; }
void fused_set_slots(Ctx* c, int slots) {
  if (c->fs) static_cast<FState*>(c->fs)->slots = slots;
}
void fused_set_lead(Ctx* c, int lead) {
  if (c->fs) static_cast<FState*>(c->fs)->lead = lead;
}
void fused_set_first_stages(Ctx* c, int s_h) {
  if (c->fs) static_cast<FState*>(c->fs)->s_h = s_h;
}

void fused_set_pf(Ctx* c, int pf) {
  if (c->fs) static_cast<FState*>(c->fs)->pf = pf;
}
void fused_set_hints(Ctx* c, int hints) {
  if (c->fs) static_cast<FState*>(c->fs)->hints = hints;
}

void fused_destroy(Ctx* c) {
  auto* f = static_cast<FState*>(c->fs);
  if (!f) return;
  // the context frees the active form's Gram slots; this frees the other's
  const bool on = c->Gpart == f->f_gpart;
  void* p[] = {f->d_seg, f->d_seg_off, on ? (void*)f->m_gpart : (void*)f->f_gpart,
               on ? (void*)f->m_gslot_off : (void*)f->f_gslot_off};
  for (void* q : p)
    if (q) cudaFree(q);
  delete f;
  c->fs = nullptr;
}

cudaError_t launch_fpass(Ctx* c) {
  auto* f = static_cast<FState*>(c->fs);
  if (!f) return cudaErrorInvalidValue;
  if (f->C == 1 && f->slots) {
    fpass_kernel<1, true><<<f->clusters, FT, f_smem_bytes<1, true>(), c->stream>>>(
        f->mapX, f->mapE, f->mapAs, f->mapXp, f->mapX64, f->d_seg, f->d_seg_off, c->T, f->s_h, f->lead, f->pf,
        f->hints, F_UNITS - f->slots, c->f_ppart, c->Gpart, c->status);
    return cudaGetLastError();
  }
  if (f->C == 1) {
    fpass_kernel<1, false><<<f->clusters, FT, f_smem_bytes<1, false>(), c->stream>>>(
        f->mapX, f->mapE, f->mapAs, f->mapXp, f->mapX64, f->d_seg, f->d_seg_off, c->T, f->s_h, f->lead, f->pf,
        f->hints, f_gops<1>(), c->f_ppart, c->Gpart, c->status);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * f->clusters);
  cfg.blockDim = dim3(FT);
  cfg.dynamicSmemBytes = f_smem_bytes<2, false>();
  cfg.stream = c->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fpass_kernel<2, false>, f->mapX, f->mapE, f->mapAs, f->mapXp, f->mapX64,
                            (const SegF*)f->d_seg, (const int*)f->d_seg_off, c->T, f->s_h, f->lead, f->pf, f->hints,
                            f_gops<2>(), c->f_ppart, c->Gpart, c->status);
}

}  // namespace srm
