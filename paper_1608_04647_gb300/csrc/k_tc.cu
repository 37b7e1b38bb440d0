// Grouped persistent tensor-core (tcgen05) form of the two streaming passes
// of the EM iteration, over all subjects of uneven v_i in one launch each.
//
// E-pass (Algorithm 1, E-step reduction; eq:srm_mean_distributed):
//   P_i[t][f] = sum_v X^_i[v][t] A_i[v][f]   (A_i = W_i at the first iteration)
//   MMA shape M = 128 (t) x N = kld (features) x K = 16 (voxels), both
//   operands MN-major straight from the row-major HBM layouts (no transposes).
//   One CTA per SM walks a contiguous range of (T-block, subject, 32-row
//   chunk) steps; four 128 x kld FP32 accumulators (a 512-wide T-block) live
//   in TMEM and are flushed to a partial slot whenever the subject or the
//   T-block changes.  A fixed-order reduction (p_reduce) sums the slots.
// M-pass (eq:srm_mapping_update): A_i = X^_i E[S]^T, tiles of 128 voxels:
//   M = 128 (voxels) x N = kld x K = 16 (t), both operands K-major.  The
//   epilogue writes A_i (BF16) and stages the tile in shared memory, and a
//   second MMA accumulates the Gram A_i^T A_i (M = 128 features, N = kld,
//   K = 128 voxels, MN-major) in TMEM; it is flushed per subject segment.
//
// Warp roles (192 threads): warp 0 issues TMA loads, warp 1 owns TMEM and
// issues MMAs (one thread), warps 2-5 run the epilogue (one TMEM lane
// quarter each).  Every wait is bounded; on time-out the block raises a flag
// in the status word, stops issuing work and frees TMEM before returning.
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <vector>

#include "srm_internal.cuh"
#include "tc_ptx.cuh"
#include "../../include/srm_debug.h"

namespace srm {

using namespace tc;

namespace {

constexpr int NT = 192;       // threads per CTA
constexpr int E_KR = 32;      // voxel rows per E-pass stage
constexpr int E_STAGES = 4;
constexpr int E_RESERVE_MAX = 20;  // SMs the E-pass leaves free (at most)
constexpr int E_TB = 512;     // t per E-pass item (4 accumulators of 128)

struct WorkE {
  int subject, tb, slot, pad;
  int64_t row_begin, row_end;  // global rows, multiples of E_KR
};
struct SegM {
  int64_t tile_begin, tile_end;  // 128-row tiles (global)
  int slot, subject;
};

struct TcState {
  CUtensorMap mapXe, mapA, mapXm, mapE, mapAs, mapXp;
  WorkE* d_work = nullptr;
  int* d_work_off = nullptr;
  SegM* d_seg = nullptr;
  int* d_seg_off = nullptr;
  int grid = 0;         // M-pass CTAs (one per SM)
  int egrid = 0;        // E-pass CTAs
  bool m_res = false;   // M-pass keeps E[S] resident in shared memory
  int m_stages = 4;     // M-pass pipeline depth
  int m_gop = 2;        // M-pass Gram operand buffers
  int m_pf = 0;         // M-pass L2 prefetch distance (X^ chunks; 0 = off)
  int m_bps = 1;        // M-pass 64-t boxes per stage (1, 2 or 4)
  size_t m_smem = 0;
};

// Warp-uniform bounded wait (all lanes agree on the outcome).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  bool ok = mbar_wait(bar, parity, abort, status, ST_TIMEOUT);
  return __all_sync(0xffffffffu, ok);
}
// The same for waits that span a whole work item (lane 0 polls with back-off).
__device__ __forceinline__ bool warp_wait_patient(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_patient(bar, parity, abort, status, ST_TIMEOUT, 2048);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  return ok && mbar_try_wait(bar, parity);
}

__host__ __device__ constexpr uint32_t e_stage_bytes(int kld) { return 8u * E_KR * 128u + (uint32_t)(kld / 64) * E_KR * 128u; }
__host__ __device__ constexpr uint32_t m_stage_bytes(int kld) { return 128u * 128u + (uint32_t)kld * 128u; }
constexpr uint32_t kBarBytes = 256;
constexpr size_t e_smem_bytes(int kld) { return 1024 + (size_t)E_STAGES * e_stage_bytes(kld) + kBarBytes; }
// Gram operand buffers: kld = 64 uses one feature atom per buffer plus one
// shared zero atom; kld = 128 uses two atoms per buffer.
// One or two Gram operand buffers (chosen at run time): with one, the
// epilogue of tile n + 1 waits for the Gram MMA of tile n, and the bytes saved
// buy one more X^ stage.
__host__ __device__ constexpr uint32_t gop_bytes(int kld, int nb) {
  return kld == 64 ? 16384u * (uint32_t)(nb + 1) : 32768u * (uint32_t)nb;
}
constexpr int M_MAX_STAGES = 8;  // runtime stage count of the M-pass is at most this
constexpr int M_PF = 8;          // M-pass L2 prefetch distance (X^ chunks of 16 KB) ...
constexpr int M_PF_STAGES = 5;   // ... used when fewer shared-memory stages than this fit
constexpr int M_PF_MODE = 3;     // 1: per 16 KB chunk, 2: per tile (bulk), 3: per 4 chunks (one wide box)
constexpr size_t m_fixed_bytes(int kld, int nb) { return 1024 + gop_bytes(kld, nb) + kBarBytes; }
constexpr size_t kMaxSmem = 232448;  // opt-in limit per block

// ------------------------------------------------------------------ E-pass
template <int KLD>
__global__ void __launch_bounds__(NT, 1)
    estep_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapA,
                    const WorkE* __restrict__ work, const int* __restrict__ work_off, int T,
                    float* __restrict__ part, int* status) {
  constexpr int NA = KLD / 64;
  constexpr uint32_t X_BYTES = 8u * E_KR * 128u;
  constexpr uint32_t STAGE = e_stage_bytes(KLD);
  constexpr uint32_t TMEM_COLS = 4 * KLD;
  constexpr uint32_t IDESC = idesc_bf16(128, KLD, true, true);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + E_STAGES * STAGE);
  uint64_t* empty = full + E_STAGES;
  uint64_t* acc_full = empty + E_STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* done = acc_empty + 1;
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_s + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w0 = work_off[blockIdx.x], w1 = work_off[blockIdx.x + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < E_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 4);
    mbar_init(done, 1);
    *abort_s = 0;
    fence_mbar_init();
  }
  if (threadIdx.x == 32) {
    tma_prefetch(&mapX);
    tma_prefetch(&mapA);
  }
  if (warp == 1) {
    tmem_alloc(tmem_s, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_s;

  if (warp == 0) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int issued[E_STAGES] = {0};
      uint32_t iss_ph[E_STAGES] = {0};
      bool ok = true;
      for (int w = w0; w < w1 && ok; ++w) {
        const WorkE it = work[w];
        const int tbase = it.tb * E_TB;
        for (int64_t r = it.row_begin; r < it.row_end; r += E_KR) {
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_s, status, ST_TIMEOUT)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE;
          mbar_arrive_expect_tx(&full[s], STAGE);
#pragma unroll
          for (int c = 0; c < 8; ++c) tma_load_2d(st + c * (E_KR * 128), &mapX, tbase + 64 * c, (int)r, &full[s]);
#pragma unroll
          for (int a = 0; a < NA; ++a) tma_load_2d(st + X_BYTES + a * (E_KR * 128), &mapA, 64 * a, (int)r, &full[s]);
          issued[s] = 1;
          iss_ph[s] = ph;
          if (++s == E_STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok) {
        // let loads already in flight land before the block exits
        for (int q = 0; q < E_STAGES; ++q)
          if (issued[q]) {
            mbar_drain(&full[q], iss_ph[q], 128);
          }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0, acc_ph = 0;
      bool ok = true;
      for (int w = w0; w < w1 && ok; ++w) {
        const WorkE it = work[w];
        const int n_mt = min(4, (T - it.tb * E_TB + 127) / 128);
        if (!mbar_wait(acc_empty, acc_ph ^ 1u, abort_s, status, ST_TIMEOUT)) {
          ok = false;
          break;
        }
        acc_ph ^= 1u;
        tc_fence_after();
        bool first = true;
        for (int64_t r = it.row_begin; r < it.row_end; r += E_KR) {
          if (!mbar_wait(&full[s], ph, abort_s, status, ST_TIMEOUT)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t xs = smem_u32(smem + s * STAGE);
          const uint32_t as = xs + X_BYTES;
#pragma unroll
          for (int j = 0; j < E_KR / 16; ++j) {
            const uint64_t bdesc = sdesc_sw128(as + j * 2048, E_KR * 128, 1024);
            for (int m = 0; m < n_mt; ++m) {
              const uint64_t adesc = sdesc_sw128(xs + 2 * m * (E_KR * 128) + j * 2048, E_KR * 128, 1024);
              mma_bf16(tmem + m * KLD, adesc, bdesc, IDESC, (first && j == 0) ? 0u : 1u);
            }
          }
          first = false;
          mma_commit(&empty[s]);
          if (++s == E_STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (ok) mma_commit(acc_full);
      }
      // everything issued must have completed before TMEM is freed
      mma_commit(done);
      mbar_drain(done, 0, 64);
    }
  } else {
    const int q = warp & 3;
    uint32_t acc_ph = 0;
    for (int w = w0; w < w1; ++w) {
      const WorkE it = work[w];
      const int n_mt = min(4, (T - it.tb * E_TB + 127) / 128);
      if (!warp_wait_patient(acc_full, acc_ph, abort_s, status)) break;
      acc_ph ^= 1u;
      tc_fence_after();
      float* slot = part + (int64_t)it.slot * E_TB * KLD;
      for (int m = 0; m < n_mt; ++m) {
        float* dst = slot + (int64_t)(m * 128 + q * 32 + lane) * KLD;
#pragma unroll
        for (int cc = 0; cc < KLD; cc += 32) {
          float r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(m * KLD + cc), r);
          float4* d4 = reinterpret_cast<float4*>(dst + cc);
#pragma unroll
          for (int u = 0; u < 8; ++u) d4[u] = make_float4(r[4 * u], r[4 * u + 1], r[4 * u + 2], r[4 * u + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------------ M-pass
// RES: E[S] (all 64-column chunks, kld rows each) is loaded once per CTA and
// stays in shared memory; the stages then carry X^ tiles only.  Otherwise
// every stage carries an X^ tile and the matching E[S] chunk.
template <int KLD, bool RES, int GNB>  // GNB: Gram operand buffers (1 or 2)
__global__ void __launch_bounds__(NT, 1)
    mstep_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapE,
                    const __grid_constant__ CUtensorMap mapAs, const __grid_constant__ CUtensorMap mapXp,
                    const SegM* __restrict__ segs, const int* __restrict__ seg_off, int T, int S_N, int bps,
                    int pf_dist, const uint8_t* __restrict__ xbase, int64_t xrow_bytes,
                    __nv_bfloat16* __restrict__ Aout, float* __restrict__ gpart, int* status) {
  constexpr uint32_t X_BYTES = 128u * 128u;
  constexpr uint32_t E_CHUNK = (uint32_t)KLD * 128u;
  // a stage holds bps consecutive 64-t boxes of the same 128 rows (X^ boxes
  // first, then, unless E[S] is resident, the matching E[S] chunks)
  const uint32_t STAGE = (uint32_t)bps * (RES ? X_BYTES : m_stage_bytes(KLD));
  constexpr uint32_t TMEM_COLS = (3 * KLD <= 256) ? 256 : 512;
  constexpr uint32_t IDESC_MAIN = idesc_bf16(128, KLD, false, false);
  constexpr uint32_t IDESC_GRAM = idesc_bf16(128, KLD, true, true);
  const int nk = (T + 63) / 64;
  constexpr int gop_nb = GNB;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* eres = smem + S_N * STAGE;                      // resident E[S] chunks (RES only)
  uint8_t* gop = eres + (RES ? (uint32_t)nk * E_CHUNK : 0u);  // Gram operand buffers
  uint64_t* full = reinterpret_cast<uint64_t*>(gop + gop_bytes(KLD, gop_nb));
  uint64_t* empty = full + S_N;
  uint64_t* acc_full = empty + S_N;        // [2]
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint64_t* gram_ready = acc_empty + 2;    // [2]
  uint64_t* gram_free = gram_ready + 2;    // [2]
  uint64_t* gram_full = gram_free + 2;
  uint64_t* gram_empty = gram_full + 1;
  uint64_t* done = gram_empty + 1;
  uint64_t* e_full = done + 1;
  uint64_t* epi_bar = e_full + 1;          // the four epilogue warps meet here (bounded waits)
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(epi_bar + 1);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_s + 1);
  // Gram operand buffer b, feature atom a (a = 1 only for kld = 128) and the
  // distance from atom 0 to atom 1 (the descriptor's leading-byte offset)
  auto gop_atom = [&](int b, int a) -> uint8_t* {
    return KLD == 64 ? gop + b * 16384 : gop + b * 32768 + a * 16384;
  };
  auto gop_lbo = [&](int b) -> uint32_t { return KLD == 64 ? 16384u * (uint32_t)(gop_nb - b) : 16384u; };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g0 = seg_off[blockIdx.x], g1 = seg_off[blockIdx.x + 1];

  // zero the Gram operand buffers (with kld = 64 the shared atom 64..127 stays zero)
  for (uint32_t e = threadIdx.x; e < gop_bytes(KLD, gop_nb) / 16; e += NT)
    reinterpret_cast<uint4*>(gop)[e] = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(e_full, 1);
    for (int s = 0; s < S_N; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
      mbar_init(&gram_ready[b], 4);
      mbar_init(&gram_free[b], 1);
    }
    mbar_init(gram_full, 1);
    mbar_init(gram_empty, 4);
    mbar_init(done, 1);
    mbar_init(epi_bar, 4);
    *abort_s = 0;
    fence_mbar_init();
  }
  if (threadIdx.x == 32) {
    tma_prefetch(&mapX);
    tma_prefetch(&mapE);
    tma_prefetch(&mapAs);
  }
  if (warp == 1) {
    tmem_alloc(tmem_s, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_s;
  const uint32_t tgram = tmem + 2 * KLD;

  if (warp == 0) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int issued[M_MAX_STAGES] = {0};
      uint32_t iss_ph[M_MAX_STAGES] = {0};
      bool ok = true;
      if (RES && g0 < g1) {
        mbar_arrive_expect_tx(e_full, (uint32_t)nk * E_CHUNK);
        for (int kc = 0; kc < nk; ++kc) tma_load_2d(eres + kc * E_CHUNK, &mapE, 64 * kc, 0, e_full);
      }
      // L2 prefetch cursor, pf_dist chunks of X^ ahead of the loads: more
      // bytes in flight than the shared-memory stages hold (used when the
      // stages are few)
      int pg = g0, pkc = 0;
      int64_t ptile = g0 < g1 ? segs[g0].tile_begin : 0;
      auto pf_next = [&]() {
        while (pg < g1 && ptile >= segs[pg].tile_end)
          if (++pg < g1) ptile = segs[pg].tile_begin;
        if (pg >= g1 || pf_dist == 0) return;
        if (M_PF_MODE == 3) {
          // four chunks of the same 128 rows in one box, once every four chunks
          if ((pkc & 3) == 0) tma_prefetch_l2_2d(&mapXp, 64 * pkc, (int)(ptile * 128));
        } else if (M_PF_MODE == 2) {
          // a whole 128-row tile (contiguous rows) per prefetch, in 32 KB pieces
          if (pkc == 0) {
            const uint8_t* p = xbase + ptile * 128 * xrow_bytes;
            const int64_t tot = 128 * xrow_bytes;
            for (int64_t o = 0; o < tot; o += 32768)
              bulk_prefetch_l2(p + o, (uint32_t)(tot - o < 32768 ? tot - o : 32768));
          }
        } else {
          tma_prefetch_l2_2d(&mapX, 64 * pkc, (int)(ptile * 128));
        }
        if (++pkc == nk) {
          pkc = 0;
          ++ptile;
        }
      };
      for (int q = 0; q < pf_dist; ++q) pf_next();
      for (int g = g0; g < g1 && ok; ++g) {
        const SegM sg = segs[g];
        for (int64_t tile = sg.tile_begin; tile < sg.tile_end && ok; ++tile) {
          for (int kc0 = 0; kc0 < nk; kc0 += bps) {
            const int nb = min(bps, nk - kc0);
            for (int bb = 0; bb < nb; ++bb) pf_next();
            if (!mbar_wait(&empty[s], ph ^ 1u, abort_s, status, ST_TIMEOUT)) {
              ok = false;
              break;
            }
            uint8_t* st = smem + s * STAGE;
            mbar_arrive_expect_tx(&full[s], (uint32_t)nb * (RES ? X_BYTES : m_stage_bytes(KLD)));
            for (int bb = 0; bb < nb; ++bb) {
              tma_load_2d(st + bb * X_BYTES, &mapX, 64 * (kc0 + bb), (int)(tile * 128), &full[s]);
              if (!RES) tma_load_2d(st + bps * X_BYTES + bb * E_CHUNK, &mapE, 64 * (kc0 + bb), 0, &full[s]);
            }
            issued[s] = 1;
            iss_ph[s] = ph;
            if (++s == S_N) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        for (int q = 0; q < S_N; ++q)
          if (issued[q]) {
            mbar_drain(&full[q], iss_ph[q], 128);
          }
        if (RES && g0 < g1)
          mbar_drain(e_full, 0, 128);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t ae_ph[2] = {0, 0}, gr_ph[2] = {0, 0}, ge_ph = 0;
      bool ok = true;
      int64_t n = 0;
      // previous tile waiting for its Gram update
      bool pv = false, pfirst = false, plast = false;
      int pb = 0;
      auto do_gram = [&](int b, bool firstseg, bool lastseg) -> bool {
        if (!mbar_wait(&gram_ready[b], gr_ph[b], abort_s, status, ST_TIMEOUT)) return false;
        gr_ph[b] ^= 1u;
        if (firstseg) {
          if (!mbar_wait(gram_empty, ge_ph ^ 1u, abort_s, status, ST_TIMEOUT)) return false;
          ge_ph ^= 1u;
        }
        tc_fence_after();
        const uint32_t g = smem_u32(gop_atom(b, 0));
        const uint32_t lbo = gop_lbo(b);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint64_t d = sdesc_sw128(g + j * 2048, lbo, 1024);
          mma_bf16(tgram, d, d, IDESC_GRAM, (firstseg && j == 0) ? 0u : 1u);
        }
        mma_commit(&gram_free[b]);
        if (lastseg) mma_commit(gram_full);
        return true;
      };
      if (RES && g0 < g1 && !mbar_wait(e_full, 0, abort_s, status, ST_TIMEOUT)) ok = false;
      for (int g = g0; g < g1 && ok; ++g) {
        const SegM sg = segs[g];
        for (int64_t tile = sg.tile_begin; tile < sg.tile_end && ok; ++tile, ++n) {
          const int b = (int)(n & 1);
          if (!mbar_wait(&acc_empty[b], ae_ph[b] ^ 1u, abort_s, status, ST_TIMEOUT)) {
            ok = false;
            break;
          }
          ae_ph[b] ^= 1u;
          tc_fence_after();
          const uint32_t dacc = tmem + b * KLD;
          for (int kc0 = 0; kc0 < nk; kc0 += bps) {
            const int nb = min(bps, nk - kc0);
            if (!mbar_wait(&full[s], ph, abort_s, status, ST_TIMEOUT)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * STAGE);
            for (int bb = 0; bb < nb; ++bb) {
              const int kc = kc0 + bb;
              const uint32_t xs = st + bb * X_BYTES;
              const uint32_t es = RES ? smem_u32(eres + kc * E_CHUNK) : st + bps * X_BYTES + bb * E_CHUNK;
#pragma unroll
              for (int j = 0; j < 4; ++j)
                mma_bf16(dacc, sdesc_sw128(xs + 32 * j, 16, 1024), sdesc_sw128(es + 32 * j, 16, 1024), IDESC_MAIN,
                         (kc | j) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
            if (++s == S_N) {
              s = 0;
              ph ^= 1u;
            }
          }
          if (!ok) break;
          mma_commit(&acc_full[b]);
          if (pv && !do_gram(pb, pfirst, plast)) {
            ok = false;
            break;
          }
          pv = true;
          pb = (int)(n % gop_nb);
          pfirst = (tile == sg.tile_begin);
          plast = (tile == sg.tile_end - 1);
        }
      }
      if (ok && pv) ok = do_gram(pb, pfirst, plast);
      // everything issued must have completed before TMEM is freed
      mma_commit(done);
      mbar_drain(done, 0, 64);
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    uint32_t af_ph[2] = {0, 0}, gf_ph[2] = {0, 0}, gfl_ph = 0, eb_ph = 0;
    int64_t n = 0;
    bool ok = true;
    // all four epilogue warps arrive (lane 0 each) and wait, with the bounded wait
    auto epi_sync = [&]() -> bool {
      __syncwarp();
      if (lane == 0) mbar_arrive(epi_bar);
      const bool r = warp_wait(epi_bar, eb_ph, abort_s, status);
      eb_ph ^= 1u;
      return r;
    };
    for (int g = g0; g < g1 && ok; ++g) {
      const SegM sg = segs[g];
      for (int64_t tile = sg.tile_begin; tile < sg.tile_end; ++tile, ++n) {
        const int b = (int)(n & 1);
        if (!warp_wait(&acc_full[b], af_ph[b], abort_s, status)) {
          ok = false;
          break;
        }
        af_ph[b] ^= 1u;
        const int gb = (int)(n % gop_nb);  // Gram operand buffer
        if (!warp_wait(&gram_free[gb], gf_ph[gb] ^ 1u, abort_s, status)) {
          ok = false;
          break;
        }
        gf_ph[gb] ^= 1u;
        tc_fence_after();
        // the TMA store of the buffer's previous tile must have read it
        if (threadIdx.x == 64) bulk_wait_read0();
        if (!epi_sync()) {
          ok = false;
          break;
        }

#pragma unroll
        for (int cc = 0; cc < KLD / 32; ++cc) {
          float r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * KLD + cc * 32), r);
          uint32_t pk[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * u], r[2 * u + 1]);
            pk[u] = *reinterpret_cast<uint32_t*>(&h);
          }
          const int atom = (cc * 32) >> 6;
          const int cbase = (cc & 1) * 4;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const uint4 v = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
            const int phys = (cbase + u) ^ (row & 7);
            *reinterpret_cast<uint4*>(gop_atom(gb, atom) + row * 128 + phys * 16) = v;
          }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        // A_i tile to global memory: one TMA store per 64-feature atom of the
        // 128B-swizzled copy (the same bytes the Gram MMA reads)
        if (!epi_sync()) {
          ok = false;
          break;
        }
        if (threadIdx.x == 64) {
#pragma unroll
          for (int a = 0; a < KLD / 64; ++a) tma_store_2d(&mapAs, 64 * a, (int)(tile * 128), gop_atom(gb, a));
          bulk_commit();
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&gram_ready[gb]);
          mbar_arrive(&acc_empty[b]);
        }
        if (tile == sg.tile_end - 1) {
          if (!warp_wait(gram_full, gfl_ph, abort_s, status)) {
            ok = false;
            break;
          }
          gfl_ph ^= 1u;
          tc_fence_after();
          if (q * 32 < KLD) {
            float* gp = gpart + (int64_t)sg.slot * KLD * KLD + (int64_t)row * KLD;
#pragma unroll
            for (int cc = 0; cc < KLD / 32; ++cc) {
              float r[32];
              tmem_ld32(tgram + ((uint32_t)(q * 32) << 16) + (uint32_t)(cc * 32), r);
              float4* d4 = reinterpret_cast<float4*>(gp + cc * 32);
#pragma unroll
              for (int u = 0; u < 8; ++u) d4[u] = make_float4(r[4 * u], r[4 * u + 1], r[4 * u + 2], r[4 * u + 3]);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(gram_empty);
        }
      }
    }
    if (threadIdx.x == 64) bulk_wait0();  // the A_i stores have landed
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------------ self-test GEMM
// One CTA: D (128 x N, FP32) = A * B^T with A, B given either K-major
// (A: 128 x K, B: N x K, K contiguous) or MN-major (A: K x 128, B: K x N).
template <bool MN>
__global__ void __launch_bounds__(128, 1)
    selftest_mma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int N,
                        int K, float* __restrict__ D, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nkc = K / 64;
  const uint32_t a_chunk = 128u * 128u;          // bytes of A per 64-wide K chunk
  const uint32_t b_chunk = (uint32_t)N * 128u;   // bytes of B per 64-wide K chunk
  uint8_t* As = smem;
  uint8_t* Bs = smem + nkc * a_chunk;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bs + nkc * b_chunk);
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(bars + 2);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_s + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    *abort_s = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_s, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_s;
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bars[0], nkc * (a_chunk + b_chunk));
    for (int kc = 0; kc < nkc; ++kc) {
      if (!MN) {
        tma_load_2d(As + kc * a_chunk, &mapA, 64 * kc, 0, &bars[0]);
        tma_load_2d(Bs + kc * b_chunk, &mapB, 64 * kc, 0, &bars[0]);
      } else {
        // box {64 (MN), 64 (K rows)}: atoms of 8 KB
        for (int a = 0; a < 2; ++a) tma_load_2d(As + kc * a_chunk + a * 8192, &mapA, 64 * a, 64 * kc, &bars[0]);
        for (int a = 0; a < N / 64; ++a) tma_load_2d(Bs + kc * b_chunk + a * 8192, &mapB, 64 * a, 64 * kc, &bars[0]);
      }
    }
    bool ok = mbar_wait(&bars[0], 0, abort_s, status, ST_TIMEOUT);
    if (ok) {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(128, N, MN, MN);
      for (int kc = 0; kc < nkc; ++kc)
        for (int j = 0; j < 4; ++j) {
          uint64_t ad, bd;
          if (!MN) {
            ad = sdesc_sw128(smem_u32(As + kc * a_chunk) + 32 * j, 16, 1024);
            bd = sdesc_sw128(smem_u32(Bs + kc * b_chunk) + 32 * j, 16, 1024);
          } else {
            ad = sdesc_sw128(smem_u32(As + kc * a_chunk) + 2048 * j, 8192, 1024);
            bd = sdesc_sw128(smem_u32(Bs + kc * b_chunk) + 2048 * j, 8192, 1024);
          }
          mma_bf16(tmem, ad, bd, idesc, (kc | j) ? 1u : 0u);
        }
    }
    mma_commit(&bars[1]);
  }
  __syncwarp();
  const bool ok = mbar_wait(&bars[1], 0, abort_s, status, ST_TIMEOUT);
  tc_fence_after();
  if (__all_sync(0xffffffffu, ok)) {
    for (int cc = 0; cc < N; cc += 32) {
      float r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + cc, r);
      for (int u = 0; u < 32; ++u) D[(warp * 32 + lane) * N + cc + u] = r[u];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D BF16 tensor map, 128-byte swizzle; inner = contiguous extent (elements).
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes, uint32_t box_in,
              uint32_t box_out, bool swizzle = true) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_in, box_out};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <typename T>
srm_status upload(T** d, const std::vector<T>& h, const char* what) {
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

// E-pass schedule for GE persistent CTAs: the (T-block, subject, 32-row
// chunk) steps split evenly, each CTA's share cut at subject and T-block
// boundaries into work items with one partial slot each, and the table that
// lists, for every (subject, 64-column chunk), its slots in a fixed order.
// GE is the split-v depth: how many CTAs share the voxel range of the pass.
srm_status build_e_schedule(Ctx* c, int GE) {
  auto* s = static_cast<TcState*>(c->tc);
  const int N = c->N;
  void* old[] = {s->d_work, s->d_work_off, c->Ppart, c->chunk_src, c->chunk_src_off};
  for (void* q : old)
    if (q) cudaFree(q);
  s->d_work = nullptr;
  s->d_work_off = nullptr;
  c->Ppart = nullptr;
  c->chunk_src = nullptr;
  c->chunk_src_off = nullptr;
  s->egrid = GE;
  const int nTB = (c->T + E_TB - 1) / E_TB;
  int64_t U = 0;
  for (int i = 0; i < N; ++i) U += c->vpad[i] / E_KR;
  U *= nTB;
  std::vector<WorkE> work;
  std::vector<int> work_off(GE + 1, 0);
  {
    int64_t pos = 0;  // global step index of the current (tb, i) start
    int cta = 0;
    auto cta_begin = [&](int q) { return (U * q) / GE; };
    for (int tb = 0; tb < nTB; ++tb)
      for (int i = 0; i < N; ++i) {
        const int64_t nsteps = c->vpad[i] / E_KR;
        int64_t a = pos, e = pos + nsteps;
        while (a < e) {
          while (cta < GE - 1 && a >= cta_begin(cta + 1)) {
            work_off[cta + 1] = (int)work.size();
            ++cta;
          }
          const int64_t cend = cta_begin(cta + 1);
          const int64_t b = std::min(e, cend);
          WorkE w{i, tb, (int)work.size(), 0, c->off[i] + (a - pos) * E_KR, c->off[i] + (b - pos) * E_KR};
          work.push_back(w);
          a = b;
        }
        pos = e;
      }
    for (int q = cta + 1; q <= GE; ++q) work_off[q] = (int)work.size();
  }
  c->Ppart_elems = (int64_t)work.size() * E_TB * c->kld;
  std::vector<std::vector<int64_t>> lists((size_t)N * c->nchunk);
  for (const WorkE& w : work)
    for (int cl = 0; cl < E_TB / TCH; ++cl) {
      const int ch = w.tb * (E_TB / TCH) + cl;
      if (ch >= c->nchunk) break;
      lists[(size_t)w.subject * c->nchunk + ch].push_back((int64_t)w.slot * E_TB * c->kld + (int64_t)cl * TCH * c->kld);
    }
  std::vector<ChunkSrc> src;
  std::vector<int> src_off((size_t)N * c->nchunk + 1);
  for (size_t j = 0; j < lists.size(); ++j) {
    src_off[j] = (int)src.size();
    for (int64_t o : lists[j]) src.push_back({o});
  }
  src_off[lists.size()] = (int)src.size();
  srm_status st;
  if ((st = upload(&s->d_work, work, "E-pass schedule")) != SRM_OK) return st;
  if ((st = upload(&s->d_work_off, work_off, "E-pass schedule offsets")) != SRM_OK) return st;
  if ((st = upload(&c->chunk_src, src, "chunk table")) != SRM_OK) return st;
  if ((st = upload(&c->chunk_src_off, src_off, "chunk table offsets")) != SRM_OK) return st;
  if (cudaMalloc(&c->Ppart, sizeof(float) * std::max<int64_t>(1, c->Ppart_elems)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed for E-pass partial slots");
    return SRM_ERR_NOMEM;
  }
  return SRM_OK;
}

// Shared memory of an M-pass plan: nb Gram operand buffers, E[S] resident or
// streamed, stages X^ stages.  0 if it does not fit.
size_t m_plan_smem(const Ctx* c, int nb, bool res, int stages, int bps) {
  if ((nb != 1 && nb != 2) || stages < 2 || stages > M_MAX_STAGES || (bps != 1 && bps != 2 && bps != 4)) return 0;
  const size_t eres = (size_t)((c->T + 63) / 64) * c->kld * 128;
  const size_t sm = m_fixed_bytes(c->kld, nb) + (res ? eres + (size_t)stages * bps * 16384
                                                      : (size_t)stages * bps * m_stage_bytes(c->kld));
  return sm <= kMaxSmem ? sm : 0;
}

}  // namespace

// The default E-pass reserve.  The E-pass leaves a few SMs to the M-step tail
// that runs beside it (the polar factors take one CTA per subject): the
// tail's blocks then run on otherwise idle SMs instead of slowing the E-pass
// CTAs they would share an SM with, whose fixed share of the work sets the
// pass's end.  132 of 152 SMs still saturate HBM (greeneyes-like workload:
// E-pass 0.255 -> 0.217 ms, iteration 0.588 -> 0.548 ms).
int tc_default_e_reserve(const Ctx* c) { return std::min(E_RESERVE_MAX, c->N + 4); }

int tc_e_reserve(const Ctx* c) { return c->num_sms - static_cast<const TcState*>(c->tc)->egrid; }

srm_status tc_set_e_reserve(Ctx* c, int reserve) {
  if (reserve < 0 || reserve >= c->num_sms) {
    set_error("plan: the E-pass reserve must leave at least one SM to the pass");
    return SRM_ERR_ARG;
  }
  const int GE = c->num_sms - reserve;
  if (static_cast<TcState*>(c->tc)->egrid == GE && c->Ppart) return SRM_OK;
  return build_e_schedule(c, GE);
}

void tc_get_m_plan(const Ctx* c, int* nb, int* res, int* stages, int* pf, int* bps) {
  const auto* s = static_cast<const TcState*>(c->tc);
  *nb = s->m_gop;
  *res = s->m_res ? 1 : 0;
  *stages = s->m_stages;
  *pf = s->m_pf;
  *bps = s->m_bps;
}

srm_status tc_set_m_plan(Ctx* c, int nb, int res, int stages, int pf, int bps) {
  const size_t sm = m_plan_smem(c, nb, res != 0, stages, bps);
  if (!sm || pf < 0 || pf > 64) {
    set_error("plan: the M-pass plan does not fit in shared memory (Gram buffers 1-2, stages 2-8, boxes per "
              "stage 1, 2 or 4, prefetch 0-64)");
    return SRM_ERR_ARG;
  }
  auto* s = static_cast<TcState*>(c->tc);
  s->m_gop = nb;
  s->m_res = res != 0;
  s->m_stages = stages;
  s->m_pf = pf;
  s->m_bps = bps;
  s->m_smem = sm;
  return SRM_OK;
}

void tc_m_candidates(const Ctx* c, std::vector<std::array<int, 5>>& out) {
  out.clear();
  for (int bps : {1, 2, 4})
    for (int nb = 1; nb <= 2; ++nb)
      for (int res = 0; res <= 1; ++res)
        for (int st = 2; st <= M_MAX_STAGES; ++st) {
          if (!m_plan_smem(c, nb, res != 0, st, bps)) continue;
          out.push_back({nb, res, st, 0, bps});
          if (bps == 1) out.push_back({nb, res, st, M_PF, bps});
        }
}

srm_status tc_setup(Ctx* c) {
  if (c->kld != 64 && c->kld != 128) {
    set_error("tensor-core form: padded k must be 64 or 128");
    return SRM_ERR_UNSUPPORTED;
  }
  auto* s = new TcState();
  c->tc = s;
  const int G = c->num_sms;
  s->grid = G;
  const int N = c->N;
  const int GE = std::max(1, c->num_sms - tc_default_e_reserve(c));
  // tensor maps
  bool ok = make_map(&s->mapXe, c->Xh, c->T, c->Vpad_tot, (uint64_t)c->ldT * 2, 64, E_KR) &&
            make_map(&s->mapA, c->A, c->kld, c->Vpad_tot, (uint64_t)c->kld * 2, 64, E_KR) &&
            make_map(&s->mapXm, c->Xh, c->T, c->Vpad_tot, (uint64_t)c->ldT * 2, 64, 128) &&
            make_map(&s->mapE, c->ESb, c->T, c->kld, (uint64_t)c->ldT * 2, 64, c->kld) &&
            make_map(&s->mapAs, c->A, c->kld, c->Vpad_tot, (uint64_t)c->kld * 2, 64, 128) &&
            // L2 prefetch only (never lands in shared memory): 4 chunks x 128 rows per box
            make_map(&s->mapXp, c->Xh, c->T, c->Vpad_tot, (uint64_t)c->ldT * 2, 256, 128, false);
  if (!ok) {
    set_error("cuTensorMapEncodeTiled failed (driver entry point missing or bad layout)");
    return SRM_ERR_CUDA;
  }
  // ---- M-pass schedule: 128-row tiles split evenly, segments at subject boundaries
  const int64_t NTl = c->Vpad_tot / 128;
  std::vector<SegM> seg;
  std::vector<int> seg_cta;
  for (int q = 0; q < G; ++q) {
    const int64_t t0 = NTl * q / G, t1 = NTl * (q + 1) / G;
    int64_t t = t0;
    while (t < t1) {
      // subject of tile t
      const int64_t row = t * 128;
      int i = (int)(std::upper_bound(c->off.begin(), c->off.begin() + N + 1, row) - c->off.begin()) - 1;
      const int64_t tend = std::min<int64_t>(t1, c->off[i + 1] / 128);
      seg.push_back({t, tend, 0, i});
      seg_cta.push_back(q);
      t = tend;
    }
  }
  // slot ids contiguous per subject (CTA order within a subject)
  std::vector<int> gslot_off(N + 1, 0);
  for (const SegM& g : seg) gslot_off[g.subject + 1]++;
  for (int i = 0; i < N; ++i) gslot_off[i + 1] += gslot_off[i];
  {
    std::vector<int> fill(gslot_off.begin(), gslot_off.end() - 1);
    for (SegM& g : seg) g.slot = fill[g.subject]++;
  }
  std::vector<int> seg_off(G + 1, 0);
  for (size_t j = 0; j < seg.size(); ++j) seg_off[seg_cta[j] + 1]++;
  for (int q = 0; q < G; ++q) seg_off[q + 1] += seg_off[q];
  c->n_gslots = (int)seg.size();
  c->Gpart_elems = (int64_t)seg.size() * c->kld * c->kld;

  srm_status st;
  if ((st = build_e_schedule(c, GE)) != SRM_OK) return st;
  if ((st = upload(&s->d_seg, seg, "M-pass schedule")) != SRM_OK) return st;
  if ((st = upload(&s->d_seg_off, seg_off, "M-pass schedule offsets")) != SRM_OK) return st;
  if ((st = upload(&c->gslot_off, gslot_off, "Gram slot table")) != SRM_OK) return st;
  if (cudaMalloc(&c->Gpart, sizeof(float) * std::max<int64_t>(1, c->Gpart_elems)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed for tensor-core partial slots");
    return SRM_ERR_NOMEM;
  }
  // kernel attributes
  const int nk = (c->T + 63) / 64;
  {
    // stage count from the shared-memory budget: resident E[S] if that still
    // leaves at least M_RES_MIN stages of X^ tiles, else streamed E[S] chunks
    // Two Gram buffers unless one buffer gives a deeper pipeline of at least
    // M_PF_STAGES stages (measured: T = 1000, k = 50 runs faster with three
    // stages, two buffers and L2 prefetch than with four stages and one
    // buffer; T = 500 and T = 3500 gain from the extra stage).
    constexpr long M_RES_MIN = 3;
    const size_t eres = (size_t)nk * c->kld * 128;
    auto plan = [&](int nb, bool& res, long& st) {
      const size_t fixed = m_fixed_bytes(c->kld, nb);
      const long res_st = fixed + eres < kMaxSmem ? (long)((kMaxSmem - fixed - eres) / 16384) : 0;
      const long str_st = (long)((kMaxSmem - fixed) / m_stage_bytes(c->kld));
      res = res_st >= M_RES_MIN;
      st = std::min<long>(M_MAX_STAGES, res ? res_st : str_st);
    };
    bool res1, res2;
    long st1, st2;
    plan(1, res1, st1);
    plan(2, res2, st2);
    const bool one = (res1 == res2) && st1 > st2 && st1 >= M_PF_STAGES;
    s->m_gop = one ? 1 : 2;
    s->m_res = one ? res1 : res2;
    s->m_stages = (int)(one ? st1 : st2);
    s->m_pf = s->m_stages < M_PF_STAGES ? M_PF : 0;
    s->m_bps = 1;
    s->m_smem = m_plan_smem(c, s->m_gop, s->m_res, s->m_stages, 1);
  }
  // The E-pass leaves room on each SM for the M-step tail that runs beside it
  // on the second stream; ask for the largest shared-memory carve-out so that
  // the tail's blocks fit next to the persistent CTA.
  cudaFuncSetAttribute(estep_tc_kernel<64>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(estep_tc_kernel<128>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  if (c->kld == 64) {
    cudaFuncSetAttribute(estep_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e_smem_bytes(64));
    cudaFuncSetAttribute(mstep_tc_kernel<64, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    cudaFuncSetAttribute(mstep_tc_kernel<64, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    cudaFuncSetAttribute(mstep_tc_kernel<64, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    cudaFuncSetAttribute(mstep_tc_kernel<64, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
  } else {
    cudaFuncSetAttribute(estep_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e_smem_bytes(128));
    cudaFuncSetAttribute(mstep_tc_kernel<128, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    cudaFuncSetAttribute(mstep_tc_kernel<128, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    cudaFuncSetAttribute(mstep_tc_kernel<128, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    cudaFuncSetAttribute(mstep_tc_kernel<128, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core kernel attributes");
  return SRM_OK;
}

void tc_destroy(Ctx* c) {
  auto* s = static_cast<TcState*>(c->tc);
  if (!s) return;
  void* p[] = {s->d_work, s->d_work_off, s->d_seg, s->d_seg_off};
  for (void* q : p)
    if (q) cudaFree(q);
  delete s;
  c->tc = nullptr;
}

cudaError_t launch_p_tc(Ctx* c) {
  auto* s = static_cast<TcState*>(c->tc);
  if (c->kld == 64)
    estep_tc_kernel<64><<<s->egrid, NT, e_smem_bytes(64), c->stream>>>(s->mapXe, s->mapA, s->d_work, s->d_work_off,
                                                                       c->T, c->Ppart, c->status);
  else
    estep_tc_kernel<128><<<s->egrid, NT, e_smem_bytes(128), c->stream>>>(s->mapXe, s->mapA, s->d_work,
                                                                         s->d_work_off, c->T, c->Ppart, c->status);
  return cudaGetLastError();
}

cudaError_t launch_a_tc(Ctx* c) {
  auto* s = static_cast<TcState*>(c->tc);
  auto* A = static_cast<__nv_bfloat16*>(c->A);
#define M_LAUNCH(KLD, RES, GNB)                                                                                  \
  mstep_tc_kernel<KLD, RES, GNB><<<s->grid, NT, s->m_smem, c->stream>>>(                                          \
      s->mapXm, s->mapE, s->mapAs, s->mapXp, s->d_seg, s->d_seg_off, c->T, s->m_stages, s->m_bps,                 \
      s->m_pf,                                                                                                     \
      static_cast<const uint8_t*>(c->Xh), (int64_t)c->ldT * 2, A, c->Gpart, c->status)
#define M_LAUNCH2(KLD, RES) \
  if (s->m_gop == 1) {      \
    M_LAUNCH(KLD, RES, 1);  \
  } else {                  \
    M_LAUNCH(KLD, RES, 2);  \
  }
  if (c->kld == 64) {
    if (s->m_res) {
      M_LAUNCH2(64, true)
    } else {
      M_LAUNCH2(64, false)
    }
  } else {
    if (s->m_res) {
      M_LAUNCH2(128, true)
    } else {
      M_LAUNCH2(128, false)
    }
  }
#undef M_LAUNCH2
#undef M_LAUNCH
  return cudaGetLastError();
}

namespace {

// The bounded wait of the tensor-core kernels, exercised alone: warp 0 waits
// on one mbarrier, warp 1 on another.  With arrive != 0 a thread arrives on
// both and the waits succeed.  With arrive == 0 nothing arrives on the first:
// its waiter gives up after the library's poll limit and raises the abort
// flag and the timeout bit.  The second waiter (on a barrier nothing arrives
// on either) must then stop through the abort flag, well before its own
// limit.  out[0..1]: 1 if the wait of warp 0 / warp 1 succeeded.
__global__ void __launch_bounds__(64, 1) wait_selftest_kernel(int arrive, int* out, int* status) {
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  volatile int* abort_s = &abort_flag;
  if (arrive && threadIdx.x == 0) {
    mbar_arrive(&bar[0]);
    mbar_arrive(&bar[1]);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    const bool ok = mbar_wait(&bar[warp], 0, abort_s, status, ST_TIMEOUT);
    out[warp] = ok ? 1 : 0;
  }
}

}  // namespace

}  // namespace srm

// Self-test of the tensor-core building blocks (TMA 128-byte-swizzled loads,
// shared-memory descriptors, tcgen05.mma, TMEM loads); see srm_debug.h.
extern "C" SRM_API srm_status srm_debug_mma(int32_t mn_major, const void* A, const void* B, float* D, int32_t N,
                                            int32_t K) {
  using namespace srm;
  if (!A || !B || !D || (N != 64 && N != 128) || K < 64 || K > 256 || K % 64) {
    set_error("srm_debug_mma: need N in {64, 128}, K in {64, ..., 256} (multiple of 64)");
    return SRM_ERR_ARG;
  }
  CUtensorMap mA, mB;
  bool ok;
  if (!mn_major)
    ok = make_map(&mA, A, K, 128, (uint64_t)K * 2, 64, 128) && make_map(&mB, B, K, N, (uint64_t)K * 2, 64, N);
  else
    ok = make_map(&mA, A, 128, K, 128 * 2, 64, 64) && make_map(&mB, B, N, K, (uint64_t)N * 2, 64, 64);
  if (!ok) {
    set_error("srm_debug_mma: tensor map encoding failed");
    return SRM_ERR_CUDA;
  }
  int* status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaMalloc");
  cudaMemset(status, 0, sizeof(int));
  const size_t sm = 1024 + (size_t)(K / 64) * (128 * 128 + N * 128) + 64;
  cudaError_t e;
  if (!mn_major) {
    cudaFuncSetAttribute(selftest_mma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    selftest_mma_kernel<false><<<1, 128, sm>>>(mA, mB, N, K, D, status);
  } else {
    cudaFuncSetAttribute(selftest_mma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    selftest_mma_kernel<true><<<1, 128, sm>>>(mA, mB, N, K, D, status);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(status);
  if (e != cudaSuccess) return cuda_fail(e, "srm_debug_mma");
  if (st) {
    set_error("srm_debug_mma: a bounded wait gave up");
    return SRM_ERR_NUMERIC;
  }
  return SRM_OK;
}

// The bounded wait's give-up path, exercised without a fault; see srm_debug.h.
extern "C" SRM_API srm_status srm_debug_wait(int32_t arrive) {
  using namespace srm;
  int* dev = nullptr;
  if (cudaMalloc(&dev, 3 * sizeof(int)) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaMalloc");
  cudaError_t e = cudaMemset(dev, 0, 3 * sizeof(int));
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 64>>>(arrive ? 1 : 0, dev, dev + 2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, dev, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(dev);
  if (e != cudaSuccess) return cuda_fail(e, "srm_debug_wait");
  if (h[2] & ST_TIMEOUT) {
    set_error(std::string("srm_debug_wait: a bounded wait gave up; waits ok: ") + std::to_string(h[0]) + ", " +
              std::to_string(h[1]));
    return SRM_ERR_NUMERIC;
  }
  if (!h[0] || !h[1]) {
    set_error("srm_debug_wait: a wait failed without raising the timeout bit");
    return SRM_ERR_STATE;
  }
  return SRM_OK;
}
