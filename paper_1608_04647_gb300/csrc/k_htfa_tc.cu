// HTFA local objective ||X_i - W_i F_i||_F^2 (Sec. III-B, the Frobenius term of
// eq:htfa_subject_update_rbfs) on the tensor cores, for K <= 128.
//
// The product W F is formed to FP32 accuracy from BF16 pieces.  Each FP32
// value is split as x = x1 + x2 + x3, with x1 = bf16(x), x2 = bf16(x - x1) and
// x3 = bf16(x - x1 - x2) (each difference exact in FP32).  BF16 keeps eight
// significant bits (unit roundoff 2^-8), so |x - x1 - x2 - x3| <= 2^-24 |x|,
// the unit roundoff of FP32 itself.  Then
//   W F = (W1F3 + W2F2 + W3F1) + (W1F2 + W2F1) + W1F1 + e,
//   |e| <= 4 u |W||F|  (u = 2^-24: the pieces' remainders and the three
//   dropped products W2F3, W3F2, W3F3),
// six tcgen05 MMAs (kind::f16, BF16 in, FP32 accumulate) per 16-wide K step.
// They accumulate into one TMEM tile, smallest terms first, so the large
// products do not swamp the small ones.  Every product of two BF16 values
// is exact in FP32; the accumulator rounds once per MMA, 6 ceil(K / 16)
// times, where the FP32 form rounds K times.
//
// Block work: one subject i, one 128-row T tile, Q consecutive 64-column V
// tiles.  Warps 0-6 convert: W_i's tile once into three K-major pieces (two
// 64-wide K atoms each, 128-byte swizzle), then each F tile into three
// MN-major pieces, double-buffered so that the next tile is converted while
// the MMAs of the current one run.  X, W and F are read with plain coalesced
// loads, since their rows need not be 16-byte aligned for TMA.  Warp 7 issues
// the MMAs into two TMEM accumulators (128 lanes x 64 columns each).  Warps
// 8-11 read an accumulator (TMEM lane = row t), subtract it from X, square,
// and sum: FP32 per thread, a fixed-order shuffle tree to one FP64 partial
// per warp and tile.  The partials are summed in a fixed order by a second
// kernel, so repeated calls give identical bits.  Every wait is bounded; a block that
// gives up raises the status bit and stops issuing work.
#include <math.h>

#include "srm_internal.cuh"
#include "tc_ptx.cuh"

namespace srm {

using namespace tc;

namespace {

constexpr int HT_M = 128;            // rows (t) per tile
constexpr int HT_N = 64;             // columns (v) per tile
constexpr int HT_THREADS = 384;      // 12 warps: 0-6 convert, 7 MMA, 8-11 epilogue
constexpr int HT_CONV = 224;         // converter threads
constexpr int HT_MMA_WARP = HT_CONV / 32;
constexpr uint32_t W_ATOM = 16384;   // 128 rows x 64 K BF16
constexpr uint32_t W_PIECE = 2 * W_ATOM;
constexpr uint32_t F_PIECE = 128 * 128;  // up to 128 K rows x 64 v BF16
constexpr int XS_LD = HT_N + 1;      // staged X rows (floats), padded against bank conflicts
constexpr uint32_t XS_BYTES = 4u * 32u * XS_LD * 4u;  // four epilogue warps x 32 rows
constexpr size_t ht_smem_bytes() {
  return 1024 + 3 * (size_t)W_PIECE + 2 * 3 * (size_t)F_PIECE + XS_BYTES + 256;
}
static_assert(ht_smem_bytes() <= 232448, "HTFA residual shared memory");

// two values -> their adjacent 2-byte slots (4-byte aligned offset off) in
// each of the three pieces, with paired conversions
__device__ __forceinline__ void store_split2(float x0, float x1, uint8_t* p0, uint32_t piece_bytes, uint32_t off) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(x0, x1);
  const float2 af = __bfloat1622float2(a);
  const float r0 = x0 - af.x, r1 = x1 - af.y;
  const __nv_bfloat162 b = __floats2bfloat162_rn(r0, r1);
  const float2 bf = __bfloat1622float2(b);
  const __nv_bfloat162 c = __floats2bfloat162_rn(r0 - bf.x, r1 - bf.y);
  *reinterpret_cast<__nv_bfloat162*>(p0 + off) = a;
  *reinterpret_cast<__nv_bfloat162*>(p0 + piece_bytes + off) = b;
  *reinterpret_cast<__nv_bfloat162*>(p0 + 2 * piece_bytes + off) = c;
}

__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort, status, ST_TIMEOUT);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// grid (ceil(tiles_v / Q), ceil(T / 128), n_subj)
__global__ void __launch_bounds__(HT_THREADS, 1)
    htfa_residual_tc_kernel(int K, int T, int V, int tiles_v, int tiles, int Q, const float* __restrict__ X,
                            const float* __restrict__ W, const float* __restrict__ F, double* __restrict__ part,
                            int* status) {
  extern __shared__ uint8_t ht_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ht_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* wp = smem;                      // [3] W pieces
  uint8_t* fp = smem + 3 * W_PIECE;        // [2][3] F pieces
  float* xs = reinterpret_cast<float*>(fp + 6 * F_PIECE);  // [4][32][XS_LD] staged X rows
  uint64_t* w_full = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(xs) + XS_BYTES);
  uint64_t* f_full = w_full + 1;           // [2]
  uint64_t* f_empty = f_full + 2;          // [2]
  uint64_t* acc_full = f_empty + 2;        // [2]
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_s = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_s + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = blockIdx.z, mt = blockIdx.y;
  const int t0 = mt * HT_M;
  const int vt0 = blockIdx.x * Q, vt1 = min(tiles_v, vt0 + Q);
  const int Kp = (K + 15) & ~15;  // K padded to whole MMA steps (zeros)
  const int ks = Kp / 16;

  if (threadIdx.x == 0) {
    mbar_init(w_full, HT_CONV / 32);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&f_full[b], HT_CONV / 32);
      mbar_init(&f_empty[b], 1);
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(done, 1);
    *abort_s = 0;
    fence_mbar_init();
  }
  if (warp == HT_MMA_WARP) {
    tmem_alloc(tmem_s, 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_s;
  const float* Xn = X + (int64_t)n * T * V;
  const float* Wn = W + (int64_t)n * T * K;
  const float* Fn = F + (int64_t)n * K * V;

  if (warp < HT_CONV / 32) {
    // ---- converters (HT_CONV threads): lane = two adjacent columns of one row,
    // so a warp's two loads cover 256 contiguous bytes; each pair is split with
    // paired conversions and stored in its 4-byte slots of the three swizzled
    // pieces.  The loads of a batch of rows are all issued before any is used,
    // and the F rows of the tile after next are requested from L2.
    const int cw = warp;  // converter warp
    constexpr int NCW = HT_CONV / 32;
    auto prefetch_f = [&](int vt) {
      if (vt >= vt1) return;
      const int v0 = vt * HT_N;
      for (int e = threadIdx.x; e < K * 2; e += HT_CONV) {  // two 128-byte lines per row of the tile
        const int k = e >> 1, h = e & 1;
        const int v = min(V - 1, v0 + 32 * h);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(Fn + (int64_t)k * V + v));
      }
    };
    prefetch_f(vt0);
    prefetch_f(vt0 + 1);
    // W tile: rows t0 .. t0 + 127 (warp cw takes rows cw, cw + NCW, ...), K padded to Kp
    for (int r0 = cw; r0 < HT_M; r0 += 8 * NCW) {
      float x[8][4];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int r = r0 + NCW * b, t = t0 + r;
#pragma unroll
        for (int h = 0; h < 4; ++h) {  // k = 64 (h / 2) + 2 lane + h % 2
          const int k = 64 * (h >> 1) + 2 * lane + (h & 1);
          x[b][h] = (r < HT_M && t < T && k < K) ? __ldg(Wn + (int64_t)t * K + k) : 0.f;
        }
      }
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int r = r0 + NCW * b;
        if (r >= HT_M) continue;
#pragma unroll
        for (int a = 0; a < 2; ++a) {  // the two K atoms
          const int k = 64 * a + 2 * lane;
          if (k >= Kp) continue;
          const int kk = 2 * lane;
          const uint32_t off = (uint32_t)a * W_ATOM + (uint32_t)r * 128u +
                               (uint32_t)((((kk >> 3) ^ (r & 7)) << 4) + ((kk & 7) << 1));
          store_split2(x[b][2 * a], x[b][2 * a + 1], wp, W_PIECE, off);
        }
      }
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(w_full);
    // F tiles: Kp rows x 64 columns; warp cw takes rows cw, cw + NCW, ...
    // A lane's whole share of a tile (at most ceil(128 / NCW) rows x 2) is
    // loaded in one batch, before the wait for the buffer it goes to: the
    // tile's bytes are all in flight at once and the wait overlaps them.
    constexpr int FR = (128 + NCW - 1) / NCW;  // rows per converter warp
    uint32_t fe_ph[2] = {0, 0};
    for (int vt = vt0, j = 0; vt < vt1; ++vt, ++j) {
      const int b = j & 1;
      const int v0 = vt * HT_N;
      float x[FR][2];  // columns 2 lane and 2 lane + 1 of each of the warp's rows
#pragma unroll
      for (int i = 0; i < FR; ++i) {
        const int k = cw + NCW * i;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int v = v0 + 2 * lane + h;
          x[i][h] = (k < K && v < V) ? __ldg(Fn + (int64_t)k * V + v) : 0.f;
        }
      }
      prefetch_f(vt + 2);
      if (j >= 2) {
        if (!warp_wait(&f_empty[b], fe_ph[b], abort_s, status)) break;
        fe_ph[b] ^= 1u;
      }
      uint8_t* fb = fp + (size_t)b * 3 * F_PIECE;
#pragma unroll
      for (int i = 0; i < FR; ++i) {
        const int k = cw + NCW * i;
        if (k >= Kp) continue;
        const int vl = 2 * lane;
        const uint32_t off = (uint32_t)k * 128u + (uint32_t)((((vl >> 3) ^ (k & 7)) << 4) + ((vl & 7) << 1));
        store_split2(x[i][0], x[i][1], fb, F_PIECE, off);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&f_full[b]);
    }
  } else if (warp == HT_MMA_WARP) {
    // ---- MMA issue: D[t][v] = sum_k W[t][k] F[k][v], six piece products per K step
    if (lane == 0) {
      constexpr uint32_t IDESC = idesc_bf16(HT_M, HT_N, false, true);  // A K-major, B MN-major
      bool ok = mbar_wait(w_full, 0, abort_s, status, ST_TIMEOUT);
      uint32_t ff_ph[2] = {0, 0}, ae_ph[2] = {0, 0};
      // piece pairs, smallest terms first: (1,3) (2,2) (3,1), (1,2) (2,1), (1,1)
      // piece of W and of F for each of the six products, 4 bits each (product 0
      // lowest): (1,3) (2,2) (3,1) (1,2) (2,1) (1,1), pieces counted from 0
      constexpr uint32_t pa = 0x010210u, pb = 0x001012u;
      for (int vt = vt0, j = 0; ok && vt < vt1; ++vt, ++j) {
        const int b = j & 1;
        if (!mbar_wait(&f_full[b], ff_ph[b], abort_s, status, ST_TIMEOUT)) break;
        ff_ph[b] ^= 1u;
        if (j >= 2) {
          if (!mbar_wait(&acc_empty[b], ae_ph[b], abort_s, status, ST_TIMEOUT)) break;
          ae_ph[b] ^= 1u;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)b * 64u;
        // descriptors of the pieces' first K step; a step's descriptor adds its
        // byte offset / 16 to the start-address field (bits 0-13), which every
        // shared-memory address here fits
        const uint64_t da0 = sdesc_sw128(smem_u32(wp), 16, 1024);
        const uint64_t db0 = sdesc_sw128(smem_u32(fp + (size_t)b * 3 * F_PIECE), F_PIECE, 1024);
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const uint32_t ia = (pa >> (4 * p)) & 15u, ib = (pb >> (4 * p)) & 15u;
#pragma unroll
          for (int st = 0; st < 8; ++st) {
            if (st >= ks) break;
            const uint64_t da = da0 + ((ia * W_PIECE + (uint32_t)(st >> 2) * W_ATOM + (uint32_t)(st & 3) * 32u) >> 4);
            const uint64_t db = db0 + ((ib * F_PIECE + (uint32_t)st * 2048u) >> 4);
            mma_bf16(d, da, db, IDESC, (p | st) ? 1u : 0u);
          }
        }
        mma_commit(&f_empty[b]);
        mma_commit(&acc_full[b]);
      }
      // everything issued has completed before TMEM is freed
      mma_commit(done);
      mbar_drain(done, 0, 64);
    }
  } else if (warp >= 8) {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows t0 + 32 q + lane)
    const int q = warp & 3;
    uint32_t af_ph[2] = {0, 0};
    float* xw = xs + (size_t)q * 32 * XS_LD;  // this warp's 32 staged rows
    {
      const int tt = t0 + 32 * q + lane;  // the first two tiles' lines of this lane's row, into L2
      for (int vt = vt0; vt < min(vt1, vt0 + 2) && tt < T; ++vt) {
        const int v0 = vt * HT_N;
        const float* nx = Xn + (int64_t)tt * V + v0;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(nx));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + min(32, V - v0 - 1)));
      }
    }
    for (int vt = vt0, j = 0; vt < vt1; ++vt, ++j) {
      const int b = j & 1;
      const int v0 = vt * HT_N;
      // the tile's X rows of this warp, coalesced (lane = column), staged in
      // shared memory: all 64 loads of a lane in flight at once, issued
      // before the wait for the product (they do not depend on it); the rows
      // of the tile after next are requested from L2 meanwhile
      {
        float x[32][2];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
          const int tt = t0 + 32 * q + rr;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int v = v0 + 32 * h + lane;
            x[rr][h] = (tt < T && v < V) ? __ldg(Xn + (int64_t)tt * V + v) : 0.f;
          }
        }
        if (vt + 2 < vt1) {
          const int tt = t0 + 32 * q + lane;  // lane: one row, its two lines of tile vt + 2
          if (tt < T) {
            const float* nx = Xn + (int64_t)tt * V + v0 + 2 * HT_N;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(nx));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + min(32, V - v0 - 2 * HT_N - 1)));
          }
        }
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
          xw[rr * XS_LD + lane] = x[rr][0];
          xw[rr * XS_LD + 32 + lane] = x[rr][1];
        }
      }
      __syncwarp();
      if (!warp_wait(&acc_full[b], af_ph[b], abort_s, status)) break;
      af_ph[b] ^= 1u;
      tc_fence_after();
      // lane = row: its staged X row against its accumulator row, in two halves
      // of 32 columns (padding rows and columns hold zeros on both sides)
      float s = 0.f;
      const float* xr = xw + lane * XS_LD;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float dv[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)b * 64u + 32u * h, dv);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const float r = xr[32 * h + c] - dv[c];
          s = fmaf(r, r, s);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);  // the accumulator is free for tile j + 2
      __syncwarp();  // the staged rows are read before the next tile overwrites them
      double dsum = s;
#pragma unroll
      for (int o = 16; o; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
      // one partial per epilogue warp (no barrier among the warps, whose waits
      // may give up independently); the sum kernel adds them in order
      if (lane == 0) part[((int64_t)n * tiles + (int64_t)mt * tiles_v + vt) * 4 + q] = dsum;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == HT_MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, 128);
  }
}

}  // namespace

size_t htfa_tc_smem_bytes() { return ht_smem_bytes(); }

bool htfa_tc_supported(int K) { return K >= 1 && K <= 128; }

int64_t htfa_tc_tiles(int T, int V) { return (int64_t)((T + HT_M - 1) / HT_M) * ((V + HT_N - 1) / HT_N); }

cudaError_t launch_htfa_residual_tc(int n_subj, int K, int T, int V, const float* X, const float* W, const float* F,
                                    double* part, int* status, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(htfa_residual_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ht_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int tiles_v = (V + HT_N - 1) / HT_N;
  const int mtiles = (T + HT_M - 1) / HT_M;
  const int tiles = tiles_v * mtiles;
  const int Q = 16;  // V tiles per block (the W tile is converted once per block)
  const dim3 grid((unsigned)((tiles_v + Q - 1) / Q), (unsigned)mtiles, (unsigned)n_subj);
  htfa_residual_tc_kernel<<<grid, HT_THREADS, ht_smem_bytes(), s>>>(K, T, V, tiles_v, tiles, Q, X, W, F, part,
                                                                    status);
  return cudaGetLastError();
}

}  // namespace srm
