// HTFA local-step evaluations (Sec. III, and the native extension modules of
// Sec. IV-A): the factor matrix F_i of Eq. 14, the residual
// ||X_i - W_i F_i||_F^2 of eq:htfa_subject_update_rbfs, and the per-voxel
// z-score.  Layouts follow the paper's HTFA notation: X_i is T x V (one
// sample per row), W_i is T x K, F_i is K x V; a batch of equal-sized
// subjects is stored back to back.
#include <algorithm>
#include <climits>
#include <string>

#include "htfa.h"
#include "srm_internal.cuh"

namespace srm {

namespace {

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

// ---------------------------------------------------------------------------
// Factor matrix (Eq. 14).  ||p - mu||^2 separates over the axes, so
//   F[k][v] = Ex[ix][k] * Ey[iy][k] * Ez[iz][k],  Ec[a][k] = exp(-(a_c - mu_kc)^2 / lambda_k).
// The first kernel evaluates the tables of every subject once (n (nx+ny+nz)
// K exponentials, laid out [n][a][Kp] with K padded to Kp, a multiple of 4,
// so that four factors of one axis position are one 16-byte load).  The
// second copies the tables of kc factors into shared memory and writes
// those kc rows of F for 1024 voxels: per four factors of a voxel, three
// 16-byte shared loads, eight multiplies and four coalesced stores.
constexpr int FV_THREADS = 256;
constexpr int F_SMEM_DEFAULT = 48 * 1024;

// a block covers 32 axis positions of one subject; a thread owns one factor
// (its center and width loaded once) and writes its 32 table entries
constexpr int TAB_ROWS = 32;

__global__ void __launch_bounds__(128) htfa_tables_kernel(int K, int Kp, int na, const float* __restrict__ axes,
                                                          int nx, int ny, const float* __restrict__ mu,
                                                          const float* __restrict__ lam, float* __restrict__ tab,
                                                          int* flag) {
  const int n = blockIdx.y;
  const int a0 = blockIdx.x * TAB_ROWS, a1 = min(na, a0 + TAB_ROWS);
  for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
    float* out = tab + (int64_t)n * na * Kp + k;
    if (k >= K) {
      for (int a = a0; a < a1; ++a) out[(int64_t)a * Kp] = 0.f;
      continue;
    }
    const int64_t f = (int64_t)n * K + k;
    const float l = lam[f];
    const bool ok = l > 0.f && l <= 3.402823466e38f;
    if (!ok && a0 == 0 && flag) atomicOr(flag, 2);
    const float m0 = mu[f * 3], m1 = mu[f * 3 + 1], m2 = mu[f * 3 + 2];
#pragma unroll 4
    for (int a = a0; a < a1; ++a) {
      const float d = axes[a] - (a < nx ? m0 : (a < nx + ny ? m1 : m2));
      out[(int64_t)a * Kp] = ok ? expf(-(d * d) / l) : qnan();
    }
  }
}

__global__ void __launch_bounds__(FV_THREADS) htfa_factors_kernel(int K, int Kp, int V, int kc, int ld, int vpt, int nx,
                                                                  int ny, int nz, const float* __restrict__ tab,
                                                                  const int* __restrict__ vox, float* __restrict__ F,
                                                                  int* flag) {
  extern __shared__ __align__(16) float ftab[];  // [na][ld], factors k0 .. k0 + kc - 1
  const int n = blockIdx.z;
  const int k0 = blockIdx.y * kc;
  const int kn = min(kc, K - k0);
  const int q4 = (kn + 3) >> 2;
  const int na = nx + ny + nz;
  // the voxels' grid indices first, so that their loads overlap the copy
  // of the tables
  const int64_t vb = (int64_t)blockIdx.x * vpt * FV_THREADS + threadIdx.x;
  int idx[4][3];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t v = r < vpt ? vb + r * FV_THREADS : V;
    const int* q = vox + ((int64_t)n * V + (v < V ? v : 0)) * 3;
    idx[r][0] = q[0];
    idx[r][1] = q[1];
    idx[r][2] = q[2];
  }
  const float* tn = tab + (int64_t)n * na * Kp + k0;
  for (int e = threadIdx.x; e < na * q4; e += FV_THREADS) {
    const int a = e / q4, j = (e - a * q4) * 4;
    *reinterpret_cast<float4*>(&ftab[a * ld + j]) = *reinterpret_cast<const float4*>(&tn[(int64_t)a * Kp + j]);
  }
  __syncthreads();
  // per voxel: its three table rows, or none (past V, or an index outside
  // its axis: that column becomes NaN)
  const float* px[4];
  const float* py[4];
  const float* pz[4];
  float* out[4];
  bool live[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t v = r < vpt ? vb + r * FV_THREADS : V;
    const int ix = idx[r][0], iy = idx[r][1], iz = idx[r][2];
    const bool inside = (unsigned)ix < (unsigned)nx && (unsigned)iy < (unsigned)ny && (unsigned)iz < (unsigned)nz;
    out[r] = F + ((int64_t)n * K + k0) * V + (v < V ? v : 0);
    live[r] = v < V && inside;
    px[r] = ftab + (inside ? ix : 0) * ld;
    py[r] = ftab + (nx + (inside ? iy : 0)) * ld;
    pz[r] = ftab + (nx + ny + (inside ? iz : 0)) * ld;
    if (v < V && !inside) {
      if (flag) atomicOr(flag, 1);
      for (int j = 0; j < kn; ++j) out[r][(int64_t)j * V] = qnan();
    }
  }
  int j = 0;
  for (; j + 4 <= kn; j += 4) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (!live[r]) continue;
      const float4 x = *reinterpret_cast<const float4*>(px[r] + j);
      const float4 y = *reinterpret_cast<const float4*>(py[r] + j);
      const float4 z = *reinterpret_cast<const float4*>(pz[r] + j);
      float* o = out[r] + (int64_t)j * V;
      o[0] = x.x * y.x * z.x;
      o[V] = x.y * y.y * z.y;
      o[2 * (int64_t)V] = x.z * y.z * z.z;
      o[3 * (int64_t)V] = x.w * y.w * z.w;
    }
  }
  for (; j < kn; ++j)
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (live[r]) out[r][(int64_t)j * V] = px[r][j] * py[r][j] * pz[r][j];
}

// factors per block (a multiple of 4) and the table row stride (an odd
// multiple of 4 floats, so that random rows spread over the banks)
struct FactorPlan {
  int Kp, kc, ld;
  size_t smem;
};

FactorPlan factor_plan(int K, int na) {
  FactorPlan p;
  p.Kp = (K + 3) & ~3;
  const int cap = F_SMEM_DEFAULT / (int)sizeof(float) / na;  // floats per table row that fit 48 KB
  int kc = std::min(p.Kp, std::max(4, (cap - 4) & ~3));
  p.kc = kc;
  p.ld = ((kc >> 2) & 1) ? kc : kc + 4;
  p.smem = (size_t)na * p.ld * sizeof(float);
  return p;
}

// ---------------------------------------------------------------------------
// Residual ||X - W F||_F^2.  A block of 128 threads owns a 64 (t) x 128 (v)
// tile of W F and a thread an 8 x 8 piece of it: rows 4 ty + i and
// 32 + 4 ty + i, columns 4 tx + j and 64 + 4 tx + j (i, j < 4; two 16-byte
// groups each way, so that a warp's shared loads are broadcasts or cover 256
// contiguous bytes).  K is consumed in chunks of 16, double-buffered in
// shared memory: the copy of the next chunk (cp.async, no registers) is in
// flight while the current one is multiplied, and one barrier per chunk
// separates the buffers.  W[t][k] is staged transposed (Ws[k][t]) and F as
// is; per k a thread does 64 FMAs for four 16-byte shared loads.  The
// squared residuals of the tile are summed in FP32 per thread and in FP64
// across the block (fixed order), one partial per tile; a second kernel
// adds the partials of a subject in fixed order.
constexpr int RT = 64, RV = 128, RK = 16, R_THREADS = 128;
constexpr int WS_LD = RT + 4, FS_LD = RV + 4;  // floats per staged row

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 4-byte global -> shared copy; ok == false writes zero and reads nothing
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 4 : 0) : "memory");
}

template <int KN>
__device__ __forceinline__ void residual_mma_chunk(const float (*Ws)[WS_LD], const float (*Fs)[FS_LD], int kn, int ty,
                                                   int tx, float (&acc)[8][8]) {
#pragma unroll
  for (int kk = 0; kk < (KN > 0 ? KN : RK); ++kk) {
    if (KN == 0 && kk >= kn) break;
    const float4 a0 = *reinterpret_cast<const float4*>(&Ws[kk][ty * 4]);
    const float4 a1 = *reinterpret_cast<const float4*>(&Ws[kk][32 + ty * 4]);
    const float4 b0 = *reinterpret_cast<const float4*>(&Fs[kk][tx * 4]);
    const float4 b1 = *reinterpret_cast<const float4*>(&Fs[kk][64 + tx * 4]);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
}

template <bool VEC>
__global__ void __launch_bounds__(R_THREADS, VEC ? 3 : 4) htfa_residual_kernel(int K, int T, int V, int tiles_v, int tiles,
                                                                     const float* __restrict__ X,
                                                                     const float* __restrict__ W,
                                                                     const float* __restrict__ F,
                                                                     double* __restrict__ part) {
  __shared__ __align__(16) float Ws[2][RK][WS_LD];
  __shared__ __align__(16) float Fs[2][RK][FS_LD];
  __shared__ double red[R_THREADS / 32];
  const int n = blockIdx.y;
  const int tile = blockIdx.x;
  const int tt = tile / tiles_v, tv = tile - tt * tiles_v;
  const int t0 = tt * RT, v0 = tv * RV;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float* Wn = W + (int64_t)n * T * K;
  const float* Fn = F + (int64_t)n * K * V;
  const float* Xn = X + (int64_t)n * T * V;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  // one chunk, global -> shared by cp.async (4-byte copies, zero-filled
  // outside the matrices).  W tile 64 t x 16 k: this thread copies column
  // k0 + wk of rows t0 + wt + 8 r (r < 8) into Ws[k][t].  F tile 16 k x
  // 128 v: this thread copies column v0 + tid of rows k0 + r (r < 16).  The
  // pointers and row predicates are formed once; a chunk only advances them.
  const int wt = tid >> 4, wk = tid & 15;
  unsigned wrows = 0;  // bit r: row t0 + wt + 8 r exists
#pragma unroll
  for (int r = 0; r < 8; ++r) wrows |= (t0 + wt + 8 * r < T ? 1u : 0u) << r;
  const float* wsrc = Wn + (int64_t)min(t0 + wt, T - 1) * K + wk;
  const int64_t wstep = (int64_t)8 * K;
  const bool fcol = v0 + tid < V;
  const float* fsrc = Fn + (fcol ? v0 + tid : 0);
  const uint32_t wdst = smem_u32(&Ws[0][wk][wt]);
  const uint32_t fdst = smem_u32(&Fs[0][0][tid]);
  constexpr uint32_t WBUF = RK * WS_LD * 4, FBUF = RK * FS_LD * 4;
  const bool interior = t0 + RT <= T && v0 + RV <= V;
  auto issue_chunk = [&](int k0, int b) {
    const uint32_t wd = wdst + b * WBUF, fd = fdst + b * FBUF;
    const float* wp = wsrc + k0;
    const float* fp = fsrc + (int64_t)k0 * V;
    if (interior && k0 + RK <= K) {
#pragma unroll
      for (int r = 0; r < 8; ++r) cp_async4(wd + 32 * r, wp + r * wstep, true);
#pragma unroll
      for (int r = 0; r < 16; ++r) cp_async4(fd + r * (FS_LD * 4), fp + (int64_t)r * V, true);
    } else {
      const bool kw = k0 + wk < K;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const bool ok = kw && ((wrows >> r) & 1u);
        cp_async4(wd + 32 * r, ok ? wp + r * wstep : Wn, ok);
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const bool ok = fcol && k0 + r < K;
        cp_async4(fd + r * (FS_LD * 4), ok ? fp + (int64_t)r * V : Fn, ok);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // the X tile is read once, after the products: ask L2 for its lines now
  // (one request per 128-byte line: threads with tx = 0 or 8)
  if ((tx & 7) == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int t = t0 + (i < 4 ? 0 : 32) + ty * 4 + (i & 3);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int vc = v0 + 64 * h + tx * 4;
        if (t < T && vc < V) asm volatile("prefetch.global.L2 [%0];" ::"l"(Xn + (int64_t)t * V + vc));
      }
    }
  }

  const int nch = (K + RK - 1) / RK;
  issue_chunk(0, 0);
  for (int c = 0; c < nch; ++c) {
    const int b = c & 1;
    // chunk c has landed; every thread is done with chunk c - 1, whose
    // buffer the copy of chunk c + 1 now overwrites
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (c + 1 < nch) issue_chunk((c + 1) * RK, b ^ 1);
    const int kn = min(RK, K - c * RK);
    if (kn == RK)
      residual_mma_chunk<RK>(Ws[b], Fs[b], kn, ty, tx, acc);
    else
      residual_mma_chunk<0>(Ws[b], Fs[b], kn, ty, tx, acc);
  }

  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int t = t0 + (i < 4 ? 0 : 32) + ty * 4 + (i & 3);
    if (t >= T) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int vc = v0 + 64 * h + tx * 4;
      const float* xr = Xn + (int64_t)t * V + vc;
      if (VEC) {
        if (vc < V) {
          const float4 x = *reinterpret_cast<const float4*>(xr);
          const float r0 = x.x - acc[i][4 * h], r1 = x.y - acc[i][4 * h + 1];
          const float r2 = x.z - acc[i][4 * h + 2], r3 = x.w - acc[i][4 * h + 3];
          s = fmaf(r0, r0, s);
          s = fmaf(r1, r1, s);
          s = fmaf(r2, r2, s);
          s = fmaf(r3, r3, s);
        }
      } else if (vc + 3 < V) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float r = xr[j] - acc[i][4 * h + j];
          s = fmaf(r, r, s);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (vc + j < V) {
            const float r = xr[j] - acc[i][4 * h + j];
            s = fmaf(r, r, s);
          }
      }
    }
  }
  double d = s;
#pragma unroll
  for (int o = 16; o; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if ((tid & 31) == 0) red[tid >> 5] = d;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < R_THREADS / 32; ++w) tot += red[w];
    part[(int64_t)n * tiles + tile] = tot;
  }
}

// out[n] = sum of subject n's `tiles` partials in a fixed order; NaN when a
// bounded wait of the tensor-core kernel gave up (status != 0).
__global__ void __launch_bounds__(256) htfa_residual_sum_kernel(int tiles, const double* __restrict__ part,
                                                                double* __restrict__ out,
                                                                const int* __restrict__ status) {
  __shared__ double red[8];
  const int n = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < tiles; i += 256) s += part[(int64_t)n * tiles + i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += red[w];
    out[n] = (status && *status) ? __longlong_as_double(0x7ff8000000000000ll) : tot;
  }
}

// ---------------------------------------------------------------------------
// z-score of every column of a T x V matrix.  A block owns 32 columns (one
// per lane); warp w reads rows w, w + 8, ...  (128 contiguous bytes per row
// and warp).  The first pass forms sums of x - x_0 and (x - x_0)^2, with x_0
// the column's first sample, so the variance E[(x-x_0)^2] - E[x-x_0]^2 does
// not cancel when the mean is large against the spread; it also tracks the
// column's minimum and maximum, so that a constant column is detected
// exactly.  With STAGE the strip is kept in shared memory and X is read from
// HBM once; otherwise the second pass reads it again.
constexpr int Z_STAGE_MAX_T = 768;  // 96 KB of staged strip

template <bool STAGE>
__global__ void __launch_bounds__(256) zscore_kernel(int T, int V, const float* X, float* Y) {
  extern __shared__ float zs_strip[];  // STAGE: [T][32]
  __shared__ float p1[8][32], p2[8][32], plo[8][32], phi[8][32];
  __shared__ float s_mean[32], s_inv[32];
  const int n = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + lane;
  const bool live = c < V;
  const float* Xn = X + (int64_t)n * T * V;
  float* Yn = Y + (int64_t)n * T * V;
  const float x0 = live ? Xn[c] : 0.f;
  float s1 = 0.f, s2 = 0.f, lo = 3.402823466e38f, hi = -3.402823466e38f;
  if (live) {
#pragma unroll 4
    for (int r = w; r < T; r += 8) {
      const float x = Xn[(int64_t)r * V + c];
      if (STAGE) zs_strip[r * 32 + lane] = x;
      const float d = x - x0;
      s1 += d;
      s2 = fmaf(d, d, s2);
      lo = fminf(lo, x);
      hi = fmaxf(hi, x);
    }
  }
  p1[w][lane] = s1;
  p2[w][lane] = s2;
  plo[w][lane] = lo;
  phi[w][lane] = hi;
  __syncthreads();
  if (w == 0) {
    float a = 0.f, b = 0.f, mn = 3.402823466e38f, mx = -3.402823466e38f;
    for (int j = 0; j < 8; ++j) {
      a += p1[j][lane];
      b += p2[j][lane];
      mn = fminf(mn, plo[j][lane]);
      mx = fmaxf(mx, phi[j][lane]);
    }
    const float m1 = a / (float)T;
    const float var = b / (float)T - m1 * m1;
    s_mean[lane] = x0 + m1;
    s_inv[lane] = (mn < mx && var > 0.f) ? 1.f / sqrtf(var) : 0.f;
  }
  __syncthreads();
  if (!live) return;
  const float mean = s_mean[lane], inv = s_inv[lane];
#pragma unroll 4
  for (int r = w; r < T; r += 8) {
    const float x = STAGE ? zs_strip[r * 32 + lane] : Xn[(int64_t)r * V + c];
    Yn[(int64_t)r * V + c] = inv == 0.f ? 0.f : (x - mean) * inv;
  }
}

srm_status launch_check(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SRM_OK : cuda_fail(e, what);
}

int64_t residual_tiles(int32_t T, int32_t V) {
  return (int64_t)((T + RT - 1) / RT) * ((V + RV - 1) / RV);
}

}  // namespace

}  // namespace srm

using namespace srm;

extern "C" size_t srm_htfa_factors_workspace(int32_t n_subj, int32_t K, int32_t nx, int32_t ny, int32_t nz) {
  if (n_subj <= 0 || K <= 0 || nx <= 0 || ny <= 0 || nz <= 0) return 0;
  return (size_t)n_subj * (size_t)(nx + ny + nz) * (size_t)((K + 3) & ~3) * sizeof(float);
}

extern "C" srm_status srm_htfa_factors(int32_t n_subj, int32_t K, int32_t V, const float* axes, int32_t nx,
                                       int32_t ny, int32_t nz, const int32_t* vox, const float* mu,
                                       const float* lambda, float* F, int32_t* flag, void* work, size_t work_bytes,
                                       void* stream) {
  if (n_subj < 0 || n_subj > 65535 || K < 1 || K > (1 << 20) || V < 0 || nx < 1 || ny < 1 || nz < 1 || nx > 4096 ||
      ny > 4096 || nz > 4096) {
    set_error("srm_htfa_factors: need 0 <= n_subj <= 65535, 1 <= K <= 2^20, V >= 0, 1 <= nx, ny, nz <= 4096");
    return SRM_ERR_ARG;
  }
  if (n_subj == 0 || V == 0) return SRM_OK;
  const size_t need = srm_htfa_factors_workspace(n_subj, K, nx, ny, nz);
  if (!axes || !vox || !mu || !lambda || !F || !work || (reinterpret_cast<uintptr_t>(work) & 15) ||
      work_bytes < need) {
    set_error("srm_htfa_factors: null pointer, workspace not 16-byte aligned or below " + std::to_string(need) +
              " bytes");
    return SRM_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int na = nx + ny + nz;
  const FactorPlan p = factor_plan(K, na);
  float* tab = static_cast<float*>(work);
  htfa_tables_kernel<<<dim3((unsigned)((na + TAB_ROWS - 1) / TAB_ROWS), (unsigned)n_subj), 128, 0, s>>>(
      K, p.Kp, na, axes, nx, ny, mu, lambda, tab, flag);
  srm_status st = launch_check("srm_htfa_factors: tables");
  if (st != SRM_OK) return st;
  if (p.smem > (size_t)F_SMEM_DEFAULT) {
    const cudaError_t e = cudaFuncSetAttribute(htfa_factors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)p.smem);
    if (e != cudaSuccess) return cuda_fail(e, "srm_htfa_factors: cudaFuncSetAttribute");
  }
  // four voxels a thread: one a thread (more, smaller blocks for a single
  // subject) measured slower, each block copying the same tables
  const int vpt = 4;
  const dim3 grid((unsigned)((V + vpt * FV_THREADS - 1) / (vpt * FV_THREADS)), (unsigned)((K + p.kc - 1) / p.kc),
                  (unsigned)n_subj);
  htfa_factors_kernel<<<grid, FV_THREADS, p.smem, s>>>(K, p.Kp, V, p.kc, p.ld, vpt, nx, ny, nz, tab, vox, F, flag);
  return launch_check("srm_htfa_factors");
}

// Partials per subject of the form that runs for K: the FP32 SIMT tiles, or
// four per tensor-core tile (one per epilogue warp).
int64_t residual_parts(int32_t K, int32_t T, int32_t V) {
  return htfa_tc_supported(K) ? 4 * htfa_tc_tiles(T, V) : residual_tiles(T, V);
}

extern "C" size_t srm_htfa_residual_workspace(int32_t n_subj, int32_t K, int32_t T, int32_t V) {
  if (n_subj <= 0 || T <= 0 || V <= 0) return 0;
  // the partials, then one status word (16 bytes) for the tensor-core form
  return (size_t)n_subj * (size_t)residual_parts(K, T, V) * sizeof(double) + 16;
}

extern "C" srm_status srm_htfa_residual(int32_t n_subj, int32_t K, int32_t T, int32_t V, const float* X,
                                        const float* W, const float* F, double* out, void* work, size_t work_bytes,
                                        void* stream) {
  if (n_subj < 0 || n_subj > 65535 || K < 1 || T < 0 || V < 0) {
    set_error("srm_htfa_residual: need 0 <= n_subj <= 65535, K >= 1, T >= 0, V >= 0");
    return SRM_ERR_ARG;
  }
  if (n_subj == 0) return SRM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!out) {
    set_error("srm_htfa_residual: null output pointer");
    return SRM_ERR_ARG;
  }
  if (T == 0 || V == 0) {
    const cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n_subj * sizeof(double), s);
    return e == cudaSuccess ? SRM_OK : cuda_fail(e, "srm_htfa_residual: cudaMemsetAsync");
  }
  const int64_t tiles = residual_parts(K, T, V);
  if (tiles > INT_MAX / 4) {
    set_error("srm_htfa_residual: T x V has too many tiles");
    return SRM_ERR_ARG;
  }
  if (!X || !W || !F || !work || (reinterpret_cast<uintptr_t>(work) & 7) ||
      work_bytes < srm_htfa_residual_workspace(n_subj, K, T, V)) {
    set_error("srm_htfa_residual: null pointer, misaligned workspace or workspace below " +
              std::to_string(srm_htfa_residual_workspace(n_subj, K, T, V)) + " bytes");
    return SRM_ERR_ARG;
  }
  double* part = static_cast<double*>(work);
  if (htfa_tc_supported(K)) {
    int* st_word = reinterpret_cast<int*>(part + (size_t)n_subj * (size_t)tiles);
    cudaError_t e = cudaMemsetAsync(st_word, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "srm_htfa_residual: cudaMemsetAsync");
    e = launch_htfa_residual_tc(n_subj, K, T, V, X, W, F, part, st_word, s);
    if (e != cudaSuccess) return cuda_fail(e, "srm_htfa_residual: tensor-core kernel");
    htfa_residual_sum_kernel<<<(unsigned)n_subj, 256, 0, s>>>((int)tiles, part, out, st_word);
    return launch_check("srm_htfa_residual: sum kernel");
  }
  const int tiles_v = (V + RV - 1) / RV;
  const dim3 grid((unsigned)tiles, (unsigned)n_subj);
  const bool vec = (V % 4 == 0) && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  if (vec)
    htfa_residual_kernel<true><<<grid, R_THREADS, 0, s>>>(K, T, V, tiles_v, (int)tiles, X, W, F, part);
  else
    htfa_residual_kernel<false><<<grid, R_THREADS, 0, s>>>(K, T, V, tiles_v, (int)tiles, X, W, F, part);
  srm_status st = launch_check("srm_htfa_residual: tile kernel");
  if (st != SRM_OK) return st;
  htfa_residual_sum_kernel<<<(unsigned)n_subj, 256, 0, s>>>((int)tiles, part, out, nullptr);
  return launch_check("srm_htfa_residual: sum kernel");
}

extern "C" srm_status srm_zscore(int32_t n_mat, int32_t T, int32_t V, const float* X, float* Y, void* stream) {
  if (n_mat < 0 || n_mat > 65535 || T < 0 || V < 0) {
    set_error("srm_zscore: need 0 <= n_mat <= 65535, T >= 0, V >= 0");
    return SRM_ERR_ARG;
  }
  if (n_mat == 0 || T == 0 || V == 0) return SRM_OK;
  if (!X || !Y) {
    set_error("srm_zscore: null pointer");
    return SRM_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const dim3 grid((unsigned)((V + 31) / 32), (unsigned)n_mat);
  if (T <= Z_STAGE_MAX_T) {
    const size_t smem = (size_t)T * 32 * sizeof(float);
    if (smem > 48 * 1024) {
      const cudaError_t attr = cudaFuncSetAttribute(zscore_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    Z_STAGE_MAX_T * 32 * (int)sizeof(float));
      if (attr != cudaSuccess) return cuda_fail(attr, "srm_zscore: cudaFuncSetAttribute");
    }
    zscore_kernel<true><<<grid, 256, smem, s>>>(T, V, X, Y);
  } else {
    zscore_kernel<false><<<grid, 256, 0, s>>>(T, V, X, Y);
  }
  return launch_check("srm_zscore");
}
