// HTFA local-step evaluations (Sec. III, and the native extension modules of
// Sec. IV-A): the factor matrix F_i of Eq. 14, the residual
// ||X_i - W_i F_i||_F^2 of eq:htfa_subject_update_rbfs, and the per-voxel
// z-score.  Layouts follow the paper's HTFA notation: X_i is T x V (one
// sample per row), W_i is T x K, F_i is K x V; a batch of equal-sized
// subjects is stored back to back.
#include <climits>
#include <string>

#include "htfa.h"
#include "srm_internal.cuh"

namespace srm {

namespace {

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

// ---------------------------------------------------------------------------
// Factor matrix (Eq. 14).  ||p - mu||^2 separates over the axes, so
//   F[k][v] = Ex[k][ix] * Ey[k][iy] * Ez[k][iz],  Ec[k][a] = exp(-(a_c - mu_kc)^2 / lambda_k).
// A block builds the tables of kc factors in shared memory (kc * (nx+ny+nz)
// exponentials), then writes those kc rows for 1024 voxels: two multiplies
// and one coalesced 4-byte store per element.
constexpr int FV_THREADS = 256;
constexpr int FV_PER_BLOCK = 4 * FV_THREADS;
constexpr int F_TABLE_FLOATS = 12288;  // 48 KB of tables per block

__global__ void __launch_bounds__(FV_THREADS) htfa_factors_kernel(int K, int V, int kc, const float* __restrict__ axes,
                                                                  int nx, int ny, int nz, const int* __restrict__ vox,
                                                                  const float* __restrict__ mu,
                                                                  const float* __restrict__ lam, float* __restrict__ F,
                                                                  int* flag) {
  extern __shared__ float ftab[];  // [kn][na]
  const int n = blockIdx.z;
  const int k0 = blockIdx.y * kc;
  const int kn = min(kc, K - k0);
  const int na = nx + ny + nz;
  for (int e = threadIdx.x; e < kn * na; e += FV_THREADS) {
    const int j = e / na, a = e - j * na;
    const int axis = a < nx ? 0 : (a < nx + ny ? 1 : 2);
    const int64_t f = (int64_t)n * K + k0 + j;
    const float l = lam[f];
    const bool ok = l > 0.f && l <= 3.402823466e38f;
    const float d = axes[a] - mu[f * 3 + axis];
    ftab[e] = ok ? expf(-(d * d) / l) : qnan();
    if (!ok && a == 0 && flag) atomicOr(flag, 2);
  }
  __syncthreads();
  const int64_t vb = (int64_t)blockIdx.x * FV_PER_BLOCK;
#pragma unroll 1
  for (int r = 0; r < 4; ++r) {
    const int64_t v = vb + r * FV_THREADS + threadIdx.x;
    if (v >= V) break;
    const int* q = vox + ((int64_t)n * V + v) * 3;
    const int ix = q[0], iy = q[1], iz = q[2];
    float* out = F + ((int64_t)n * K + k0) * V + v;
    if ((unsigned)ix < (unsigned)nx && (unsigned)iy < (unsigned)ny && (unsigned)iz < (unsigned)nz) {
      const float* px = ftab + ix;
      const float* py = ftab + nx + iy;
      const float* pz = ftab + nx + ny + iz;
      for (int j = 0; j < kn; ++j) out[(int64_t)j * V] = px[j * na] * py[j * na] * pz[j * na];
    } else {
      if (flag) atomicOr(flag, 1);
      for (int j = 0; j < kn; ++j) out[(int64_t)j * V] = qnan();
    }
  }
}

// ---------------------------------------------------------------------------
// Residual ||X - W F||_F^2.  A block owns a 64 (t) x 64 (v) tile of W F and
// a thread a 4 x 4 piece of it (rows 4 ty .. 4 ty + 3, columns 4 tx ..
// 4 tx + 3).  K is consumed in chunks of 16: W[t][k] is staged transposed
// (Ws[k][t]) and F[k][v] as is, each thread then does 16 FMAs per pair of
// 16-byte shared loads.  The squared residuals of the tile are summed in
// FP32 per thread and in FP64 across the block (fixed order), one partial
// per tile; a second kernel adds the partials of a subject in fixed order.
constexpr int RT = 64, RV = 64, RK = 16, RPAD = 4;

template <bool VEC>
__global__ void __launch_bounds__(256, 3) htfa_residual_kernel(int K, int T, int V, int tiles_v, int tiles,
                                                               const float* __restrict__ X,
                                                               const float* __restrict__ W,
                                                               const float* __restrict__ F,
                                                               double* __restrict__ part) {
  __shared__ __align__(16) float Ws[RK][RT + RPAD];
  __shared__ __align__(16) float Fs[RK][RV + RPAD];
  __shared__ double red[8];
  const int n = blockIdx.y;
  const int tile = blockIdx.x;
  const int tt = tile / tiles_v, tv = tile - tt * tiles_v;
  const int t0 = tt * RT, v0 = tv * RV;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float* Wn = W + (int64_t)n * T * K;
  const float* Fn = F + (int64_t)n * K * V;
  const float* Xn = X + (int64_t)n * T * V;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < K; k0 += RK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r;          // 0 .. 1023
      const int wt = e >> 4, wk = e & 15;   // W tile: 64 t x 16 k, k fastest in memory
      const int t = t0 + wt, k = k0 + wk;
      Ws[wk][wt] = (t < T && k < K) ? Wn[(int64_t)t * K + k] : 0.f;
      const int fk = e >> 6, fv = e & 63;   // F tile: 16 k x 64 v, v fastest in memory
      const int kf = k0 + fk, v = v0 + fv;
      Fs[fk][fv] = (kf < K && v < V) ? Fn[(int64_t)kf * V + v] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < RK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&Ws[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Fs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }

  float s = 0.f;
  const int vc = v0 + tx * 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t = t0 + ty * 4 + i;
    if (t >= T) break;
    const float* xr = Xn + (int64_t)t * V + vc;
    if (VEC && vc < V) {
      const float4 x = *reinterpret_cast<const float4*>(xr);
      const float r0 = x.x - acc[i][0], r1 = x.y - acc[i][1], r2 = x.z - acc[i][2], r3 = x.w - acc[i][3];
      s = fmaf(r0, r0, s);
      s = fmaf(r1, r1, s);
      s = fmaf(r2, r2, s);
      s = fmaf(r3, r3, s);
    } else if (!VEC) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (vc + j < V) {
          const float r = xr[j] - acc[i][j];
          s = fmaf(r, r, s);
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
    for (int w = 0; w < 8; ++w) tot += red[w];
    part[(int64_t)n * tiles + tile] = tot;
  }
}

__global__ void __launch_bounds__(256) htfa_residual_sum_kernel(int tiles, const double* __restrict__ part,
                                                                double* __restrict__ out) {
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
    out[n] = tot;
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

extern "C" srm_status srm_htfa_factors(int32_t n_subj, int32_t K, int32_t V, const float* axes, int32_t nx,
                                       int32_t ny, int32_t nz, const int32_t* vox, const float* mu,
                                       const float* lambda, float* F, int32_t* flag, void* stream) {
  if (n_subj < 0 || n_subj > 65535 || K < 1 || V < 0 || nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 ||
      nz > 4096) {
    set_error("srm_htfa_factors: need 0 <= n_subj <= 65535, K >= 1, V >= 0, 1 <= nx, ny, nz <= 4096");
    return SRM_ERR_ARG;
  }
  if (n_subj == 0 || V == 0) return SRM_OK;
  if (!axes || !vox || !mu || !lambda || !F) {
    set_error("srm_htfa_factors: null pointer");
    return SRM_ERR_ARG;
  }
  const int na = nx + ny + nz;
  const int kc = std::max(1, std::min<int>(K, F_TABLE_FLOATS / na));
  const dim3 grid((unsigned)((V + FV_PER_BLOCK - 1) / FV_PER_BLOCK), (unsigned)((K + kc - 1) / kc),
                  (unsigned)n_subj);
  if (grid.y > 65535) {
    set_error("srm_htfa_factors: too many factor chunks (K = " + std::to_string(K) + ")");
    return SRM_ERR_ARG;
  }
  htfa_factors_kernel<<<grid, FV_THREADS, (size_t)kc * na * sizeof(float), static_cast<cudaStream_t>(stream)>>>(
      K, V, kc, axes, nx, ny, nz, vox, mu, lambda, F, flag);
  return launch_check("srm_htfa_factors");
}

extern "C" size_t srm_htfa_residual_workspace(int32_t n_subj, int32_t K, int32_t T, int32_t V) {
  (void)K;
  if (n_subj <= 0 || T <= 0 || V <= 0) return 0;
  return (size_t)n_subj * (size_t)residual_tiles(T, V) * sizeof(double);
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
  const int64_t tiles = residual_tiles(T, V);
  if (tiles > INT_MAX) {
    set_error("srm_htfa_residual: T x V has more than 2^31 - 1 tiles of 64 x 64");
    return SRM_ERR_ARG;
  }
  if (!X || !W || !F || !work || (reinterpret_cast<uintptr_t>(work) & 7) ||
      work_bytes < srm_htfa_residual_workspace(n_subj, K, T, V)) {
    set_error("srm_htfa_residual: null pointer, misaligned workspace or workspace below " +
              std::to_string(srm_htfa_residual_workspace(n_subj, K, T, V)) + " bytes");
    return SRM_ERR_ARG;
  }
  double* part = static_cast<double*>(work);
  const int tiles_v = (V + RV - 1) / RV;
  const dim3 grid((unsigned)tiles, (unsigned)n_subj);
  const bool vec = (V % 4 == 0) && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  if (vec)
    htfa_residual_kernel<true><<<grid, 256, 0, s>>>(K, T, V, tiles_v, (int)tiles, X, W, F, part);
  else
    htfa_residual_kernel<false><<<grid, 256, 0, s>>>(K, T, V, tiles_v, (int)tiles, X, W, F, part);
  srm_status st = launch_check("srm_htfa_residual: tile kernel");
  if (st != SRM_OK) return st;
  htfa_residual_sum_kernel<<<(unsigned)n_subj, 256, 0, s>>>((int)tiles, part, out);
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
