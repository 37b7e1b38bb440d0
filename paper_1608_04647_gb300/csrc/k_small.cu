// The k x k and k x T steps of one EM iteration (everything but the two
// streaming passes over X^).
//
// E-step (Algorithm 1, master process):
//   p_reduce : Z_i = rho_i^-2 M_i P_i from the E-pass partials, using
//              W_i^T X^_i = M_i (A_i^T X^_i)        (eq:srm_mean_distributed),
//              summed over groups of subjects (FP64, subjects in order)
//   phi      : rho_0 = sum_i rho_i^-2 (eq:srm_wt_psi_w) and
//              Phi = (Sigma_s^-1 + rho_0 I)^-1 (eq:srm_inversion_opt), written
//              as the matrix function Phi = g(Sigma_s), g(x) = x / (1 + rho_0 x),
//              of the FP64 eigen-decomposition of Sigma_s kept from the M-step;
//              ln det(I + rho_0 Sigma_s) = sum ln(1 + rho_0 lambda) for the
//              log-likelihood.  Phi equals the paper's
//              Sigma_s^T [I - rho_0 (Sigma_s^-1 + rho_0 I)^-1].
//   es       : E[S] = Phi y, the operand copies for the M-pass, and per-block
//              partials of E[S] E[S]^T and <y, Phi y>   (FP64)
//   sigma    : Sigma_s^new = Phi + E[S] E[S]^T / T
//              (eq:srm_variance_update_optimized) and the log-likelihood
// M-step (per subject, plus Sigma_s^new as one more symmetric matrix):
//   eig      : G_i = A_i^T A_i from the Gram partials; cyclic Jacobi in FP32,
//              warm-started from the previous eigenvectors
//   refine   : FP64 re-orthonormalisation U = U_0 (3I - U_0^T U_0)/2 and
//              G' = U^T G U (off-diagonal part E of order 1e-6 |G|)
//   rho      : first-order (Daleckii-Krein) correction of a matrix function
//              f(G) = U (f(Lambda) + F o E) U^T with the divided differences
//              F_ab = f[lambda_a, lambda_b]; for f(x) = x^-1/2 this gives
//              M_i = (A_i^T A_i)^-1/2 to FP64 accuracy (error O(|E|^2)),
//              ||A_i||_* = tr (A_i^T A_i)^1/2 = sum sqrt(lambda) + O(|E|^2), and
//              rho_i^2 = (||X^_i||^2 - 2 ||A_i||_* + T tr Sigma_s^new)/(T v_i)
//              (eq:srm_rho_update, with tr(W_i^T A_i) = ||A_i||_* for the
//              polar factor W_i of eq:srm_mapping_update).
#include <math.h>

#include <algorithm>

#include "kk_util.cuh"

namespace srm {

namespace {

// ------------------------------------------------------------------ E-step
// p_reduce: grid (nchunk, G), 256 threads.  Block (c, g) takes the subjects
// [N g / G, N (g + 1) / G) in order.  For each it sums the subject's partial
// blocks of t-chunk c in slot order into P (TCH x kld), forms
// Z_i = rho_i^-2 M_i P in FP32 (sum over m in order) and adds it to an
// error-free FP32 accumulator (hi + lo); the block then writes ypart[g][f][t].
// Thread (tx, ty) of the 16 x 16 grid holds the 4 x FW tile t = tx + 16 u,
// f = ty + 16 w, which reads P and M from shared memory at one load per two
// FMAs without bank conflicts (P rows padded to an odd stride, M stored
// m-major).
// es: y = sum_g ypart[g] (groups in order), E[S] = Phi y, the operand copies
// and the E[S] E[S]^T / <y, E[S]> partials of ES_T columns per block, in FP32
// (FP64 runs at about 2 FMA per clock per SM on this part).  Sigma_s^new and
// the log-likelihood (sigma_kernel) are left to the M-step tail, which runs
// beside the next E-pass: the M-pass needs only E[S].
constexpr int PR_MAX_SLOTS = 64;  // slot offsets staged in shared memory per (subject, chunk)

struct EReduceArgs {
  int N, G, T, k, nchunk;
  const float* part;
  const ChunkSrc* src;
  const int* src_off;
  const float* M32;
  const double* rho2;
  float2* ypart;           // [G][k][T] (hi, lo)
};

template <int FW>  // kld = 16 FW
__global__ void __launch_bounds__(256, FW <= 4 ? 3 : 2) p_reduce_kernel(EReduceArgs ar) {
  const int N = ar.N, G = ar.G, T = ar.T, k = ar.k, nchunk = ar.nchunk;
  const float* __restrict__ part = ar.part;
  const ChunkSrc* __restrict__ src = ar.src;
  const int* __restrict__ src_off = ar.src_off;
  const float* __restrict__ M32 = ar.M32;
  const double* __restrict__ rho2 = ar.rho2;
  float2* __restrict__ ypart = ar.ypart;
  constexpr int KLD = 16 * FW;
  constexpr int SPT = TCH + 4;  // row stride of Ps (16-byte rows, conflict-free float4 stores)
  extern __shared__ __align__(16) float pr_smem[];
  float* Ms = pr_smem;                 // [KLD][KLD]: Ms[m * KLD + f] = M_i[m][f] = M_i[f][m]
  float* Ps = pr_smem + KLD * KLD;     // [KLD][SPT]: Ps[m * SPT + t] = P[t][m]
  // the slot sum as loaded, P0[t * (KLD + 1) + m] ([TCH][KLD + 1]); for
  // kld = 128 it shares M_i's space (M_i is then loaded after the transpose)
  constexpr bool P0_IN_MS = FW > 4;
  float* P0 = P0_IN_MS ? Ms : Ps + KLD * SPT;
  static_assert(!P0_IN_MS || TCH * (KLD + 1) <= KLD * KLD, "P0 fits in M_i's space");
  const int c = blockIdx.x, g = blockIdx.y;
  const int t0 = c * TCH;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = (int)(((int64_t)N * g) / G), i1 = (int)(((int64_t)N * (g + 1)) / G);
  // thread (tx, ty) owns t = 4 tx + u (u < 4) and f = FW ty + w (w < FW):
  // per m one float4 of P (t) and FW consecutive floats of M (f)
  float acc[4][FW], accl[4][FW];  // hi + lo (error-free FP32 accumulation)
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < FW; ++w) acc[u][w] = accl[u][w] = 0.f;
  static_assert(TCH * KLD / 4 == 256 * FW, "a thread owns FW float4 positions of a slot block");
  // M_i (symmetric: row m read as column m): KLD^2 / 4 float4, all of a thread's loads in flight
  auto load_m = [&](int i) {
    {
      constexpr int NM4 = KLD * KLD / 4;          // 64 FW^2
      constexpr int MJ = (NM4 + 255) / 256;
      const float4* Mi4 = reinterpret_cast<const float4*>(M32 + (int64_t)i * KLD * KLD);
      float4 mv[MJ];
#pragma unroll
      for (int j = 0; j < MJ; ++j)
        mv[j] = (tid + 256 * j < NM4) ? __ldg(Mi4 + tid + 256 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < MJ; ++j) {
        if (tid + 256 * j >= NM4) continue;
        const int e = 4 * (tid + 256 * j), m = e / KLD, f = e - m * KLD;
        const bool rm = m < k;
        float4 v = mv[j];
        v.x = (rm && f < k) ? v.x : 0.f;
        v.y = (rm && f + 1 < k) ? v.y : 0.f;
        v.z = (rm && f + 2 < k) ? v.z : 0.f;
        v.w = (rm && f + 3 < k) ? v.w : 0.f;
        *reinterpret_cast<float4*>(Ms + e) = v;
      }
    }
  };
  for (int i = i0; i < i1; ++i) {
    __syncthreads();  // the previous subject's tiles have been read
    if (!P0_IN_MS) load_m(i);
    const int b = src_off[i * nchunk + c], en = src_off[i * nchunk + c + 1];
    // slot offsets of this (subject, chunk) staged in shared memory
    __shared__ int64_t s_off[PR_MAX_SLOTS];
    const int ns = en - b;
    for (int q = tid; q < ns && q < PR_MAX_SLOTS; q += 256) s_off[q] = src[b + q].off;
    __syncthreads();
    // a thread's FW float4 positions (4 consecutive m of one t; lanes take
    // consecutive positions, so the loads are coalesced), two slots at a
    // time: 2 FW loads in flight, summed in slot order
    float4 a4[FW];
#pragma unroll
    for (int j = 0; j < FW; ++j) a4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < ns; q += 2) {
      const int64_t o0 = q < PR_MAX_SLOTS ? s_off[q] : src[b + q].off;
      const bool two = q + 1 < ns;
      const int64_t o1 = two ? (q + 1 < PR_MAX_SLOTS ? s_off[q + 1] : src[b + q + 1].off) : o0;
      float4 v0[FW], v1[FW];
#pragma unroll
      for (int j = 0; j < FW; ++j) {
        v0[j] = __ldg(reinterpret_cast<const float4*>(part + o0) + tid + 256 * j);
        v1[j] = two ? __ldg(reinterpret_cast<const float4*>(part + o1) + tid + 256 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < FW; ++j) {
        a4[j].x += v0[j].x;
        a4[j].y += v0[j].y;
        a4[j].z += v0[j].z;
        a4[j].w += v0[j].w;
        if (two) {
          a4[j].x += v1[j].x;
          a4[j].y += v1[j].y;
          a4[j].z += v1[j].z;
          a4[j].w += v1[j].w;
        }
      }
    }
    // as loaded (t-major, odd row stride: conflict-free scalar stores) ...
#pragma unroll
    for (int j = 0; j < FW; ++j) {
      const int e = 4 * (tid + 256 * j), t = e / KLD, m = e - t * KLD;
      float* d = P0 + t * (KLD + 1) + m;
      d[0] = a4[j].x;
      d[1] = a4[j].y;
      d[2] = a4[j].z;
      d[3] = a4[j].w;
    }
    __syncthreads();
    // ... then feature-major: thread (m, 4-t group) reads down a column of P0
    // (lanes take consecutive m: distinct banks) and stores one float4
#pragma unroll
    for (int j = 0; j < FW; ++j) {
      const int e = tid + 256 * j, m = e % KLD, tq = e / KLD;
      const float* sp = P0 + 4 * tq * (KLD + 1) + m;
      *reinterpret_cast<float4*>(Ps + m * SPT + 4 * tq) =
          make_float4(sp[0], sp[KLD + 1], sp[2 * (KLD + 1)], sp[3 * (KLD + 1)]);
    }
    if (P0_IN_MS) {
      __syncthreads();  // P0 has been read
      load_m(i);
    }
    __syncthreads();
    float z[4][FW];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < FW; ++w) z[u][w] = 0.f;
    for (int m = 0; m < k; ++m) {
      const float4 p4 = *reinterpret_cast<const float4*>(Ps + m * SPT + 4 * tx);
      const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
      float mv[FW];
      const float* mrow = Ms + m * KLD + FW * ty;
      if constexpr (FW % 4 == 0) {
#pragma unroll
        for (int w = 0; w < FW; w += 4) {
          const float4 q4 = *reinterpret_cast<const float4*>(mrow + w);
          mv[w] = q4.x;
          mv[w + 1] = q4.y;
          mv[w + 2] = q4.z;
          mv[w + 3] = q4.w;
        }
      } else if constexpr (FW % 2 == 0) {
#pragma unroll
        for (int w = 0; w < FW; w += 2) {
          const float2 q2 = *reinterpret_cast<const float2*>(mrow + w);
          mv[w] = q2.x;
          mv[w + 1] = q2.y;
        }
      } else {
#pragma unroll
        for (int w = 0; w < FW; ++w) mv[w] = mrow[w];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < FW; ++w) z[u][w] = fmaf(mv[w], pv[u], z[u][w]);
    }
    const float rinv = (float)(1.0 / rho2[i]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < FW; ++w) {
        float hs, he;
        two_sum(acc[u][w], __fmul_rn(rinv, z[u][w]), hs, he);  // the product rounded on its own, never fused
        acc[u][w] = hs;
        accl[u][w] += he;
      }
  }
  const int64_t kT = (int64_t)k * T;
  float2* out = ypart + (int64_t)g * kT;
#pragma unroll
  for (int w = 0; w < FW; ++w) {
    const int f = FW * ty + w;
    if (f >= k) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + 4 * tx + u;
      if (t < T) out[(int64_t)f * T + t] = make_float2(acc[u][w], accl[u][w]);
    }
  }
}



// p_sum: grid (nchunk, N), 256 threads.  Block (c, i) sums subject i's
// partial blocks of t-chunk c in slot order (the order p_reduce uses) into
// psum[i][c].  It needs no M_i, so it runs beside the polar factors; p_reduce
// then reads one block per (subject, chunk), and 0 + psum = psum exactly:
// the result is bitwise that of p_reduce on the slots.
template <int FW>
__global__ void __launch_bounds__(256) p_sum_kernel(int nchunk, const float* __restrict__ part,
                                                    const ChunkSrc* __restrict__ src,
                                                    const int* __restrict__ src_off, float* __restrict__ psum) {
  constexpr int KLD = 16 * FW;
  const int c = blockIdx.x, i = blockIdx.y, tid = threadIdx.x;
  const int b = src_off[i * nchunk + c], en = src_off[i * nchunk + c + 1];
  float4 a4[FW];
#pragma unroll
  for (int j = 0; j < FW; ++j) a4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int q = b; q < en; q += 2) {
    const int64_t o0 = src[q].off;
    const bool two = q + 1 < en;
    const int64_t o1 = two ? src[q + 1].off : o0;
    float4 v0[FW], v1[FW];
#pragma unroll
    for (int j = 0; j < FW; ++j) {
      v0[j] = __ldg(reinterpret_cast<const float4*>(part + o0) + tid + 256 * j);
      v1[j] = two ? __ldg(reinterpret_cast<const float4*>(part + o1) + tid + 256 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < FW; ++j) {
      a4[j].x += v0[j].x;
      a4[j].y += v0[j].y;
      a4[j].z += v0[j].z;
      a4[j].w += v0[j].w;
      if (two) {
        a4[j].x += v1[j].x;
        a4[j].y += v1[j].y;
        a4[j].z += v1[j].z;
        a4[j].w += v1[j].w;
      }
    }
  }
  float4* out = reinterpret_cast<float4*>(psum + ((int64_t)i * nchunk + c) * TCH * KLD);
#pragma unroll
  for (int j = 0; j < FW; ++j) out[tid + 256 * j] = a4[j];
}

// Block reduction of three doubles over blockDim.x (a power of two <= 256) threads.
__device__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double red[3][256];
  const int tid = threadIdx.x;
  red[0][tid] = a;
  red[1][tid] = b;
  red[2][tid] = c;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      red[0][tid] += red[0][tid + s];
      red[1][tid] += red[1][tid + s];
      red[2][tid] += red[2][tid + s];
    }
    __syncthreads();
  }
  a = red[0][0];
  b = red[1][0];
  c = red[2][0];
  __syncthreads();
}

// grid k blocks (row a of Phi), 256 threads.
//   Sigma_s = U (Lambda + E) U^T with U = Us, G' = Lambda + E = Gp (k x k).
//   Phi = U (g(Lambda) + F o E) U^T,  g(x) = x/(1 + rho0 x),
//   F_bd = g[lambda_b, lambda_d] = 1 / ((1 + rho0 lambda_b)(1 + rho0 lambda_d)).
// U is staged in shared memory beside G' when both fit (u_smem), else read
// from global memory (k close to 128).
// With sums != nullptr (a sharded E-step) rho_0 and the likelihood's sums
// over subjects are taken from sums = {sum rho_i^-2, sum v_i ln rho_i^2,
// sum ||X^_i||^2 / rho_i^2, sum v_i} over all shards instead of this
// context's subjects.
__global__ void __launch_bounds__(256) phi_kernel(int N, int k, const double* __restrict__ rho2,
                                                  const double* __restrict__ sqnorm,
                                                  const int64_t* __restrict__ vox, const double* __restrict__ Us,
                                                  const double* __restrict__ Gp, double* __restrict__ Phi,
                                                  float* __restrict__ Phi32, double* __restrict__ scal, int u_smem,
                                                  int* status, double vtot, const double* __restrict__ sums) {
  extern __shared__ double ph_smem[];
  double* w = ph_smem;          // [k]  1 / (1 + rho0 lambda)
  double* ua = w + k;           // [k]  row a of U
  double* tv = ua + k;          // [k]  (U[a,:] B)
  double* Gps = tv + k;         // [k][k] G', symmetrised
  double* Uss = Gps + k * k;    // [k][k] U (u_smem only)
  const int a = blockIdx.x, tid = threadIdx.x;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int b = e / k, d = e % k;
    Gps[e] = 0.5 * (Gp[b * k + d] + Gp[d * k + b]);
    if (u_smem) Uss[e] = Us[e];
  }
  const double* Ur = u_smem ? Uss : Us;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (sums) {
    s0 = sums[0];
    s1 = sums[1];
    s2 = sums[2];
    vtot = sums[3];
    if (!(s0 > 0.0) || !isfinite(s0) || !isfinite(s1) || !isfinite(s2) || !(vtot > 0.0)) flag(status, ST_NONFINITE);
  } else {
    for (int i = tid; i < N; i += blockDim.x) {
      const double r = rho2[i];
      s0 += 1.0 / r;
      if (a == 0) {
        if (!(r > 0.0) || !isfinite(r)) flag(status, ST_NONFINITE);
        s1 += (double)vox[i] * log(r);
        s2 += sqnorm[i] / r;
      }
    }
    block_sum3(s0, s1, s2);
  }
  const double rho0 = s0;
  for (int b = tid; b < k; b += blockDim.x) {
    w[b] = 1.0 / (1.0 + rho0 * Gp[b * k + b]);
    ua[b] = Us[a * k + b];
  }
  __syncthreads();
  // tv[d] = sum_b U[a][b] B[b][d],  B_bd = (b == d) ? lambda_b w_b : w_b w_d G'_bd
  for (int d = tid; d < k; d += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < k; ++b) s = fma(ua[b] * w[b], Gps[b * k + d], s);
    // the diagonal term: lambda_d w_d (not w_d^2 lambda_d)
    s = (s - ua[d] * w[d] * Gps[d * k + d]) * w[d] + ua[d] * Gps[d * k + d] * w[d];
    tv[d] = s;
  }
  __syncthreads();
  for (int cc = tid; cc < k; cc += blockDim.x) {
    double s = 0.0;
    for (int d = 0; d < k; ++d) s = fma(tv[d], Ur[cc * k + d], s);
    if (!isfinite(s)) flag(status, ST_NONFINITE);
    Phi[a * k + cc] = s;
    Phi32[a * k + cc] = (float)s;
  }
  if (a == 0) {
    double ld = 0.0;
    for (int b = tid; b < k; b += blockDim.x) {
      const double lam = Gp[b * k + b];
      if (!(lam > 0.0)) flag(status, ST_NOT_PD);
      ld += log1p(rho0 * lam);
    }
    double z0 = 0.0, z1 = 0.0;
    block_sum3(ld, z0, z1);
    if (tid == 0) {
      scal[SC_RHO0] = rho0;
      scal[SC_LOGDET] = ld;
      scal[SC_VLOGRHO] = s1;
      scal[SC_SQRHO] = s2;
      scal[SC_VTOT] = vtot;
    }
  }
}

// A sharded E-step (Algorithm 1's Reduce, done by the caller between
// shards): this context's share of y = sum_i rho_i^-2 W_i^T X^_i, the group
// partials summed in group order exactly as es_kernel sums them (error-free
// FP32), written as FP64 hi + lo; one thread per (f, t).
__global__ void __launch_bounds__(256) ysum_kernel(int G, int k, int T, const float2* __restrict__ ypart,
                                                   double* __restrict__ y) {
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x, kT = (int64_t)k * T;
  if (e >= kT) return;
  float yh = 0.f, yl = 0.f;
  for (int q = 0; q < G; ++q) {
    const float2 v = __ldcg(ypart + (int64_t)q * kT + e);
    float hs, he;
    two_sum(yh, v.x, hs, he);
    yh = hs;
    yl += he + v.y;
  }
  y[e] = (double)yh + (double)yl;
}

// This context's share of the E-step's sums over subjects:
// {sum rho_i^-2 (eq:srm_wt_psi_w), sum v_i ln rho_i^2, sum ||X^_i||^2 / rho_i^2,
// sum v_i}; one block, a fixed-order tree.
__global__ void __launch_bounds__(256) shard_sums_kernel(int N, const double* __restrict__ rho2,
                                                         const double* __restrict__ sqnorm,
                                                         const int64_t* __restrict__ vox, double* __restrict__ out) {
  __shared__ double v4[256];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int i = threadIdx.x; i < N; i += 256) {
    const double r = rho2[i];
    s0 += 1.0 / r;
    s1 += (double)vox[i] * log(r);
    s2 += sqnorm[i] / r;
    s3 += (double)vox[i];
  }
  block_sum3(s0, s1, s2);
  v4[threadIdx.x] = s3;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) v4[threadIdx.x] += v4[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
    out[3] = v4[0];
  }
}

constexpr int ES_T = 8;  // columns of E[S] per es block

__global__ void __launch_bounds__(256) es_kernel(int G, int k, int T, int kld, int ldT, const float* __restrict__ Phi32,
                                                 const float2* __restrict__ ypart, double* __restrict__ ES64,
                                                 float* __restrict__ ESt, __nv_bfloat16* __restrict__ ESb,
                                                 float* __restrict__ sPart, double* __restrict__ yePart,
                                                 const double* __restrict__ y64) {
  __shared__ float Ys[KMAX][ES_T];
  __shared__ float Es[KMAX][ES_T];
  __shared__ double red[256];
  extern __shared__ float es_smem[];
  float* Ps = es_smem;  // [k][k] Phi (symmetrised, FP32)
  const int t0 = blockIdx.x * ES_T, tid = threadIdx.x;
  const int64_t kT = (int64_t)k * T;
  for (int e = tid; e < k * k; e += 256) {
    const int f = e / k, m = e - f * k;
    Ps[e] = 0.5f * (Phi32[e] + Phi32[m * k + f]);
  }
  // y: each thread owns up to two (f, t) elements; all group loads of a step in flight
  for (int e = tid; e < k * ES_T; e += 256) {
    const int f = e / ES_T, tt = e - f * ES_T, t = t0 + tt;
    float yv = 0.f;
    if (t < T && y64) {
      yv = (float)y64[(int64_t)f * T + t];  // the y of a sharded E-step, reduced over the shards
    } else if (t < T) {
      const float2* zp = ypart + (int64_t)f * T + t;
      float yh = 0.f, yl = 0.f;
      int q = 0;
      for (; q + 8 <= G; q += 8) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(zp + (int64_t)(q + u) * kT);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float hs, he;
          two_sum(yh, v[u].x, hs, he);
          yh = hs;
          yl += he + v[u].y;
        }
      }
      for (; q < G; ++q) {
        const float2 v = __ldcg(zp + (int64_t)q * kT);
        float hs, he;
        two_sum(yh, v.x, hs, he);
        yh = hs;
        yl += he + v.y;
      }
      yv = yh + yl;
    }
    Ys[f][tt] = yv;
  }
  __syncthreads();
  double ye = 0.0;
  for (int e = tid; e < k * ES_T; e += 256) {
    const int f = e / ES_T, tt = e - f * ES_T, t = t0 + tt;
    float s = 0.f;
    for (int m = 0; m < k; ++m) s = fmaf(Ps[f * k + m], Ys[m][tt], s);
    if (t >= T) s = 0.f;
    Es[f][tt] = s;
    if (t < T) {
      ye += (double)Ys[f][tt] * (double)s;
      ES64[(int64_t)f * T + t] = (double)s;
      if (ESt) ESt[(int64_t)t * kld + f] = s;
      if (ESb) ESb[(int64_t)f * ldT + t] = __float2bfloat16_rn(s);
    }
  }
  __syncthreads();
  float* pc = sPart + (int64_t)blockIdx.x * k * k;
  for (int e = tid; e < k * k; e += 256) {
    const int a = e / k, b = e - a * k;
    if (b < a) continue;
    float sab = 0.f;
#pragma unroll
    for (int tt = 0; tt < ES_T; ++tt) sab = fmaf(Es[a][tt], Es[b][tt], sab);
    pc[a * k + b] = sab;
    pc[b * k + a] = sab;
  }
  red[tid] = ye;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st) red[tid] += red[tid + st];
    __syncthreads();
  }
  if (tid == 0) yePart[blockIdx.x] = red[0];
}

// Sigma_s^new = Phi + E[S] E[S]^T / T (eq:srm_variance_update_optimized) from
// the chunk partials (summed in chunk order, error-free FP32 accumulation),
// and the log-likelihood of the E-step that produced them.  grid k blocks
// (row a), 256 threads; block 0 also finishes the likelihood.
__global__ void __launch_bounds__(256) sigma_kernel(int k, int T, int nchunk, const double* __restrict__ Phi,
                                                    const float* __restrict__ sPart,
                                                    const double* __restrict__ yePart, double* __restrict__ SigmaNext,
                                                    double* __restrict__ scal, double* __restrict__ ll, int* iter,
                                                    int max_iter, int* status) {
  const int a = blockIdx.x, tid = threadIdx.x;
  const int64_t kk2 = (int64_t)k * k;
  // four threads per element (adjacent lanes), each a contiguous quarter of
  // the partials; the quarters are then added in order
  const int sub = tid & 3;
  const int q0 = (nchunk * sub) / 4, q1 = (nchunk * (sub + 1)) / 4;
  for (int b0 = 0; b0 < k; b0 += 64) {
    const int b = b0 + (tid >> 2);
    const bool in = b < k;
    const int e = a * k + (in ? b : 0);
    float sh = 0.f, sl = 0.f;
    int q = q0;
    for (; q + 8 <= q1; q += 8) {  // eight loads in flight
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = sPart[(int64_t)(q + u) * kk2 + e];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float hs, he;
        two_sum(sh, v[u], hs, he);
        sh = hs;
        sl += he;
      }
    }
    for (; q < q1; ++q) {
      float hs, he;
      two_sum(sh, sPart[(int64_t)q * kk2 + e], hs, he);
      sh = hs;
      sl += he;
    }
    // combine the four quarters in order (lanes 4j .. 4j + 3)
    const int base = (tid & 31) & ~3;
    float h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      h[u] = __shfl_sync(0xffffffffu, sh, base + u);
      l[u] = __shfl_sync(0xffffffffu, sl, base + u);
    }
    if (sub == 0 && in) {
      float th = h[0], tl = l[0];
#pragma unroll
      for (int u = 1; u < 4; ++u) {
        float hs, he;
        two_sum(th, h[u], hs, he);
        th = hs;
        tl += he + l[u];
      }
      const double v = 0.5 * (Phi[a * k + b] + Phi[b * k + a]) + ((double)th + (double)tl) / (double)T;
      if (!isfinite(v)) flag(status, ST_NONFINITE);
      SigmaNext[e] = v;
    }
  }
  if (a != 0) return;
  // <y, Phi y>: the per-block partials summed by a fixed-order tree
  __shared__ double yred[256];
  double ys = 0.0;
  for (int q = tid; q < nchunk; q += 256) ys += yePart[q];
  yred[tid] = ys;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st) yred[tid] += yred[tid + st];
    __syncthreads();
  }
  if (tid == 0) {
    const double yes = yred[0];
    scal[SC_YPHIY] = yes;
    const double Vtot = scal[SC_VTOT];  // all subjects' voxels (all shards' in a sharded E-step)
    const double L = -0.5 * ((double)T * Vtot * 1.8378770664093454835606594728112 + (double)T * scal[SC_VLOGRHO] +
                             (double)T * scal[SC_LOGDET] + scal[SC_SQRHO] - yes);
    if (!isfinite(L)) flag(status, ST_NONFINITE);
    const int it = *iter;
    if (it >= 0 && it < max_iter) ll[it] = L;
    *iter = it + 1;
  }
}

// ------------------------------------------------------------------ M-step
constexpr int JAC_MAX_SWEEPS = 24;

// One block per symmetric matrix: blocks 0..N-1 take G_i from the Gram
// partials, block N takes Sigma_s^new.  FP32 one-sided (Hestenes) Jacobi:
// the columns of Y = G V are made mutually orthogonal by plane rotations
// applied to the columns of Y and V alike, starting from V = U_w (the
// previous eigenvectors).  When they are orthogonal, V diagonalises G^2 and
// hence G (G is symmetric positive semi-definite).  Round-robin ordering of
// the column pairs; one warp owns one pair in a round: it holds the two
// columns of Y and of V in registers, forms their Gram entries with warp
// reductions, rotates, and writes them back; one barrier per round.
// Convergence is tested between sweeps by one parallel pass over all pairs
// (no rotations, so every thread takes its own pairs without barriers): the
// loop ends as soon as no pair has |y_p.y_q| > OSJ_STOP |y_p| |y_q|, which
// with a good warm start is often before the first sweep; a sweep rotates
// every pair above OSJ_TOL.  At most JAC_MAX_SWEEPS sweeps.  The residual
// off-diagonal part E of V^T G V is then bounded by OSJ_STOP min(lambda_p,
// lambda_q) pair by pair; the FP64 refinement removes it to first order, so
// what is left of it in G^{-1/2}, tr G^{1/2} and log det is of relative size
// k OSJ_STOP^2 (about 5e-7 for k = 50).  Output U_0 = V (FP64).
constexpr float OSJ_TOL = 1e-5f;
constexpr float OSJ_STOP = 1e-4f;

template <int RPL>  // rows per lane: kk <= 32 * RPL
__global__ void __launch_bounds__(1024) eig_kernel(int N, int k, int kld, const float* __restrict__ gpart,
                                                   const int* __restrict__ gslot_off,
                                                   const double* __restrict__ SigmaNext, double* __restrict__ G64,
                                                   const float* __restrict__ Uwarm, double* __restrict__ U64,
                                                   int* __restrict__ sweeps_out, int* status, int first,
                                                   const int* __restrict__ only) {
  extern __shared__ float eig_smem[];
  const int kk = k + (k & 1);
  float* Gs = eig_smem;           // [kk][kk] G (symmetric)
  float* Yc = Gs + kk * kk;       // columns of Y: column j at Yc + j * kk
  float* Vc = Yc + kk * kk;       // columns of V
  uint16_t* tab = reinterpret_cast<uint16_t*>(Vc + kk * kk);  // [kk-1][kk/2]: p | q << 8
  float* nrm = Vc + kk * kk + ((kk - 1) * (kk / 2) + 1) / 2;    // [kk] |y_p|^2
  const int i = blockIdx.x + first, tid = threadIdx.x, nt = blockDim.x;
  if (only && i < N && only[i] == 0) return;  // this subject's polar factor is already certified
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  double* Gi = G64 + (int64_t)i * k * k;
  const float* Uw = Uwarm + (int64_t)i * k * k;
  const int npair = kk / 2;
  for (int e = tid; e < (kk - 1) * npair; e += nt) {
    const int round = e / npair, j = e - round * npair;
    const int pa = (j == 0) ? 0 : 1 + ((j - 1 + round) % (kk - 1));
    const int pb = 1 + ((kk - 2 - j + round) % (kk - 1));
    tab[e] = (uint16_t)(min(pa, pb) | (max(pa, pb) << 8));
  }
  if (i < N) {
    const int s0 = gslot_off[i], s1 = gslot_off[i + 1];
    for (int e = tid; e < k * k; e += nt) {
      const int a = e / k, b = e % k;
      double sum = 0.0;
      for (int q = s0; q < s1; ++q) sum += (double)gpart[(int64_t)q * kld * kld + a * kld + b];
      Gi[e] = sum;
    }
  } else {
    for (int e = tid; e < k * k; e += nt) Gi[e] = SigmaNext[e];
  }
  // scale: max |G_ab|, so that the FP32 Jacobi works on entries of order 1
  // (Gram entries of large subjects exceed 1e12, and |y|^2 products would
  // overflow FP32); the eigenvectors do not change
  __shared__ unsigned gmax_bits;
  if (tid == 0) gmax_bits = 0u;
  __syncthreads();
  {
    float mx = 0.f;
    for (int e = tid; e < k * k; e += nt) mx = fmaxf(mx, (float)fabs(Gi[e]));
    atomicMax(&gmax_bits, __float_as_uint(mx));  // non-negative floats order as their bit patterns
  }
  __syncthreads();
  const float gm = __uint_as_float(gmax_bits);
  const double gsc = (gm > 0.f && isfinite(gm)) ? 1.0 / (double)gm : 1.0;
  // Gs = G / max |G| (symmetrised, FP32; the padding row/column is zero), Vc = U_w (padded with e_k)
  for (int e = tid; e < kk * kk; e += nt) {
    const int a = e / kk, b = e % kk;
    float g = 0.f, u;
    if (a < k && b < k) {
      g = (float)(0.5 * (Gi[a * k + b] + Gi[b * k + a]) * gsc);
      u = Uw[a * k + b];
    } else {
      u = (a == b) ? 1.f : 0.f;
    }
    if (!isfinite(g)) flag(status, ST_NONFINITE);
    Gs[a * kk + b] = g;
    Vc[b * kk + a] = u;  // column b, row a
  }
  __syncthreads();
  // Y = G V (column-major)
  for (int e = tid; e < kk * kk; e += nt) {
    const int j = e / kk, r = e % kk;
    float sum = 0.f;
    for (int m = 0; m < kk; ++m) sum = fmaf(Gs[r * kk + m], Vc[j * kk + m], sum);
    Yc[j * kk + r] = sum;
  }
  bool converged = false;
  int sweep = 0;
  for (;;) {
    // convergence test: count the pairs with |y_p.y_q| > OSJ_STOP |y_p| |y_q|
    __syncthreads();
    for (int p = tid; p < kk; p += nt) {
      float a = 0.f;
      for (int r = 0; r < kk; ++r) a = fmaf(Yc[p * kk + r], Yc[p * kk + r], a);
      nrm[p] = a;
    }
    __syncthreads();
    bool above = false;
    for (int e = tid; e < kk * kk; e += nt) {
      const int p = e / kk, q = e - p * kk;
      if (q <= p || q >= k) continue;
      const float* yp = Yc + p * kk;
      const float* yq = Yc + q * kk;
      float g0 = 0.f, g1 = 0.f;
      int r = 0;
      for (; r + 1 < kk; r += 2) {
        g0 = fmaf(yp[r], yq[r], g0);
        g1 = fmaf(yp[r + 1], yq[r + 1], g1);
      }
      if (r < kk) g0 = fmaf(yp[r], yq[r], g0);
      const float g = g0 + g1;
      if (g * g > OSJ_STOP * OSJ_STOP * nrm[p] * nrm[q] && fabsf(g) > 1e-30f) above = true;
    }
    if (__syncthreads_or(above) == 0) {
      converged = true;
      break;
    }
    if (sweep == JAC_MAX_SWEEPS) break;
    ++sweep;
    for (int round = 0; round < kk - 1; ++round) {
      for (int j = warp; j < npair; j += nw) {
        const uint16_t tq = tab[round * npair + j];
        const int p = tq & 255, q = tq >> 8;
        float yp[RPL], yq[RPL], vp[RPL], vq[RPL];
        float a = 0.f, b = 0.f, g = 0.f;
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int r = lane + 32 * u;
          const bool in = r < kk;
          yp[u] = in ? Yc[p * kk + r] : 0.f;
          yq[u] = in ? Yc[q * kk + r] : 0.f;
          vp[u] = in ? Vc[p * kk + r] : 0.f;
          vq[u] = in ? Vc[q * kk + r] : 0.f;
          a = fmaf(yp[u], yp[u], a);
          b = fmaf(yq[u], yq[u], b);
          g = fmaf(yp[u], yq[u], g);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        const float ag = fabsf(g), sab = sqrtf(a * b);
        if (q < k && ag > OSJ_TOL * sab && ag > 1e-30f) {
          const float tau = (b - a) * __fdividef(1.f, 2.f * g);
          const float w = 1.f + tau * tau;
          const float t = copysignf(__fdividef(1.f, fabsf(tau) + w * rsqrtf(w)), tau);
          const float c = rsqrtf(1.f + t * t), sn = t * c;
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int r = lane + 32 * u;
            if (r < kk) {
              Yc[p * kk + r] = c * yp[u] - sn * yq[u];
              Yc[q * kk + r] = sn * yp[u] + c * yq[u];
              Vc[p * kk + r] = c * vp[u] - sn * vq[u];
              Vc[q * kk + r] = sn * vp[u] + c * vq[u];
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (!converged && tid == 0) flag(status, ST_EIG_NOCONV);
  if (tid == 0 && sweeps_out) sweeps_out[i] = sweep + (only ? 256 : 0);
  // U_0 = V
  double* Uo = U64 + (int64_t)i * k * k;
  for (int e = tid; e < k * k; e += nt) {
    const int a = e / k, b = e % k;
    Uo[e] = (double)Vc[b * kk + a];
  }
}

size_t eig_smem_bytes(int k) {
  const int kk = k + (k & 1);
  return sizeof(float) * (3 * kk * kk + ((kk - 1) * (kk / 2) + 1) / 2 + kk) + 16;
}

int eig_threads(int k) {
  const int npair = (k + (k & 1)) / 2;
  return 32 * (npair < 32 ? (npair < 1 ? 1 : npair) : 32);
}

// D_b = alpha op(A_b) op(B_b) + beta C_b for a batch of k x k FP64 matrices.
// grid (nband, nbatch), 256 threads.  op(B) is staged in shared memory as
// [m][c] and the band of op(A) as [r][m]; with sym != 0 only c >= r is
// computed and mirrored (the product is known to be symmetric).  With
// only != nullptr, matrices b with only[b] == 0 are skipped.
__global__ void __launch_bounds__(256) bgemm64_kernel(int k, int nband, const double* __restrict__ A, int tA,
                                                      const double* __restrict__ B, int tB, double alpha,
                                                      const double* __restrict__ C, double beta,
                                                      double* __restrict__ D, int sym,
                                                      const int* __restrict__ only) {
  extern __shared__ double bg_smem[];
  if (only && only[blockIdx.y] == 0) return;  // matrix not selected
  const int ldb = k + 1;
  double* Bs = bg_smem;              // [k][k+1]
  double* As = Bs + k * ldb;         // [band][k+1]
  const int b = blockIdx.y;
  const int r0 = (k * blockIdx.x) / nband, r1 = (k * (blockIdx.x + 1)) / nband;
  const int nr = r1 - r0;
  const int64_t base = (int64_t)b * k * k;
  const double* Ab = A + base;
  const double* Bb = B + base;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int m = e / k, c = e % k;
    Bs[m * ldb + c] = tB ? Bb[c * k + m] : Bb[e];
  }
  for (int e = threadIdx.x; e < nr * k; e += blockDim.x) {
    const int r = e / k, m = e % k;
    As[r * ldb + m] = tA ? Ab[m * k + r0 + r] : Ab[(r0 + r) * k + m];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * k; e += blockDim.x) {
    const int r = e / k, c = e % k;
    if (sym && c < r0 + r) continue;
    double s = 0.0;
    const double* ar = As + r * ldb;
    for (int m = 0; m < k; ++m) s = fma(ar[m], Bs[m * ldb + c], s);
    double out = alpha * s;
    if (C) out += beta * C[base + (r0 + r) * k + c];
    D[base + (r0 + r) * k + c] = out;
    if (sym) D[base + c * k + r0 + r] = out;
  }
}

// Per matrix: eigenvalues lambda = diag(G'), G' = U^T G U (FP64); for the
// subjects (i < N) the Daleckii-Krein matrix for f(x) = x^-1/2,
//   B = diag(lambda^-1/2) + F o E,  F_ab = -1 / (s_a s_b (s_a + s_b)), s = sqrt(lambda),
// the nuclear norm sum s_a and the rho update.  Block 0 commits
// Sigma_s <- Sigma_s^new.  Block N (Sigma_s^new) only checks its eigenvalues.
__global__ void __launch_bounds__(128) dk_rho_kernel(int N, int k, int T, const double* __restrict__ Gp,
                                                     double* __restrict__ Bout, double* __restrict__ eigv,
                                                     const double* __restrict__ sqnorm,
                                                     const int64_t* __restrict__ vox,
                                                     const double* __restrict__ SigmaNext, double* __restrict__ Sigma,
                                                     double* __restrict__ rho2, double* __restrict__ scal,
                                                     int* status, const int* __restrict__ only) {
  __shared__ double sq[KMAX];
  if (only && (blockIdx.x >= N || only[blockIdx.x] == 0)) return;  // subject not selected
  __shared__ double red[3][128];
  const int i = blockIdx.x, tid = threadIdx.x;
  const double* G = Gp + (int64_t)i * k * k;
  // lambda = diag(G'), its maximum, tr Sigma_s^new (parallel, fixed-order tree)
  double lam = 0.0, lm = 0.0, tr = 0.0;
  if (tid < k) {
    lam = G[tid * k + tid];
    lm = lam;
    tr = SigmaNext[tid * k + tid];
  }
  red[0][tid] = lm;
  red[1][tid] = tr;
  __syncthreads();
  for (int st = 64; st > 0; st >>= 1) {
    if (tid < st) {
      red[0][tid] = fmax(red[0][tid], red[0][tid + st]);
      red[1][tid] += red[1][tid + st];
    }
    __syncthreads();
  }
  const double lmax = red[0][0], trS = red[1][0];
  if (tid < k) {
    if (!(lam > 1e-12 * lmax) || !isfinite(lam)) flag(status, i < N ? ST_RANK : ST_NOT_PD);
    sq[tid] = sqrt(lam > 1e-300 ? lam : 1e-300);
    eigv[(int64_t)i * k + tid] = lam;
  }
  if (i == 0)
    for (int e = tid; e < k * k; e += blockDim.x) Sigma[e] = SigmaNext[e];
  if (i >= N) return;
  __syncthreads();
  // off-diagonal divided differences are multiplied by E = O(1e-6 |G|), so
  // FP32 factors keep B to FP64 accuracy
  double* Bm = Bout + (int64_t)i * k * k;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e - a * k;
    double v;
    if (a == b) {
      v = 1.0 / sq[a];
    } else {
      const float sa = (float)sq[a], sb = (float)sq[b];
      const float f = -1.f / (sa * sb * (sa + sb));
      v = (double)f * (0.5 * (G[a * k + b] + G[b * k + a]));
    }
    Bm[e] = v;
  }
  red[2][tid] = (tid < k) ? sq[tid] : 0.0;
  __syncthreads();
  for (int st = 64; st > 0; st >>= 1) {
    if (tid < st) red[2][tid] += red[2][tid + st];
    __syncthreads();
  }
  if (tid == 0) {
    const double r = (sqnorm[i] - 2.0 * red[2][0] + (double)T * trS) / ((double)T * (double)vox[i]);
    if (!(r > 0.0) || !isfinite(r)) flag(status, ST_NONFINITE);
    rho2[i] = r;
    if (i == 0) scal[SC_TRSIG] = trS;
  }
}

// ---------------------------------------------------------------- polar factor by Newton-Schulz
// For k <= NS_KMAX: M_i = (A_i^T A_i)^-1/2 and ||A_i||_* without an
// eigen-decomposition when A_i^T A_i is well conditioned.  One CTA per
// subject.  With G = A_i^T A_i (error-free sum of the Gram partials) and
// c = min(||G||_F, ||G||_inf) >= lambda_max, the coupled Newton-Schulz
// iteration on A = G / c,
//     P = Z Y,  T = (3 I - P) / 2,  Y <- Y T,  Z <- T Z,   Y_0 = A, Z_0 = I,
// converges quadratically to Y = A^1/2, Z = A^-1/2 for a symmetric positive
// definite A (eigenvalues in (0, 1]); it is the stable, coupled form.  It
// stops one update after max |P - I| < NS_TOL; M_0 = Z / sqrt(c).
//
// FP32 arithmetic leaves M_0 with an error of about eps cond(G) in the
// directions of the small eigenvalues, so each result is certified: with
// E = M_0 G M_0 - I and delta = M_0 - G^-1/2, first order gives
// E_ab = (sqrt(lambda_a) + sqrt(lambda_b)) delta_ab in the eigenbasis of G,
// while the polar factor's error A_i delta has entries sqrt(lambda_a)
// delta_ab; so ||A_i delta||_F <= ||E||_F.  For the FP32 store E is formed
// in compensated FP32 (error-free products and sums, G split into two FP32
// parts); for the BF16 store, whose threshold is 50 times larger, in plain
// FP32 (its rounding, about k eps sqrt(cond G) per entry, can only make a
// subject fail).  A subject with ||E||_F > cert sqrt(k) (or no convergence)
// is marked for the eigen-decomposition path (Jacobi + FP64 refinement),
// which then overwrites its M_i and rho_i^2.
//
// ||A_i||_* = tr(W^T A_i) for the polar factor W.  With W~ = A_i M_0 and
// W = W~ (I + E)^-1/2 (orthonormal), tr(W^T A_i) = tr(M_0 G) - tr(E M_0 G)/2
// + O(|E|^2), stationary at the exact M (the trace is maximal there).
//
// Matrices are KP x KP (KP = k rounded up to 4) FP32 in shared memory with
// zero padding; the products use 4 x 4 register tiles whose operands are
// read as float4 (the left operand as its transpose, which for these
// symmetric matrices is itself), each tile's inner index split over 2 or 4
// lanes.
constexpr int NS_KMAX = 64;


constexpr int NS_THREADS = 512;

__device__ __forceinline__ float block_max_ns(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = red[0];
#pragma unroll
  for (int w = 1; w < NS_THREADS / 32; ++w) r = fmaxf(r, red[w]);
  __syncthreads();
  return r;
}

// Sums of two floats over the NS_THREADS threads (fixed-order shuffle tree,
// then the warp partials in warp order); every thread gets the totals.
__device__ void block_sum2f_ns(float& a, float& b, float (*red)[NS_THREADS / 32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  a = red[0][0];
  b = red[1][0];
#pragma unroll
  for (int w = 1; w < NS_THREADS / 32; ++w) {
    a += red[0][w];
    b += red[1][w];
  }
  __syncthreads();
}

// ---- 4 x 4 register tiles of C = A^T B split over KS lanes along the inner
// index (lanes l ^ 1, l ^ 2, ... hold the parts of one tile and add them by
// shuffles).  With COMP the products are error-free (A^T B_hi in hi + lo
// plus A^T B_lo), as in ns_mm2.
template <int KS, bool COMP>
__device__ __forceinline__ void tile_part(const float* __restrict__ A, const float* __restrict__ Bh,
                                          const float* __restrict__ Bl, int KP, int tr, int tc, int q, bool valid,
                                          float (&hi)[4][4], float (&lo)[4][4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) hi[u][v] = lo[u][v] = 0.f;
  if (!valid) return;
  const int KQ = ((KP / 4 + KS - 1) / KS) * 4;
  const int m0 = q * KQ, m1 = min(KP, m0 + KQ);
#pragma unroll 2
  for (int m = m0; m < m1; ++m) {
    const float4 a = *reinterpret_cast<const float4*>(A + m * KP + 4 * tr);
    const float4 b = *reinterpret_cast<const float4*>(Bh + m * KP + 4 * tc);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
    if (!COMP) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) hi[u][v] = fmaf(av[u], bv[v], hi[u][v]);
    } else {
      const float4 bl = *reinterpret_cast<const float4*>(Bl + m * KP + 4 * tc);
      const float lv[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          // rounded on its own (never fused into the sum below), so that
          // p + pe is the exact product and two_sum stays error-free
          const float p = __fmul_rn(av[u], bv[v]);
          const float pe = fmaf(av[u], bv[v], -p);  // exact product error
          float sm, se;
          two_sum(hi[u][v], p, sm, se);
          hi[u][v] = sm;
          lo[u][v] += se + pe;
          lo[u][v] = fmaf(av[u], lv[v], lo[u][v]);
        }
    }
  }
}
// C = A^T B for KP x KP operands whose product is symmetric (here: A, B
// commuting symmetric polynomials of the same matrix, so C = A B = B A):
// the upper tiles only, mirrored.  Threads [base, base + nth) of the block,
// nth a multiple of 32; tiles from the upper-tile table `ut` (nut entries).
template <int KS>
__device__ __forceinline__ void sym_mm(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C,
                                       int KP, const uint16_t* __restrict__ ut, int nut, int base, int nth) {
  const int lt = (int)threadIdx.x - base;
  if (lt < 0 || lt >= nth) return;  // whole warps
  const int per = nth / KS;
  const int q = lt % KS;
  for (int t0 = 0; t0 < nut; t0 += per) {
    const int t = t0 + lt / KS;
    const bool valid = t < nut;
    const int tr = valid ? (ut[t] & 0xff) : 0, tc = valid ? (ut[t] >> 8) : 0;
    float hi[4][4], lo[4][4];
    tile_part<KS, false>(A, B, nullptr, KP, tr, tc, q, valid, hi, lo);
    tile_combine<KS, false>(hi, lo);
    if (valid && q == 0) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        *reinterpret_cast<float4*>(C + (4 * tr + u) * KP + 4 * tc) = make_float4(hi[u][0], hi[u][1], hi[u][2], hi[u][3]);
      if (tc != tr) {
#pragma unroll
        for (int v = 0; v < 4; ++v)
          *reinterpret_cast<float4*>(C + (4 * tc + v) * KP + 4 * tr) = make_float4(hi[0][v], hi[1][v], hi[2][v], hi[3][v]);
      }
    }
  }
}

// FP64 arithmetic runs at about 2 FMA per clock per SM on this GPU, so the
// kernel keeps it to O(k) scalar work: sums of Gram partials, the
// symmetrised G and tr(M_0 G) are carried as FP32 hi + lo pairs (error-free
// transformations), the rest is plain FP32.  All iterates Y, Z, T are
// polynomials in G, so every product of the iteration is symmetric and only
// its upper 4 x 4 tiles are computed.  The certificate's products are
// error-free for the FP32 store (comp = 1); for the BF16 store, whose
// threshold is 50 times larger, plain FP32 products suffice (comp = 0).
constexpr int NS_GE = 8;  // Gram elements per thread (KP * KP <= NS_GE * NS_THREADS)
static_assert(NS_GE * NS_THREADS >= NS_KMAX * NS_KMAX, "polar: Gram elements per thread");

template <bool COMP>
__device__ __forceinline__ void ns_certificate(const float* __restrict__ Mb, const float* __restrict__ Gh,
                                               const float* __restrict__ Gl, float* __restrict__ Ph,
                                               float* __restrict__ Pl, int k, int KP,
                                               const uint16_t* __restrict__ ut, int nut, float& e2, float& corr) {
  const int tid = threadIdx.x, nt4 = KP / 4;
  // R = M_0 G (all tiles), stored transposed: P = R^T = G M_0
  {
    constexpr int KS = 2;
    const int per = NS_THREADS / KS, q = tid % KS, ntile = nt4 * nt4;
    for (int t0 = 0; t0 < ntile; t0 += per) {
      const int t = t0 + tid / KS;
      const bool valid = t < ntile;
      const int tr = valid ? t / nt4 : 0, tc = valid ? t - (t / nt4) * nt4 : 0;
      float hi[4][4], lo[4][4];
      tile_part<KS, COMP>(Mb, Gh, Gl, KP, tr, tc, q, valid, hi, lo);
      tile_combine<KS, COMP>(hi, lo);
      if (valid && q == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            Ph[(4 * tc + v) * KP + 4 * tr + u] = hi[u][v];
            if (COMP) Pl[(4 * tc + v) * KP + 4 * tr + u] = lo[u][v];
          }
      }
    }
  }
  __syncthreads();
  // E = M_0 P - I (symmetric: upper tiles), ||E||_F^2 and
  // tr(E M_0 G) = sum_ab E_ab R_ba = sum_ab E_ab P_ab
  {
    constexpr int KS = 4;
    const int per = NS_THREADS / KS, q = tid % KS;
    for (int t0 = 0; t0 < nut; t0 += per) {
      const int t = t0 + tid / KS;
      const bool valid = t < nut;
      const int tr = valid ? (ut[t] & 0xff) : 0, tc = valid ? (ut[t] >> 8) : 0;
      float hi[4][4], lo[4][4];
      tile_part<KS, COMP>(Mb, Ph, Pl, KP, tr, tc, q, valid, hi, lo);
      tile_combine<KS, COMP>(hi, lo);
      if (valid && q == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int a = 4 * tr + u, b = 4 * tc + v;
            if (a >= k || b >= k || b < a) continue;
            const float ev = (hi[u][v] - (a == b ? 1.f : 0.f)) + lo[u][v];
            if (a == b) {
              e2 = fmaf(ev, ev, e2);
              corr = fmaf(ev, Ph[a * KP + a], corr);
            } else {
              e2 = fmaf(2.f * ev, ev, e2);
              corr = fmaf(ev, Ph[a * KP + b] + Ph[b * KP + a], corr);
            }
          }
      }
    }
  }
}

// MINB CTAs per SM: 1 when every subject has an SM of its own (latency), 2
// when subjects outnumber the SMs (throughput: half the waves, at the cost of
// a few spilled registers)
template <int MINB>
__global__ void __launch_bounds__(NS_THREADS, MINB) polar_ns_kernel(int N, int k, int kld, int T, const float* __restrict__ gpart,
                                                       const int* __restrict__ gslot_off,
                                                       double* __restrict__ M64, float* __restrict__ M32,
                                                       const double* __restrict__ sqnorm,
                                                       const int64_t* __restrict__ vox,
                                                       const double* __restrict__ SigmaNext,
                                                       double* __restrict__ Sigma, double* __restrict__ rho2,
                                                       double* __restrict__ scal, int* __restrict__ iters_out,
                                                       int* __restrict__ fallback, double cert, int comp,
                                                       int* status) {
  extern __shared__ __align__(16) float ns_smem[];
  __shared__ float redf[NS_THREADS / 32];
  __shared__ float red2[2][NS_THREADS / 32];
  __shared__ double trS_s;
  __shared__ float tmg_s[2];
  __shared__ uint16_t ut[(NS_KMAX / 4) * (NS_KMAX / 4 + 1) / 2];
  const int KP = (k + 3) & ~3;
  const int KK = KP * KP;
  const int nt4 = KP / 4, nut = nt4 * (nt4 + 1) / 2;
  float* Y = ns_smem;
  float* Z = Y + KK;
  float* Tm = Z + KK;
  float* W = Tm + KK;
  float* Xb = W + KK;
  float* Gh = Xb + KK;  // sym(G) = Gh + Gl, kept for the certificate
  float* Gl = Gh + KK;
  const int i = blockIdx.x, tid = threadIdx.x;
  for (int t = tid; t < nut; t += NS_THREADS) {  // upper tiles, row by row
    int r = 0, rem = t;
    while (rem >= nt4 - r) {
      rem -= nt4 - r;
      ++r;
    }
    ut[t] = (uint16_t)(r | ((r + rem) << 8));
  }
  // G = hi + lo from the Gram partials (slot order, error-free; loads of
  // four slots x NS_GE elements in flight); ||G||_F^2 from hi
  const int s0 = gslot_off[i], s1 = gslot_off[i + 1];
  const int64_t sst = (int64_t)kld * kld;
  float fro = 0.f, unused = 0.f;
  {
    float gh[NS_GE], gl[NS_GE];
    int off[NS_GE];
#pragma unroll
    for (int j = 0; j < NS_GE; ++j) {
      const int e = tid + j * NS_THREADS;
      const int a = e / KP, b = e - (e / KP) * KP;
      off[j] = (e < KK && a < k && b < k) ? a * kld + b : -1;
      gh[j] = gl[j] = 0.f;
    }
    for (int q = s0; q < s1; q += 4) {
      float g[NS_GE][4];
#pragma unroll
      for (int j = 0; j < NS_GE; ++j)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          g[j][jj] = (off[j] >= 0 && q + jj < s1) ? __ldg(gpart + (q + jj) * sst + off[j]) : 0.f;
#pragma unroll
      for (int j = 0; j < NS_GE; ++j)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          float sm, se;
          two_sum(gh[j], g[j][jj], sm, se);
          gh[j] = sm;
          gl[j] += se;
        }
    }
#pragma unroll
    for (int j = 0; j < NS_GE; ++j) {
      const int e = tid + j * NS_THREADS;
      if (e < KK) {
        float sm, se;
        two_sum(gh[j], gl[j], sm, se);
        W[e] = sm;  // raw G (hi, lo) until symmetrised below
        Xb[e] = se;
        fro = fmaf(sm, sm, fro);
      }
    }
  }
  // tr Sigma_s^new: one warp, fixed-order FP64 tree over the diagonal
  if (tid < 32) {
    double t = 0.0;
    for (int a = tid; a < k; a += 32) t += SigmaNext[a * k + a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (tid == 0) trS_s = t;
  }
  block_sum2f_ns(fro, unused, red2);  // (its barriers also publish W, Xb, trS_s, ut)
  const double trS = trS_s;
  // sym(G) in float-float into Gh, Gl; Y = sym(G) / c below; Z = I
  float rowmax = 0.f;
  for (int a = tid; a < k; a += NS_THREADS) {
    float rs = 0.f;
    for (int b = 0; b < k; ++b) rs += 0.5f * (fabsf(W[a * KP + b]) + fabsf(W[b * KP + a]));
    rowmax = fmaxf(rowmax, rs);
  }
  for (int e = tid; e < KK; e += NS_THREADS) {
    const int a = e / KP, b = e - (e / KP) * KP;
    float h = W[e], l = Xb[e];
    ff_add(h, l, W[b * KP + a], Xb[b * KP + a]);
    Gh[e] = 0.5f * h;  // exact scaling
    Gl[e] = 0.5f * l;
  }
  const float ginf = block_max_ns(rowmax, redf);  // (its barriers also publish Gh, Gl)
  // both bound lambda_max from above (the margin covers FP32 rounding of the bounds)
  const double c = fmin(sqrt((double)fro), (double)ginf) * (1.0 + 1e-5);
  const bool good_c = isfinite(c) && c > 0.0;
  const float cinv = good_c ? (float)(1.0 / c) : 0.f;
  for (int e = tid; e < KK; e += NS_THREADS) {
    const int a = e / KP, b = e - (e / KP) * KP;
    Y[e] = (Gh[e] + Gl[e]) * cinv;
    Z[e] = (a == b && a < k) ? 1.f : 0.f;
  }
  __syncthreads();
  int it = 0, extra = -1;
  bool conv = false;
  for (; good_c && it < NS_MAXIT; ++it) {
    // one update after max |P - I| < NS_TOL the iterates have converged (the
    // error of P squares per step); the certificate checks the result
    if (extra == 0) {
      conv = true;
      break;
    }
    sym_mm<4>(Z, Y, Tm, KP, ut, nut, 0, NS_THREADS);  // P = Z Y
    __syncthreads();
    // T = (3I - P) / 2 on the k block (zero elsewhere); e = max |P - I|
    float emax = 0.f;
    for (int e = tid; e < KK; e += NS_THREADS) {
      const int a = e / KP, b = e - (e / KP) * KP;
      float t = 0.f;
      if (a < k && b < k) {
        const float d = (a == b) ? 1.f : 0.f;
        const float pab = Tm[e];
        emax = fmaxf(emax, fabsf(pab - d));
        t = 1.5f * d - 0.5f * pab;
      }
      Tm[e] = t;
    }
    const float err = block_max_ns(emax, redf);
    if (!(err == err)) break;  // non-finite
    if (extra < 0 && err < NS_TOL) extra = 1;
    if (extra > 0) --extra;
    // Y T and T Z at once, each by half of the block
    sym_mm<2>(Y, Tm, W, KP, ut, nut, 0, NS_THREADS / 2);
    sym_mm<2>(Tm, Z, Xb, KP, ut, nut, NS_THREADS / 2, NS_THREADS / 2);
    __syncthreads();
    float* t = Y;
    Y = W;
    W = t;
    t = Z;
    Z = Xb;
    Xb = t;
  }
  // M_0 = Z / sqrt(c) into W; the certificate's product P = G M_0 into the
  // buffers of Y (hi) and T (lo)
  float* Mb = W;
  {
    const float sc = good_c ? (float)sqrt(1.0 / c) : 0.f;
    for (int e = tid; e < KK; e += NS_THREADS) Mb[e] = Z[e] * sc;
  }
  __syncthreads();
  float* Ph = Y;
  float* Pl = Tm;
  float e2 = 0.f, corr = 0.f;
  if (comp)
    ns_certificate<true>(Mb, Gh, Gl, Ph, Pl, k, KP, ut, nut, e2, corr);
  else
    ns_certificate<false>(Mb, Gh, Gl, Ph, Pl, k, KP, ut, nut, e2, corr);
  // tr(M_0 G) = tr P in float-float (hi + lo with comp, hi alone without)
  if (tid < 32) {
    float h = 0.f, l = 0.f;
    for (int a = tid; a < k; a += 32) ff_add(h, l, Ph[a * KP + a], comp ? Pl[a * KP + a] : 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
      ff_add(h, l, oh, ol);
    }
    if (tid == 0) {
      tmg_s[0] = h;
      tmg_s[1] = l;
    }
  }
  block_sum2f_ns(e2, corr, red2);
  const double tmg = (double)tmg_s[0] + (double)tmg_s[1];
  const double enorm = sqrt((double)e2);
  const bool ok = conv && good_c && enorm <= cert * sqrt((double)k) && isfinite(enorm);
  if (tid == 0) {
    if (iters_out) iters_out[i] = it;
    fallback[i] = ok ? 0 : 1;
    if (ok) {
      const double nuc = tmg - 0.5 * (double)corr;
      const double r = (sqnorm[i] - 2.0 * nuc + (double)T * trS) / ((double)T * (double)vox[i]);
      if (!(r > 0.0) || !isfinite(r)) flag(status, ST_NONFINITE);
      rho2[i] = r;
    }
    if (i == 0) scal[SC_TRSIG] = trS;
  }
  if (ok) {
    double* Mi = M64 + (int64_t)i * k * k;
    float* M32i = M32 + (int64_t)i * kld * kld;
    for (int e = tid; e < k * k; e += NS_THREADS) {
      const int a = e / k, b = e - a * k;
      const float m = Mb[a * KP + b];
      Mi[e] = (double)m;
      M32i[a * kld + b] = m;
    }
  }
  if (i == 0)
    for (int e = tid; e < k * k; e += NS_THREADS) Sigma[e] = SigmaNext[e];
}

size_t ns_smem_bytes(int k) {
  const int KP = (k + 3) & ~3;
  return sizeof(float) * 7 * (size_t)KP * KP;
}

// ---------------------------------------------------------------- fused M-step tail
// refine + rho for k <= MT_KMAX in one launch: a cluster of MT_C CTAs per
// symmetric matrix (subjects 0..N-1, Sigma_s^new as matrix N).  CTA r of a
// cluster owns the rows a = r (mod MT_C) of every intermediate; each product
// reads its right operand in full from global memory (L2), written there by
// the whole cluster before a cluster barrier (release/acquire at cluster
// scope; the loads bypass L1).  FP64 throughout, as in the unfused path:
//   H  = U0^T U0                     (symmetric: upper triangle, mirrored)
//   X  = 1.5 U0 - 0.5 U0 H           (re-orthonormalised eigenvectors)
//   H' = G X,  G' = X^T H'           (symmetric)
//   lambda = diag G', B = f(lambda) + F o E (Daleckii-Krein, f(x) = x^-1/2),
//   rho_i^2 from sum sqrt(lambda)    (subjects)
//   M  = X B X^T                     (symmetric; subjects only)
// and the FP32 copies M32 and Uwarm.  The products' left operands and
// outputs are this CTA's rows; the column loop runs over the lanes, so the
// right operand (row-major, odd row stride in shared memory) is read without
// bank conflicts and the left one is broadcast.
constexpr int MT_C = 8;
constexpr int MT_KMAX = 64;
constexpr int MT_RMAX = (MT_KMAX + MT_C - 1) / MT_C;

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __cluster_dims__(MT_C, 1, 1) __launch_bounds__(256)
    mtail_kernel(int N, int k, int kld, int T, const double* __restrict__ U64, double* __restrict__ G64,
                 double* __restrict__ H64, double* __restrict__ Xr64, double* __restrict__ M64,
                 float* __restrict__ M32, float* __restrict__ Uwarm, double* __restrict__ eigv,
                 const double* __restrict__ sqnorm, const int64_t* __restrict__ vox,
                 const double* __restrict__ SigmaNext, double* __restrict__ Sigma, double* __restrict__ rho2,
                 double* __restrict__ scal, int* status, int first, const int* __restrict__ only) {
  extern __shared__ double mt_smem[];
  const int kp = k | 1;                  // odd row stride
  double* Xs = mt_smem;                  // [k][kp] X
  double* Bs = Xs + k * kp;              // [k][kp] right operand
  double* Rs = Bs + k * kp;              // [MT_RMAX][kp] own rows
  double* sq = Rs + MT_RMAX * kp;        // [k] sqrt(lambda)
  __shared__ double red[3][256];
  const int r = blockIdx.x, i = blockIdx.y + first, tid = threadIdx.x;
  if (only && i < N && only[i] == 0) return;  // whole cluster: same i
  const int nr = (k - r + MT_C - 1) / MT_C;  // own rows: a = r + MT_C * al
  const int64_t kk2 = (int64_t)k * k;
  const double* Ui = U64 + i * kk2;
  double* Gi = G64 + i * kk2;
  double* Hi = H64 + i * kk2;
  double* Xi = Xr64 + i * kk2;
  // U0 -> Bs; own rows of U0 -> Rs
  for (int e = tid; e < k * k; e += 256) Bs[(e / k) * kp + e % k] = Ui[e];
  __syncthreads();
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, m = e - al * k;
    Rs[al * kp + m] = Bs[(r + MT_C * al) * kp + m];
  }
  // H = U0^T U0 (rows a, columns c >= a, mirrored)
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, c = e - al * k, a = r + MT_C * al;
    if (c < a) continue;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s = fma(Bs[m * kp + a], Bs[m * kp + c], s);
    Hi[a * k + c] = s;
    Hi[c * k + a] = s;
  }
  cluster_barrier();
  // X = 1.5 U0 - 0.5 U0 H
  for (int e = tid; e < k * k; e += 256) Bs[(e / k) * kp + e % k] = __ldcg(Hi + e);
  __syncthreads();
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, c = e - al * k, a = r + MT_C * al;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s = fma(Rs[al * kp + m], Bs[m * kp + c], s);
    const double x = 1.5 * Rs[al * kp + c] - 0.5 * s;
    Xi[a * k + c] = x;
    Uwarm[i * kk2 + a * k + c] = (float)x;
  }
  cluster_barrier();
  // H' = G X (own rows of G; all of X)
  for (int e = tid; e < k * k; e += 256) Xs[(e / k) * kp + e % k] = __ldcg(Xi + e);
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, m = e - al * k;
    Rs[al * kp + m] = Gi[(r + MT_C * al) * k + m];
  }
  __syncthreads();
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, c = e - al * k, a = r + MT_C * al;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s = fma(Rs[al * kp + m], Xs[m * kp + c], s);
    Hi[a * k + c] = s;
  }
  cluster_barrier();
  // G' = X^T H' (symmetric), into G64
  for (int e = tid; e < k * k; e += 256) Bs[(e / k) * kp + e % k] = __ldcg(Hi + e);
  __syncthreads();
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, c = e - al * k, a = r + MT_C * al;
    if (c < a) continue;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s = fma(Xs[m * kp + a], Bs[m * kp + c], s);
    Gi[a * k + c] = s;
    Gi[c * k + a] = s;
  }
  cluster_barrier();
  // lambda = diag G'; its maximum, sum sqrt(lambda), tr Sigma_s^new (fixed-order tree)
  double lam = 0.0, lm = 0.0, tr = 0.0, sl = 0.0;
  if (tid < k) {
    lam = __ldcg(Gi + tid * k + tid);
    lm = lam;
    tr = SigmaNext[tid * k + tid];
    sl = sqrt(lam > 1e-300 ? lam : 1e-300);
    sq[tid] = sl;
  }
  red[0][tid] = lm;
  red[1][tid] = tr;
  red[2][tid] = (tid < k) ? sl : 0.0;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st) {
      red[0][tid] = fmax(red[0][tid], red[0][tid + st]);
      red[1][tid] += red[1][tid + st];
      red[2][tid] += red[2][tid + st];
    }
    __syncthreads();
  }
  const double lmax = red[0][0], trS = red[1][0], ssum = red[2][0];
  if (r == 0) {
    if (tid < k) {
      if (!(lam > 1e-12 * lmax) || !isfinite(lam)) flag(status, i < N ? ST_RANK : ST_NOT_PD);
      eigv[(int64_t)i * k + tid] = lam;
    }
    if (i == 0)
      for (int e = tid; e < k * k; e += 256) Sigma[e] = SigmaNext[e];
    if (i < N && tid == 0) {
      const double rr = (sqnorm[i] - 2.0 * ssum + (double)T * trS) / ((double)T * (double)vox[i]);
      if (!(rr > 0.0) || !isfinite(rr)) flag(status, ST_NONFINITE);
      rho2[i] = rr;
      if (i == 0) scal[SC_TRSIG] = trS;
    }
  }
  if (i >= N) return;  // Sigma_s: X and G' are kept for the next E-step
  // B = f(lambda) + F o E into H64: the off-diagonal divided differences
  // multiply E = O(1e-4 |G|) and are taken in FP32
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, c = e - al * k, a = r + MT_C * al;
    double v;
    if (a == c) {
      v = 1.0 / sq[a];
    } else {
      const float sa = (float)sq[a], sb = (float)sq[c];
      const float f = -1.f / (sa * sb * (sa + sb));
      v = (double)f * __ldcg(Gi + a * k + c);
    }
    Hi[a * k + c] = v;
  }
  cluster_barrier();
  // T1 = X B (own rows, kept in Rs), then M = T1 X^T (symmetric)
  for (int e = tid; e < k * k; e += 256) Bs[(e / k) * kp + e % k] = __ldcg(Hi + e);
  __syncthreads();
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, c = e - al * k, a = r + MT_C * al;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s = fma(Xs[a * kp + m], Bs[m * kp + c], s);
    Rs[al * kp + c] = s;
  }
  __syncthreads();
  double* Mi = M64 + i * kk2;
  float* M32i = M32 + (int64_t)i * kld * kld;
  for (int e = tid; e < nr * k; e += 256) {
    const int al = e / k, c = e - al * k, a = r + MT_C * al;
    if (c < a) continue;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s = fma(Rs[al * kp + m], Xs[c * kp + m], s);
    Mi[a * k + c] = s;
    Mi[c * k + a] = s;
    M32i[a * kld + c] = (float)s;
    M32i[c * kld + a] = (float)s;
  }
}

size_t mtail_smem_bytes(int k) {
  const int kp = k | 1;
  return sizeof(double) * ((size_t)2 * k * kp + (size_t)MT_RMAX * kp + k);
}

// M32 (padded, FP32) from M64; Uwarm <- FP32 copy of the refined U (N + 1
// matrices, or the subjects selected by only).
__global__ void finish_m_kernel(int N, int k, int kld, const double* __restrict__ M64, const double* __restrict__ U,
                                float* __restrict__ M32, float* __restrict__ Uwarm, const int* __restrict__ only) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)(N + 1) * k * k) return;
  const int64_t i = e / ((int64_t)k * k);
  if (only && (i >= N || only[i] == 0)) return;  // subject not selected
  const int w = (int)(e % ((int64_t)k * k));
  const int a = w / k, b = w % k;
  if (i < N) M32[i * kld * kld + a * kld + b] = (float)M64[e];
  Uwarm[e] = (float)U[e];
}

// transform: S[f][t] = sum_m M[f][m] sum_s part[s][c][t][m]
__global__ void __launch_bounds__(256) transform_finish_kernel(int k, int kld, int T, int nsplit, int nchunk,
                                                               const float* __restrict__ part,
                                                               const float* __restrict__ M, float* __restrict__ S) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * T) return;
  const int f = (int)(e / T), t = (int)(e % T);
  const int c = t / TCH, tt = t % TCH;
  float acc = 0.f;
  for (int m = 0; m < k; ++m) {
    float p = 0.f;
    for (int s = 0; s < nsplit; ++s) p += part[(((int64_t)s * nchunk + c) * TCH + tt) * kld + m];
    acc = fmaf(M[f * kld + m], p, acc);
  }
  S[e] = acc;
}

int g_max_smem = 232448;  // opt-in shared memory per block (set by prepare_small_kernels)

int refine_bands(const Ctx* c, int nbatch) {
  int nb = (2 * c->num_sms + nbatch - 1) / nbatch;
  nb = nb < 1 ? 1 : nb;
  const int mx = c->k / 4 > 0 ? c->k / 4 : 1;
  nb = nb > mx ? mx : nb;
  // B (k x (k+1)) and one band of A must fit in shared memory: at k = 128
  // with many matrices (one band each) they would not
  const int band_max = g_max_smem / (int)(sizeof(double) * (c->k + 1)) - c->k;
  const int nb_min = band_max > 0 ? (c->k + band_max - 1) / band_max : c->k;
  return nb < nb_min ? nb_min : nb;
}

cudaError_t bgemm(Ctx* c, int nbatch, const double* A, int tA, const double* B, int tB, double alpha,
                  const double* C, double beta, double* D, int sym, const int* only = nullptr) {
  const int k = c->k;
  const int nb = refine_bands(c, nbatch);
  const int band = (k + nb - 1) / nb;
  const size_t sm = sizeof(double) * (size_t)(k + band) * (k + 1);
  bgemm64_kernel<<<dim3(nb, nbatch), 256, sm, c->stream>>>(k, nb, A, tA, B, tB, alpha, C, beta, D, sym, only);
  return cudaGetLastError();
}

}  // namespace


void prepare_small_kernels(int max_smem) {
  g_max_smem = max_smem;
  prepare_tail_kernels();
  cudaFuncSetAttribute(es_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float) * KMAX * KMAX));
  // (these kernels also hold a few KB of static shared memory)
  cudaFuncSetAttribute(p_reduce_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 8 * 1024);
  cudaFuncSetAttribute(p_reduce_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 8 * 1024);
  cudaFuncSetAttribute(p_reduce_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 8 * 1024);
  cudaFuncSetAttribute(p_reduce_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 8 * 1024);
  cudaFuncSetAttribute(p_reduce_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 8 * 1024);
  cudaFuncSetAttribute(eig_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 4 * 1024);
  cudaFuncSetAttribute(eig_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 4 * 1024);
  cudaFuncSetAttribute(eig_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 4 * 1024);
  cudaFuncSetAttribute(bgemm64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  // these run beside the E-pass: take the SM's full shared-memory carve-out too
  cudaFuncSetAttribute(eig_kernel<1>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(eig_kernel<2>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(eig_kernel<4>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(bgemm64_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(mtail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mtail_smem_bytes(MT_KMAX));
  cudaFuncSetAttribute(polar_ns_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ns_smem_bytes(NS_KMAX));
  cudaFuncSetAttribute(polar_ns_kernel<1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(polar_ns_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ns_smem_bytes(NS_KMAX));
  cudaFuncSetAttribute(polar_ns_kernel<2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(mtail_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(phi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 8 * 1024);
}

// p_reduce's shared memory: M_i, the feature-major P and (kld <= 64) the
// slot sum as loaded.
size_t p_reduce_smem_bytes(int kld) {
  return sizeof(float) * ((size_t)kld * kld + (size_t)kld * (TCH + 4) + (kld <= 64 ? (size_t)TCH * (kld + 1) : 0));
}

// Subject groups of the E-step reduction: one wave of its (chunk, group)
// blocks at the kernel's occupancy (each group's subjects run in series in
// one block, so a partial second wave would double the time).
int zsum_groups(int N, int nchunk, int num_sms, int kld) {
  const size_t sm = p_reduce_smem_bytes(kld);
  int bps = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (kld) {
#define ZG_CASE(FW)                                                                                   \
  case 16 * FW:                                                                                       \
    if (sm > 48 * 1024)                                                                               \
      cudaFuncSetAttribute(p_reduce_kernel<FW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p_reduce_kernel<FW>, 256, sm);            \
    break;
    ZG_CASE(1) ZG_CASE(2) ZG_CASE(3) ZG_CASE(4) ZG_CASE(5) ZG_CASE(6) ZG_CASE(7) ZG_CASE(8)
#undef ZG_CASE
    default: break;
  }
  if (e != cudaSuccess || bps < 1) {
    cudaGetLastError();
    bps = 2;
  }
  const int want = (bps * num_sms + nchunk - 1) / nchunk;
  return std::max(1, std::min(N, std::min(128, want)));
}

cudaError_t launch_p_sum(Ctx* c) {
  const dim3 grid(c->nchunk, c->N);
  switch (c->kld) {
#define PS_CASE(FW) \
  case 16 * FW: p_sum_kernel<FW><<<grid, 256, 0, c->stream>>>(c->nchunk, c->f_ppart, c->f_chunk_src, c->f_chunk_src_off, c->psum); break;
    PS_CASE(4)
#undef PS_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_p_reduce(Ctx* c) { return launch_p_reduce_from(c, false); }

cudaError_t launch_p_reduce_from(Ctx* c, bool from_sums) {
  const cudaError_t e = launch_p_reduce_part(c, from_sums);
  return e != cudaSuccess ? e : launch_p_reduce_finish(c);
}

cudaError_t launch_p_reduce_part(Ctx* c, bool from_sums) {
  const size_t sm = p_reduce_smem_bytes(c->kld);
  const dim3 grid(c->nchunk, c->zgroups);
  EReduceArgs ar;
  ar.N = c->N;
  ar.G = c->zgroups;
  ar.T = c->T;
  ar.k = c->k;
  ar.nchunk = c->nchunk;
  ar.part = from_sums ? c->psum : c->p_from_f ? c->f_ppart : c->Ppart;
  ar.src = from_sums ? c->psum_src : c->p_from_f ? c->f_chunk_src : c->chunk_src;
  ar.src_off = from_sums ? c->psum_src_off : c->p_from_f ? c->f_chunk_src_off : c->chunk_src_off;
  ar.M32 = c->M32;
  ar.rho2 = c->rho2;
  ar.ypart = c->Ypart;
  cudaError_t e;
  switch (c->kld) {
#define PR_CASE(FW) \
  case 16 * FW: p_reduce_kernel<FW><<<grid, 256, sm, c->stream>>>(ar); break;
    PR_CASE(1) PR_CASE(2) PR_CASE(3) PR_CASE(4) PR_CASE(5) PR_CASE(6) PR_CASE(7) PR_CASE(8)
#undef PR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_p_reduce_finish(Ctx* c) {
  cudaError_t e;
  if (c->shard_y) {
    // a sharded E-step stops at this context's share of y and of the sums
    ysum_kernel<<<nblocks((int64_t)c->k * c->T, 256), 256, 0, c->stream>>>(c->zgroups, c->k, c->T, c->Ypart,
                                                                              c->shard_y);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    shard_sums_kernel<<<1, 256, 0, c->stream>>>(c->N, c->rho2, c->sqnorm, c->d_v, c->shard_sums);
    return cudaGetLastError();
  }
  es_kernel<<<c->nes_blk, 256, sizeof(float) * c->k * c->k, c->stream>>>(
      c->zgroups, c->k, c->T, c->kld, c->ldT, c->Phi32, c->Ypart, c->ES64, c->batched ? nullptr : c->ESt,
      c->batched ? c->ESb : nullptr, c->sPart, c->esPart, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_estep_finish(Ctx* c, const double* y, const double* sums) {
  cudaError_t e = launch_phi_from(c, sums);
  if (e != cudaSuccess) return e;
  es_kernel<<<c->nes_blk, 256, sizeof(float) * c->k * c->k, c->stream>>>(
      c->zgroups, c->k, c->T, c->kld, c->ldT, c->Phi32, c->Ypart, c->ES64, c->batched ? nullptr : c->ESt,
      c->batched ? c->ESb : nullptr, c->sPart, c->esPart, y);
  return cudaGetLastError();
}

int es_blocks(int T) { return (T + ES_T - 1) / ES_T; }

cudaError_t launch_sigma(Ctx* c) {
  sigma_kernel<<<c->k, 256, 0, c->stream>>>(c->k, c->T, c->nes_blk, c->Phi, c->sPart, c->esPart,
                                            c->SigmaNext, c->scal, c->ll, c->iter, c->max_iter, c->status);
  return cudaGetLastError();
}

cudaError_t launch_phi(Ctx* c) { return launch_phi_from(c, nullptr); }

cudaError_t launch_phi_from(Ctx* c, const double* sums) {
  if (!sigma_eig_supported(c)) return launch_phi_chol(c, sums);
  const int64_t kk = (int64_t)c->k * c->k;
  // U in shared memory beside G' when both fit (k <= 119 on this part)
  const size_t sm1 = sizeof(double) * (3 * c->k + c->k * c->k);
  const bool u_smem = sm1 + sizeof(double) * c->k * c->k + 8 * 1024 <= (size_t)g_max_smem;
  const size_t sm = u_smem ? sm1 + sizeof(double) * c->k * c->k : sm1;
  phi_kernel<<<c->k, 256, sm, c->stream>>>(c->N, c->k, c->rho2, c->sqnorm, c->d_v, c->Xr64 + c->N * kk,
                                           c->G64 + c->N * kk, c->Phi, c->Phi32, c->scal, u_smem ? 1 : 0,
                                           c->status, (double)c->Vtot, sums);
  return cudaGetLastError();
}

// Eigen-decompositions of matrices first .. first + count - 1 (subjects
// 0..N-1, Sigma_s = N); with only != nullptr, subjects whose flag is 0 skip.
cudaError_t launch_eig_from(Ctx* c, int first, int count, const int* only) {
  const size_t sm = eig_smem_bytes(c->k);
  const int nt = eig_threads(c->k);
  const int kk = c->k + (c->k & 1);
  const unsigned nb = (unsigned)count;
  if (kk <= 32)
    eig_kernel<1><<<nb, nt, sm, c->stream>>>(c->N, c->k, c->kld, c->Gpart, c->gslot_off, c->SigmaNext, c->G64,
                                             c->Uwarm, c->U64, c->jac_sweeps, c->status, first, only);
  else if (kk <= 64)
    eig_kernel<2><<<nb, nt, sm, c->stream>>>(c->N, c->k, c->kld, c->Gpart, c->gslot_off, c->SigmaNext, c->G64,
                                             c->Uwarm, c->U64, c->jac_sweeps, c->status, first, only);
  else
    eig_kernel<4><<<nb, nt, sm, c->stream>>>(c->N, c->k, c->kld, c->Gpart, c->gslot_off, c->SigmaNext, c->G64,
                                             c->Uwarm, c->U64, c->jac_sweeps, c->status, first, only);
  return cudaGetLastError();
}

cudaError_t launch_eig(Ctx* c) { return launch_eig_from(c, 0, c->N + 1, nullptr); }
cudaError_t launch_eig_sigma(Ctx* c) { return launch_eig_from(c, c->N, 1, nullptr); }
cudaError_t launch_eig_fallback(Ctx* c) { return launch_eig_from(c, 0, c->N, c->ns_fb); }

// The FP64 refinement of the Jacobi eigenvectors: N + 1 matrices, or the
// subjects selected by only (n1 = N).
cudaError_t launch_refine_from(Ctx* c, const int* only) {
  const int n1 = only ? c->N : c->N + 1;
  cudaError_t e;
  // H = U0^T U0 (symmetric)
  if ((e = bgemm(c, n1, c->U64, 1, c->U64, 0, 1.0, nullptr, 0.0, c->H64, 1, only)) != cudaSuccess) return e;
  // X = U0 (3I - U0^T U0) / 2 = 1.5 U0 - 0.5 U0 H
  if ((e = bgemm(c, n1, c->U64, 0, c->H64, 0, -0.5, c->U64, 1.5, c->Xr64, 0, only)) != cudaSuccess) return e;
  // H = G X
  if ((e = bgemm(c, n1, c->G64, 0, c->Xr64, 0, 1.0, nullptr, 0.0, c->H64, 0, only)) != cudaSuccess) return e;
  // G' = X^T H (symmetric)
  return bgemm(c, n1, c->Xr64, 1, c->H64, 0, 1.0, nullptr, 0.0, c->G64, 1, only);
}

cudaError_t launch_refine(Ctx* c) { return launch_refine_from(c, nullptr); }

cudaError_t launch_rho_from(Ctx* c, const int* only);

// Newton-Schulz polar factors: one CTA per subject for k <= 64, a cluster per
// subject above (k_tail.cu).
bool ns_supported(const Ctx* c) { return (c->k <= NS_KMAX && c->k <= MT_KMAX) || polar_cl_supported(c); }

// Sigma_s's eigen-decomposition (and Phi from it) for k <= 64; above, Phi
// comes from a Cholesky factorisation and Sigma_s is not decomposed.
bool sigma_eig_supported(const Ctx* c) { return c->k <= MT_KMAX; }

cudaError_t launch_polar(Ctx* c) {
  const size_t sm = ns_smem_bytes(c->k);
  // a negative threshold fails every certificate (all subjects take the
  // eigen-decomposition path)
  const double cert = c->force_eig_polar ? -1.0 : c->store == SRM_BF16 ? NS_CERT_BF16 : NS_CERT_F32;
  const int comp = c->store == SRM_BF16 ? 0 : 1;
  if (c->k > NS_KMAX) return launch_polar_cl(c, cert, comp);
  // two CTAs per SM when the subjects outnumber the SMs and two fit
  if (c->N > c->num_sms && 2 * (sm + 1024) <= (size_t)g_max_smem)
    polar_ns_kernel<2><<<c->N, NS_THREADS, sm, c->stream>>>(
        c->N, c->k, c->kld, c->T, c->Gpart, c->gslot_off, c->M64, c->M32, c->sqnorm, c->d_v, c->SigmaNext,
        c->Sigma, c->rho2, c->scal, c->jac_sweeps, c->ns_fb, cert, comp, c->status);
  else
    polar_ns_kernel<1><<<c->N, NS_THREADS, sm, c->stream>>>(
        c->N, c->k, c->kld, c->T, c->Gpart, c->gslot_off, c->M64, c->M32, c->sqnorm, c->d_v, c->SigmaNext,
        c->Sigma, c->rho2, c->scal, c->jac_sweeps, c->ns_fb, cert, comp, c->status);
  return cudaGetLastError();
}

bool mtail_supported(const Ctx* c) { return c->k <= MT_KMAX; }

cudaError_t launch_mtail_from(Ctx* c, int first, int count, const int* only) {
  mtail_kernel<<<dim3(MT_C, count), 256, mtail_smem_bytes(c->k), c->stream>>>(
      c->N, c->k, c->kld, c->T, c->U64, c->G64, c->H64, c->Xr64, c->M64, c->M32, c->Uwarm, c->eigv, c->sqnorm, c->d_v,
      c->SigmaNext, c->Sigma, c->rho2, c->scal, c->status, first, only);
  return cudaGetLastError();
}

cudaError_t launch_mtail(Ctx* c) { return launch_mtail_from(c, 0, c->N + 1, nullptr); }
cudaError_t launch_mtail_sigma(Ctx* c) { return launch_mtail_from(c, c->N, 1, nullptr); }
cudaError_t launch_mtail_fallback(Ctx* c) {
  if (mtail_supported(c)) return launch_mtail_from(c, 0, c->N, c->ns_fb);
  // k > 64: the FP64 refinement and M_i, rho_i^2 for the subjects whose
  // Newton-Schulz certificate failed
  cudaError_t e = launch_refine_from(c, c->ns_fb);
  if (e != cudaSuccess) return e;
  return launch_rho_from(c, c->ns_fb);
}

cudaError_t launch_rho_from(Ctx* c, const int* only) {
  const int k = c->k, N = c->N;
  dk_rho_kernel<<<only ? N : N + 1, 128, 0, c->stream>>>(N, k, c->T, c->G64, c->H64, c->eigv, c->sqnorm, c->d_v,
                                                          c->SigmaNext, c->Sigma, c->rho2, c->scal, c->status, only);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // subjects only; entry N of G64 / Xr64 (Sigma_s) is kept for the next E-step.
  // T1 = X B (into G64) ; M = T1 X^T (symmetric)
  if ((e = bgemm(c, N, c->Xr64, 0, c->H64, 0, 1.0, nullptr, 0.0, c->G64, 0, only)) != cudaSuccess) return e;
  if ((e = bgemm(c, N, c->G64, 0, c->Xr64, 1, 1.0, nullptr, 0.0, c->M64, 1, only)) != cudaSuccess) return e;
  const int64_t n = (int64_t)(N + 1) * k * k;
  finish_m_kernel<<<nblocks(n, 256), 256, 0, c->stream>>>(N, k, c->kld, c->M64, c->Xr64, c->M32, c->Uwarm, only);
  return cudaGetLastError();
}

cudaError_t launch_rho(Ctx* c) { return launch_rho_from(c, nullptr); }

cudaError_t launch_transform_finish(Ctx* c, int i, const float* part, int nsplit, int T_new, float* S_out) {
  const int nchunk = (T_new + TCH - 1) / TCH;
  const int64_t n = (int64_t)c->k * T_new;
  transform_finish_kernel<<<nblocks(n, 256), 256, 0, c->stream>>>(
      c->k, c->kld, T_new, nsplit, nchunk, part, c->M32 + (int64_t)i * c->kld * c->kld, S_out);
  return cudaGetLastError();
}

}  // namespace srm
