// The k x k and k x T steps of one EM iteration (everything but the two
// streaming passes over X^).  FP64 is used where the paper's reduced
// E-step and M-step need it; k x k eigen-work runs in FP32 and is refined to
// FP64 accuracy with FP64 matrix products.
//
//  E-step (Algorithm 1, master process):
//    p_reduce : Z_i = rho_i^-2 M_i P_i  from the E-pass partials, with
//               W_i^T X^_i = M_i (A_i^T X^_i)  (eq:srm_mean_distributed)
//    y_sum    : y = sum_i Z_i                               (FP64)
//    chol     : rho_0 = sum_i rho_i^-2 (eq:srm_wt_psi_w), Cholesky of
//               I + rho_0 Sigma_s, ln det, likelihood scalars
//    phi      : Phi = (Sigma_s^-1 + rho_0 I)^-1 = (I + rho_0 Sigma_s)^-1 Sigma_s
//               (eq:srm_inversion_opt), one right-hand side per block
//    es       : E[S] = Phi y (eq:srm_mean_distributed; Phi equals
//               Sigma_s^T [I - rho_0 (Sigma_s^-1 + rho_0 I)^-1]), the operand
//               copies for the M-pass, and per-block partials of
//               E[S] E[S]^T and <y, Phi y>
//    sigma    : Sigma_s^new = Phi + E[S] E[S]^T / T
//               (eq:srm_variance_update_optimized) and the log-likelihood
//  M-step (per subject, after the M-pass):
//    eig      : G_i = A_i^T A_i from the Gram partials; FP32 cyclic Jacobi
//               (warm-started from the previous eigenvectors)
//    refine   : FP64 refinement of the eigenvectors, then
//               M_i = (A_i^T A_i)^-1/2 through the Daleckii-Krein first-order
//               correction, ||A_i||_* = tr (A_i^T A_i)^1/2, and
//               rho_i^2 = (||X^_i||^2 - 2 ||A_i||_* + T tr Sigma_s^new)/(T v_i)
//               (eq:srm_rho_update with tr(W_i^T A_i) = ||A_i||_* for the
//               polar factor W_i of eq:srm_mapping_update)
#include <math.h>

#include "srm_internal.cuh"

namespace srm {

namespace {

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename K>
void set_smem_once(K kernel, size_t bytes) {
  // cudaFuncSetAttribute is not a stream operation; calling it once per
  // kernel and size is enough.
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

__device__ __forceinline__ void flag(int* status, int bits) { atomicOr(status, bits); }

// ------------------------------------------------------------------ E-step
// grid (nchunk, N), 256 threads.  Sums the subject's partial blocks for one
// 64-wide t-chunk in a fixed order, then Z = rho^-2 M P.
__global__ void __launch_bounds__(256) p_reduce_kernel(int N, int T, int k, int kld, int nchunk,
                                                       const float* __restrict__ part,
                                                       const ChunkSrc* __restrict__ src,
                                                       const int* __restrict__ src_off,
                                                       const float* __restrict__ M32,
                                                       const double* __restrict__ rho2, float* __restrict__ Z) {
  extern __shared__ float pr_smem[];
  float* Ms = pr_smem;                  // [k][k+1]
  float* Ps = pr_smem + k * (k + 1);    // [TCH][kld+1]
  const int c = blockIdx.x, i = blockIdx.y;
  const int t0 = c * TCH;
  const float* Mi = M32 + (int64_t)i * kld * kld;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Ms[(e / k) * (k + 1) + e % k] = Mi[(e / k) * kld + e % k];
  for (int e = threadIdx.x; e < TCH * kld; e += blockDim.x) Ps[(e / kld) * (kld + 1) + e % kld] = 0.f;
  __syncthreads();
  const int b = src_off[i * nchunk + c], en = src_off[i * nchunk + c + 1];
  for (int s = b; s < en; ++s) {
    const float* p = part + src[s].off;
    for (int e = threadIdx.x; e < TCH * kld; e += blockDim.x) Ps[(e / kld) * (kld + 1) + e % kld] += p[e];
  }
  __syncthreads();
  const float rinv = (float)(1.0 / rho2[i]);
  for (int e = threadIdx.x; e < k * TCH; e += blockDim.x) {
    const int f = e / TCH, t = e % TCH;
    if (t0 + t >= T) continue;
    float z = 0.f;
    const float* mr = Ms + f * (k + 1);
    const float* pr = Ps + t * (kld + 1);
    for (int m = 0; m < k; ++m) z = fmaf(mr[m], pr[m], z);
    Z[((int64_t)i * k + f) * T + t0 + t] = rinv * z;
  }
}

// y[f][t] = sum_i Z_i[f][t] in FP64, subjects in order.
__global__ void __launch_bounds__(256) y_sum_kernel(int N, int64_t kT, const float* __restrict__ Z,
                                                    double* __restrict__ Y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kT) return;
  double acc = 0.0;
  for (int i = 0; i < N; ++i) acc += (double)Z[(int64_t)i * kT + e];
  Y[e] = acc;
}

// scal[] layout
enum { SC_RHO0 = 0, SC_LOGDET = 1, SC_VLOGRHO = 2, SC_SQRHO = 3, SC_YPHIY = 4, SC_TRSIG = 5 };

// One block: rho_0 and likelihood sums over subjects, Cholesky of
// C = I + rho_0 Sigma_s (lower, in place), ln det C.
__global__ void __launch_bounds__(256) chol_kernel(int N, int k, const double* __restrict__ rho2,
                                                   const double* __restrict__ sqnorm,
                                                   const int64_t* __restrict__ vox,
                                                   const double* __restrict__ Sigma, double* __restrict__ Lout,
                                                   double* __restrict__ scal, int* status) {
  extern __shared__ double C[];  // [k][k+1] (chol_kernel only)
  __shared__ double red[3][256];
  const int tid = threadIdx.x;
  double a = 0, b = 0, d = 0;
  for (int i = tid; i < N; i += blockDim.x) {
    const double r = rho2[i];
    if (!(r > 0.0) || !isfinite(r)) flag(status, ST_NONFINITE);
    a += 1.0 / r;
    b += (double)vox[i] * log(r);
    d += sqnorm[i] / r;
  }
  red[0][tid] = a;
  red[1][tid] = b;
  red[2][tid] = d;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s)
      for (int q = 0; q < 3; ++q) red[q][tid] += red[q][tid + s];
    __syncthreads();
  }
  const double rho0 = red[0][0];
  const int ld = k + 1;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int r = e / k, cc = e % k;
    C[r * ld + cc] = (r == cc ? 1.0 : 0.0) + rho0 * Sigma[e];
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const double p = C[j * ld + j];
      if (!(p > 0.0) || !isfinite(p)) flag(status, ST_NOT_PD);
      C[j * ld + j] = sqrt(p > 1e-300 ? p : 1e-300);
    }
    __syncthreads();
    const double piv = C[j * ld + j];
    for (int r = j + 1 + tid; r < k; r += blockDim.x) C[r * ld + j] /= piv;
    __syncthreads();
    for (int r = j + 1 + warp; r < k; r += nw) {
      const double lr = C[r * ld + j];
      for (int cc = j + 1 + lane; cc <= r; cc += 32) C[r * ld + cc] -= lr * C[cc * ld + j];
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int r = e / k, cc = e % k;
    Lout[e] = (cc <= r) ? C[r * ld + cc] : 0.0;
  }
  if (tid == 0) {
    double ld2 = 0.0;
    for (int j = 0; j < k; ++j) ld2 += log(C[j * ld + j]);
    scal[SC_RHO0] = rho0;
    scal[SC_LOGDET] = 2.0 * ld2;
    scal[SC_VLOGRHO] = red[1][0];
    scal[SC_SQRHO] = red[2][0];
  }
}

// Phi[:, j] = L^-T L^-1 Sigma_s[:, j]; one warp per right-hand side.
__global__ void __launch_bounds__(32) phi_kernel(int k, const double* __restrict__ L,
                                                 const double* __restrict__ Sigma, double* __restrict__ Phi) {
  __shared__ double z[KMAX];
  const int j = blockIdx.x, lane = threadIdx.x;
  for (int r = 0; r < k; ++r) {
    double s = 0.0;
    for (int m = lane; m < r; m += 32) s += L[r * k + m] * z[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) z[r] = (Sigma[r * k + j] - s) / L[r * k + r];
    __syncwarp();
  }
  for (int r = k - 1; r >= 0; --r) {
    double s = 0.0;
    for (int m = r + 1 + lane; m < k; m += 32) s += L[m * k + r] * z[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) z[r] = (z[r] - s) / L[r * k + r];
    __syncwarp();
  }
  for (int r = lane; r < k; r += 32) Phi[r * k + j] = z[r];
}

constexpr int ES_T = 32;  // t per es block

// E[S][:, t0:t0+32] = Phi_sym y[:, t0:t0+32]; partial E E^T and <y, E>.
__global__ void __launch_bounds__(256) es_kernel(int k, int T, int kld, int ldT, const double* __restrict__ Phi,
                                                 const double* __restrict__ Y, double* __restrict__ ES64,
                                                 float* __restrict__ ESt, __nv_bfloat16* __restrict__ ESb,
                                                 double* __restrict__ part) {
  extern __shared__ double es_smem[];
  double* Ps = es_smem;              // [k][k]
  double* Ys = Ps + k * k;           // [k][ES_T]
  double* Es = Ys + k * ES_T;        // [k][ES_T]
  const int t0 = blockIdx.x * ES_T;
  const int tid = threadIdx.x;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e % k;
    Ps[e] = 0.5 * (Phi[a * k + b] + Phi[b * k + a]);
  }
  for (int e = tid; e < k * ES_T; e += blockDim.x) {
    const int f = e / ES_T, tt = e % ES_T;
    Ys[e] = (t0 + tt < T) ? Y[(int64_t)f * T + t0 + tt] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < k * ES_T; e += blockDim.x) {
    const int f = e / ES_T, tt = e % ES_T;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s += Ps[f * k + m] * Ys[m * ES_T + tt];
    Es[e] = s;
    const int t = t0 + tt;
    if (t < T) {
      ES64[(int64_t)f * T + t] = s;
      if (ESt) ESt[(int64_t)t * kld + f] = (float)s;
      if (ESb) ESb[(int64_t)f * ldT + t] = __float2bfloat16_rn((float)s);
    }
  }
  __syncthreads();
  double* out = part + (int64_t)blockIdx.x * (k * k + 1);
  for (int e = tid; e < k * (k + 1) / 2; e += blockDim.x) {
    // e -> (a, b) with a <= b, row-major upper triangle
    int a = 0, rem = e;
    while (rem >= k - a) {
      rem -= k - a;
      ++a;
    }
    const int b = a + rem;
    double s = 0.0;
    for (int tt = 0; tt < ES_T; ++tt) s += Es[a * ES_T + tt] * Es[b * ES_T + tt];
    out[a * k + b] = s;
    out[b * k + a] = s;
  }
  if (tid < 32) {
    double s = 0.0;
    for (int e = tid; e < k * ES_T; e += 32) s += Ys[e] * Es[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) out[k * k] = s;
  }
}

// grid k blocks (row a of Sigma_s^new); block 0 also finishes the likelihood.
__global__ void __launch_bounds__(128) sigma_kernel(int k, int T, int nblk, double Vtot, const double* __restrict__ Phi,
                                                    const double* __restrict__ part, double* __restrict__ SigmaNext,
                                                    double* __restrict__ scal, double* __restrict__ ll, int* iter,
                                                    int max_iter, int* status) {
  const int a = blockIdx.x;
  for (int b = threadIdx.x; b < k; b += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nblk; ++q) s += part[(int64_t)q * (k * k + 1) + a * k + b];
    const double v = 0.5 * (Phi[a * k + b] + Phi[b * k + a]) + s / (double)T;
    if (!isfinite(v)) flag(status, ST_NONFINITE);
    SigmaNext[a * k + b] = v;
  }
  if (a == 0 && threadIdx.x == 0) {
    double ye = 0.0;
    for (int q = 0; q < nblk; ++q) ye += part[(int64_t)q * (k * k + 1) + k * k];
    scal[SC_YPHIY] = ye;
    const double L = -0.5 * ((double)T * Vtot * 1.8378770664093454835606594728112 + (double)T * scal[SC_VLOGRHO] +
                             (double)T * scal[SC_LOGDET] + scal[SC_SQRHO] - ye);
    if (!isfinite(L)) flag(status, ST_NONFINITE);
    const int it = *iter;
    if (it >= 0 && it < max_iter) ll[it] = L;
    *iter = it + 1;
  }
}

// ------------------------------------------------------------------ M-step
// One block per subject.  G_i (FP64) = sum of Gram partials; FP32 Jacobi on
// U_w^T G U_w (U_w = previous eigenvectors); U_0 = U_w V written to U64.
__global__ void __launch_bounds__(256) eig_kernel(int k, int kld, const float* __restrict__ gpart,
                                                  const int* __restrict__ gslot_off, double* __restrict__ G64,
                                                  float* __restrict__ Uwarm, double* __restrict__ U64,
                                                  int* status) {
  extern __shared__ float eig_smem[];
  const int kk = k + (k & 1);   // even size for the round-robin schedule
  const int ld = kk + 1;
  float* Gs = eig_smem;         // [kk][ld]
  float* Vs = Gs + kk * ld;     // [kk][ld]
  float* Us = Vs + kk * ld;     // [kk][ld]
  __shared__ float cs[KMAX / 2][2];
  __shared__ int pq[KMAX / 2][2];
  __shared__ float redf[2][256];
  const int i = blockIdx.x, tid = threadIdx.x;
  const int s0 = gslot_off[i], s1 = gslot_off[i + 1];
  double* Gi = G64 + (int64_t)i * k * k;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e % k;
    double s = 0.0;
    for (int q = s0; q < s1; ++q) s += (double)gpart[(int64_t)q * kld * kld + a * kld + b];
    Gi[e] = s;
  }
  __syncthreads();
  // symmetrise in FP64 (both triangles were accumulated separately)
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e % k;
    const float g = (float)(0.5 * (Gi[a * k + b] + Gi[b * k + a]));
    if (!isfinite(g)) flag(status, ST_NONFINITE);
    Gs[a * ld + b] = g;
    Us[a * ld + b] = Uwarm[(int64_t)i * k * k + e];
  }
  for (int e = tid; e < kk * kk; e += blockDim.x) {
    const int a = e / kk, b = e % kk;
    if (a >= k || b >= k) {
      Gs[a * ld + b] = (a == b) ? 1.f : 0.f;
      Us[a * ld + b] = (a == b) ? 1.f : 0.f;
    }
  }
  __syncthreads();
  // Vs = G U ; Gs = U^T Vs   (rotate into the warm basis)
  for (int e = tid; e < kk * kk; e += blockDim.x) {
    const int a = e / kk, b = e % kk;
    float s = 0.f;
    for (int m = 0; m < kk; ++m) s = fmaf(Gs[a * ld + m], Us[m * ld + b], s);
    Vs[a * ld + b] = s;
  }
  __syncthreads();
  for (int e = tid; e < kk * kk; e += blockDim.x) {
    const int a = e / kk, b = e % kk;
    float s = 0.f;
    for (int m = 0; m < kk; ++m) s = fmaf(Us[m * ld + a], Vs[m * ld + b], s);
    Gs[a * ld + b] = s;
  }
  __syncthreads();
  for (int e = tid; e < kk * kk; e += blockDim.x) {
    const int a = e / kk, b = e % kk;
    Vs[a * ld + b] = (a == b) ? 1.f : 0.f;
  }
  __syncthreads();
  // cyclic Jacobi, round-robin ordering: kk/2 disjoint rotations per round
  const int npair = kk / 2;
  bool converged = false;
  for (int sweep = 0; sweep < 30 && !converged; ++sweep) {
    float off = 0.f, dg = 0.f;
    for (int e = tid; e < k * k; e += blockDim.x) {
      const int a = e / k, b = e % k;
      const float g = Gs[a * ld + b];
      if (a == b) dg += g * g;
      else off += g * g;
    }
    redf[0][tid] = off;
    redf[1][tid] = dg;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (tid < s) {
        redf[0][tid] += redf[0][tid + s];
        redf[1][tid] += redf[1][tid + s];
      }
      __syncthreads();
    }
    converged = !(redf[0][0] > 1e-11f * redf[1][0]);
    __syncthreads();
    if (converged) break;
    for (int round = 0; round < kk - 1; ++round) {
      if (tid < npair) {
        const int j = tid;
        const int pa = (j == 0) ? 0 : 1 + ((j - 1 + round) % (kk - 1));
        const int pb_pos = kk - 1 - j;
        const int pb = 1 + ((pb_pos - 1 + round) % (kk - 1));
        const int p = min(pa, pb), q = max(pa, pb);
        float c = 1.f, s = 0.f;
        if (q < k) {
          const float gpq = Gs[p * ld + q];
          const float gpp = Gs[p * ld + p], gqq = Gs[q * ld + q];
          if (fabsf(gpq) > 1e-30f + 1e-9f * sqrtf(fabsf(gpp * gqq))) {
            const float tau = (gqq - gpp) / (2.f * gpq);
            const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            s = t * c;
          }
        }
        cs[j][0] = c;
        cs[j][1] = s;
        pq[j][0] = p;
        pq[j][1] = q;
      }
      __syncthreads();
      for (int e = tid; e < npair * kk; e += blockDim.x) {
        const int j = e / kk, col = e % kk;
        const float c = cs[j][0], s = cs[j][1];
        if (s == 0.f) continue;
        const int p = pq[j][0], q = pq[j][1];
        const float gp = Gs[p * ld + col], gq = Gs[q * ld + col];
        Gs[p * ld + col] = c * gp - s * gq;
        Gs[q * ld + col] = s * gp + c * gq;
      }
      __syncthreads();
      for (int e = tid; e < npair * kk; e += blockDim.x) {
        const int j = e / kk, row = e % kk;
        const float c = cs[j][0], s = cs[j][1];
        if (s == 0.f) continue;
        const int p = pq[j][0], q = pq[j][1];
        const float gp = Gs[row * ld + p], gq = Gs[row * ld + q];
        Gs[row * ld + p] = c * gp - s * gq;
        Gs[row * ld + q] = s * gp + c * gq;
        const float vp = Vs[row * ld + p], vq = Vs[row * ld + q];
        Vs[row * ld + p] = c * vp - s * vq;
        Vs[row * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (!converged && tid == 0) {
    // FP32 Jacobi reaching its sweep cap is only a precision loss (the FP64
    // refinement follows); a large remaining off-diagonal is a failure.
    if (redf[0][0] > 1e-6f * redf[1][0]) flag(status, ST_EIG_NOCONV);
  }
  // U_0 = U_w V
  double* Uo = U64 + (int64_t)i * k * k;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e % k;
    float s = 0.f;
    for (int m = 0; m < kk; ++m) s = fmaf(Us[a * ld + m], Vs[m * ld + b], s);
    Uo[e] = (double)s;
  }
}

// D_b = alpha op(A_b) op(B_b) + beta C_b for a batch of k x k FP64 matrices.
// grid (nband, nbatch); block 256; rows of the band split across threads.
__global__ void __launch_bounds__(256) bgemm64_kernel(int k, int nband, const double* __restrict__ A, int tA,
                                                      const double* __restrict__ B, int tB, double alpha,
                                                      const double* __restrict__ C, double beta,
                                                      double* __restrict__ D) {
  const int b = blockIdx.y;
  const int r0 = (k * blockIdx.x) / nband, r1 = (k * (blockIdx.x + 1)) / nband;
  const int64_t base = (int64_t)b * k * k;
  const double* Ab = A + base;
  const double* Bb = B + base;
  for (int e = threadIdx.x; e < (r1 - r0) * k; e += blockDim.x) {
    const int r = r0 + e / k, c = e % k;
    double s = 0.0;
    for (int m = 0; m < k; ++m) {
      const double a = tA ? Ab[m * k + r] : Ab[r * k + m];
      const double bb = tB ? Bb[c * k + m] : Bb[m * k + c];
      s = fma(a, bb, s);
    }
    double out = alpha * s;
    if (C) out += beta * C[base + r * k + c];
    D[base + r * k + c] = out;
  }
}

// Per subject: eigenvalues lambda = diag(G'), G' = U^T G U; the Daleckii-Krein
// matrix B = diag(lambda^-1/2) + F o E with F_ab = -1/(s_a s_b (s_a + s_b)),
// s = sqrt(lambda), E = off-diagonal part of G'; nuclear norm and rho update.
// Block 0 also commits Sigma_s <- Sigma_s^new.
__global__ void __launch_bounds__(128) dk_rho_kernel(int N, int k, int T, const double* __restrict__ Gp,
                                                     double* __restrict__ Bout, double* __restrict__ eigv,
                                                     const double* __restrict__ sqnorm,
                                                     const int64_t* __restrict__ vox,
                                                     const double* __restrict__ SigmaNext, double* __restrict__ Sigma,
                                                     double* __restrict__ rho2, double* __restrict__ scal,
                                                     int* status) {
  __shared__ double sq[KMAX];
  __shared__ double red[128];
  const int i = blockIdx.x, tid = threadIdx.x;
  const double* G = Gp + (int64_t)i * k * k;
  double* Bm = Bout + (int64_t)i * k * k;
  double lmax = 0.0;
  for (int a = 0; a < k; ++a) lmax = fmax(lmax, G[a * k + a]);
  for (int a = tid; a < k; a += blockDim.x) {
    const double l = G[a * k + a];
    if (!(l > 1e-12 * lmax) || !isfinite(l)) flag(status, ST_RANK);
    const double lc = l > 1e-300 ? l : 1e-300;
    sq[a] = sqrt(lc);
    eigv[(int64_t)i * k + a] = l;
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e % k;
    double v;
    if (a == b) v = 1.0 / sq[a];
    else v = -0.5 * (G[a * k + b] + G[b * k + a]) / (sq[a] * sq[b] * (sq[a] + sq[b]));
    Bm[e] = v;
  }
  double nuc = 0.0;
  for (int a = tid; a < k; a += blockDim.x) nuc += sq[a];
  red[tid] = nuc;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  if (tid == 0) {
    double tr = 0.0;
    for (int a = 0; a < k; ++a) tr += SigmaNext[a * k + a];
    const double r = (sqnorm[i] - 2.0 * red[0] + (double)T * tr) / ((double)T * (double)vox[i]);
    if (!(r > 0.0) || !isfinite(r)) flag(status, ST_NONFINITE);
    rho2[i] = r;
    if (i == 0) scal[SC_TRSIG] = tr;
  }
  if (i == 0)
    for (int e = tid; e < k * k; e += blockDim.x) Sigma[e] = SigmaNext[e];
}

// M32 (padded, FP32), M64 stays; Uwarm <- FP32 copy of the refined U.
__global__ void finish_m_kernel(int N, int k, int kld, const double* __restrict__ M64, const double* __restrict__ U,
                                float* __restrict__ M32, float* __restrict__ Uwarm) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)N * k * k) return;
  const int64_t i = e / ((int64_t)k * k);
  const int w = (int)(e % ((int64_t)k * k));
  const int a = w / k, b = w % k;
  M32[i * kld * kld + a * kld + b] = (float)M64[e];
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

int refine_bands(const Ctx* c) {
  int nb = (2 * c->num_sms + c->N - 1) / c->N;
  nb = nb < 1 ? 1 : nb;
  const int mx = c->k / 4 > 0 ? c->k / 4 : 1;
  return nb > mx ? mx : nb;
}

}  // namespace

void prepare_small_kernels(int max_smem) {
  set_smem_once(p_reduce_kernel, max_smem);
  set_smem_once(chol_kernel, max_smem - 8 * 1024);
  set_smem_once(es_kernel, max_smem);
  set_smem_once(eig_kernel, max_smem - 4 * 1024);
}

cudaError_t launch_p_reduce(Ctx* c) {
  const size_t sm = sizeof(float) * (c->k * (c->k + 1) + TCH * (c->kld + 1));
  p_reduce_kernel<<<dim3(c->nchunk, c->N), 256, sm, c->stream>>>(c->N, c->T, c->k, c->kld, c->nchunk, c->Ppart,
                                                                  c->chunk_src, c->chunk_src_off, c->M32, c->rho2,
                                                                  c->Zbuf);
  return cudaGetLastError();
}

cudaError_t launch_y_sum(Ctx* c) {
  const int64_t kT = (int64_t)c->k * c->T;
  y_sum_kernel<<<nblocks(kT, 256), 256, 0, c->stream>>>(c->N, kT, c->Zbuf, c->Y);
  return cudaGetLastError();
}

cudaError_t launch_chol(Ctx* c) {
  const size_t sm = sizeof(double) * c->k * (c->k + 1);
  chol_kernel<<<1, 256, sm, c->stream>>>(c->N, c->k, c->rho2, c->sqnorm, c->d_v, c->Sigma, c->L, c->scal, c->status);
  return cudaGetLastError();
}

cudaError_t launch_phi(Ctx* c) {
  phi_kernel<<<c->k, 32, 0, c->stream>>>(c->k, c->L, c->Sigma, c->Phi);
  return cudaGetLastError();
}

cudaError_t launch_es(Ctx* c) {
  const size_t sm = sizeof(double) * (c->k * c->k + 2 * c->k * ES_T);
  es_kernel<<<c->nes_blk, 256, sm, c->stream>>>(c->k, c->T, c->kld, c->ldT, c->Phi, c->Y, c->ES64,
                                                c->batched ? nullptr : c->ESt,
                                                c->batched ? c->ESb : nullptr, c->esPart);
  return cudaGetLastError();
}

cudaError_t launch_sigma(Ctx* c) {
  sigma_kernel<<<c->k, 128, 0, c->stream>>>(c->k, c->T, c->nes_blk, (double)c->Vtot, c->Phi, c->esPart, c->SigmaNext,
                                            c->scal, c->ll, c->iter, c->max_iter, c->status);
  return cudaGetLastError();
}

cudaError_t launch_eig(Ctx* c) {
  const int kk = c->k + (c->k & 1);
  const size_t sm = sizeof(float) * 3 * kk * (kk + 1);
  eig_kernel<<<c->N, 256, sm, c->stream>>>(c->k, c->kld, c->Gpart, c->gslot_off, c->G64, c->Uwarm, c->U64,
                                           c->status);
  return cudaGetLastError();
}

cudaError_t launch_refine(Ctx* c) {
  const int k = c->k, N = c->N;
  const int nb = refine_bands(c);
  dim3 g(nb, N);
  // H = U0^T U0 - I
  // (the identity is subtracted by the next step: U1 = U0 - 1/2 U0 (U0^T U0 - I)
  //  = 1.5 U0 - 0.5 U0 (U0^T U0))
  bgemm64_kernel<<<g, 256, 0, c->stream>>>(k, nb, c->U64, 1, c->U64, 0, 1.0, nullptr, 0.0, c->H64);
  // X = 1.5 U0 - 0.5 U0 H   (first-order re-orthonormalisation)
  bgemm64_kernel<<<g, 256, 0, c->stream>>>(k, nb, c->U64, 0, c->H64, 0, -0.5, c->U64, 1.5, c->Xr64);
  // H = G X
  bgemm64_kernel<<<g, 256, 0, c->stream>>>(k, nb, c->G64, 0, c->Xr64, 0, 1.0, nullptr, 0.0, c->H64);
  // G' = X^T H
  bgemm64_kernel<<<g, 256, 0, c->stream>>>(k, nb, c->Xr64, 1, c->H64, 0, 1.0, nullptr, 0.0, c->G64);
  return cudaGetLastError();
}

cudaError_t launch_rho(Ctx* c) {
  const int k = c->k, N = c->N;
  const int nb = refine_bands(c);
  dim3 g(nb, N);
  dk_rho_kernel<<<N, 128, 0, c->stream>>>(N, k, c->T, c->G64, c->H64, c->eigv, c->sqnorm, c->d_v, c->SigmaNext,
                                          c->Sigma, c->rho2, c->scal, c->status);
  // T1 = X B ; M = T1 X^T
  bgemm64_kernel<<<g, 256, 0, c->stream>>>(k, nb, c->Xr64, 0, c->H64, 0, 1.0, nullptr, 0.0, c->G64);
  bgemm64_kernel<<<g, 256, 0, c->stream>>>(k, nb, c->G64, 0, c->Xr64, 1, 1.0, nullptr, 0.0, c->M64);
  const int64_t n = (int64_t)N * k * k;
  finish_m_kernel<<<nblocks(n, 256), 256, 0, c->stream>>>(N, k, c->kld, c->M64, c->Xr64, c->M32, c->Uwarm);
  return cudaGetLastError();
}

cudaError_t launch_transform_finish(Ctx* c, int i, const float* part, int nsplit, int T_new, float* S_out) {
  const int nchunk = (T_new + TCH - 1) / TCH;
  const int64_t n = (int64_t)c->k * T_new;
  transform_finish_kernel<<<nblocks(n, 256), 256, 0, c->stream>>>(
      c->k, c->kld, T_new, nsplit, nchunk, part, c->M32 + (int64_t)i * c->kld * c->kld, S_out);
  return cudaGetLastError();
}

}  // namespace srm
