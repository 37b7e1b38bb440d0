// The k x k steps of an EM iteration for 64 < k <= 128 that would otherwise
// take an eigen-decomposition per subject and one of Sigma_s (Algorithm 1):
//
// polar_ns_cl  the M-step's polar factor W_i = A_i (A_i^T A_i)^-1/2
//              (eq:srm_mapping_update), ||A_i||_* and rho_i^2 (eq:srm_rho_update)
//              by the certified coupled Newton-Schulz iteration, on a cluster
//              of 8 or 4 CTAs per subject (the matrices of one subject do not
//              fit one CTA's shared memory at k = 128);
// phi_chol,    the E-step's Phi = (Sigma_s^-1 + rho_0 I)^-1 (eq:srm_inversion_opt)
// phi_solve    written as B^-1 Sigma_s with B = I + rho_0 Sigma_s, from the
//              Cholesky factor B = L L^T in float-float arithmetic; ln det B =
//              sum ln L_jj^2 gives the log-likelihood's ln det(I + rho_0
//              Sigma_s), and a failed factorisation reports B as not positive
//              definite.
//
// Newton-Schulz (as for k <= 64): with G = A_i^T A_i (error-free sum of the
// Gram partials, symmetrised) and c = min(||G||_F, ||G||_inf) >= lambda_max,
// the iteration on A = G / c,
//     P = Z Y,  T = (3 I - P) / 2,  Y <- T Y,  Z <- T Z,   Y_0 = A, Z_0 = I,
// converges to Y = A^1/2, Z = A^-1/2 (all iterates are polynomials in G, so
// T Y = Y T); it stops one update after max |P - I| < NS_TOL; M_0 = Z / sqrt(c).
// The certificate E = M_0 G M_0 - I bounds the polar factor's error
// (||A_i (M_0 - G^-1/2)||_F <= ||E||_F to first order); a subject with
// ||E||_F > cert sqrt(k) goes through the eigen-decomposition path.  For the
// FP32 store E is formed in float-float arithmetic (G kept as hi + lo), for
// the BF16 store, whose threshold is 50 times larger, in plain FP32.
// ||A_i||_* = tr(M_0 G) - tr(E M_0 G) / 2 + O(|E|^2).
//
// Cluster layout: CTA r of a cluster of C CTAs owns the 4-row tiles tr = r + C l of
// every matrix (rows a = 4 tr + u).  Each CTA keeps full copies of Y and Z
// (the right operands) and computes its own rows of each product; after a
// step the new rows are stored into every CTA's copies (distributed shared
// memory) between cluster barriers.  Every control decision is taken from
// values that all CTAs reduce in the same order, so the CTAs of a cluster
// run the same sequence of barriers.
#include <math.h>

#include "kk_util.cuh"
#include "tc_ptx.cuh"

namespace srm {

namespace {

using tc::cluster_ctarank;
using tc::cluster_sync_all;
using tc::mapa_shared;
using tc::smem_u32;

__device__ __forceinline__ void st_cluster_f4(uint32_t raddr, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(raddr), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void st_cluster_f32(uint32_t raddr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(raddr), "f"(v) : "memory");
}

constexpr int NC_KMAX = 128;
constexpr int NC_THREADS = 512;
constexpr int NC_NW = NC_THREADS / 32;

// Own rows per CTA for a cluster of C CTAs: the 4-row tiles tr = r + C l.
template <int C>
struct NcGeom {
  static constexpr int TRMAX = (NC_KMAX / 4 + C - 1) / C;
  static constexpr int RMAX = 4 * TRMAX;
};

// 4 x 4 tile C[u][v] = sum_m A[m][ac + u] B[m][bc + v], m < KP, over this
// lane's share of m: the KS adjacent lanes of a tile take m = q, q + KS, ...,
// so that they read KS consecutive rows at once; with row strides that are
// odd multiples of 4 floats those rows start in different bank groups.  A is
// m-major with leading dimension lda, B row-major with leading dimension ldb.
// With CA (CB) A (B) carries a low part: the products of the high parts are
// error-free (hi + lo), the low parts' products are added to lo.
template <int KS, bool CA, bool CB>
__device__ __forceinline__ void cl_tile(const float* __restrict__ Ah, const float* __restrict__ Al, int lda, int ac,
                                        const float* __restrict__ Bh, const float* __restrict__ Bl, int ldb, int bc,
                                        int KP, int q, bool valid, float (&hi)[4][4], float (&lo)[4][4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) hi[u][v] = lo[u][v] = 0.f;
  if (!valid) return;
#pragma unroll 4
  for (int m = q; m < KP; m += KS) {
    const float4 a = *reinterpret_cast<const float4*>(Ah + m * lda + ac);
    const float4 b = *reinterpret_cast<const float4*>(Bh + m * ldb + bc);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
    if (!CA && !CB) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) hi[u][v] = fmaf(av[u], bv[v], hi[u][v]);
    } else {
      float alv[4] = {0.f, 0.f, 0.f, 0.f}, blv[4] = {0.f, 0.f, 0.f, 0.f};
      if (CA) {
        const float4 t = *reinterpret_cast<const float4*>(Al + m * lda + ac);
        alv[0] = t.x, alv[1] = t.y, alv[2] = t.z, alv[3] = t.w;
      }
      if (CB) {
        const float4 t = *reinterpret_cast<const float4*>(Bl + m * ldb + bc);
        blv[0] = t.x, blv[1] = t.y, blv[2] = t.z, blv[3] = t.w;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float p = __fmul_rn(av[u], bv[v]);
          const float pe = fmaf(av[u], bv[v], -p);  // exact product error
          float sm, se;
          two_sum(hi[u][v], p, sm, se);
          hi[u][v] = sm;
          lo[u][v] += se + pe;
          if (CB) lo[u][v] = fmaf(av[u], blv[v], lo[u][v]);
          if (CA) lo[u][v] = fmaf(alv[u], bv[v], lo[u][v]);
        }
    }
  }
}

__device__ __forceinline__ float block_max_cl(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = red[0];
#pragma unroll
  for (int w = 1; w < NC_NW; ++w) r = fmaxf(r, red[w]);
  __syncthreads();
  return r;
}

// Sums of two floats over the block (fixed-order shuffle tree, then the warp
// partials in warp order); every thread gets the totals.
__device__ __forceinline__ void block_sum2_cl(float& a, float& b, float (*red)[NC_NW]) {
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
  for (int w = 1; w < NC_NW; ++w) {
    a += red[0][w];
    b += red[1][w];
  }
  __syncthreads();
}

// Stores `v` into slots[idx] in every CTA of the cluster.
template <int C>
__device__ __forceinline__ void cl_publish(float* slots, int idx, float v) {
  const uint32_t a = smem_u32(slots + idx);
#pragma unroll
  for (int d = 0; d < C; ++d) st_cluster_f32(mapa_shared(a, (uint32_t)d), v);
}

// Copies this CTA's rows of S (row-major [own row][KP]) into rows 4 tr + u of
// the full matrix F (leading dimension ldf) in every CTA of the cluster.
template <int C>
__device__ __forceinline__ void cl_broadcast_rows(const float* __restrict__ S, float* F, int KP, int ldf, uint32_t r,
                                                  int nown) {
  const int nq = KP / 4;
  const int n = nown * 4 * nq;
  for (int e = threadIdx.x; e < n; e += NC_THREADS) {
    const int lr = e / nq, j = e - lr * nq;
    const int a = 4 * ((int)r + C * (lr >> 2)) + (lr & 3);
    const float4 v = *reinterpret_cast<const float4*>(S + lr * KP + 4 * j);
    const uint32_t dst = smem_u32(F + a * ldf + 4 * j);
#pragma unroll
    for (int d = 0; d < C; ++d) st_cluster_f4(mapa_shared(dst, (uint32_t)d), v);
  }
}

// One triangle of the k x k block of a full matrix (leading dimension ld)
// copied onto the other: from_lower sets F_ab = F_ba (a < b),
// otherwise F_ba = F_ab.  With T and Y symmetric, (T Y)^T = Y T, so after the
// exchange the lower triangle of T Y is the upper triangle of Y T: mirrored,
// it gives the update Y <- Y T of the coupled iteration, and the upper
// triangle of T Z mirrored gives Z <- T Z, both symmetric as the iteration's
// exact iterates are.  Every CTA holds the same copy and gets the same
// result.
__device__ __forceinline__ void cl_mirror(float* F, int k, int ld, bool from_lower) {
  // warps over rows a, lanes over the columns b > a
  for (int a = threadIdx.x >> 5; a < k - 1; a += NC_NW)
    for (int b = a + 1 + (threadIdx.x & 31); b < k; b += 32) {
      if (from_lower)
        F[a * ld + b] = F[b * ld + a];
      else
        F[b * ld + a] = F[a * ld + b];
    }
}

// Products of this CTA's tiles: the KS-lane groups walk the own tiles (lt,
// tc), lt < nown, tc < nt4, in passes of NTH / KS tiles (NTH threads from
// thread `base`); f(lt, tc, hi, lo) consumes a finished tile (lane q == 0).
template <int KS, bool CA, bool CB, typename F>
__device__ __forceinline__ void cl_product(const float* Ah, const float* Al, int lda, bool a_full, int r, int C,
                                           const float* Bh, const float* Bl, int ldb, int KP, int nown, int base,
                                           int nth, F f) {
  const int lt0 = (int)threadIdx.x - base;
  if (lt0 < 0 || lt0 >= nth) return;  // whole warps
  const int nt4 = KP / 4, ntile = nown * nt4, per = nth / KS, q = lt0 % KS;
  for (int t0 = 0; t0 < ntile; t0 += per) {
    const int t = t0 + lt0 / KS;
    const bool valid = t < ntile;
    const int lt = valid ? t / nt4 : 0, tc = valid ? t - (t / nt4) * nt4 : 0;
    const int ac = a_full ? 4 * (r + C * lt) : 4 * lt;
    float hi[4][4], lo[4][4];
    cl_tile<KS, CA, CB>(Ah, Al, lda, ac, Bh, Bl, ldb, 4 * tc, KP, q, valid, hi, lo);
    tile_combine<KS, CA || CB>(hi, lo);
    if (valid && q == 0) f(lt, tc, hi, lo);
  }
}

// grid (C, N), cluster (C, 1, 1), NC_THREADS threads.  gscr: per subject
// 2 k^2 floats (sym(G) hi, lo; compact k x k) of scratch.  Shared memory:
// full Y and Z, with comp a third full matrix (sym(G) lo in the
// certificate), and three own-row buffers.
template <int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(NC_THREADS, 1)
    polar_ns_cl_kernel(int N, int k, int kld, int T, const float* __restrict__ gpart,
                       const int* __restrict__ gslot_off, float* __restrict__ gscr, double* __restrict__ M64,
                       float* __restrict__ M32, const double* __restrict__ sqnorm, const int64_t* __restrict__ vox,
                       const double* __restrict__ SigmaNext, double* __restrict__ Sigma, double* __restrict__ rho2,
                       double* __restrict__ scal, int* __restrict__ iters_out, int* __restrict__ fallback,
                       double cert, int comp, int* status) {
  constexpr int RMAX = NcGeom<C>::RMAX;
  constexpr int LDT = RMAX + 4;  // transposed own rows: an odd multiple of 4 floats
  extern __shared__ __align__(16) float nc_smem[];
  __shared__ float redf[NC_NW];
  __shared__ float red2[2][NC_NW];
  __shared__ float sl_fro[C], sl_inf[C], sl_err[C * NC_NW];
  __shared__ float sl_e2[C], sl_corr[C], sl_th[C], sl_tl[C];
  __shared__ double trS_s;
  const uint32_t r = cluster_ctarank();
  const int i = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KP = (k + 3) & ~3, KK = KP * KP, nt4 = KP / 4;
  const int LDZ = KP + ((nt4 & 1) ? 0 : 4);  // Z / M_0 are read by columns: an odd multiple of 4 floats
  const int nown = (nt4 - (int)r + C - 1) / C;  // own tile rows (>= 2 for k > 64)
  float* F0 = nc_smem;                     // Y (full)   | sym(G) hi (certificate); read by rows
  float* F1 = F0 + KK;                     // Z (full)   | M_0 (full); leading dimension LDZ
  float* F2 = F1 + KP * LDZ;               // (comp)       sym(G) lo (certificate)
  float* S0 = F2 + (comp ? KK : 0);        // T^T: [KP][LDT] (own rows as columns)
  float* S1 = S0 + LDT * KP;               // new Y rows [RMAX][KP] | R^T hi [KP][LDT]
  float* S2 = S1 + LDT * KP;               // new Z rows [RMAX][KP] | R^T lo [KP][LDT]
  float* gh_g = gscr + (int64_t)i * 2 * k * k;
  float* gl_g = gh_g + (int64_t)k * k;
  auto own_row = [&](int lr) { return 4 * ((int)r + C * (lr >> 2)) + (lr & 3); };
  cluster_sync_all();  // every CTA of the cluster has started before any remote store

  // ---- G: this CTA's rows a and the transposed entries G(b, a), summed over
  // the Gram partials in slot order (error-free FP32), then sym(G) = (G + G^T)/2
  // in float-float.  Scratch (direct hi, lo; transposed hi, lo) in F0 and F1,
  // which hold nothing yet.
  float* Dh = F0;
  float* Dl = Dh + RMAX * KP;
  float* Th = Dl + RMAX * KP;
  float* Tl = Th + RMAX * KP;
  {
    const int s0 = gslot_off[i], s1 = gslot_off[i + 1];
    const int64_t sst = (int64_t)kld * kld;
    const int nq = nt4;
    // direct: own row lr, columns 4j..4j+3; transposed: row b, columns 4 tr..4 tr+3
    for (int e = tid; e < 2 * nown * 4 * nq; e += NC_THREADS) {
      const bool dir = e < nown * 4 * nq;
      const int ee = dir ? e : e - nown * 4 * nq;
      int lr = 0, j = 0, b = 0, tl = 0;
      int64_t off;
      bool ok;
      if (dir) {
        lr = ee / nq;
        j = ee - lr * nq;
        const int a = own_row(lr);
        ok = a < k;
        off = (int64_t)a * kld + 4 * j;
      } else {
        b = ee / nown;
        tl = ee - b * nown;
        ok = b < k;
        off = (int64_t)b * kld + 4 * ((int)r + C * tl);
      }
      float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
      for (int q = s0; q < s1; q += 4) {
        float4 g[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          g[jj] = (ok && q + jj < s1) ? __ldg(reinterpret_cast<const float4*>(gpart + (q + jj) * sst + off))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const float x[4] = {g[jj].x, g[jj].y, g[jj].z, g[jj].w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float sm, se;
            two_sum(h[u], x[u], sm, se);
            h[u] = sm;
            l[u] += se;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float sm, se;
        two_sum(h[u], l[u], sm, se);
        if (dir) {
          const bool in = ok && 4 * j + u < k;
          Dh[lr * KP + 4 * j + u] = in ? sm : 0.f;
          Dl[lr * KP + 4 * j + u] = in ? se : 0.f;
        } else {  // G(b, 4 tr + u) -> transposed entry of own row (tl, u)
          const bool in = ok && 4 * ((int)r + C * tl) + u < k;
          Th[(4 * tl + u) * KP + b] = in ? sm : 0.f;
          Tl[(4 * tl + u) * KP + b] = in ? se : 0.f;
        }
      }
    }
  }
  if (r == 0 && tid < 32) {  // tr Sigma_s^new: fixed-order FP64 tree over the diagonal
    double t = 0.0;
    for (int a = tid; a < k; a += 32) t += SigmaNext[a * k + a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (tid == 0) trS_s = t;
  }
  __syncthreads();
  // sym(G) own rows -> S1 (hi), S2 (lo) and the global scratch; ||G||_F^2
  // and the largest absolute row sum over the own rows
  float fro = 0.f, rowmax = 0.f;
  for (int e = tid; e < nown * 4 * KP; e += NC_THREADS) {
    const int lr = e / KP, b = e - (e / KP) * KP;
    float h = Dh[e], l = Dl[e];
    ff_add(h, l, Th[e], Tl[e]);
    h *= 0.5f;  // exact scaling
    l *= 0.5f;
    S1[e] = h;
    S2[e] = l;
    const int a = own_row(lr);
    if (a < k && b < k) {
      gh_g[a * k + b] = h;
      gl_g[a * k + b] = l;
    }
    fro = fmaf(h, h, fro);
  }
  __syncthreads();
  for (int lr = warp; lr < nown * 4; lr += NC_NW) {  // one warp per own row
    float sum = 0.f;
    for (int b = lane; b < KP; b += 32) sum += fabsf(S1[lr * KP + b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    rowmax = fmaxf(rowmax, sum);
  }
  float unused = 0.f;
  block_sum2_cl(fro, unused, red2);
  rowmax = block_max_cl(rowmax, redf);
  if (tid == 0) {
    cl_publish<C>(sl_fro, (int)r, fro);
    cl_publish<C>(sl_inf, (int)r, rowmax);
  }
  cluster_sync_all();
  float fro_t = 0.f, ginf = 0.f;
#pragma unroll
  for (int d = 0; d < C; ++d) {
    fro_t += sl_fro[d];
    ginf = fmaxf(ginf, sl_inf[d]);
  }
  // both bound lambda_max from above (the margin covers FP32 rounding of the bounds)
  const double c = fmin(sqrt((double)fro_t), (double)ginf) * (1.0 + 1e-5);
  const bool good_c = isfinite(c) && c > 0.0;
  const float cinv = good_c ? (float)(1.0 / c) : 0.f;
  // Y_0 = sym(G) / c (own rows, into every CTA's copy); Z_0 = I
  for (int e = tid; e < nown * 4 * KP; e += NC_THREADS) S1[e] = (S1[e] + S2[e]) * cinv;
  for (int e = tid; e < KK; e += NC_THREADS) {
    const int a = e / KP, b = e - (e / KP) * KP;
    F1[a * LDZ + b] = (a == b && a < k) ? 1.f : 0.f;
  }
  __syncthreads();
  cl_broadcast_rows<C>(S1, F0, KP, KP, r, nown);
  cluster_sync_all();

  float* Y = F0;
  float* Z = F1;
  int it = 0, extra = -1;
  bool conv = false;
  for (; good_c && it < NS_MAXIT; ++it) {
    // one update after max |P - I| < NS_TOL the iterates have converged (the
    // error of P squares per step); the certificate checks the result
    if (extra == 0) {
      conv = true;
      break;
    }
    // P = Z Y with its upper triangle mirrored (own rows, into S1), one tile
    // product over the whole block: a tile on or above the diagonal (tc >= tr)
    // is (Z Y)_ab, a tile below it (Y Z)_ab, and a diagonal tile's lower half
    // is its own upper half transposed (Y and Z symmetric, so rows are read as
    // columns).  Element (a, b) of Z Y and element (b, a) of Y Z are the same
    // products summed in the same order, so P and T = (3I - P)/2 are exactly
    // symmetric across the CTAs: the symmetric form of the one-CTA kernel.  A
    // T that is not symmetric does not commute with G and breaks the
    // invariant Y = G Z / c of the coupled iteration, and the mean
    // (Z Y + Y Z)/2, though symmetric, diverged on Grams of condition 10^3
    // where this form converges.
    {
      constexpr int KS = 4;
      const int per = NC_THREADS / KS, q = tid % KS, ntile = nown * nt4;
      for (int t0 = 0; t0 < ntile; t0 += per) {
        const int t = t0 + tid / KS;
        const bool valid = t < ntile;
        const int lt = valid ? t / nt4 : 0, tc = valid ? t - (t / nt4) * nt4 : 0;
        const int tr = (int)r + C * lt;
        const bool upper = tc >= tr;
        float hi[4][4], lo[4][4];
        cl_tile<KS, false, false>(upper ? Z : Y, nullptr, upper ? LDZ : KP, 4 * tr, upper ? Y : Z, nullptr,
                                  upper ? KP : LDZ, 4 * tc, KP, q, valid, hi, lo);
        tile_combine<KS, false>(hi, lo);
        if (valid && q == 0) {
          if (tc == tr) {  // the diagonal tile: lower half from the upper half
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < u; ++v) hi[u][v] = hi[v][u];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            *reinterpret_cast<float4*>(S1 + (4 * lt + u) * KP + 4 * tc) =
                make_float4(hi[u][0], hi[u][1], hi[u][2], hi[u][3]);
        }
      }
    }
    __syncthreads();
    // T = (3I - P)/2 on the k block, stored transposed in S0; e = max |P - I|
    float emax = 0.f;
    for (int e = tid; e < nown * 4 * KP; e += NC_THREADS) {
      const int lr = e / KP, b = e - (e / KP) * KP;
      const int a = own_row(lr);
      float t = 0.f;
      if (a < k && b < k) {
        const float d = (a == b) ? 1.f : 0.f;
        const float pab = S1[e];
        emax = fmaxf(emax, fabsf(pab - d));
        t = 1.5f * d - 0.5f * pab;
      }
      S0[b * LDT + lr] = t;
    }
    // the warp's largest |P - I| into every CTA's slots (warp-level, no block barrier)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if (lane == 0) cl_publish<C>(sl_err, (int)r * NC_NW + warp, emax);
    __syncthreads();
    // T Y and T Z at once, each by half of the block
    {
      auto store_rows = [&](float* out) {
        return [&, out](int lt, int tc, float (&hi)[4][4], float (&)[4][4]) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            *reinterpret_cast<float4*>(out + (4 * lt + u) * KP + 4 * tc) =
                make_float4(hi[u][0], hi[u][1], hi[u][2], hi[u][3]);
        };
      };
      cl_product<2, false, false>(S0, nullptr, LDT, false, (int)r, C, Y, nullptr, KP, KP, nown, 0, NC_THREADS / 2,
                                  store_rows(S1));
      cl_product<2, false, false>(S0, nullptr, LDT, false, (int)r, C, Z, nullptr, LDZ, KP, nown, NC_THREADS / 2,
                                  NC_THREADS / 2, store_rows(S2));
    }
    __syncthreads();
    cluster_sync_all();  // every CTA has read Y and Z; the errors are published
    float err = 0.f;
    for (int d = lane; d < C * NC_NW; d += 32) err = fmaxf(err, sl_err[d]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) err = fmaxf(err, __shfl_xor_sync(0xffffffffu, err, o));
    if (!(err == err)) break;  // non-finite (the same value in every thread of the cluster)
    if (extra < 0 && err < NS_TOL) extra = 1;
    if (extra > 0) --extra;
    cl_broadcast_rows<C>(S1, Y, KP, KP, r, nown);
    cl_broadcast_rows<C>(S2, Z, KP, LDZ, r, nown);
    cluster_sync_all();
    cl_mirror(Y, k, KP, true);    // Y <- Y T
    cl_mirror(Z, k, LDZ, false);  // Z <- T Z
    __syncthreads();
  }

  // ---- certificate.  M_0 = Z / sqrt(c) (full, in F1); sym(G) hi / lo from
  // the global scratch into F0 / F2.  R = M_0 G (own rows, stored transposed
  // in S1 / S2); E = R M_0 - I (own rows); ||E||_F^2, tr(E R^T) =
  // sum_ab E_ab R_ab (E symmetric) and tr R = tr(M_0 G).
  float* Mb = F1;
  {
    const float sc = good_c ? (float)sqrt(1.0 / c) : 0.f;
    for (int e = tid; e < KK; e += NC_THREADS) {
      const int a = e / KP, b = e - (e / KP) * KP;
      const bool in = a < k && b < k;
      Mb[a * LDZ + b] *= sc;
      F0[e] = in ? __ldcg(gh_g + a * k + b) : 0.f;
      if (comp) F2[e] = in ? __ldcg(gl_g + a * k + b) : 0.f;
    }
  }
  __syncthreads();
  {
    auto store_rt = [&](int lt, int tc, float (&hi)[4][4], float (&lo)[4][4]) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int b = 4 * tc + v;
        *reinterpret_cast<float4*>(S1 + b * LDT + 4 * lt) = make_float4(hi[0][v], hi[1][v], hi[2][v], hi[3][v]);
        *reinterpret_cast<float4*>(S2 + b * LDT + 4 * lt) =
            comp ? make_float4(lo[0][v], lo[1][v], lo[2][v], lo[3][v]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    if (comp)
      cl_product<4, false, true>(Mb, nullptr, LDZ, true, (int)r, C, F0, F2, KP, KP, nown, 0, NC_THREADS, store_rt);
    else
      cl_product<4, false, false>(Mb, nullptr, LDZ, true, (int)r, C, F0, nullptr, KP, KP, nown, 0, NC_THREADS,
                                  store_rt);
  }
  __syncthreads();
  float e2 = 0.f, corr = 0.f;
  {
    auto acc_e = [&](int lt, int tc, float (&hi)[4][4], float (&lo)[4][4]) {
      const int tr = (int)r + C * lt;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int a = 4 * tr + u, b = 4 * tc + v;
          if (a >= k || b >= k) continue;
          const float ev = (hi[u][v] - (a == b ? 1.f : 0.f)) + lo[u][v];
          e2 = fmaf(ev, ev, e2);
          corr = fmaf(ev, S1[b * LDT + 4 * lt + u], corr);
        }
    };
    if (comp)
      cl_product<4, true, false>(S1, S2, LDT, false, (int)r, C, Mb, nullptr, LDZ, KP, nown, 0, NC_THREADS, acc_e);
    else
      cl_product<4, false, false>(S1, nullptr, LDT, false, (int)r, C, Mb, nullptr, LDZ, KP, nown, 0, NC_THREADS,
                                  acc_e);
  }
  // tr R over the own rows in float-float (one warp)
  if (tid < 32) {
    float h = 0.f, l = 0.f;
    for (int lr = tid; lr < nown * 4; lr += 32) {
      const int a = own_row(lr);
      if (a < k) ff_add(h, l, S1[a * LDT + lr], S2[a * LDT + lr]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
      ff_add(h, l, oh, ol);
    }
    if (tid == 0) {
      cl_publish<C>(sl_th, (int)r, h);
      cl_publish<C>(sl_tl, (int)r, l);
    }
  }
  block_sum2_cl(e2, corr, red2);
  if (tid == 0) {
    cl_publish<C>(sl_e2, (int)r, e2);
    cl_publish<C>(sl_corr, (int)r, corr);
  }
  cluster_sync_all();  // the last exchange: no remote access follows
  float e2t = 0.f, corrt = 0.f, th = 0.f, tl = 0.f;
#pragma unroll
  for (int d = 0; d < C; ++d) {
    e2t += sl_e2[d];
    corrt += sl_corr[d];
    ff_add(th, tl, sl_th[d], sl_tl[d]);
  }
  const double enorm = sqrt((double)e2t);
  const bool ok = conv && good_c && enorm <= cert * sqrt((double)k) && isfinite(enorm);
  if (r == 0 && tid == 0) {
    const double trS = trS_s;
    if (iters_out) iters_out[i] = it;
    fallback[i] = ok ? 0 : 1;
    if (ok) {
      const double nuc = ((double)th + (double)tl) - 0.5 * (double)corrt;
      const double rr = (sqnorm[i] - 2.0 * nuc + (double)T * trS) / ((double)T * (double)vox[i]);
      if (!(rr > 0.0) || !isfinite(rr)) flag(status, ST_NONFINITE);
      rho2[i] = rr;
    }
    if (i == 0) scal[SC_TRSIG] = trS;
  }
  if (ok) {
    double* Mi = M64 + (int64_t)i * k * k;
    float* M32i = M32 + (int64_t)i * kld * kld;
    for (int e = tid; e < nown * 4 * k; e += NC_THREADS) {
      const int lr = e / k, b = e - (e / k) * k;
      const int a = own_row(lr);
      if (a >= k) continue;
      const float m = Mb[a * LDZ + b];
      Mi[a * k + b] = (double)m;
      M32i[a * kld + b] = m;
    }
  }
  if (i == 0 && r == 0)
    for (int e = tid; e < k * k; e += NC_THREADS) Sigma[e] = SigmaNext[e];
}

template <int C>
size_t ns_cl_smem_bytes(int k, int comp) {
  const int KP = (k + 3) & ~3, nt4 = KP / 4;
  const int LDZ = KP + ((nt4 & 1) ? 0 : 4);
  return sizeof(float) * ((size_t)(1 + (comp ? 1 : 0)) * KP * KP + (size_t)KP * LDZ +
                          3 * (size_t)(NcGeom<C>::RMAX + 4) * KP);
}

// ---------------------------------------------------------------- Phi by Cholesky
// Phi = B^-1 Sigma_s and ln det B with B = I + rho_0 sym(Sigma_s), in
// float-float arithmetic: each value is an unevaluated sum h + l of two FP32
// numbers (about 48 significant bits), with error-free products (the FMA
// gives a h b exactly as p + fma(a, b, -p)) and error-free sums (two_sum).
// FP64 runs at a small fraction of the FP32 rate on this part, so the
// factorisation and the solves, whose steps form long dependent chains, take
// FP32 operations only; every product that feeds an error-free transformation
// is rounded on its own (__fmul_rn), never fused with a following add.

// s + e == a + b exactly, for |a| >= |b| or a == 0
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// (h, l) = (ah, al) (bh, bl), renormalised
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  fast_two_sum(p, e, h, l);
}

// (h, l) -= (ah, al) (bh, bl)
__device__ __forceinline__ void ff_fnms(float& h, float& l, float ah, float al, float bh, float bl) {
  float ph, pl;
  ff_mul(ah, al, bh, bl, ph, pl);
  ff_add(h, l, -ph, -pl);
}

// 1 / sqrt(d) for d = dh + dl > 0: the FP32 rsqrtf estimate y (about 22
// correct bits) and one Newton-Raphson step y + y (1 - d y^2) / 2, with the
// residual 1 - d y^2 formed in float-float (about 44 correct bits)
__device__ __forceinline__ void ff_rsqrt(float dh, float dl, float& h, float& l) {
  const float y = rsqrtf(dh);
  float th, tl;
  ff_mul(dh, dl, y, 0.f, th, tl);
  ff_mul(th, tl, y, 0.f, th, tl);
  const float e = __fsub_rn(__fsub_rn(1.f, th), tl);
  fast_two_sum(y, __fmul_rn(0.5f * y, e), h, l);
}

// One CTA.  rho_0 = sum_i rho_i^-2 (eq:srm_wt_psi_w) and the likelihood's sums
// over subjects (or, for a sharded E-step, sums = {sum rho_i^-2,
// sum v_i ln rho_i^2, sum ||X^_i||^2 / rho_i^2, sum v_i} over all shards);
// B in shared memory (column-major, hi and lo planes), factorised
// right-looking: step j scales column j by 1 / sqrt(d_j) into L (and a
// shared copy), then the trailing lower triangle takes the rank-1 update
// B_ic -= L_ij L_cj.  L goes to Lh / Ll (column-major), 1 / L_jj to Dh / Dl,
// and ln det B = sum_j ln d_j is summed in FP64 after the loop.
constexpr int PC_THREADS = 512;  // each warp repeats a step's prologue: 16 warps balance it against latency

__global__ void __launch_bounds__(PC_THREADS) phi_chol_kernel(int N, int k, const double* __restrict__ rho2,
                                                              const double* __restrict__ sqnorm,
                                                              const int64_t* __restrict__ vox,
                                                              const double* __restrict__ Sigma, float* __restrict__ Lh,
                                                              float* __restrict__ Ll, float* __restrict__ Dh,
                                                              float* __restrict__ Dl, double* __restrict__ scal,
                                                              int* status, double vtot, const double* __restrict__ sums) {
  extern __shared__ float pc_smem[];
  float* Bh = pc_smem;       // [k][k] column-major: (i, c) at c * k + i
  float* Bl = Bh + k * k;
  float* ch = Bl + k * k;    // [k] column j of L
  float* cl = ch + k;
  float* ph = cl + k;        // [k] pivots d_j
  float* pl = ph + k;
  __shared__ double red[3][PC_THREADS];
  const int tid = threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (sums) {
    s0 = sums[0];
    s1 = sums[1];
    s2 = sums[2];
    vtot = sums[3];
    if (!(s0 > 0.0) || !isfinite(s0) || !isfinite(s1) || !isfinite(s2) || !(vtot > 0.0)) flag(status, ST_NONFINITE);
  } else {
    for (int i = tid; i < N; i += PC_THREADS) {
      const double r = rho2[i];
      if (!(r > 0.0) || !isfinite(r)) flag(status, ST_NONFINITE);
      s0 += 1.0 / r;
      s1 += (double)vox[i] * log(r);
      s2 += sqnorm[i] / r;
    }
    red[0][tid] = s0;
    red[1][tid] = s1;
    red[2][tid] = s2;
    __syncthreads();
    for (int st = PC_THREADS / 2; st > 0; st >>= 1) {
      if (tid < st) {
        red[0][tid] += red[0][tid + st];
        red[1][tid] += red[1][tid + st];
        red[2][tid] += red[2][tid + st];
      }
      __syncthreads();
    }
    s0 = red[0][0];
    s1 = red[1][0];
    s2 = red[2][0];
    __syncthreads();  // red is reused below
  }
  const double rho0 = s0;
  for (int e = tid; e < k * k; e += PC_THREADS) {
    const int c = e / k, i = e - c * k;
    const double x = (i == c ? 1.0 : 0.0) + rho0 * (0.5 * (Sigma[i * k + c] + Sigma[c * k + i]));
    const float h = (float)x;
    Bh[e] = h;
    Bl[e] = (float)(x - (double)h);
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  bool pd = true;
  int jdone = 0;
  for (int j = 0; j < k; ++j) {
    const float dh = Bh[j * k + j], dl = Bl[j * k + j];
    if (!(dh > 0.f) || !isfinite(dh)) {  // the same value in every thread
      pd = false;
      break;
    }
    float ih, il;
    ff_rsqrt(dh, dl, ih, il);
    for (int i = j + tid; i < k; i += PC_THREADS) {
      float h, l;
      ff_mul(Bh[j * k + i], Bl[j * k + i], ih, il, h, l);
      ch[i] = h;
      cl[i] = l;
      Lh[j * k + i] = h;
      Ll[j * k + i] = l;
    }
    if (tid == 0) {
      ph[j] = dh;
      pl[j] = dl;
      Dh[j] = ih;
      Dl[j] = il;
    }
    __syncthreads();
    for (int cc = j + 1 + warp; cc < k; cc += PC_THREADS / 32) {
      const float lh = ch[cc], ll = cl[cc];
      float* bh = Bh + cc * k;
      float* bl = Bl + cc * k;
      for (int i = cc + lane; i < k; i += 32) {
        float h = bh[i], l = bl[i];
        ff_fnms(h, l, ch[i], cl[i], lh, ll);
        bh[i] = h;
        bl[i] = l;
      }
    }
    __syncthreads();
    jdone = j + 1;
  }
  // ln det B = sum_j ln d_j (fixed-order tree over the block)
  double ld = 0.0;
  for (int j = tid; j < jdone; j += PC_THREADS) ld += log((double)ph[j] + (double)pl[j]);
  red[0][tid] = ld;
  __syncthreads();
  for (int st = PC_THREADS / 2; st > 0; st >>= 1) {
    if (tid < st) red[0][tid] += red[0][tid + st];
    __syncthreads();
  }
  if (tid == 0) {
    if (!pd) flag(status, ST_NOT_PD);
    scal[SC_RHO0] = rho0;
    scal[SC_LOGDET] = red[0][0];
    scal[SC_VLOGRHO] = s1;
    scal[SC_SQRHO] = s2;
    scal[SC_VTOT] = vtot;
  }
}

// grid k blocks, PS_THREADS threads.  Block j stages L (hi and lo planes,
// column-major with an odd leading dimension so that rows and columns are
// both read without bank conflicts) and one warp solves L L^T x =
// sym(Sigma_s)[:, j] in float-float by forward and backward substitution,
// lane l holding entries l + 32 u, by 32-row blocks: the block's triangle
// step by step (only that block's entries are in the dependent chain), then
// the other blocks take its contribution.  Phi's row j = x (Phi = B^-1
// Sigma_s is symmetric), in FP64 and FP32.
constexpr int PS_THREADS = 128;

template <int R>  // entries per lane: k <= 32 R
__global__ void __launch_bounds__(PS_THREADS) phi_solve_kernel(int k, const float* __restrict__ Lh,
                                                               const float* __restrict__ Ll,
                                                               const float* __restrict__ Dh,
                                                               const float* __restrict__ Dl,
                                                               const double* __restrict__ Sigma,
                                                               double* __restrict__ Phi, float* __restrict__ Phi32,
                                                               int* status) {
  extern __shared__ float ps_smem[];
  const int ld = k | 1;
  float* Sh = ps_smem;        // [k][ld]: (i, m) at m * ld + i
  float* Sl = Sh + k * ld;
  float* dh = Sl + k * ld;    // [k] 1 / L_mm
  float* dl = dh + k;
  const int j = blockIdx.x, tid = threadIdx.x;
  // L from L2 with 16-byte loads (both planes start on 16-byte boundaries),
  // four per plane in flight per thread; the last k^2 mod 4 elements singly
  const int n4 = (k * k) / 4;
  for (int e0 = tid; e0 < n4; e0 += 4 * PS_THREADS) {
    float4 vh[4], vl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * PS_THREADS;
      vh[u] = e < n4 ? __ldg(reinterpret_cast<const float4*>(Lh) + e) : make_float4(0.f, 0.f, 0.f, 0.f);
      vl[u] = e < n4 ? __ldg(reinterpret_cast<const float4*>(Ll) + e) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * PS_THREADS;
      if (e >= n4) continue;
      const float hv[4] = {vh[u].x, vh[u].y, vh[u].z, vh[u].w}, lv[4] = {vl[u].x, vl[u].y, vl[u].z, vl[u].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int f = 4 * e + q, m = f / k, i = f - m * k;
        const bool low = i >= m;
        Sh[m * ld + i] = low ? hv[q] : 0.f;
        Sl[m * ld + i] = low ? lv[q] : 0.f;
      }
    }
  }
  for (int f = 4 * n4 + tid; f < k * k; f += PS_THREADS) {
    const int m = f / k, i = f - m * k;
    const bool low = i >= m;
    Sh[m * ld + i] = low ? Lh[f] : 0.f;
    Sl[m * ld + i] = low ? Ll[f] : 0.f;
  }
  for (int m = tid; m < k; m += PS_THREADS) {
    dh[m] = Dh[m];
    dl[m] = Dl[m];
  }
  __syncthreads();
  if (tid >= 32) return;
  const int lane = tid;
  float yh[R], yl[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = lane + 32 * u;
    const double x = i < k ? 0.5 * (Sigma[i * k + j] + Sigma[j * k + i]) : 0.0;
    yh[u] = (float)x;
    yl[u] = (float)(x - (double)yh[u]);
  }
  // L z = y
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int iu = lane + 32 * u;
    for (int s = 0; s < 32; ++s) {
      const int m = 32 * u + s;
      if (m >= k) break;
      float zh, zl;
      ff_mul(__shfl_sync(0xffffffffu, yh[u], s), __shfl_sync(0xffffffffu, yl[u], s), dh[m], dl[m], zh, zl);
      if (lane == s) {
        yh[u] = zh;
        yl[u] = zl;
      }
      if (iu > m && iu < k) ff_fnms(yh[u], yl[u], Sh[m * ld + iu], Sl[m * ld + iu], zh, zl);
    }
    if (u + 1 < R) {
      for (int s = 0; s < 32; ++s) {
        const int m = 32 * u + s;
        if (m >= k) break;
        const float zh = __shfl_sync(0xffffffffu, yh[u], s), zl = __shfl_sync(0xffffffffu, yl[u], s);
#pragma unroll
        for (int w = u + 1; w < R; ++w) {
          const int i = lane + 32 * w;
          if (i < k) ff_fnms(yh[w], yl[w], Sh[m * ld + i], Sl[m * ld + i], zh, zl);
        }
      }
    }
  }
  // L^T x = z (column m of L^T is row m of L), blocks from the last
#pragma unroll
  for (int u = R - 1; u >= 0; --u) {
    const int iu = lane + 32 * u;
    for (int s = 31; s >= 0; --s) {
      const int m = 32 * u + s;
      if (m >= k) continue;
      float xh, xl;
      ff_mul(__shfl_sync(0xffffffffu, yh[u], s), __shfl_sync(0xffffffffu, yl[u], s), dh[m], dl[m], xh, xl);
      if (lane == s) {
        yh[u] = xh;
        yl[u] = xl;
      }
      if (iu < m) ff_fnms(yh[u], yl[u], Sh[iu * ld + m], Sl[iu * ld + m], xh, xl);
    }
    if (u > 0) {
      for (int s = 0; s < 32; ++s) {
        const int m = 32 * u + s;
        if (m >= k) break;
        const float xh = __shfl_sync(0xffffffffu, yh[u], s), xl = __shfl_sync(0xffffffffu, yl[u], s);
#pragma unroll
        for (int w = 0; w < u; ++w) {
          const int i = lane + 32 * w;
          ff_fnms(yh[w], yl[w], Sh[i * ld + m], Sl[i * ld + m], xh, xl);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = lane + 32 * u;
    if (i < k) {
      const double x = (double)yh[u] + (double)yl[u];
      if (!isfinite(x)) flag(status, ST_NONFINITE);
      Phi[j * k + i] = x;
      Phi32[j * k + i] = (float)x;
    }
  }
}

size_t phi_chol_smem_bytes(int k) { return sizeof(float) * (2 * (size_t)k * k + 4 * k); }
size_t phi_solve_smem_bytes(int k) { return sizeof(float) * (2 * (size_t)k * (k | 1) + 2 * k); }

}  // namespace

bool polar_cl_supported(const Ctx* c) { return c->k > 64 && c->k <= NC_KMAX; }

void prepare_tail_kernels() {
  cudaFuncSetAttribute(polar_ns_cl_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ns_cl_smem_bytes<8>(NC_KMAX, 1));
  cudaFuncSetAttribute(polar_ns_cl_kernel<8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  // four-CTA clusters: up to k = 128 without the third full matrix, k <= 112 with it
  cudaFuncSetAttribute(polar_ns_cl_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ns_cl_smem_bytes<4>(NC_KMAX, 0));
  cudaFuncSetAttribute(polar_ns_cl_kernel<4>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(phi_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)phi_chol_smem_bytes(KMAX));
  cudaFuncSetAttribute(phi_solve_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)phi_solve_smem_bytes(KMAX));
}

namespace {

// Clusters of 8 CTAs run as many subjects at once as the GPU holds such
// clusters (15 on a 152-SM part with one cluster of this size per 8 SMs of a
// GPC); with more subjects, clusters of 4 (twice the rows per CTA) take fewer
// waves when their shared memory fits.  The choice is made once per context
// from the occupancy calculator.
int polar_cl_waves(const void* fn, int C, int N, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, N);
  cfg.blockDim = dim3(NC_THREADS);
  cfg.dynamicSmemBytes = smem;
  int active = 0;
  if (cudaOccupancyMaxActiveClusters(&active, fn, &cfg) != cudaSuccess || active <= 0) {
    cudaGetLastError();
    return -1;
  }
  return (N + active - 1) / active;
}

}  // namespace

void choose_polar_cl(Ctx* c) {
  const int comp = c->store == SRM_BF16 ? 0 : 1;
  const size_t sm8 = ns_cl_smem_bytes<8>(c->k, comp), sm4 = ns_cl_smem_bytes<4>(c->k, comp);
  c->ns_cl_c = 8;
  if (sm4 <= ns_cl_smem_bytes<4>(NC_KMAX, 0)) {
    const int w8 = polar_cl_waves(reinterpret_cast<const void*>(polar_ns_cl_kernel<8>), 8, c->N, sm8);
    const int w4 = polar_cl_waves(reinterpret_cast<const void*>(polar_ns_cl_kernel<4>), 4, c->N, sm4);
    if (w4 > 0 && (w8 < 0 || w4 < w8)) c->ns_cl_c = 4;
  }
}

cudaError_t launch_polar_cl(Ctx* c, double cert, int comp) {
  const size_t sm8 = ns_cl_smem_bytes<8>(c->k, comp), sm4 = ns_cl_smem_bytes<4>(c->k, comp);
  // sym(G) hi / lo per subject in the G64 buffer (k^2 doubles = 2 k^2 floats),
  // which the eigen-decomposition fallback overwrites only afterwards
  float* gscr = reinterpret_cast<float*>(c->G64);
  if (c->ns_cl_c == 4)
    polar_ns_cl_kernel<4><<<dim3(4, c->N), NC_THREADS, sm4, c->stream>>>(
        c->N, c->k, c->kld, c->T, c->Gpart, c->gslot_off, gscr, c->M64, c->M32, c->sqnorm, c->d_v, c->SigmaNext,
        c->Sigma, c->rho2, c->scal, c->jac_sweeps, c->ns_fb, cert, comp, c->status);
  else
    polar_ns_cl_kernel<8><<<dim3(8, c->N), NC_THREADS, sm8, c->stream>>>(
        c->N, c->k, c->kld, c->T, c->Gpart, c->gslot_off, gscr, c->M64, c->M32, c->sqnorm, c->d_v, c->SigmaNext,
        c->Sigma, c->rho2, c->scal, c->jac_sweeps, c->ns_fb, cert, comp, c->status);
  return cudaGetLastError();
}

// Phi and ln det(I + rho_0 Sigma_s) from the committed Sigma_s.  The Cholesky
// factor (hi and lo planes, each padded to a multiple of 4 floats) and its
// reciprocal diagonal go to the H64 buffer (at most 2 k^2 + 2 k + 6 floats of
// (N + 1) k^2 doubles), which nothing else reads
// between an M-step tail and the next.
cudaError_t launch_phi_chol(Ctx* c, const double* sums) {
  const int k = c->k;
  if (k > 128) return cudaErrorInvalidValue;
  const int64_t kk4 = ((int64_t)k * k + 3) & ~(int64_t)3;  // planes on 16-byte boundaries
  float* Lh = reinterpret_cast<float*>(c->H64);
  float* Ll = Lh + kk4;
  float* Dh = Ll + kk4;
  float* Dl = Dh + k;
  phi_chol_kernel<<<1, PC_THREADS, phi_chol_smem_bytes(k), c->stream>>>(
      c->N, k, c->rho2, c->sqnorm, c->d_v, c->Sigma, Lh, Ll, Dh, Dl, c->scal, c->status, (double)c->Vtot, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  phi_solve_kernel<4><<<k, PS_THREADS, phi_solve_smem_bytes(k), c->stream>>>(k, Lh, Ll, Dh, Dl, c->Sigma, c->Phi,
                                                                             c->Phi32, c->status);
  return cudaGetLastError();
}

}  // namespace srm
