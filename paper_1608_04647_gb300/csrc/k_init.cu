// Algorithm 1's initialisation of the mappings inside the library: "initialise
// W_i to a random orthogonal matrix", drawn here from the Haar distribution
// on v_i x k matrices with orthonormal columns as the Q factor (with a
// positive-diagonal R) of a matrix of independent standard normal entries.
//
// The normal entries come from a counter-based generator, so that any other
// implementation of the same definition draws the same W^0:
//   Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
//   easy as 1, 2, 3", SC 2011): key (seed, 0), counter (b, i, 0, 0) for
//   block b of subject i; each 64-bit output word w gives the uniform
//   u = ((w >> 12) + 1/2) 2^-52 in (0, 1); the words (w0, w1) and (w2, w3) of
//   a block give four normals by the Box-Muller transform
//   sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b); block b supplies entries
//   4b .. 4b + 3 of the v_i x k matrix G_i in row-major order.
// Q is formed by Cholesky QR applied twice in FP64: C = G^T G = L L^T,
// Q = G L^-T, then the same on Q.  Cholesky's L has a positive diagonal, so
// R = L_2^T L_1^T does too, and Q is the unique such Q factor of G.
#include <math.h>

#include <algorithm>

#include "srm_internal.cuh"

namespace srm {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Ten rounds of Philox4x64 on counter c with key (k0, k1): the multipliers
// and the key increments (the golden ratio and sqrt(3) - 1 in 64-bit fixed
// point) of the published definition.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// exact in FP64: in [2^-53, 1 - 2^-53]
__device__ __forceinline__ double unit_open(uint64_t w) { return ((double)(w >> 12) + 0.5) * 0x1.0p-52; }

// G[e], e < n = v k: the standard normal entries of subject `subject`.
__global__ void __launch_bounds__(256) haar_normal_kernel(uint64_t seed, int subject, int64_t n,
                                                          double* __restrict__ G) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * b >= n) return;
  uint64_t c[4] = {(uint64_t)b, (uint64_t)subject, 0ull, 0ull};
  philox4x64_10(c, seed, 0ull);
  double z[4];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const double r = sqrt(-2.0 * log(unit_open(c[2 * p])));
    double s, co;
    sincospi(2.0 * unit_open(c[2 * p + 1]), &s, &co);
    z[2 * p] = r * co;
    z[2 * p + 1] = r * s;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (4 * b + q < n) G[4 * b + q] = z[q];
}

// part[s][a][b] = sum over rows r of split s of G[r][a] G[r][b]: grid
// (splits, tiles of 32 x 32 entries), 256 threads with 2 x 2 entries each.
constexpr int GT = 32, GR = 64;
__global__ void __launch_bounds__(256) gram64_part_kernel(const double* __restrict__ G, int64_t v, int k,
                                                          int nsplit, double* __restrict__ part) {
  __shared__ double Ga[GR][GT + 1], Gb[GR][GT + 1];
  const int s = blockIdx.x;
  const int ntb = (k + GT - 1) / GT;
  const int a0 = (blockIdx.y / ntb) * GT, b0 = (blockIdx.y % ntb) * GT;
  const int64_t r0 = v * s / nsplit, r1 = v * (s + 1) / nsplit;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t rb = r0; rb < r1; rb += GR) {
    for (int e = threadIdx.x; e < GR * GT; e += 256) {
      const int rr = e / GT, cc = e % GT;
      const int64_t r = rb + rr;
      Ga[rr][cc] = (r < r1 && a0 + cc < k) ? G[r * k + a0 + cc] : 0.0;
      Gb[rr][cc] = (r < r1 && b0 + cc < k) ? G[r * k + b0 + cc] : 0.0;
    }
    __syncthreads();
    for (int rr = 0; rr < GR; ++rr)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = fma(Ga[rr][ty + 16 * i], Gb[rr][tx + 16 * j], acc[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < k && b < k) part[((int64_t)s * k + a) * k + b] = acc[i][j];
    }
}

// C[a][b] = sum of the splits' partials (in split order), symmetrised; one
// thread per entry.
__global__ void __launch_bounds__(256) gram64_sum_kernel(const double* __restrict__ part, int nsplit, int k,
                                                         double* __restrict__ C) {
  const int64_t kk = (int64_t)k * k;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kk) return;
  const int a = (int)(e / k), b = (int)(e % k);
  double x = 0.0, y = 0.0;
  for (int s = 0; s < nsplit; ++s) {
    x += part[s * kk + (int64_t)a * k + b];
    y += part[s * kk + (int64_t)b * k + a];
  }
  C[e] = 0.5 * (x + y);
}

// One block: the Cholesky factor L of C (C = L L^T, positive diagonal, in
// place in C's lower triangle) and Linv = L^-1, FP64.  A non-positive pivot
// sets ST_NOT_PD.
__global__ void __launch_bounds__(256) chol_inv_kernel(int k, double* __restrict__ C, double* __restrict__ Linv,
                                                       int* status) {
  const int tid = threadIdx.x;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  // right-looking Cholesky in place (lower triangle of C becomes L)
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const double d = C[(int64_t)j * k + j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        C[(int64_t)j * k + j] = 1.0;
      } else {
        C[(int64_t)j * k + j] = sqrt(d);
      }
    }
    __syncthreads();
    const double ljj = C[(int64_t)j * k + j];
    for (int i = j + 1 + tid; i < k; i += 256) C[(int64_t)i * k + j] /= ljj;
    __syncthreads();
    const int m = k - j - 1;
    for (int64_t e = tid; e < (int64_t)m * m; e += 256) {
      const int i = j + 1 + (int)(e / m), c2 = j + 1 + (int)(e % m);
      if (c2 <= i) C[(int64_t)i * k + c2] -= C[(int64_t)i * k + j] * C[(int64_t)c2 * k + j];
    }
    __syncthreads();
  }
  if (tid == 0 && bad) atomicOr(status, ST_NOT_PD);
  // Linv column by column (forward substitution), one thread per column
  for (int jc = tid; jc < k; jc += 256) {
    for (int i = 0; i < k; ++i) {
      double s = (i == jc) ? 1.0 : 0.0;
      for (int m = jc; m < i; ++m) s -= C[(int64_t)i * k + m] * Linv[(int64_t)m * k + jc];
      Linv[(int64_t)i * k + jc] = (i < jc) ? 0.0 : s / C[(int64_t)i * k + i];
    }
  }
}

// Q[r][c] = sum_{j <= c} G[r][j] Linv[c][j]  (Q = G L^-T), one thread per entry.
__global__ void __launch_bounds__(256) apply_linv_kernel(const double* __restrict__ G, int64_t v, int k,
                                                         const double* __restrict__ Linv, double* __restrict__ Q) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= v * k) return;
  const int64_t r = e / k;
  const int c = (int)(e % k);
  const double* g = G + r * k;
  const double* l = Linv + (int64_t)c * k;
  double s = 0.0;
  for (int j = 0; j <= c; ++j) s = fma(g[j], __ldg(l + j), s);
  Q[e] = s;
}

__global__ void __launch_bounds__(256) to_f32_kernel(const double* __restrict__ Q, int64_t n, float* __restrict__ W) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) W[e] = (float)Q[e];
}

// Row splits of the Gram: enough blocks for about four per SM (FP64 runs at
// about 2 FMA per clock per SM on this part), at least 64 rows each.
int gram_splits(int64_t v, int k, int num_sms) {
  const int tiles = ((k + GT - 1) / GT) * ((k + GT - 1) / GT);
  const int want = (4 * num_sms + tiles - 1) / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, v / 64));
}

}  // namespace

size_t haar_workspace_bytes(const Ctx* c) {
  int64_t vmax = 0;
  for (int i = 0; i < c->N; ++i) vmax = std::max(vmax, c->v[i]);
  const int64_t kk = (int64_t)c->k * c->k;
  const int64_t nf = ((vmax * c->k + 1) / 2) * 2;  // FP32 W^0, padded to keep the FP64 workspace aligned
  return (size_t)(2 * vmax * c->k) * sizeof(double) + (size_t)nf * sizeof(float) +
         (size_t)(gram_splits(vmax, c->k, c->num_sms) * kk + 2 * kk) * sizeof(double);
}

cudaError_t launch_haar_w0(Ctx* c, int i, uint64_t seed, void* work) {
  const int64_t v = c->v[i], n = v * c->k;
  const int k = c->k;
  int64_t vmax = 0;
  for (int q = 0; q < c->N; ++q) vmax = std::max(vmax, c->v[q]);
  double* G = static_cast<double*>(work);
  double* Q = G + vmax * k;
  float* Wf = reinterpret_cast<float*>(Q + vmax * k);
  double* part = reinterpret_cast<double*>(Wf + ((vmax * k + 1) / 2) * 2);
  const int ns = gram_splits(v, k, c->num_sms);
  const int64_t kk = (int64_t)k * k;
  double* C = part + ns * kk;
  double* Linv = C + kk;
  const int ntb = (k + GT - 1) / GT;
  haar_normal_kernel<<<nblk((n + 3) / 4, 256), 256, 0, c->stream>>>(seed, i, n, G);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // two Cholesky-QR passes: G -> Q -> G (the second result lands in G)
  for (int pass = 0; pass < 2; ++pass) {
    const double* src = pass == 0 ? G : Q;
    double* dst = pass == 0 ? Q : G;
    gram64_part_kernel<<<dim3(ns, ntb * ntb), 256, 0, c->stream>>>(src, v, k, ns, part);
    gram64_sum_kernel<<<nblk(kk, 256), 256, 0, c->stream>>>(part, ns, k, C);
    chol_inv_kernel<<<1, 256, 0, c->stream>>>(k, C, Linv, c->status);
    apply_linv_kernel<<<nblk(n, 256), 256, 0, c->stream>>>(src, v, k, Linv, dst);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  to_f32_kernel<<<nblk(n, 256), 256, 0, c->stream>>>(G, n, Wf);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_load_w0(c, i, Wf);
}

}  // namespace srm
