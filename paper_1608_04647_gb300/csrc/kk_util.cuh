// Device helpers shared by the k x k kernels of an EM iteration (k_small.cu,
// k_tail.cu): status flags, error-free FP32 sums, the scal[] layout and the
// Newton-Schulz polar-factor constants.
#pragma once

#include "srm_internal.cuh"

namespace srm {
namespace {

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ void flag(int* status, int bits) { atomicOr(status, bits); }

// Error-free sum: s + e == a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// (h, l) += (bh, bl) in float-float arithmetic (renormalised)
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e += l + bl;
  two_sum(s, e, h, l);
}

// scal[] layout
enum { SC_RHO0 = 0, SC_LOGDET = 1, SC_VLOGRHO = 2, SC_SQRHO = 3, SC_YPHIY = 4, SC_TRSIG = 5, SC_VTOT = 6 };

// Newton-Schulz polar factor: iteration limit, stopping tolerance on
// max |P - I|, and the accepted certificate ||E||_F / sqrt(k) for the FP32
// store (results compared at 1e-5) and the BF16 store (2e-2)
constexpr int NS_MAXIT = 40;
constexpr float NS_TOL = 1e-4f;
constexpr double NS_CERT_F32 = 2e-6;
constexpr double NS_CERT_BF16 = 1e-4;

// Adds the partial 4 x 4 tiles that KS adjacent lanes hold (lanes l ^ 1,
// l ^ 2, ...), in float-float arithmetic with COMP.
template <int KS, bool COMP>
__device__ __forceinline__ void tile_combine(float (&hi)[4][4], float (&lo)[4][4]) {
#pragma unroll
  for (int o = 1; o < KS; o <<= 1)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi[u][v], o);
        if (COMP) {
          const float ol = __shfl_xor_sync(0xffffffffu, lo[u][v], o);
          ff_add(hi[u][v], lo[u][v], oh, ol);
        } else {
          hi[u][v] += oh;
        }
      }
}

}  // namespace
}  // namespace srm
