// srm_transform_noalloc: the shared-space projection of srm_transform with
// no allocation at all.  srm_transform keeps a centred copy of the new data
// and its split-v partial sums in buffers it allocates (and grows) on
// demand; this variant centres on the fly and keeps the row means and the
// partial sums in one fixed device array that lives as long as the library
// is loaded.  The paper has no counterpart; this exists for callers that must
// not allocate device memory.
#include <algorithm>
#include <mutex>
#include <string>

#include "srm_internal.cuh"

namespace srm {

namespace {

// Fixed scratch: the row means of the new data, then the split-v partials.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ float ld_f(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_f(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

// mu[r] = mean_t X[r][t]: one warp per row, per-lane compensated FP32 sums and
// an FP64 warp reduction (the same arithmetic as the centring pre-pass).
template <typename TX>
__global__ void __launch_bounds__(256) rowmean_kernel(const TX* __restrict__ X, int64_t rows, int T,
                                                      float* __restrict__ mu) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  if (r >= rows) return;
  const TX* xr = X + r * T;
  float s = 0.f, cmp = 0.f;
  for (int t = lane; t < T; t += 32) {
    float y = ld_f(xr, t) - cmp;
    float tt = s + y;
    cmp = (tt - s) - y;
    s = tt;
  }
  double ds = (double)s - (double)cmp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, o);
  if (lane == 0) mu[r] = (float)(ds / (double)T);
}

__device__ __forceinline__ float ld_a(const float* A, int64_t i) { return A[i]; }
__device__ __forceinline__ float ld_a(const __nv_bfloat16* A, int64_t i) { return __bfloat162float(A[i]); }

// part[s][c][t][f] = sum over the rows of split s of A[r][f] (X[r][t0 + t] - mu[r]).
// Same tiling as the plain E-pass: a block owns a 64-wide t-chunk of one
// v-split, each thread a (KQ/16) x 4 register tile.
template <int KQ, typename TA, typename TX>
__global__ void __launch_bounds__(256) p_centred_kernel(const TA* __restrict__ A, int kld, const TX* __restrict__ X,
                                                        const float* __restrict__ mu, int64_t rows, int T,
                                                        int nsplit, float* __restrict__ part) {
  constexpr int FJ = KQ / 16;
  constexpr int R = 32;
  __shared__ float As[R][KQ];
  __shared__ __align__(16) float Xs[R][TCH];
  const int cT = blockIdx.x, s = blockIdx.y, nchunk = gridDim.x;
  const int t0 = cT * TCH;
  const int64_t rb = rows * s / nsplit, re = rows * (s + 1) / nsplit;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float acc[FJ][4];
#pragma unroll
  for (int j = 0; j < FJ; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  for (int64_t r0 = rb; r0 < re; r0 += R) {
    for (int e = tid; e < R * KQ; e += 256) {
      const int rr = e / KQ, f = e % KQ;
      const int64_t r = r0 + rr;
      As[rr][f] = (r < re && f < kld) ? ld_a(A, r * kld + f) : 0.f;
    }
    for (int e = tid; e < R * TCH; e += 256) {
      const int rr = e / TCH, t = e % TCH;
      const int64_t r = r0 + rr;
      Xs[rr][t] = (r < re && t0 + t < T) ? ld_f(X, r * (int64_t)T + t0 + t) - mu[r] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < R; ++rr) {
      const float4 xv = *reinterpret_cast<const float4*>(&Xs[rr][tx * 4]);
#pragma unroll
      for (int j = 0; j < FJ; ++j) {
        const float a = As[rr][ty + 16 * j];
        acc[j][0] = fmaf(a, xv.x, acc[j][0]);
        acc[j][1] = fmaf(a, xv.y, acc[j][1]);
        acc[j][2] = fmaf(a, xv.z, acc[j][2]);
        acc[j][3] = fmaf(a, xv.w, acc[j][3]);
      }
    }
    __syncthreads();
  }
  float* out = part + ((int64_t)s * nchunk + cT) * TCH * kld;
#pragma unroll
  for (int j = 0; j < FJ; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(tx * 4 + q) * kld + ty + 16 * j] = acc[j][q];
}

template <typename TA, typename TX>
cudaError_t launch_p_centred(int kld, dim3 grid, cudaStream_t st, const TA* A, const TX* X, const float* mu,
                             int64_t rows, int T, int nsplit, float* part) {
  switch (kld) {
#define PC_CASE(KQ) \
  case KQ: p_centred_kernel<KQ, TA, TX><<<grid, 256, 0, st>>>(A, kld, X, mu, rows, T, nsplit, part); break;
    PC_CASE(16) PC_CASE(32) PC_CASE(48) PC_CASE(64) PC_CASE(80) PC_CASE(96) PC_CASE(112) PC_CASE(128)
#undef PC_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename TA>
cudaError_t launch_p_centred_x(srm_dtype xt, int kld, dim3 grid, cudaStream_t st, const TA* A, const void* X,
                               const float* mu, int64_t rows, int T, int nsplit, float* part) {
  if (xt == SRM_BF16)
    return launch_p_centred<TA, __nv_bfloat16>(kld, grid, st, A, static_cast<const __nv_bfloat16*>(X), mu, rows, T,
                                               nsplit, part);
  return launch_p_centred<TA, float>(kld, grid, st, A, static_cast<const float*>(X), mu, rows, T, nsplit, part);
}

// Device address of the scratch array on device `dev`, looked up once per
// device and cached.  The caller has made `dev` the current device.
srm_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("srm_transform_noalloc: device ordinal out of range");
    return SRM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "srm_transform_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SRM_OK;
}

}  // namespace
}  // namespace srm

using namespace srm;

extern "C" srm_status srm_transform_noalloc(srm_ctx* c, int32_t subject, const void* X_new, int32_t T_new,
                                            float* S_out) {
  if (!c) {
    set_error("srm_transform_noalloc: null context");
    return SRM_ERR_ARG;
  }
  if (subject < 0 || subject >= c->N || !X_new || !S_out || T_new < 1) {
    set_error("srm_transform_noalloc: bad subject, pointer or T_new");
    return SRM_ERR_ARG;
  }
  const int64_t v = c->v[subject];
  const int nchunk = (T_new + TCH - 1) / TCH;
  const size_t mu_bytes = (((size_t)v * sizeof(float)) + 255) & ~size_t(255);
  const size_t split_bytes = (size_t)nchunk * TCH * c->kld * sizeof(float);
  if (mu_bytes + split_bytes > kNoAllocScratchBytes) {
    set_error("srm_transform_noalloc: v_i = " + std::to_string(v) + " voxels and T_new = " + std::to_string(T_new) +
              " need " + std::to_string(mu_bytes + split_bytes) + " bytes of scratch; the fixed array holds " +
              std::to_string(kNoAllocScratchBytes) + " (use srm_transform)");
    return SRM_ERR_ARG;
  }
  int ns = std::max(1, 2 * c->num_sms / nchunk);
  ns = (int)std::min<int64_t>(ns, std::max<int64_t>(1, v / 64));
  ns = (int)std::min<int64_t>(ns, (int64_t)((kNoAllocScratchBytes - mu_bytes) / split_bytes));
  // the array's address belongs to the context's device, which must be current
  // (launches on the context's stream need it too)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != c->device) {
    set_error("srm_transform_noalloc: the context lives on device " + std::to_string(c->device) + " but device " +
              std::to_string(dev) + " is current; make the context's device current first");
    return SRM_ERR_ARG;
  }
  void* base = nullptr;
  srm_status st = scratch_address(c->device, &base);
  if (st != SRM_OK) return st;
  // the transform reads the current A_i and M_i
  st = flush_pending(c);
  if (st != SRM_OK) return st;
  float* mu = static_cast<float*>(base);
  float* part = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + mu_bytes);
  const unsigned g = (unsigned)((v + 7) / 8);
  if (c->in_dtype == SRM_BF16)
    rowmean_kernel<__nv_bfloat16><<<g, 256, 0, c->stream>>>(static_cast<const __nv_bfloat16*>(X_new), v, T_new, mu);
  else
    rowmean_kernel<float><<<g, 256, 0, c->stream>>>(static_cast<const float*>(X_new), v, T_new, mu);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "srm_transform_noalloc: row means");
  const dim3 grid(nchunk, ns);
  if (c->batched)
    e = launch_p_centred_x(c->in_dtype, c->kld, grid, c->stream,
                           static_cast<const __nv_bfloat16*>(c->A) + c->off[subject] * c->kld, X_new, mu, v, T_new,
                           ns, part);
  else
    e = launch_p_centred_x(c->in_dtype, c->kld, grid, c->stream,
                           static_cast<const float*>(c->A) + c->off[subject] * c->kld, X_new, mu, v, T_new, ns, part);
  if (e != cudaSuccess) return cuda_fail(e, "srm_transform_noalloc: projection");
  e = launch_transform_finish(c, subject, part, ns, T_new, S_out);
  if (e != cudaSuccess) return cuda_fail(e, "srm_transform_noalloc: finish");
  return SRM_OK;
}
