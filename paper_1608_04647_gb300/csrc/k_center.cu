// Centring pre-pass, parameter initialisation and W_i materialisation.
//
// Centring (Algorithm 1, initialisation; Sec. II-B): mu_i = (1/T) sum_t x_it
// and x^_it = x_it - mu_i, written once into the resident copy in the store
// dtype (BF16 values are rounded after centring, so the per-voxel mean does
// not eat the BF16 mantissa), with ||X^_i||_F^2 of the stored values
// accumulated per row for the rho update (eq:srm_rho_update) and the
// log-likelihood.
#include "srm_internal.cuh"

namespace srm {

namespace {

__device__ __forceinline__ float ld_as_float(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_as_float(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}
__device__ __forceinline__ void st_from_float(float* p, int64_t i, float x) { p[i] = x; }
__device__ __forceinline__ void st_from_float(__nv_bfloat16* p, int64_t i, float x) {
  p[i] = __float2bfloat16_rn(x);
}
__device__ __forceinline__ float rt(float x, const float*) { return x; }
__device__ __forceinline__ float rt(float x, const __nv_bfloat16*) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// One warp per row.  Rows in [v, vpad) are padding and are zeroed; columns in
// [T, ldo) are zeroed.  Sums use per-lane compensated (Kahan) FP32 followed by
// an FP64 warp reduction.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) center_kernel(const Tin* __restrict__ X, int64_t ldx, int64_t v,
                                                     int64_t vpad, int T, int64_t ldo,
                                                     Tout* __restrict__ out, double* __restrict__ rowsq) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  if (r >= vpad) return;
  Tout* orow = out + r * ldo;
  if (r >= v) {
    for (int64_t t = lane; t < ldo; t += 32) st_from_float(orow, t, 0.f);
    if (lane == 0 && rowsq) rowsq[r] = 0.0;
    return;
  }
  const Tin* xr = X + r * ldx;
  float s = 0.f, cmp = 0.f;
  for (int t = lane; t < T; t += 32) {
    float y = ld_as_float(xr, t) - cmp;
    float tt = s + y;
    cmp = (tt - s) - y;
    s = tt;
  }
  double ds = (double)s - (double)cmp;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, o);
  const float mu = (float)(ds / (double)T);
  float q = 0.f, qc = 0.f;
  for (int64_t t = lane; t < ldo; t += 32) {
    if (t < T) {
      float xh = ld_as_float(xr, t) - mu;
      float st = rt(xh, orow);
      st_from_float(orow, t, xh);
      float y = st * st - qc;
      float tt = q + y;
      qc = (tt - q) - y;
      q = tt;
    } else {
      st_from_float(orow, t, 0.f);
    }
  }
  double dq = (double)q - (double)qc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dq += __shfl_xor_sync(0xffffffffu, dq, o);
  if (lane == 0 && rowsq) rowsq[r] = dq;
}

// Fixed-order tree sum of a subject's per-row squares -> ||X^_i||_F^2.
__global__ void __launch_bounds__(256) sqnorm_kernel(const double* __restrict__ rowsq,
                                                     const int64_t* __restrict__ off,
                                                     const int64_t* __restrict__ v, double* __restrict__ out) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  const double* p = rowsq + off[i];
  const int64_t n = v[i];
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += 256) acc += p[r];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = red[0];
}

template <typename TA>
__global__ void load_w0_kernel(const float* __restrict__ W0, int64_t v, int64_t vpad, int k, int kld,
                               TA* __restrict__ A) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vpad * kld) return;
  const int64_t r = idx / kld;
  const int f = (int)(idx % kld);
  float x = (r < v && f < k) ? W0[r * k + f] : 0.f;
  if constexpr (sizeof(TA) == 2) A[idx] = __float2bfloat16_rn(x);
  else A[idx] = x;
}

// W_i = A_i M_i (eq:srm_mapping_update with M_i = (A_i^T A_i)^-1/2), one thread
// per output element, M_i staged in shared memory.
template <typename TA>
__global__ void __launch_bounds__(256) get_w_kernel(const TA* __restrict__ A, int64_t v, int k, int kld,
                                                    const float* __restrict__ M, float* __restrict__ W) {
  extern __shared__ float Ms[];
  for (int e = threadIdx.x; e < k * kld; e += blockDim.x) Ms[e] = M[(e / kld) * kld + (e % kld)];
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= v * k) return;
  const int64_t r = idx / k;
  const int f = (int)(idx % k);
  const TA* ar = A + r * kld;
  float acc = 0.f;
  for (int m = 0; m < k; ++m) {
    float a;
    if constexpr (sizeof(TA) == 2) a = __bfloat162float(ar[m]);
    else a = ar[m];
    acc = fmaf(a, Ms[m * kld + f], acc);
  }
  W[idx] = acc;
}

// rho_i^2 = 1, Sigma_s = I (Algorithm 1 initialisation), M_i = I (the
// starting W_i are orthonormal), identity eigen-bases, and the
// eigen-decomposition of Sigma_s = I kept for the first Phi.
__global__ void init_params_kernel(int N, int k, int kld, double* rho2, double* Sigma, double* M64,
                                   float* M32, float* Uwarm, double* G64, double* Xr64, int* iter, int* status) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t kk = (int64_t)k * k;
  for (int64_t e = tid; e < N; e += stride) rho2[e] = 1.0;
  for (int64_t e = tid; e < kk; e += stride) {
    const double d = (e / k == e % k) ? 1.0 : 0.0;
    Sigma[e] = d;
    G64[N * kk + e] = d;
    Xr64[N * kk + e] = d;
  }
  for (int64_t e = tid; e < (int64_t)(N + 1) * kk; e += stride) {
    const int64_t w = e % kk;
    const double d = (w / k == w % k) ? 1.0 : 0.0;
    if (e < (int64_t)N * kk) M64[e] = d;
    Uwarm[e] = (float)d;
  }
  for (int64_t e = tid; e < (int64_t)N * kld * kld; e += stride) {
    const int64_t w = e % ((int64_t)kld * kld);
    const int a = (int)(w / kld), b = (int)(w % kld);
    M32[e] = (a == b && a < k) ? 1.f : 0.f;
  }
  if (tid == 0) {
    *iter = 0;
    *status = 0;
  }
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_center(Ctx* c, int i, const void* X, srm_dtype in_dtype, int64_t ldx) {
  const int64_t v = c->v[i], vp = c->vpad[i];
  const unsigned g = nblocks(vp, 8);
  double* rq = c->rowsq + c->off[i];
  if (c->store == SRM_BF16) {
    auto* out = static_cast<__nv_bfloat16*>(c->Xh) + c->off[i] * c->ldT;
    if (in_dtype == SRM_F32)
      center_kernel<float, __nv_bfloat16><<<g, 256, 0, c->stream>>>(static_cast<const float*>(X), ldx, v, vp, c->T,
                                                                    c->ldT, out, rq);
    else
      center_kernel<__nv_bfloat16, __nv_bfloat16><<<g, 256, 0, c->stream>>>(
          static_cast<const __nv_bfloat16*>(X), ldx, v, vp, c->T, c->ldT, out, rq);
  } else {
    auto* out = static_cast<float*>(c->Xh) + c->off[i] * c->ldT;
    if (in_dtype == SRM_F32)
      center_kernel<float, float><<<g, 256, 0, c->stream>>>(static_cast<const float*>(X), ldx, v, vp, c->T, c->ldT,
                                                            out, rq);
    else
      center_kernel<__nv_bfloat16, float><<<g, 256, 0, c->stream>>>(static_cast<const __nv_bfloat16*>(X), ldx, v,
                                                                     vp, c->T, c->ldT, out, rq);
  }
  return cudaGetLastError();
}

cudaError_t launch_center_generic(const void* X, srm_dtype in_dtype, int64_t rows, int T, int64_t ldx, float* out,
                                  int64_t ldo, double* rowsq, cudaStream_t s) {
  const unsigned g = nblocks(rows, 8);
  if (in_dtype == SRM_F32)
    center_kernel<float, float><<<g, 256, 0, s>>>(static_cast<const float*>(X), ldx, rows, rows, T, ldo, out, rowsq);
  else
    center_kernel<__nv_bfloat16, float><<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(X), ldx, rows, rows, T,
                                                          ldo, out, rowsq);
  return cudaGetLastError();
}

cudaError_t launch_sqnorm_reduce(Ctx* c) {
  sqnorm_kernel<<<c->N, 256, 0, c->stream>>>(c->rowsq, c->d_off, c->d_v, c->sqnorm);
  return cudaGetLastError();
}

cudaError_t launch_load_w0(Ctx* c, int i, const float* W0) {
  const int64_t n = c->vpad[i] * c->kld;
  if (c->batched) {
    auto* A = static_cast<__nv_bfloat16*>(c->A) + c->off[i] * c->kld;
    load_w0_kernel<__nv_bfloat16><<<nblocks(n, 256), 256, 0, c->stream>>>(W0, c->v[i], c->vpad[i], c->k, c->kld, A);
  } else {
    auto* A = static_cast<float*>(c->A) + c->off[i] * c->kld;
    load_w0_kernel<float><<<nblocks(n, 256), 256, 0, c->stream>>>(W0, c->v[i], c->vpad[i], c->k, c->kld, A);
  }
  return cudaGetLastError();
}

void prepare_center_kernels(int max_smem) {
  (void)max_smem;
  const int need = (int)(sizeof(float) * KMAX * KMAX);
  cudaFuncSetAttribute(get_w_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
  cudaFuncSetAttribute(get_w_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
}

cudaError_t launch_get_w(Ctx* c, int i, float* W) {
  const int64_t n = c->v[i] * c->k;
  const size_t sm = sizeof(float) * c->k * c->kld;
  const float* M = c->M32 + (int64_t)i * c->kld * c->kld;
  if (c->batched) {
    auto* A = static_cast<const __nv_bfloat16*>(c->A) + c->off[i] * c->kld;
    get_w_kernel<__nv_bfloat16><<<nblocks(n, 256), 256, sm, c->stream>>>(A, c->v[i], c->k, c->kld, M, W);
  } else {
    auto* A = static_cast<const float*>(c->A) + c->off[i] * c->kld;
    get_w_kernel<float><<<nblocks(n, 256), 256, sm, c->stream>>>(A, c->v[i], c->k, c->kld, M, W);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_params(Ctx* c) {
  init_params_kernel<<<64, 256, 0, c->stream>>>(c->N, c->k, c->kld, c->rho2, c->Sigma, c->M64, c->M32, c->Uwarm,
                                                c->G64, c->Xr64, c->iter, c->status);
  return cudaGetLastError();
}

}  // namespace srm
