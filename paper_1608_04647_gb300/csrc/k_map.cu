// srm_map: new data of subject i mapped into subject j's voxel space through
// the shared space, Y = W_j W_i^T (x - mean_t x) (Sec. II-A: the orthogonal
// mappings make this a projection to the feature space followed by the
// other subject's mapping).  With W = A M (A = X^ E[S]^T from the last
// M-step, M = (A^T A)^-1/2):
//   S = W_i^T (x - mean)      (srm_transform)
//   Z = M_j S                 (k x T_new)
//   Y = A_j Z                 (v_j x T_new, the bytes that matter)
#include <algorithm>
#include <string>

#include "srm_internal.cuh"

namespace srm {

namespace {

// Z[f][t] = sum_m M[f][m] S[m][t]: one thread per column t.
__global__ void __launch_bounds__(256) mz_kernel(int k, int kld, int T, const float* __restrict__ M,
                                                 const float* __restrict__ S, float* __restrict__ Z) {
  extern __shared__ float mz_smem[];
  float* Ms = mz_smem;  // [k][k]
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Ms[e] = M[(e / k) * kld + e % k];
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  float s[KMAX];
  for (int m = 0; m < k; ++m) s[m] = S[(int64_t)m * T + t];
  for (int f = 0; f < k; ++f) {
    float z = 0.f;
    for (int m = 0; m < k; ++m) z = fmaf(Ms[f * k + m], s[m], z);
    Z[(int64_t)f * T + t] = z;
  }
}

__device__ __forceinline__ float ld_a(const float* A, int64_t i) { return A[i]; }
__device__ __forceinline__ float ld_a(const __nv_bfloat16* A, int64_t i) { return __bfloat162float(A[i]); }

// Y[r][t] = sum_f A[r][f] Z[f][t]: a block owns 32 rows x 64 columns, a
// thread a 2 x 4 tile (rows ty, ty + 16; columns 4 tx .. 4 tx + 3).
template <typename TA>
__global__ void __launch_bounds__(256) map_out_kernel(int k, int kld, int64_t rows, int T, const TA* __restrict__ A,
                                                      const float* __restrict__ Z, float* __restrict__ Y) {
  extern __shared__ float mo_smem[];
  float* Zs = mo_smem;               // [k][64]
  float* As = Zs + (size_t)k * 64;   // [32][k + 1]
  const int t0 = blockIdx.x * 64;
  const int64_t r0 = (int64_t)blockIdx.y * 32;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < k * 64; e += 256) {
    const int f = e >> 6, t = e & 63;
    Zs[e] = (t0 + t < T) ? Z[(int64_t)f * T + t0 + t] : 0.f;
  }
  for (int e = tid; e < 32 * k; e += 256) {
    const int rr = e / k, f = e - rr * k;
    As[rr * (k + 1) + f] = (r0 + rr < rows) ? ld_a(A, (r0 + rr) * kld + f) : 0.f;
  }
  __syncthreads();
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  for (int f = 0; f < k; ++f) {
    const float4 z = *reinterpret_cast<const float4*>(Zs + f * 64 + 4 * tx);
    const float a0 = As[ty * (k + 1) + f], a1 = As[(ty + 16) * (k + 1) + f];
    acc[0][0] = fmaf(a0, z.x, acc[0][0]);
    acc[0][1] = fmaf(a0, z.y, acc[0][1]);
    acc[0][2] = fmaf(a0, z.z, acc[0][2]);
    acc[0][3] = fmaf(a0, z.w, acc[0][3]);
    acc[1][0] = fmaf(a1, z.x, acc[1][0]);
    acc[1][1] = fmaf(a1, z.y, acc[1][1]);
    acc[1][2] = fmaf(a1, z.z, acc[1][2]);
    acc[1][3] = fmaf(a1, z.w, acc[1][3]);
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t r = r0 + ty + 16 * h;
    if (r >= rows) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = t0 + 4 * tx + q;
      if (t < T) Y[r * T + t] = acc[h][q];
    }
  }
}

}  // namespace
}  // namespace srm

using namespace srm;

extern "C" srm_status srm_map(srm_ctx* c, int32_t from, int32_t to, const void* X_new, int32_t T_new, float* Y_out) {
  if (!c) {
    set_error("srm_map: null context");
    return SRM_ERR_ARG;
  }
  if (from < 0 || from >= c->N || to < 0 || to >= c->N || !X_new || !Y_out || T_new < 1) {
    set_error("srm_map: bad subject, pointer or T_new");
    return SRM_ERR_ARG;
  }
  // S and Z in one scratch allocation owned by the context
  const int64_t need = (int64_t)2 * c->k * T_new;
  if (need > c->map_elems) {
    if (c->map_buf) cudaFree(c->map_buf);
    c->map_buf = nullptr;
    c->map_elems = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&c->map_buf), sizeof(float) * need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("srm_map: cudaMalloc of " + std::to_string(sizeof(float) * need) + " bytes failed");
      return SRM_ERR_NOMEM;
    }
    c->map_elems = need;
  }
  float* S = c->map_buf;
  float* Z = c->map_buf + (int64_t)c->k * T_new;
  srm_status st = srm_transform(c, from, X_new, T_new, S);
  if (st != SRM_OK) return st;
  const int k = c->k;
  mz_kernel<<<(T_new + 255) / 256, 256, sizeof(float) * k * k, c->stream>>>(
      k, c->kld, T_new, c->M32 + (int64_t)to * c->kld * c->kld, S, Z);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "srm_map: M_j S");
  const int64_t rows = c->v[to];
  const dim3 grid((T_new + 63) / 64, (unsigned)((rows + 31) / 32));
  const size_t sm = sizeof(float) * ((size_t)k * 64 + 32 * (k + 1));
  if (c->batched)
    map_out_kernel<__nv_bfloat16><<<grid, 256, sm, c->stream>>>(
        k, c->kld, rows, T_new, static_cast<const __nv_bfloat16*>(c->A) + c->off[to] * c->kld, Z, Y_out);
  else
    map_out_kernel<float><<<grid, 256, sm, c->stream>>>(k, c->kld, rows, T_new,
                                                        static_cast<const float*>(c->A) + c->off[to] * c->kld, Z,
                                                        Y_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "srm_map: A_j Z");
  return SRM_OK;
}
