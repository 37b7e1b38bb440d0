// Plain per-subject FP32 form of the two contractions (CUDA cores, no tensor
// cores).  It is the comparison point for the batched BF16 tensor-core form
// and the path that carries the 1e-5 accuracy bar.
//
//  * E-pass (Algorithm 1, E-step reduction; eq:srm_mean_distributed):
//    P_i = B_i^T X^_i (k x T) with B_i = W_i at the first iteration and A_i
//    afterwards (W_i = A_i M_i is never formed; M_i is applied to the small
//    k x T result).  The long v axis is split across blocks; each block keeps
//    its k x 64 tile in registers and writes it to a partial slot that a
//    fixed-order reduction sums (no atomics, bitwise reproducible).
//  * M-pass (eq:srm_mapping_update): A_i = X^_i E[S]^T (v_i x k) with the
//    Gram A_i^T A_i accumulated per block from the tile just produced.
//    E[S]^T chunks are staged in shared memory by bulk asynchronous copies
//    (cp.async.bulk + mbarrier), double buffered.
#include "srm_internal.cuh"

namespace srm {

namespace {

constexpr int P_ROWS = 32;   // rows of X staged per step in the E-pass
constexpr int A_ROWS = 64;   // rows per M-pass tile
constexpr int A_TCH = 32;    // t per M-pass stage

__device__ __forceinline__ float a_load(const float* A, int64_t i) { return A[i]; }
__device__ __forceinline__ float a_load(const __nv_bfloat16* A, int64_t i) { return __bfloat162float(A[i]); }

// part layout: [nsplit][nchunk][TCH][kld]
template <int KQ, typename TA>
__global__ void __launch_bounds__(256) p_simt_kernel(const TA* __restrict__ A, int kld, const float* __restrict__ X,
                                                     int64_t ldx, int64_t rows, int T, int nsplit,
                                                     float* __restrict__ part) {
  constexpr int FJ = KQ / 16;
  __shared__ float As[P_ROWS][KQ];
  __shared__ __align__(16) float Xs[P_ROWS][TCH];
  const int cT = blockIdx.x, s = blockIdx.y, nchunk = gridDim.x;
  const int t0 = cT * TCH;
  const int64_t rb = rows * s / nsplit, re = rows * (s + 1) / nsplit;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float acc[FJ][4];
#pragma unroll
  for (int j = 0; j < FJ; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;

  for (int64_t r0 = rb; r0 < re; r0 += P_ROWS) {
    for (int e = tid; e < P_ROWS * KQ; e += 256) {
      const int rr = e / KQ, f = e % KQ;
      const int64_t r = r0 + rr;
      As[rr][f] = (r < re && f < kld) ? a_load(A, r * kld + f) : 0.f;
    }
    for (int e = tid; e < P_ROWS * TCH; e += 256) {
      const int rr = e / TCH, t = e % TCH;
      const int64_t r = r0 + rr;
      Xs[rr][t] = (r < re && t0 + t < T) ? __ldg(X + r * ldx + t0 + t) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < P_ROWS; ++rr) {
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

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait on an mbarrier phase; returns false (and flags the status word)
// if the phase did not complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  const uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) {
      const unsigned long long now = global_ns();
      if (t0 == 0)
        t0 = now;
      else if (now - t0 > kWaitLimitNs)
        break;
      __nanosleep(64);
    }
  }
  atomicOr(status, ST_TIMEOUT);
  return false;
}

template <int KQ>
__global__ void __launch_bounds__(256) a_simt_kernel(const float* __restrict__ X, int64_t ldx, int64_t vpad, int T,
                                                     const float* __restrict__ ESt, int kld,
                                                     float* __restrict__ A, float* __restrict__ gpart,
                                                     int* status) {
  constexpr int FJ = KQ / 16;
  // dynamic shared memory: Es[2][A_TCH][KQ] | Xs[A_ROWS][A_TCH+1] | Ts[A_ROWS][KQ+1] | bar[2]
  extern __shared__ __align__(128) unsigned char a_smem[];
  auto Es = reinterpret_cast<float (*)[A_TCH][KQ]>(a_smem);
  auto Xs = reinterpret_cast<float (*)[A_TCH + 1]>(a_smem + sizeof(float) * 2 * A_TCH * KQ);
  auto Ts = reinterpret_cast<float (*)[KQ + 1]>(a_smem + sizeof(float) * (2 * A_TCH * KQ + A_ROWS * (A_TCH + 1)));
  auto bar = reinterpret_cast<uint64_t*>(
      a_smem + ((sizeof(float) * (2 * A_TCH * KQ + A_ROWS * (A_TCH + 1) + A_ROWS * (KQ + 1)) + 7) & ~size_t(7)));
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int nch = (T + A_TCH - 1) / A_TCH;
  const uint32_t ebytes = (uint32_t)(A_TCH * KQ * sizeof(float));
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase[2] = {0u, 0u};
  int inflight[2] = {0, 0};  // meaningful in thread 0 only: copies issued and not yet waited for
  bool ok = true;
  float g[FJ][FJ];
#pragma unroll
  for (int a = 0; a < FJ; ++a)
#pragma unroll
    for (int b = 0; b < FJ; ++b) g[a][b] = 0.f;

  const int64_t ntile = vpad / A_ROWS;
  for (int64_t tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
    const int64_t r0 = tile * A_ROWS;
    float acc[4][FJ];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < FJ; ++j) acc[q][j] = 0.f;
    // prefetch chunk 0
    if (tid == 0) {
      inflight[0] = 1;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar[0])), "r"(ebytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(&Es[0][0][0])),
          "l"(ESt), "r"(ebytes), "r"(smem_u32(&bar[0]))
          : "memory");
    }
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      const int tc0 = ch * A_TCH;
      for (int e = tid; e < A_ROWS * A_TCH; e += 256) {
        const int rr = e / A_TCH, t = e % A_TCH;
        Xs[rr][t] = (tc0 + t < T) ? __ldg(X + (r0 + rr) * ldx + tc0 + t) : 0.f;
      }
      const bool got = mbar_wait_bounded(&bar[buf], phase[buf], status);
      phase[buf] ^= 1u;
      if (tid == 0) inflight[buf] = 0;
      ok = __syncthreads_and(got) != 0;
      // issue next chunk into the other buffer (its previous use ended at the
      // __syncthreads that closed the previous iteration)
      if (tid == 0 && ch + 1 < nch && ok) {
        const int nb = buf ^ 1;
        inflight[nb] = 1;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar[nb])), "r"(ebytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(&Es[nb][0][0])),
            "l"(ESt + (int64_t)(tc0 + A_TCH) * kld), "r"(ebytes), "r"(smem_u32(&bar[nb]))
            : "memory");
      }
      if (ok) {
#pragma unroll 4
        for (int t = 0; t < A_TCH; ++t) {
          float xv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) xv[q] = Xs[ty * 4 + q][t];
#pragma unroll
          for (int j = 0; j < FJ; ++j) {
            const float e = Es[buf][t][tx + 16 * j];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q][j] = fmaf(xv[q], e, acc[q][j]);
          }
        }
      }
      __syncthreads();
    }
    if (!ok) break;
    // write the A tile and stage it for the Gram update
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float* arow = A + (r0 + ty * 4 + q) * kld;
#pragma unroll
      for (int j = 0; j < FJ; ++j) {
        arow[tx + 16 * j] = acc[q][j];
        Ts[ty * 4 + q][tx + 16 * j] = acc[q][j];
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < A_ROWS; ++r) {
      float ra[FJ], rb[FJ];
#pragma unroll
      for (int a = 0; a < FJ; ++a) {
        ra[a] = Ts[r][ty + 16 * a];
        rb[a] = Ts[r][tx + 16 * a];
      }
#pragma unroll
      for (int a = 0; a < FJ; ++a)
#pragma unroll
        for (int b = 0; b < FJ; ++b) g[a][b] = fmaf(ra[a], rb[b], g[a][b]);
    }
    __syncthreads();
  }
  if (!ok) {
    // a wait gave up: give the copies still in flight one more bounded wait
    // so that none lands in shared memory after the block has exited
    if (tid == 0)
      for (int b = 0; b < 2; ++b)
        if (inflight[b]) mbar_wait_bounded(&bar[b], phase[b], status);
    return;
  }
  float* gp = gpart + (int64_t)blockIdx.x * kld * kld;
#pragma unroll
  for (int a = 0; a < FJ; ++a)
#pragma unroll
    for (int b = 0; b < FJ; ++b) gp[(ty + 16 * a) * kld + tx + 16 * b] = g[a][b];
}

constexpr size_t a_simt_smem(int KQ) {
  return ((sizeof(float) * (2 * A_TCH * KQ + A_ROWS * (A_TCH + 1) + A_ROWS * (KQ + 1)) + 7) & ~size_t(7)) +
         2 * sizeof(uint64_t);
}

template <typename TA>
cudaError_t p_dispatch(int kq, dim3 grid, cudaStream_t s, const TA* A, int kld, const float* X, int64_t ldx,
                       int64_t rows, int T, int nsplit, float* part) {
  switch (kq) {
#define P_CASE(KQ) \
  case KQ: p_simt_kernel<KQ, TA><<<grid, 256, 0, s>>>(A, kld, X, ldx, rows, T, nsplit, part); break;
    P_CASE(16) P_CASE(32) P_CASE(48) P_CASE(64) P_CASE(80) P_CASE(96) P_CASE(112) P_CASE(128)
#undef P_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_p_simt_generic(const void* A, bool a_bf16, int kld, int kq, const float* X, int64_t ldx,
                                  int64_t rows, int T, int nsplit, float* part, cudaStream_t s) {
  const int nchunk = (T + TCH - 1) / TCH;
  dim3 grid(nchunk, nsplit);
  if (a_bf16)
    return p_dispatch<__nv_bfloat16>(kq, grid, s, static_cast<const __nv_bfloat16*>(A), kld, X, ldx, rows, T, nsplit,
                                     part);
  return p_dispatch<float>(kq, grid, s, static_cast<const float*>(A), kld, X, ldx, rows, T, nsplit, part);
}

cudaError_t launch_p_simt(Ctx* c, int i) {
  const float* X = static_cast<const float*>(c->Xh) + c->off[i] * c->ldT;
  const float* A = static_cast<const float*>(c->A) + c->off[i] * c->kld;
  return launch_p_simt_generic(A, false, c->kld, c->kld, X, c->ldT, c->vpad[i], c->T, c->p_nsplit[i],
                               c->Ppart + c->p_slot_base[i], c->stream);
}

void prepare_simt_kernels(int max_smem) {
  (void)max_smem;
#define A_ATTR(KQ) \
  cudaFuncSetAttribute(a_simt_kernel<KQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a_simt_smem(KQ));
  A_ATTR(16) A_ATTR(32) A_ATTR(48) A_ATTR(64) A_ATTR(80) A_ATTR(96) A_ATTR(112) A_ATTR(128)
#undef A_ATTR
}

cudaError_t launch_a_simt(Ctx* c, int i) {
  const float* X = static_cast<const float*>(c->Xh) + c->off[i] * c->ldT;
  float* A = static_cast<float*>(c->A) + c->off[i] * c->kld;
  float* gp = c->Gpart + (int64_t)c->g_slot_base[i] * c->kld * c->kld;
  const int nb = c->a_nblk[i];
  switch (c->kld) {
#define A_CASE(KQ)                                                                                           \
  case KQ: {                                                                                                 \
    const size_t sm = a_simt_smem(KQ);                                                                       \
    a_simt_kernel<KQ><<<nb, 256, sm, c->stream>>>(X, c->ldT, c->vpad[i], c->T, c->ESt, c->kld, A, gp,       \
                                                  c->status);                                                \
    break;                                                                                                   \
  }
    A_CASE(16) A_CASE(32) A_CASE(48) A_CASE(64) A_CASE(80) A_CASE(96) A_CASE(112) A_CASE(128)
#undef A_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace srm
