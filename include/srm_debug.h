/*
 * srm_debug.h -- self-test entry point of libsrm's tensor-core building
 * blocks (not part of the EM method; the paper has no counterpart).
 *
 * srm_debug_mma computes, on one CTA of the current device,
 *   D (128 x N, FP32, row-major) = A * B^T
 * with BF16 operands loaded by TMA into 128-byte-swizzled shared memory and
 * multiplied by tcgen05.mma with the FP32 accumulator in tensor memory.
 *   mn_major == 0: A is 128 x K and B is N x K (K contiguous, "K-major"),
 *                  the layout of the M-pass operands X^_i and E[S].
 *   mn_major != 0: A is K x 128 and B is K x N (M / N contiguous, "MN-major"),
 *                  the layout of the E-pass operands X^_i and A_i.
 *   N in {64, 128}; K in {64, 128, 192, 256}.  A, B, D are device pointers
 *   owned by the caller (A and B 16-byte aligned).  Synchronous; returns
 *   SRM_ERR_ARG on bad sizes or pointers, SRM_ERR_CUDA on a CUDA error.
 */
#ifndef SRM_DEBUG_H
#define SRM_DEBUG_H
#include "srm.h"
#ifdef __cplusplus
extern "C" {
#endif
SRM_API srm_status srm_debug_mma(int32_t mn_major, const void* A, const void* B, float* D, int32_t N, int32_t K);

/*
 * srm_debug_eig_sweeps -- diagnostics of the last M-step, one int per
 * symmetric matrix.  Entries 0..N-1 (the subjects' A_i^T A_i): the number of
 * Newton-Schulz steps of the polar factor, or 256 + the number of Jacobi
 * sweeps when that result failed its accuracy certificate and the
 * eigen-decomposition path took over.  Entry N (Sigma_s): Jacobi sweeps for
 * k <= 64; for k > 64 Sigma_s is not decomposed (Phi comes from a Cholesky
 * factorisation) and entry N is not defined.  Writes min(n, N + 1) ints to
 * the host array out.  Synchronises.
 */
SRM_API srm_status srm_debug_eig_sweeps(srm_ctx* ctx, int32_t* out, int32_t n);

/*
 * srm_debug_force_eig_polar -- with on != 0, every later M-step of ctx fails
 * each subject's Newton-Schulz certificate on purpose, so that all polar
 * factors (eq:srm_mapping_update) and rho_i^2 come from the
 * eigen-decomposition path (Jacobi + FP64 refinement) that otherwise serves
 * only the subjects whose certificate fails; on == 0 restores the default.
 * For tests of that path.  Flushes pending work; returns SRM_ERR_ARG for a
 * bad context.
 */
SRM_API srm_status srm_debug_force_eig_polar(srm_ctx* ctx, int32_t on);

/*
 * srm_debug_wait -- the bounded mbarrier wait of the tensor-core kernels,
 * exercised on one CTA of the current device without any fault.  Two warps
 * each wait on an mbarrier.  With arrive != 0 a thread arrives on both: the
 * call returns SRM_OK.  With arrive == 0 nothing arrives.  The first waiter
 * gives up after the library's limit of one second, raises the block's
 * abort flag and the device status bit of a
 * timed-out wait.  The other waiter stops on the abort flag.  The call then
 * returns SRM_ERR_NUMERIC and srm_last_error() says which waits succeeded.
 * Synchronous; the device stays usable afterwards.
 */
SRM_API srm_status srm_debug_wait(int32_t arrive);
#ifdef __cplusplus
}
#endif
#endif
