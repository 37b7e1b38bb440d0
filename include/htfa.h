/*
 * htfa.h -- C ABI of libsrm's HTFA local-step evaluations.
 *
 * Method: Anderson et al., "Enabling Factor Analysis on Thousand-Subject
 * Neuroimaging Datasets" (arXiv 1608.04647), Sec. III (HTFA) and the native
 * extension modules listed in Sec. IV-A.
 *
 *   model (eq:htfa_factor_analysis):  X_i = W_i F_i + E_i,
 *       X_i (T x V, one fMRI sample per row), W_i (T x K), F_i (K x V).
 *   factor k of subject i (Eq. 14, eq:htfa_factor), at voxel position p:
 *       F_i[k][v] = exp(-||p_v - mu_{i,k}||^2 / lambda_{i,k}).
 *   residual (the Frobenius term of eq:htfa_subject_update_rbfs, evaluated
 *   by the NLLS solver for every trial of centers and widths):
 *       r_i = ||X_i - W_i F_i||_F^2.
 *   z-score (Sec. IV-A, data standardisation): every voxel (column of X_i)
 *       mapped to mean 0 and unit population variance over its T samples.
 *
 * Conventions (shared with srm.h):
 *   - A call works on a batch of n_subj subjects of equal sizes, stored
 *     back to back: X is [n_subj][T][V], W [n_subj][T][K], F [n_subj][K][V]
 *     (row-major, the last index contiguous).
 *   - "_dev" pointers are device pointers on the current device, owned by
 *     the caller.  The calls are asynchronous on `stream` (a cudaStream_t;
 *     NULL is the legacy default stream) and allocate nothing.
 *   - Bad sizes or null pointers return SRM_ERR_ARG before any launch; a
 *     failed launch returns SRM_ERR_CUDA.  srm_last_error() describes both.
 *     Empty batches (n_subj, T or V zero) launch nothing, except that the
 *     residual of an empty X is written as 0.
 */
#ifndef HTFA_H
#define HTFA_H
#include "srm.h"
#ifdef __cplusplus
extern "C" {
#endif

/*
 * srm_htfa_factors -- F_i for every subject of the batch (Eq. 14).
 *
 * Voxel positions lie on a grid (Sec. III-C): axes_dev holds the distinct
 * coordinates along x (nx values), then y (ny), then z (nz), and vox_dev
 * ([n_subj][V][3] int32) gives voxel v's index along each axis, so
 * p_v = (axes[ix], axes[nx + iy], axes[nx + ny + iz]).  mu_dev is
 * [n_subj][K][3] (centers, same units as the axes), lambda_dev [n_subj][K]
 * (widths, > 0), F_dev [n_subj][K][V].
 *
 * Because ||p - mu||^2 is a sum over the axes, each factor is the product of
 * one table entry per axis, exp(-(a - mu_c)^2 / lambda); the tables take
 * O(nx + ny + nz) exponentials per factor (the paper's per-axis cache of
 * squared differences, carried through the exponential) and are built once
 * per call in work_dev.
 *
 * flag_dev (one device int32, may be NULL) is OR-ed on the device with 1
 * when a voxel index lies outside its axis (that voxel's column of F is set
 * to NaN) and with 2 when a width is not a positive finite number (that
 * factor's row is set to NaN).  work_dev is caller-owned scratch for the
 * tables, at least srm_htfa_factors_workspace() bytes, 16-byte aligned.
 * Requires 1 <= K <= 2^20, 1 <= nx, ny, nz <= 4096, n_subj <= 65535,
 * V <= 2^31 - 1.  Two launches: the tables, then F.
 */
SRM_API size_t srm_htfa_factors_workspace(int32_t n_subj, int32_t K, int32_t nx, int32_t ny, int32_t nz);
SRM_API srm_status srm_htfa_factors(int32_t n_subj, int32_t K, int32_t V, const float* axes_dev, int32_t nx,
                                    int32_t ny, int32_t nz, const int32_t* vox_dev, const float* mu_dev,
                                    const float* lambda_dev, float* F_dev, int32_t* flag_dev, void* work_dev,
                                    size_t work_bytes, void* stream);

/*
 * srm_htfa_residual -- out_dev[i] = ||X_i - W_i F_i||_F^2 (FP64 result of
 * FP32 products; the sum over tiles runs in a fixed order, so repeated calls
 * give identical bits).
 *
 * work_dev is caller-owned scratch of at least srm_htfa_residual_workspace()
 * bytes (8-byte aligned).  Requires 1 <= K, n_subj <= 65535, T and V
 * <= 2^31 - 1.  X, W and F are read only.
 */
SRM_API size_t srm_htfa_residual_workspace(int32_t n_subj, int32_t K, int32_t T, int32_t V);
SRM_API srm_status srm_htfa_residual(int32_t n_subj, int32_t K, int32_t T, int32_t V, const float* X_dev,
                                     const float* W_dev, const float* F_dev, double* out_dev, void* work_dev,
                                     size_t work_bytes, void* stream);

/*
 * srm_zscore -- Y_i[t][v] = (X_i[t][v] - m_v) / s_v for each of n_mat
 * matrices [n_mat][T][V], with m_v and s_v the mean and population standard
 * deviation of column v.  A column whose T values are all equal becomes
 * zeros.  Y_dev may equal X_dev (in place); otherwise the two must not
 * overlap.  Requires n_mat <= 65535 and T, V <= 2^31 - 1.
 */
SRM_API srm_status srm_zscore(int32_t n_mat, int32_t T, int32_t V, const float* X_dev, float* Y_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif
