// Internal declarations shared by the translation units of libsrm.
// Method: probabilistic SRM EM iteration, Sec. II and Algorithm 1 of
// Anderson et al. (arXiv 1608.04647).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include "../../include/srm.h"

namespace srm {

constexpr int KMAX = 128;         // largest k supported
constexpr int ROW_PAD = 128;      // each subject's rows are padded to a multiple of this
constexpr int TCH = 64;           // t-chunk width of the partial-sum slots and reductions

// Device-side status bits (ctx->status word).
enum : int {
  ST_NONFINITE = 1,     // a NaN / Inf reached a k x k step
  ST_NOT_PD = 2,        // Cholesky met a non-positive pivot
  ST_EIG_NOCONV = 4,    // Jacobi sweep cap reached
  ST_RANK = 8,          // A_i^T A_i numerically singular (polar factor undefined)
  ST_TIMEOUT = 16,      // a bounded wait inside a tensor-core kernel gave up
  ST_BOUNDS = 32,       // a kernel's own index check refused an access
};

// Bounded waits give up after this much elapsed time (the global timer).
// Each mbarrier.try_wait may itself suspend the thread for a while, so a
// limit on the number of polls alone would be far longer than it looks (2^24
// polls measured about 63 s); the poll counts that remain are backstops.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s
#ifdef __CUDACC__
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#endif

// Kernel kinds for SRM_PROFILE timing.
enum KernelKind : int {
  KK_CENTER = 0,
  KK_P_SIMT,
  KK_P_TC,
  KK_P_REDUCE,
  KK_SIGMA,
  KK_PHI,
  KK_A_SIMT,
  KK_A_TC,
  KK_EIG,
  KK_REFINE,
  KK_RHO,
  KK_MTAIL,
  KK_POLAR,
  KK_FPASS,
  KK_P_SUM,
  KK_COUNT
};
extern const char* const kKernelNames[KK_COUNT];

// One source of a (subject, t-chunk) partial: float offset of the [TCH][kld]
// block inside the partial buffer.
struct ChunkSrc {
  int64_t off;
};

struct Ctx {
  // ---- configuration
  int N = 0, T = 0, k = 0;
  int kld = 0;        // leading dimension of A rows / partial rows (k padded)
  int ldT = 0;        // row stride of resident X^ (T padded to 8)
  int nchunk = 0;     // ceil(T / TCH)
  int zgroups = 0;    // subject groups of the E-step reduction
  srm_dtype in_dtype = SRM_F32, store = SRM_F32;
  uint32_t flags = 0;
  bool batched = false;
  int max_iter = 1024;
  int device = 0, num_sms = 0;
  std::vector<int64_t> v, vpad, off;  // per subject: rows, padded rows, row offset
  int64_t Vtot = 0, Vpad_tot = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;          // second stream for the M-step tail
  cudaStream_t side2 = nullptr;         // third stream (Sigma_s eigen-decomposition)
  cudaEvent_t ev_join2 = nullptr, ev_sig = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_polar = nullptr;  // the polar factors are done (M_i, rho_i^2), Phi may still run
  bool side_pending = false;            // an M-step's tail has not run yet
  bool sigma_pending = false;           // an E-step's Sigma_s^new / log-likelihood have not been formed yet

  // ---- resident data
  void* Xh = nullptr;        // [Vpad_tot][ldT] store dtype, demeaned, zero padded
  void* A = nullptr;         // [Vpad_tot][kld]: FP32 (plain) or BF16 (batched)
  double* sqnorm = nullptr;  // [N] ||X^_i||_F^2
  double* rowsq = nullptr;   // [Vpad_tot] per-row sum of squares (init scratch)
  int64_t* d_off = nullptr;  // [N+1] row offsets
  int64_t* d_v = nullptr;    // [N]

  // ---- EM parameters (device)
  double* rho2 = nullptr;       // [N]
  double* Sigma = nullptr;      // [k][k]
  double* SigmaNext = nullptr;  // [k][k]
  double* L = nullptr;          // [k][k] Cholesky factor of I + rho0 Sigma
  double* Phi = nullptr;        // [k][k]
  float* Phi32 = nullptr;       // [k][k] FP32 copy (the E[S] product)
  double* scal = nullptr;       // [16] scalars of the current E-step (see k_small.cu)
  double* M64 = nullptr;        // [N][k][k] (A_i^T A_i)^-1/2
  float* M32 = nullptr;         // [N][kld][kld] FP32 copy used by the reduction
  // entries 0..N-1: subjects' Gram matrices; entry N: Sigma_s
  float* Uwarm = nullptr;       // [N+1][k][k] last eigenvectors (Jacobi warm start)
  double* G64 = nullptr;        // [N+1][k][k] Gram / Sigma_s^new, then U^T G U; entry N kept for Phi
  double* U64 = nullptr;        // [N+1][k][k] FP32 Jacobi eigenvectors (promoted)
  double* H64 = nullptr;        // [N+1][k][k] scratch
  double* Xr64 = nullptr;       // [N+1][k][k] re-orthonormalised eigenvectors; entry N kept for Phi
  double* eigv = nullptr;       // [N+1][k] eigenvalues
  int* jac_sweeps = nullptr;    // [N+1] Jacobi sweeps of the last M-step (diagnostics)
  int* ns_fb = nullptr;         // [N] 1 = the subject's Newton-Schulz polar factor failed its certificate
  double* Y = nullptr;          // [k][T] FP64 reduction sum_i rho_i^-2 W_i^T X^_i
  double* ES64 = nullptr;       // [k][T] E[S]
  float* ESt = nullptr;         // [ldT][kld] FP32 E[S]^T (plain-path operand)
  __nv_bfloat16* ESb = nullptr; // [kld][ldT] BF16 E[S] (tensor-core operand)
  double* esPart = nullptr;     // [nes_blk] <y, E[S]> of each es block
  int nes_blk = 0;
  double* ll = nullptr;         // [max_iter]
  int* iter = nullptr;          // device E-step counter (index into ll)
  int* status = nullptr;        // device status word

  // ---- partial sums of the two contractions
  float* Ppart = nullptr;       // E-pass partial blocks [..][TCH][kld]
  int64_t Ppart_elems = 0;
  ChunkSrc* chunk_src = nullptr;  // device table
  int* chunk_src_off = nullptr;   // [N * nchunk + 1]
  float2* Ypart = nullptr;      // [zgroups][k][T] sum of rho_i^-2 M_i P_i over a group of subjects (hi, lo)
  float* sPart = nullptr;       // [nes_blk][k*k] E[S] E[S]^T of each es block
  float* Gpart = nullptr;       // M-pass Gram partials [..][kld][kld]
  int64_t Gpart_elems = 0;
  int* gslot_off = nullptr;     // [N+1] Gram slot ranges per subject
  int n_gslots = 0;

  // plain-path launch geometry (per subject)
  std::vector<int> p_nsplit;        // E-pass v-splits per subject
  std::vector<int64_t> p_slot_base; // float offset of subject's first partial block
  std::vector<int> a_nblk;          // M-pass blocks per subject
  std::vector<int> g_slot_base;     // first Gram slot per subject

  // tensor-core path state (k_tc.cu)
  void* tc = nullptr;
  // single-pass form (k_fused.cu): its state, its P partials and their table
  void* fs = nullptr;
  bool fused = false;
  bool p_from_f = false;      // the current P partials come from the single pass
  bool sig_eig_done = false;  // Sigma_s^new and its eigen-decomposition already ran beside that pass
  bool force_eig_polar = false;  // every polar factor through the eigen-decomposition path
  int ns_cl_c = 0;  // CTAs per subject of the clustered polar factor (0: not chosen yet)
  float* f_ppart = nullptr;
  ChunkSrc* f_chunk_src = nullptr;
  int* f_chunk_src_off = nullptr;
  // its partials summed per (subject, chunk) and the one-source table over them
  float* psum = nullptr;
  ChunkSrc* psum_src = nullptr;
  int* psum_src_off = nullptr;

  // ---- sharded E-step (srm_estep_partial / srm_estep_finish)
  double* shard_y = nullptr;     // caller's k x T buffer while a partial E-step is launched
  double* shard_sums = nullptr;  // caller's 4 sums while a partial E-step is launched
  bool shard_partial = false;    // a partial E-step awaits srm_estep_finish

  // ---- host bookkeeping
  int n_ll = 0;            // E-steps launched
  bool have_estep = false; // an E-step result is pending for an M-step
  bool have_es = false;    // E[S] exists
  int64_t iters_done = 0;

  // graph
  cudaGraphExec_t graph_exec = nullptr;

  // profiling
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  struct PendingTiming { int kind; int ev0, ev1; };
  std::vector<PendingTiming> pending;
  int ev_next = 0;
  int64_t prof_launches[KK_COUNT] = {0};
  double prof_ms[KK_COUNT] = {0};

  // transform scratch
  float* tr_buf = nullptr;
  int64_t tr_elems = 0;
  float* tr_part = nullptr;
  int64_t tr_part_elems = 0;
  float* map_buf = nullptr;       // srm_map scratch (S and Z)
  int64_t map_elems = 0;
};

// runs a deferred M-step tail (api.cu)
srm_status flush_pending(Ctx* c);
// n_iter EM iterations through the graph path when enabled (api.cu)
srm_status run_iterations(Ctx* c, int n_iter);
// synchronises the stream and returns (and clears) the device status (api.cu)
srm_status device_status(Ctx* c);
// destroys the instantiated iteration graph, if any (api.cu)
void drop_graph(Ctx* c);

// error helpers (api.cu)
void set_error(const std::string& msg);
srm_status cuda_fail(cudaError_t e, const char* what);

// profiling bracket (api.cu)
void prof_begin(Ctx* c, int kind, int* ev0);
void prof_end(Ctx* c, int kind, int ev0);

// ---- launchers (return cudaError_t of the launch)
// k_center.cu
cudaError_t launch_center(Ctx* c, int subject, const void* X, srm_dtype in_dtype, int64_t ldx);
cudaError_t launch_center_generic(const void* X, srm_dtype in_dtype, int64_t rows, int T, int64_t ldx,
                                  float* out, int64_t ldo, double* rowsq, cudaStream_t s);
cudaError_t launch_sqnorm_reduce(Ctx* c);
cudaError_t launch_load_w0(Ctx* c, int subject, const float* W0);
cudaError_t launch_get_w(Ctx* c, int subject, float* W);
// k_htfa_tc.cu: the HTFA residual on the tensor cores (K <= 128)
bool htfa_tc_supported(int K);
int64_t htfa_tc_tiles(int T, int V);
size_t htfa_tc_smem_bytes();
cudaError_t launch_htfa_residual_tc(int n_subj, int K, int T, int V, const float* X, const float* W, const float* F,
                                    double* part, int* status, cudaStream_t s);
// k_init.cu: Algorithm 1's random orthogonal W^0 drawn in the library (seeded Haar)
size_t haar_workspace_bytes(const Ctx* c);
cudaError_t launch_haar_w0(Ctx* c, int subject, uint64_t seed, void* work);
cudaError_t launch_init_params(Ctx* c);

// k_simt.cu (plain per-subject FP32 form)
cudaError_t launch_p_simt(Ctx* c, int subject);
cudaError_t launch_p_simt_generic(const void* A, bool a_bf16, int kld, int kq, const float* X, int64_t ldx,
                                  int64_t rows, int T, int nsplit, float* part, cudaStream_t s);
cudaError_t launch_a_simt(Ctx* c, int subject);

// k_small.cu
int zsum_groups(int N, int nchunk, int num_sms, int kld);
int es_blocks(int T);
cudaError_t launch_p_reduce(Ctx* c);
// the single pass's slot sums (beside the polar factors), then the reduction from them
cudaError_t launch_p_sum(Ctx* c);
cudaError_t launch_p_reduce_from(Ctx* c, bool from_sums);
// its two halves: the subject-group reduction (needs M_i and rho_i^2), then
// E[S] = Phi y (needs Phi) or, for a sharded E-step, this context's share
cudaError_t launch_p_reduce_part(Ctx* c, bool from_sums);
cudaError_t launch_p_reduce_finish(Ctx* c);
cudaError_t launch_sigma(Ctx* c);
cudaError_t launch_phi(Ctx* c);
// Phi and the likelihood's scalars from sums over all shards (sums != nullptr)
cudaError_t launch_phi_from(Ctx* c, const double* sums);
// the rest of a sharded E-step: Phi from the reduced sums, E[S] = Phi y
cudaError_t launch_estep_finish(Ctx* c, const double* y, const double* sums);
cudaError_t launch_eig(Ctx* c);
cudaError_t launch_refine(Ctx* c);
cudaError_t launch_rho(Ctx* c);
bool mtail_supported(const Ctx* c);
cudaError_t launch_mtail(Ctx* c);
cudaError_t launch_mtail_sigma(Ctx* c);
cudaError_t launch_eig_sigma(Ctx* c);
cudaError_t launch_eig_fallback(Ctx* c);
cudaError_t launch_mtail_fallback(Ctx* c);
bool ns_supported(const Ctx* c);
bool sigma_eig_supported(const Ctx* c);
// k_tail.cu: 64 < k <= 128
bool polar_cl_supported(const Ctx* c);
void prepare_tail_kernels();
void choose_polar_cl(Ctx* c);
cudaError_t launch_polar_cl(Ctx* c, double cert, int comp);
cudaError_t launch_phi_chol(Ctx* c, const double* sums);
cudaError_t launch_polar(Ctx* c);
cudaError_t launch_transform_finish(Ctx* c, int subject, const float* part, int nsplit, int T_new, float* S_out);

// one-time kernel attributes (dynamic shared memory limits); called by srm_init
void prepare_small_kernels(int max_smem);
void prepare_center_kernels(int max_smem);
void prepare_simt_kernels(int max_smem);

// k_tc.cu (grouped persistent tensor-core form)
srm_status tc_setup(Ctx* c);
void tc_destroy(Ctx* c);
int tc_default_e_reserve(const Ctx* c);
int tc_e_reserve(const Ctx* c);
srm_status tc_set_e_reserve(Ctx* c, int reserve);  // rebuilds the E-pass schedule
void tc_get_m_plan(const Ctx* c, int* gram_bufs, int* resident_es, int* stages, int* prefetch, int* boxes);
srm_status tc_set_m_plan(Ctx* c, int gram_bufs, int resident_es, int stages, int prefetch, int boxes);
// every M-pass plan that fits in shared memory: {gram_bufs, resident_es, stages, prefetch, boxes per stage}
void tc_m_candidates(const Ctx* c, std::vector<std::array<int, 5>>& out);
cudaError_t launch_p_tc(Ctx* c);
cudaError_t launch_a_tc(Ctx* c);

// k_fused.cu (single pass over X^ per iteration)
bool fused_supported(const Ctx* c);
srm_status fused_setup(Ctx* c);
void fused_destroy(Ctx* c);
void fused_select(Ctx* c, bool on);  // points the context at the single-pass (on) or two-pass Gram slots
int fused_get_pf(const Ctx* c);
void fused_set_pf(Ctx* c, int pf);
int fused_get_hints(const Ctx* c);     // L2 eviction hints of the single pass (bits, 0..7)
void fused_set_hints(Ctx* c, int hints);
int fused_get_first_stages(const Ctx* c);  // stages of the single pass's first-read ring (1..3 of 4)
void fused_set_first_stages(Ctx* c, int s_h);
int fused_get_lead(const Ctx* c);          // tiles the first read may lead phase 2 (0: no limit)
void fused_set_lead(Ctx* c, int lead);
int fused_get_slots(const Ctx* c);         // 0: four 32 KB stages; 8 or 9: 16 KB slots
void fused_set_slots(Ctx* c, int slots);
bool fused_fine_supported(const Ctx* c);   // the 16 KB-slot form (one CTA per tile: T <= 512)
int fused_get_reserve(const Ctx* c);       // SMs the single pass leaves to the Sigma_s chain beside it
srm_status fused_set_reserve(Ctx* c, int reserve);  // rebuilds the pass's schedule
cudaError_t launch_fpass(Ctx* c);

}  // namespace srm

// The opaque handle of the C ABI is the context itself.
struct srm_ctx : public srm::Ctx {};
