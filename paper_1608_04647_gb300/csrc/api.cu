// C ABI of libsrm: context life cycle, memory layout, and the order of the
// launches of one EM iteration (Algorithm 1 of Anderson et al., arXiv
// 1608.04647: E-step reduction -> E[S] on the "master" -> Sigma_s -> W_i and
// rho_i^2 per subject).  On one GPU the paper's MPI Reduce/Bcast become
// device-resident reductions; nothing leaves HBM inside an iteration.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "srm_internal.cuh"
#include "../../include/srm_debug.h"

namespace srm {

namespace {
thread_local std::string g_err;
}

const char* const kKernelNames[KK_COUNT] = {
    "center", "estep_simt", "estep_tc", "ereduce", "sigma", "phi",
    "mstep_simt", "mstep_tc", "eig", "refine", "rho", "mtail", "polar", "fpass_tc", "psum"};

void set_error(const std::string& msg) { g_err = msg; }

srm_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return SRM_ERR_CUDA;
}

void prof_begin(Ctx* c, int kind, int* ev0) {
  (void)kind;
  if ((int)c->ev_pool.size() <= c->ev_next + 1) {
    for (int q = 0; q < 256; ++q) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->ev_pool.push_back(e);
    }
  }
  *ev0 = c->ev_next++;
  cudaEventRecord(c->ev_pool[*ev0], c->stream);
}

// CUDA kernels behind one launcher call of each kind
static const int kKernelsPerKind[KK_COUNT] = {1, 1, 1, 2, 1, 1, 1, 1, 1, 4, 4, 1, 1, 1, 1};

void prof_end(Ctx* c, int kind, int ev0) {
  const int ev1 = c->ev_next++;
  cudaEventRecord(c->ev_pool[ev1], c->stream);
  c->pending.push_back({kind, ev0, ev1});
}

namespace {

template <typename T>
srm_status dalloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMalloc failed for ") + what + " (" + std::to_string(count * sizeof(T)) + " bytes): " +
              cudaGetErrorString(e));
    return SRM_ERR_NOMEM;
  }
  return SRM_OK;
}

__global__ void cast_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = (float)a[e];
}

#define CK(expr)                                               \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr);        \
  } while (0)

#define TRY(expr)                         \
  do {                                    \
    srm_status _s = (expr);               \
    if (_s != SRM_OK) return _s;          \
  } while (0)

#define LAUNCH(c, kind, expr)                              \
  do {                                                     \
    int _ev0 = -1;                                         \
    if ((c)->profile) prof_begin((c), (kind), &_ev0);      \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr);    \
    if ((c)->profile) prof_end((c), (kind), _ev0);         \
  } while (0)

void free_all(Ctx* c) {
  if (c->fs) fused_destroy(c);
  if (c->tc) tc_destroy(c);
  void* ptrs[] = {c->Xh, c->A, c->sqnorm, c->rowsq, c->d_off, c->d_v, c->rho2, c->Sigma, c->SigmaNext, c->L,
                  c->Phi, c->scal, c->M64, c->M32, c->Uwarm, c->G64, c->U64, c->H64, c->Xr64, c->eigv, c->Y,
                  c->ES64, c->ESt, c->ESb, c->esPart, c->ll, c->iter, c->status, c->Ppart, c->chunk_src, c->jac_sweeps, c->ns_fb,
                  c->chunk_src_off, c->Ypart, c->sPart, c->map_buf, c->Phi32, c->Gpart, c->gslot_off, c->tr_buf, c->tr_part,
                  c->f_ppart, c->f_chunk_src, c->f_chunk_src_off, c->psum, c->psum_src, c->psum_src_off};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->side2) cudaStreamDestroy(c->side2);
  if (c->ev_join2) cudaEventDestroy(c->ev_join2);
  if (c->ev_sig) cudaEventDestroy(c->ev_sig);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_polar) cudaEventDestroy(c->ev_polar);
}

// Plain path: per-subject launch geometry and the partial-slot tables.
srm_status setup_plain(Ctx* c) {
  const int N = c->N;
  c->p_nsplit.resize(N);
  c->p_slot_base.resize(N);
  c->a_nblk.resize(N);
  c->g_slot_base.resize(N);
  int64_t pbase = 0;
  int gbase = 0;
  const int target = 2 * c->num_sms;
  std::vector<int> gslot_off(N + 1);
  std::vector<ChunkSrc> src;
  std::vector<int> src_off(N * c->nchunk + 1);
  for (int i = 0; i < N; ++i) {
    int ns = std::max(1, target / c->nchunk);
    ns = (int)std::min<int64_t>(ns, std::max<int64_t>(1, c->vpad[i] / 64));
    c->p_nsplit[i] = ns;
    c->p_slot_base[i] = pbase;
    pbase += (int64_t)ns * c->nchunk * TCH * c->kld;
    const int64_t ntile = c->vpad[i] / 64;
    c->a_nblk[i] = (int)std::min<int64_t>(ntile, target);
    c->g_slot_base[i] = gbase;
    gslot_off[i] = gbase;
    gbase += c->a_nblk[i];
  }
  gslot_off[N] = gbase;
  for (int i = 0; i < N; ++i)
    for (int ch = 0; ch < c->nchunk; ++ch) {
      src_off[i * c->nchunk + ch] = (int)src.size();
      for (int s = 0; s < c->p_nsplit[i]; ++s)
        src.push_back({c->p_slot_base[i] + ((int64_t)s * c->nchunk + ch) * TCH * c->kld});
    }
  src_off[N * c->nchunk] = (int)src.size();
  c->Ppart_elems = pbase;
  c->n_gslots = gbase;
  c->Gpart_elems = (int64_t)gbase * c->kld * c->kld;
  TRY(dalloc(&c->Ppart, c->Ppart_elems, "E-pass partials"));
  TRY(dalloc(&c->Gpart, c->Gpart_elems, "Gram partials"));
  TRY(dalloc(&c->chunk_src, src.size(), "chunk table"));
  TRY(dalloc(&c->chunk_src_off, src_off.size(), "chunk table offsets"));
  TRY(dalloc(&c->gslot_off, gslot_off.size(), "Gram slot table"));
  CK(cudaMemcpy(c->chunk_src, src.data(), src.size() * sizeof(ChunkSrc), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->chunk_src_off, src_off.data(), src_off.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->gslot_off, gslot_off.data(), gslot_off.size() * sizeof(int), cudaMemcpyHostToDevice));
  return SRM_OK;
}

srm_status check_status(Ctx* c) {
  int st = 0;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    std::string m = "device reported a numerical failure:";
    if (st & ST_NONFINITE) m += " non-finite value;";
    if (st & ST_NOT_PD) m += " I + rho0 Sigma_s not positive definite;";
    if (st & ST_EIG_NOCONV) m += " Jacobi eigen-solver did not converge;";
    if (st & ST_RANK) m += " A_i^T A_i numerically singular (polar factor undefined);";
    if (st & ST_TIMEOUT) m += " a bounded wait in a tensor-core kernel gave up;";
    if (st & ST_BOUNDS) m += " a kernel index check refused an access;";
    set_error(m);
    CK(cudaMemset(c->status, 0, sizeof(int)));
    return SRM_ERR_NUMERIC;
  }
  return SRM_OK;
}

// Launches on `s` until destruction: the launchers use c->stream.
struct OnStream {
  Ctx* c;
  cudaStream_t saved;
  OnStream(Ctx* cc, cudaStream_t s) : c(cc), saved(cc->stream) { c->stream = s; }
  ~OnStream() { c->stream = saved; }
};

// The per-subject tail of an M-step (eigen-decompositions, M_i, rho_i^2,
// the Sigma_s eigen-basis) and the Phi of the next E-step.  None of it is
// needed by the next E-pass (which reads only A_i), so it runs on a second
// stream beside that pass when an iteration follows.
srm_status do_sigma_eig(Ctx* c) {
  if (!sigma_eig_supported(c)) return SRM_OK;  // k > 64: Phi by Cholesky, after the polar factors
  LAUNCH(c, KK_EIG, launch_eig_sigma(c));
  LAUNCH(c, KK_MTAIL, launch_mtail_sigma(c));
  return SRM_OK;
}

// Newton-Schulz polar factors; subjects whose result fails its certificate
// go through the eigen-decomposition path (the launches skip the others).
srm_status do_polar(Ctx* c) {
  LAUNCH(c, KK_POLAR, launch_polar(c));
  LAUNCH(c, KK_EIG, launch_eig_fallback(c));
  LAUNCH(c, KK_MTAIL, launch_mtail_fallback(c));
  return SRM_OK;
}

srm_status do_side_chain(Ctx* c) {
  if (ns_supported(c)) {
    TRY(do_sigma_eig(c));
    TRY(do_polar(c));
  } else {
    LAUNCH(c, KK_EIG, launch_eig(c));
    if (mtail_supported(c)) {
      LAUNCH(c, KK_MTAIL, launch_mtail(c));
    } else {
      LAUNCH(c, KK_REFINE, launch_refine(c));
      LAUNCH(c, KK_RHO, launch_rho(c));
    }
  }
  LAUNCH(c, KK_PHI, launch_phi(c));
  return SRM_OK;
}

}  // namespace

// Runs a pending M-step tail on the main stream (before anything that reads
// rho^2, M_i or Sigma_s).
srm_status flush_pending(Ctx* c) {
  if (c->sigma_pending) {
    LAUNCH(c, KK_SIGMA, launch_sigma(c));
    c->sigma_pending = false;
  }
  if (!c->side_pending) return SRM_OK;
  if (c->sig_eig_done) {
    // single-pass form: Sigma_s's part of the tail already ran beside the pass
    TRY(do_polar(c));
    LAUNCH(c, KK_PHI, launch_phi(c));
  } else {
    TRY(do_side_chain(c));
  }
  c->side_pending = false;
  c->sig_eig_done = false;
  return SRM_OK;
}

namespace {

// Single-pass form.  The M-step's pass leaves A_i^T X^_i behind, so the
// E-step reads no X^: the polar factors (which need the pass's Gram) and Phi
// run first, then the reduction.  Sigma_s^new and its eigen-decomposition ran
// beside the pass.
srm_status do_estep_fused(Ctx* c) {
  if (c->p_from_f && c->side_pending && c->sig_eig_done && !c->sigma_pending && c->psum) {
    // after a single pass: its slot sums (which need no M_i) on the context
    // stream beside the polar factors and Phi on the second; the reduction
    // from the sums once the polar factors are done (beside Phi), E[S] = Phi y
    // once Phi is
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    {
      OnStream on(c, c->side);
      TRY(do_polar(c));
      CK(cudaEventRecord(c->ev_polar, c->side));
      LAUNCH(c, KK_PHI, launch_phi(c));
    }
    CK(cudaEventRecord(c->ev_join, c->side));
    LAUNCH(c, KK_P_SUM, launch_p_sum(c));
    CK(cudaStreamWaitEvent(c->stream, c->ev_polar, 0));
    c->side_pending = false;
    c->sig_eig_done = false;
    LAUNCH(c, KK_P_REDUCE, launch_p_reduce_part(c, true));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    LAUNCH(c, KK_P_REDUCE, launch_p_reduce_finish(c));
    c->sigma_pending = true;
    return SRM_OK;
  }
  if (c->side_pending || c->sigma_pending) TRY(flush_pending(c));
  if (!c->p_from_f) LAUNCH(c, KK_P_TC, launch_p_tc(c));
  LAUNCH(c, KK_P_REDUCE, launch_p_reduce(c));
  c->sigma_pending = true;
  return SRM_OK;
}

srm_status do_mstep_fused(Ctx* c) {
  // Sigma_s^new (from the E-step just done) and its eigen-decomposition on a
  // third stream beside the pass, joined at its end
  CK(cudaEventRecord(c->ev_fork, c->stream));
  CK(cudaStreamWaitEvent(c->side2, c->ev_fork, 0));
  {
    OnStream on(c, c->side2);
    if (c->sigma_pending) {
      LAUNCH(c, KK_SIGMA, launch_sigma(c));
      c->sigma_pending = false;
    }
    if (ns_supported(c)) TRY(do_sigma_eig(c));
  }
  CK(cudaEventRecord(c->ev_join2, c->side2));
  LAUNCH(c, KK_FPASS, launch_fpass(c));
  CK(cudaStreamWaitEvent(c->stream, c->ev_join2, 0));
  c->side_pending = true;
  c->sig_eig_done = ns_supported(c);
  c->p_from_f = true;
  return SRM_OK;
}

srm_status do_estep(Ctx* c) {
  if (c->fused) return do_estep_fused(c);
  const bool overlap = c->side_pending;
  if (!overlap && c->sigma_pending) {
    // an E-step followed by another without an M-step in between
    LAUNCH(c, KK_SIGMA, launch_sigma(c));
    c->sigma_pending = false;
  }
  if (overlap) {
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    if (c->sigma_pending) {
      OnStream on(c, c->side);
      LAUNCH(c, KK_SIGMA, launch_sigma(c));
      c->sigma_pending = false;
    }
    if (ns_supported(c)) {
      // Sigma_s's eigen-decomposition on a third stream, the subjects' polar
      // factors on the second; Phi waits for both
      CK(cudaEventRecord(c->ev_sig, c->side));
      CK(cudaStreamWaitEvent(c->side2, c->ev_sig, 0));
      {
        OnStream on(c, c->side2);
        TRY(do_sigma_eig(c));
      }
      CK(cudaEventRecord(c->ev_join2, c->side2));
      OnStream on(c, c->side);
      TRY(do_polar(c));
      CK(cudaStreamWaitEvent(c->side, c->ev_join2, 0));
      LAUNCH(c, KK_PHI, launch_phi(c));
    } else {
      OnStream on(c, c->side);
      TRY(do_side_chain(c));
    }
    CK(cudaEventRecord(c->ev_join, c->side));
    c->side_pending = false;
  }
  if (c->batched) {
    LAUNCH(c, KK_P_TC, launch_p_tc(c));
  } else {
    for (int i = 0; i < c->N; ++i) LAUNCH(c, KK_P_SIMT, launch_p_simt(c, i));
  }
  if (overlap) CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  LAUNCH(c, KK_P_REDUCE, launch_p_reduce(c));
  c->sigma_pending = true;
  return SRM_OK;
}

srm_status do_mstep(Ctx* c) {
  if (c->fused) return do_mstep_fused(c);
  if (c->batched) {
    LAUNCH(c, KK_A_TC, launch_a_tc(c));
  } else {
    for (int i = 0; i < c->N; ++i) LAUNCH(c, KK_A_SIMT, launch_a_simt(c, i));
  }
  c->side_pending = true;
  return SRM_OK;
}

// A partial (sharded) E-step must be finished before anything else steps the EM.
srm_status no_partial(srm_ctx* c, const char* who) {
  if (c->shard_partial) {
    set_error(std::string(who) + ": a sharded E-step awaits srm_estep_finish");
    return SRM_ERR_STATE;
  }
  return SRM_OK;
}

srm_status valid_ctx(srm_ctx* ctx) {
  if (!ctx) {
    set_error("null context");
    return SRM_ERR_ARG;
  }
  return SRM_OK;
}

struct StateHeader {
  uint64_t magic;
  int32_t version, N, T, k, kld, batched, n_ll;
  int64_t iters_done, Vpad_tot;
};
constexpr uint64_t kStateMagic = 0x314d5253'50534743ull;

}  // namespace

srm_status device_status(Ctx* c) { return check_status(c); }

void drop_graph(Ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
}

// n_iter EM iterations (E-step then M-step each); the M-step tail of the last
// one stays pending.  With SRM_GRAPH the steady-state iteration is replayed
// as one CUDA graph.
srm_status run_iterations(Ctx* c, int n_iter) {
  const bool use_graph = (c->flags & SRM_GRAPH) && !c->profile;
  for (int it = 0; it < n_iter; ++it) {
    if (use_graph && c->side_pending) {
      if (!c->graph_exec) {
        // one steady-state iteration: [pending M-step tail || E-pass] -> E-step
        // k x k work -> M-pass (whose tail stays pending)
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        srm_status s1 = do_estep(c);
        srm_status s2 = s1 == SRM_OK ? do_mstep(c) : s1;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->side_pending = true;
        if (s2 != SRM_OK) {
          if (g) cudaGraphDestroy(g);
          return s2;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          c->graph_exec = nullptr;
          return cuda_fail(e, "cudaGraphInstantiate");
        }
      }
      CK(cudaGraphLaunch(c->graph_exec, c->stream));
    } else {
      TRY(do_estep(c));
      TRY(do_mstep(c));
    }
    c->n_ll++;
    c->iters_done++;
  }
  return SRM_OK;
}
}  // namespace srm

using namespace srm;


extern "C" {

const char* srm_last_error(void) { return g_err.c_str(); }

srm_status srm_init(const srm_config* cfg, const void* const* X, const float* const* W0_dev, void* stream,
                    srm_ctx** out) {
  g_err.clear();
  if (!cfg || !X || !out || !cfg->voxels) {
    set_error("srm_init: null argument");
    return SRM_ERR_ARG;
  }
  *out = nullptr;
  if (cfg->n_subjects < 1 || cfg->k < 1 || cfg->k > KMAX || cfg->T < 2 || cfg->k > cfg->T) {
    set_error("srm_init: need N >= 1, 1 <= k <= 128, T >= 2, k <= T");
    return SRM_ERR_ARG;
  }
  if ((cfg->in_dtype != SRM_F32 && cfg->in_dtype != SRM_BF16) ||
      (cfg->store_dtype != SRM_F32 && cfg->store_dtype != SRM_BF16)) {
    set_error("srm_init: unknown dtype");
    return SRM_ERR_ARG;
  }
  const bool batched = (cfg->flags & SRM_BATCHED) != 0;
  if (batched != (cfg->store_dtype == SRM_BF16)) {
    set_error("srm_init: SRM_BATCHED requires store_dtype SRM_BF16 and the plain form requires SRM_F32");
    return SRM_ERR_ARG;
  }
  const uint32_t known = SRM_BATCHED | SRM_GRAPH | SRM_FINAL_LL | SRM_HOST_INPUT | SRM_PROFILE | SRM_SINGLE_PASS;
  if (cfg->flags & ~known) {
    set_error("srm_init: unknown flag bits");
    return SRM_ERR_ARG;
  }
  for (int i = 0; i < cfg->n_subjects; ++i) {
    if (cfg->voxels[i] < cfg->k || cfg->voxels[i] > (int64_t)1 << 31) {
      set_error("srm_init: voxel count of subject " + std::to_string(i) + " must be in [k, 2^31]");
      return SRM_ERR_ARG;
    }
    if (!X[i] || (W0_dev && !W0_dev[i])) {
      set_error("srm_init: null data or W0 pointer for subject " + std::to_string(i));
      return SRM_ERR_ARG;
    }
  }
  srm_ctx* c = new srm_ctx();
  srm_status st = SRM_OK;
  auto fail = [&](srm_status s) {
    free_all(c);
    delete c;
    return s;
  };
  c->N = cfg->n_subjects;
  c->T = cfg->T;
  c->k = cfg->k;
  c->in_dtype = cfg->in_dtype;
  c->store = cfg->store_dtype;
  c->flags = cfg->flags;
  c->batched = batched;
  c->profile = (cfg->flags & SRM_PROFILE) != 0;
  c->max_iter = cfg->max_iter > 0 ? cfg->max_iter : 1024;
  cudaError_t ce = cudaGetDevice(&c->device);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "cudaGetDevice"));
  cudaDeviceProp prop;
  ce = cudaGetDeviceProperties(&prop, c->device);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "cudaGetDeviceProperties"));
  c->num_sms = prop.multiProcessorCount;
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    ce = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return fail(cuda_fail(ce, "cudaStreamCreate"));
    c->own_stream = true;
  }
  ce = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->ev_sig, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&c->ev_polar, cudaEventDisableTiming);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "side stream / events"));
  c->kld = batched ? (c->k <= 64 ? 64 : 128) : ((c->k + 15) / 16) * 16;
  c->ldT = ((c->T + 7) / 8) * 8;
  c->nchunk = (c->T + TCH - 1) / TCH;
  c->nes_blk = es_blocks(c->T);  // E[S] partials: one per es block
  c->zgroups = zsum_groups(c->N, c->nchunk, c->num_sms, c->kld);
  c->v.resize(c->N);
  c->vpad.resize(c->N);
  c->off.resize(c->N + 1);
  int64_t acc = 0;
  for (int i = 0; i < c->N; ++i) {
    c->v[i] = cfg->voxels[i];
    c->vpad[i] = ((c->v[i] + ROW_PAD - 1) / ROW_PAD) * ROW_PAD;
    c->off[i] = acc;
    acc += c->vpad[i];
    c->Vtot += c->v[i];
  }
  c->off[c->N] = acc;
  c->Vpad_tot = acc;

  const int N = c->N, k = c->k, T = c->T;
  const size_t xel = c->store == SRM_BF16 ? 2 : 4;
  const size_t ael = batched ? 2 : 4;
  const int64_t ldTt = ((T + 63) / 64) * 64;  // rows of E[S]^T, padded for whole 32-wide chunks
  if ((st = dalloc(reinterpret_cast<char**>(&c->Xh), (size_t)c->Vpad_tot * c->ldT * xel, "resident X^")) != SRM_OK)
    return fail(st);
  if ((st = dalloc(reinterpret_cast<char**>(&c->A), (size_t)c->Vpad_tot * c->kld * ael, "A_i")) != SRM_OK)
    return fail(st);
#define AL(ptr, n, what) \
  if ((st = dalloc(&c->ptr, (size_t)(n), what)) != SRM_OK) return fail(st);
  AL(sqnorm, N, "norms");
  AL(rowsq, c->Vpad_tot, "row norms");
  AL(d_off, N + 1, "offsets");
  AL(d_v, N, "voxel counts");
  AL(rho2, N, "rho2");
  AL(Sigma, k * k, "Sigma");
  AL(SigmaNext, k * k, "Sigma next");
  AL(L, k * k, "L");
  AL(Phi, k * k, "Phi");
  AL(scal, 16, "scalars");
  AL(M64, (int64_t)N * k * k, "M64");
  AL(M32, (int64_t)N * c->kld * c->kld, "M32");
  AL(Uwarm, (int64_t)(N + 1) * k * k, "Uwarm");
  AL(G64, (int64_t)(N + 1) * k * k, "G64");
  AL(U64, (int64_t)(N + 1) * k * k, "U64");
  AL(H64, (int64_t)(N + 1) * k * k, "H64");
  AL(Xr64, (int64_t)(N + 1) * k * k, "Xr64");
  AL(eigv, (int64_t)(N + 1) * k, "eigenvalues");
  AL(jac_sweeps, N + 1, "Jacobi sweep counts");
  AL(ns_fb, N, "polar-factor fallback flags");
  AL(Y, (int64_t)k * T, "y");
  AL(ES64, (int64_t)k * T, "E[S]");
  AL(ll, c->max_iter, "ll trace");
  AL(iter, 1, "iteration counter");
  AL(status, 1, "status");
  AL(esPart, c->nes_blk, "<y, E[S]> partials");
  AL(Phi32, (int64_t)k * k, "Phi (FP32)");
  AL(sPart, (int64_t)c->nes_blk * k * k, "E[S] E[S]^T partials");
  AL(Ypart, (int64_t)c->zgroups * k * T, "subject-group reductions");
  if (batched) {
    AL(ESb, (int64_t)c->kld * c->ldT, "E[S] bf16");
    ce = cudaMemset(c->ESb, 0, (size_t)c->kld * c->ldT * 2);
  } else {
    AL(ESt, (int64_t)ldTt * c->kld, "E[S]^T fp32");
    ce = cudaMemset(c->ESt, 0, (size_t)ldTt * c->kld * 4);
  }
#undef AL
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "cudaMemset"));
  ce = cudaMemcpy(c->d_off, c->off.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(c->d_v, c->v.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "cudaMemcpy"));

  prepare_small_kernels(prop.sharedMemPerBlockOptin);
  if (polar_cl_supported(c)) choose_polar_cl(c);
  prepare_center_kernels(prop.sharedMemPerBlockOptin);
  prepare_simt_kernels(prop.sharedMemPerBlockOptin);
  if (batched) {
    if ((st = tc_setup(c)) != SRM_OK) return fail(st);
    if ((cfg->flags & SRM_SINGLE_PASS) && fused_supported(c)) {
      if ((st = fused_setup(c)) != SRM_OK) return fail(st);
      fused_select(c, true);
    }
  } else {
    if ((st = setup_plain(c)) != SRM_OK) return fail(st);
  }
  ce = cudaMemsetAsync(c->A, 0, (size_t)c->Vpad_tot * c->kld * ael, c->stream);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "cudaMemsetAsync"));

  // centre the data.  Host input is streamed through two staging buffers:
  // the copies of consecutive subjects alternate between the two side
  // streams (two transfers in flight), and subject i's centring waits for its
  // copy while the next copy proceeds; a buffer is refilled only after the
  // centring that read it.
  const size_t iel = cfg->in_dtype == SRM_BF16 ? 2 : 4;
  void* stage[2] = {nullptr, nullptr};
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
  if (cfg->flags & SRM_HOST_INPUT) {
    int64_t vmax = 0;
    for (int i = 0; i < N; ++i) vmax = std::max(vmax, c->v[i]);
    const int nstage = N > 1 ? 2 : 1;
    for (int b = 0; b < nstage && ce == cudaSuccess; ++b) {
      ce = cudaMalloc(&stage[b], (size_t)vmax * T * iel);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&consumed[b], cudaEventDisableTiming);
    }
    if (ce != cudaSuccess) {
      cudaGetLastError();
      for (int b = 0; b < 2; ++b) {
        if (stage[b]) cudaFree(stage[b]);
        if (copied[b]) cudaEventDestroy(copied[b]);
        if (consumed[b]) cudaEventDestroy(consumed[b]);
      }
      set_error("srm_init: cannot allocate the host-input staging buffers");
      return fail(SRM_ERR_NOMEM);
    }
  }
  auto free_stages = [&]() {
    for (int b = 0; b < 2; ++b) {
      if (stage[b]) cudaFree(stage[b]);
      if (copied[b]) cudaEventDestroy(copied[b]);
      if (consumed[b]) cudaEventDestroy(consumed[b]);
    }
  };
  // Algorithm 1's random orthogonal W^0 drawn here when the caller gives none
  void* haar_work = nullptr;
  if (!W0_dev && ce == cudaSuccess) {
    ce = cudaMalloc(&haar_work, haar_workspace_bytes(c));
    if (ce != cudaSuccess) {
      cudaGetLastError();
      free_stages();
      set_error("srm_init: cannot allocate the workspace of the random initial mappings");
      return fail(SRM_ERR_NOMEM);
    }
  }
  for (int i = 0; i < N; ++i) {
    const void* src = X[i];
    if (stage[0]) {
      const int b = stage[1] ? (i & 1) : 0;
      cudaStream_t cs = b ? c->side2 : c->side;
      if (i >= (stage[1] ? 2 : 1)) ce = cudaStreamWaitEvent(cs, consumed[b], 0);  // the centring that read it
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(stage[b], X[i], (size_t)c->v[i] * T * iel, cudaMemcpyHostToDevice, cs);
      if (ce == cudaSuccess) ce = cudaEventRecord(copied[b], cs);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(c->stream, copied[b], 0);
      if (ce != cudaSuccess) break;
      src = stage[b];
    }
    int ev0 = -1;
    if (c->profile) prof_begin(c, KK_CENTER, &ev0);
    ce = launch_center(c, i, src, cfg->in_dtype, T);
    if (ce != cudaSuccess) break;
    if (stage[0]) {
      ce = cudaEventRecord(consumed[stage[1] ? (i & 1) : 0], c->stream);
      if (ce != cudaSuccess) break;
    }
    if (c->profile) prof_end(c, KK_CENTER, ev0);
    ce = W0_dev ? launch_load_w0(c, i, W0_dev[i]) : launch_haar_w0(c, i, cfg->seed, haar_work);
    if (ce != cudaSuccess) break;
  }
  if (ce == cudaSuccess) ce = launch_sqnorm_reduce(c);
  if (ce == cudaSuccess) ce = launch_init_params(c);
  if (ce == cudaSuccess) ce = launch_phi(c);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (stage[0]) {  // the side streams' copies all precede the last centring
    cudaStreamSynchronize(c->side);
    cudaStreamSynchronize(c->side2);
  }
  free_stages();
  if (haar_work) cudaFree(haar_work);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "srm_init: centring / initialisation"));
  cudaFree(c->rowsq);
  c->rowsq = nullptr;
  if ((st = check_status(c)) != SRM_OK) return fail(st);
  *out = c;
  return SRM_OK;
}

srm_status srm_estep(srm_ctx* c) {
  TRY(valid_ctx(c));
  TRY(no_partial(c, "srm_estep"));
  if (c->n_ll >= c->max_iter) {
    set_error("srm_estep: log-likelihood trace is full (raise max_iter)");
    return SRM_ERR_STATE;
  }
  TRY(do_estep(c));
  c->n_ll++;
  c->have_estep = true;
  c->have_es = true;
  return SRM_OK;
}

srm_status srm_mstep(srm_ctx* c) {
  TRY(valid_ctx(c));
  TRY(no_partial(c, "srm_mstep"));
  if (!c->have_estep) {
    set_error("srm_mstep: no E-step precedes this M-step");
    return SRM_ERR_STATE;
  }
  TRY(do_mstep(c));
  c->have_estep = false;
  c->iters_done++;
  return SRM_OK;
}

srm_status srm_fit(srm_ctx* c, int32_t n_iter, double* ll_host) {
  TRY(valid_ctx(c));
  TRY(no_partial(c, "srm_fit"));
  if (n_iter < 0) {
    set_error("srm_fit: n_iter < 0");
    return SRM_ERR_ARG;
  }
  const bool final_ll = (c->flags & SRM_FINAL_LL) != 0;
  const int need = n_iter + (final_ll ? 1 : 0);
  if (c->n_ll + need > c->max_iter) {
    set_error("srm_fit: log-likelihood trace capacity exceeded (raise max_iter)");
    return SRM_ERR_STATE;
  }
  const int ll0 = c->n_ll;
  TRY(run_iterations(c, n_iter));
  TRY(flush_pending(c));
  c->have_estep = false;
  if (n_iter > 0) c->have_es = true;
  if (final_ll) {
    // one more E-step for the likelihood of the final parameters; E[S] of the
    // last iteration is kept (saved and restored around it)
    double* save = nullptr;
    if (c->have_es) {
      CK(cudaMallocAsync(&save, sizeof(double) * c->k * c->T, c->stream));
      CK(cudaMemcpyAsync(save, c->ES64, sizeof(double) * c->k * c->T, cudaMemcpyDeviceToDevice, c->stream));
    }
    TRY(do_estep(c));
    LAUNCH(c, KK_SIGMA, launch_sigma(c));  // its log-likelihood
    c->sigma_pending = false;
    c->n_ll++;
    if (save) {
      CK(cudaMemcpyAsync(c->ES64, save, sizeof(double) * c->k * c->T, cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaFreeAsync(save, c->stream));
    }
    c->have_es = true;
  }
  if (ll_host) {
    CK(cudaMemcpyAsync(ll_host, c->ll + ll0, sizeof(double) * (c->n_ll - ll0), cudaMemcpyDeviceToHost, c->stream));
    TRY(check_status(c));
  }
  return SRM_OK;
}

srm_status srm_estep_partial(srm_ctx* c, double* y, double* sums) {
  TRY(valid_ctx(c));
  TRY(no_partial(c, "srm_estep_partial"));
  if (!y || !sums) {
    set_error("srm_estep_partial: null y or sums");
    return SRM_ERR_ARG;
  }
  if (c->n_ll >= c->max_iter) {
    set_error("srm_estep_partial: log-likelihood trace is full (raise max_iter)");
    return SRM_ERR_STATE;
  }
  c->shard_y = y;
  c->shard_sums = sums;
  const srm_status st = do_estep(c);
  c->shard_y = nullptr;
  c->shard_sums = nullptr;
  // nothing of E[S] exists yet: Sigma_s^new and the likelihood follow srm_estep_finish
  c->sigma_pending = false;
  if (st != SRM_OK) return st;
  c->shard_partial = true;
  return SRM_OK;
}

srm_status srm_estep_finish(srm_ctx* c, const double* y, const double* sums) {
  TRY(valid_ctx(c));
  if (!c->shard_partial) {
    set_error("srm_estep_finish: no srm_estep_partial awaits its finish");
    return SRM_ERR_STATE;
  }
  if (!y || !sums) {
    set_error("srm_estep_finish: null y or sums");
    return SRM_ERR_ARG;
  }
  LAUNCH(c, KK_PHI, launch_estep_finish(c, y, sums));
  c->shard_partial = false;
  c->sigma_pending = true;
  c->n_ll++;
  c->have_estep = true;
  c->have_es = true;
  return SRM_OK;
}

srm_status srm_transform(srm_ctx* c, int32_t subject, const void* X_new, int32_t T_new, float* S_out) {
  TRY(valid_ctx(c));
  if (subject < 0 || subject >= c->N || !X_new || !S_out || T_new < 1) {
    set_error("srm_transform: bad subject, pointer or T_new");
    return SRM_ERR_ARG;
  }
  TRY(flush_pending(c));
  const int64_t v = c->v[subject];
  const int64_t ldn = ((T_new + 7) / 8) * 8;
  const int nchunk = (T_new + TCH - 1) / TCH;
  int ns = std::max(1, 2 * c->num_sms / nchunk);
  ns = (int)std::min<int64_t>(ns, std::max<int64_t>(1, v / 64));
  const int64_t need_buf = v * ldn, need_part = (int64_t)ns * nchunk * TCH * c->kld;
  if (need_buf > c->tr_elems) {
    if (c->tr_buf) cudaFree(c->tr_buf);
    c->tr_buf = nullptr;
    c->tr_elems = 0;
    TRY(dalloc(&c->tr_buf, need_buf, "transform buffer"));
    c->tr_elems = need_buf;
  }
  if (need_part > c->tr_part_elems) {
    if (c->tr_part) cudaFree(c->tr_part);
    c->tr_part = nullptr;
    c->tr_part_elems = 0;
    TRY(dalloc(&c->tr_part, need_part, "transform partials"));
    c->tr_part_elems = need_part;
  }
  CK(launch_center_generic(X_new, c->in_dtype, v, T_new, T_new, c->tr_buf, ldn, nullptr, c->stream));
  const char* A = static_cast<const char*>(c->A) + c->off[subject] * c->kld * (c->batched ? 2 : 4);
  CK(launch_p_simt_generic(A, c->batched, c->kld, c->kld, c->tr_buf, ldn, v, T_new, ns, c->tr_part, c->stream));
  CK(launch_transform_finish(c, subject, c->tr_part, ns, T_new, S_out));
  return SRM_OK;
}

srm_status srm_get_w(srm_ctx* c, int32_t subject, float* W) {
  TRY(valid_ctx(c));
  if (subject < 0 || subject >= c->N || !W) {
    set_error("srm_get_w: bad subject or null pointer");
    return SRM_ERR_ARG;
  }
  TRY(flush_pending(c));
  CK(launch_get_w(c, subject, W));
  return SRM_OK;
}

srm_status srm_get_s(srm_ctx* c, float* S) {
  TRY(valid_ctx(c));
  if (!S) {
    set_error("srm_get_s: null pointer");
    return SRM_ERR_ARG;
  }
  if (!c->have_es) {
    set_error("srm_get_s: no E-step has run");
    return SRM_ERR_STATE;
  }
  const int64_t n = (int64_t)c->k * c->T;
  cast_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->ES64, S, n);
  CK(cudaGetLastError());
  return SRM_OK;
}

srm_status srm_get_params(srm_ctx* c, double* rho2, double* sigma) {
  TRY(valid_ctx(c));
  TRY(flush_pending(c));
  TRY(check_status(c));
  if (rho2) CK(cudaMemcpy(rho2, c->rho2, sizeof(double) * c->N, cudaMemcpyDeviceToHost));
  if (sigma) CK(cudaMemcpy(sigma, c->Sigma, sizeof(double) * c->k * c->k, cudaMemcpyDeviceToHost));
  return SRM_OK;
}

srm_status srm_get_ll(srm_ctx* c, double* ll_host, int32_t* n) {
  TRY(valid_ctx(c));
  if (!n) {
    set_error("srm_get_ll: null count");
    return SRM_ERR_ARG;
  }
  TRY(flush_pending(c));
  TRY(check_status(c));
  const int m = std::min(*n, c->n_ll);
  if (ll_host && m > 0) CK(cudaMemcpy(ll_host, c->ll, sizeof(double) * m, cudaMemcpyDeviceToHost));
  *n = c->n_ll;
  return SRM_OK;
}

srm_status srm_synchronize(srm_ctx* c) {
  TRY(valid_ctx(c));
  TRY(flush_pending(c));
  return check_status(c);
}

srm_status srm_get_state(srm_ctx* c, void* buf, size_t* bytes) {
  TRY(valid_ctx(c));
  TRY(no_partial(c, "srm_get_state"));
  if (!bytes) {
    set_error("srm_get_state: null size");
    return SRM_ERR_ARG;
  }
  const int N = c->N, k = c->k;
  const size_t ael = c->batched ? 2 : 4;
  const size_t nA = (size_t)c->Vpad_tot * c->kld * ael;
  const size_t need = sizeof(StateHeader) + sizeof(double) * (N + 3 * k * k + (size_t)N * k * k + c->n_ll) +
                      sizeof(float) * ((size_t)(N + 1) * k * k + (size_t)N * c->kld * c->kld) + nA;
  if (!buf) {
    *bytes = need;
    return SRM_OK;
  }
  if (*bytes < need) {
    set_error("srm_get_state: buffer too small");
    *bytes = need;
    return SRM_ERR_ARG;
  }
  if (c->have_estep) {
    set_error("srm_get_state: an E-step is pending; checkpoint between iterations");
    return SRM_ERR_STATE;
  }
  TRY(flush_pending(c));
  TRY(check_status(c));
  StateHeader h{kStateMagic, 2, N, c->T, k, c->kld, c->batched ? 1 : 0, c->n_ll, c->iters_done, c->Vpad_tot};
  char* p = static_cast<char*>(buf);
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  auto get = [&](const void* d, size_t nb) -> cudaError_t {
    cudaError_t e = cudaMemcpy(p, d, nb, cudaMemcpyDeviceToHost);
    p += nb;
    return e;
  };
  CK(get(c->rho2, sizeof(double) * N));
  CK(get(c->Sigma, sizeof(double) * k * k));
  CK(get(c->M64, sizeof(double) * N * k * k));
  CK(get(c->ll, sizeof(double) * c->n_ll));
  CK(get(c->G64 + (size_t)N * k * k, sizeof(double) * k * k));
  CK(get(c->Xr64 + (size_t)N * k * k, sizeof(double) * k * k));
  CK(get(c->Uwarm, sizeof(float) * (N + 1) * k * k));
  CK(get(c->M32, sizeof(float) * N * c->kld * c->kld));
  CK(get(c->A, nA));
  *bytes = need;
  return SRM_OK;
}

srm_status srm_set_state(srm_ctx* c, const void* buf, size_t bytes) {
  TRY(valid_ctx(c));
  TRY(no_partial(c, "srm_set_state"));
  if (!buf || bytes < sizeof(StateHeader)) {
    set_error("srm_set_state: buffer too small");
    return SRM_ERR_ARG;
  }
  StateHeader h;
  memcpy(&h, buf, sizeof h);
  if (h.magic != kStateMagic || h.version != 2 || h.N != c->N || h.T != c->T || h.k != c->k || h.kld != c->kld ||
      h.batched != (c->batched ? 1 : 0) || h.Vpad_tot != c->Vpad_tot || h.n_ll < 0 || h.n_ll > c->max_iter) {
    set_error("srm_set_state: checkpoint does not match this context's configuration");
    return SRM_ERR_ARG;
  }
  const int N = c->N, k = c->k;
  const size_t ael = c->batched ? 2 : 4;
  const size_t nA = (size_t)c->Vpad_tot * c->kld * ael;
  const size_t need = sizeof(StateHeader) + sizeof(double) * (N + 3 * k * k + (size_t)N * k * k + h.n_ll) +
                      sizeof(float) * ((size_t)(N + 1) * k * k + (size_t)N * c->kld * c->kld) + nA;
  if (bytes != need) {
    set_error("srm_set_state: size mismatch");
    return SRM_ERR_ARG;
  }
  CK(cudaStreamSynchronize(c->stream));
  const char* p = static_cast<const char*>(buf) + sizeof h;
  auto put = [&](void* d, size_t nb) -> cudaError_t {
    cudaError_t e = cudaMemcpy(d, p, nb, cudaMemcpyHostToDevice);
    p += nb;
    return e;
  };
  CK(put(c->rho2, sizeof(double) * N));
  CK(put(c->Sigma, sizeof(double) * k * k));
  CK(put(c->M64, sizeof(double) * N * k * k));
  CK(put(c->ll, sizeof(double) * h.n_ll));
  CK(put(c->G64 + (size_t)N * k * k, sizeof(double) * k * k));
  CK(put(c->Xr64 + (size_t)N * k * k, sizeof(double) * k * k));
  CK(put(c->Uwarm, sizeof(float) * (N + 1) * k * k));
  CK(put(c->M32, sizeof(float) * N * c->kld * c->kld));
  CK(put(c->A, nA));
  const int it = h.n_ll;
  CK(cudaMemcpy(c->iter, &it, sizeof(int), cudaMemcpyHostToDevice));
  c->n_ll = h.n_ll;
  c->iters_done = h.iters_done;
  c->have_estep = false;
  c->have_es = false;
  c->side_pending = false;
  c->sigma_pending = false;
  c->sig_eig_done = false;
  c->p_from_f = false;  // A_i changed: the next E-step streams X^ again
  CK(launch_phi(c));
  return check_status(c);
}

srm_status srm_get_kernel_times(srm_ctx* c, const char** names, int64_t* launches, double* ms, int32_t* n,
                                int32_t reset) {
  TRY(valid_ctx(c));
  if (!n) {
    set_error("srm_get_kernel_times: null count");
    return SRM_ERR_ARG;
  }
  CK(cudaStreamSynchronize(c->stream));
  for (const auto& p : c->pending) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->ev_pool[p.ev0], c->ev_pool[p.ev1]));
    c->prof_launches[p.kind] += kKernelsPerKind[p.kind];
    c->prof_ms[p.kind] += t;
  }
  c->pending.clear();
  c->ev_next = 0;
  const int m = std::min<int>(*n, KK_COUNT);
  for (int j = 0; j < m; ++j) {
    if (names) names[j] = kKernelNames[j];
    if (launches) launches[j] = c->prof_launches[j];
    if (ms) ms[j] = c->prof_ms[j];
  }
  *n = KK_COUNT;
  if (reset) {
    for (int j = 0; j < KK_COUNT; ++j) {
      c->prof_launches[j] = 0;
      c->prof_ms[j] = 0;
    }
  }
  return SRM_OK;
}

srm_status srm_layout(srm_ctx* c, int64_t* out, int32_t n) {
  TRY(valid_ctx(c));
  if (!out) {
    set_error("srm_layout: null output");
    return SRM_ERR_ARG;
  }
  const int64_t vals[6] = {c->ldT, c->kld, c->Vpad_tot,
                           c->Vpad_tot * c->ldT * (c->store == SRM_BF16 ? 2 : 4),
                           c->Vpad_tot * c->kld * (c->batched ? 2 : 4), c->fused ? 1 : 0};
  for (int j = 0; j < n && j < 6; ++j) out[j] = vals[j];
  return SRM_OK;
}

srm_status srm_debug_eig_sweeps(srm_ctx* c, int32_t* out, int32_t n) {
  TRY(valid_ctx(c));
  if (!out || n < 0) {
    set_error("srm_debug_eig_sweeps: null output");
    return SRM_ERR_ARG;
  }
  TRY(flush_pending(c));
  TRY(check_status(c));
  const int m = std::min(n, c->N + 1);
  if (m > 0) CK(cudaMemcpy(out, c->jac_sweeps, sizeof(int) * m, cudaMemcpyDeviceToHost));
  return SRM_OK;
}

srm_status srm_debug_force_eig_polar(srm_ctx* c, int32_t on) {
  TRY(valid_ctx(c));
  TRY(flush_pending(c));
  c->force_eig_polar = on != 0;
  drop_graph(c);  // a captured iteration holds the launch arguments
  return SRM_OK;
}

void srm_destroy(srm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  free_all(c);
  delete c;
}

}  // extern "C"
