// Launch plans of the batched form and the autotuner that picks one per
// (v_i, T, k) on the device at hand.
//
// The plan decides how the two streaming contractions of an EM iteration
// (Algorithm 1: the E-step reduction sum_i W_i^T X^_i and the M-step's
// A_i = X^_i E[S]^T with its Gram) are cut and pipelined: the E-pass CTA
// count (its split-v depth, set by the SMs it leaves to the M-step tail that
// runs beside it), the M-pass's stage count, Gram buffers, E[S] residency
// and L2 prefetch distance, and whether the single-pass form replaces the
// two passes.  None of it changes the mathematics; the tuner times the
// candidates on the resident data and keeps the fastest.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "srm_internal.cuh"

namespace srm {
namespace {

#define TCK(expr)                                     \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr); \
  } while (0)
#define TTRY(expr)                   \
  do {                               \
    srm_status _s = (expr);          \
    if (_s != SRM_OK) return _s;     \
  } while (0)

srm_plan current_plan(const Ctx* c) {
  srm_plan p{};
  p.single_pass = c->fused ? 1 : 0;
  p.e_reserve = tc_e_reserve(c);
  tc_get_m_plan(c, &p.m_gram_bufs, &p.m_resident_es, &p.m_stages, &p.m_prefetch, &p.m_boxes);
  p.f_prefetch = fused_get_pf(c);
  p.f_l2_hints = fused_get_hints(c);
  p.f_first_stages = fused_get_first_stages(c);
  p.f_reserve = fused_get_reserve(c);
  p.f_lead = fused_get_lead(c);
  p.f_slots = fused_get_slots(c);
  return p;
}

srm_status apply_plan(Ctx* c, const srm_plan& p) {
  const bool fine = p.f_slots != 0;
  if ((p.single_pass != 0 && p.single_pass != 1) || p.f_prefetch < 0 || p.f_prefetch > 16 || p.f_l2_hints < 0 ||
      p.f_l2_hints > 7 || (fine && p.f_slots != 8 && p.f_slots != 9) || p.f_first_stages < (fine ? 2 : 1) ||
      p.f_first_stages > (fine ? p.f_slots - 2 : 4) || p.f_lead < 0 || p.f_lead > 4) {
    set_error("srm_set_plan: field out of range (single_pass 0/1, f_prefetch 0-16, f_l2_hints 0-7, "
              "f_slots 0/8/9, f_first_stages 1-4 with f_slots 0 or 2..f_slots-2, f_lead 0-4)");
    return SRM_ERR_ARG;
  }
  if (p.single_pass && !fused_supported(c)) {
    set_error("srm_set_plan: the single-pass form needs k <= 64 and T <= 1024");
    return SRM_ERR_UNSUPPORTED;
  }
  if (fine && !fused_fine_supported(c)) {
    set_error("srm_set_plan: f_slots 8 or 9 needs the single-pass form's one-CTA tiles (k <= 64, T <= 512)");
    return SRM_ERR_UNSUPPORTED;
  }
  // a pending M-step tail reads the Gram slots of the form that produced them
  TTRY(flush_pending(c));
  TCK(cudaStreamSynchronize(c->stream));
  TCK(cudaStreamSynchronize(c->side));
  TCK(cudaStreamSynchronize(c->side2));
  int nb, res, st, pf, bx;
  tc_get_m_plan(c, &nb, &res, &st, &pf, &bx);
  srm_status s = tc_set_m_plan(c, p.m_gram_bufs, p.m_resident_es, p.m_stages, p.m_prefetch, p.m_boxes);
  if (s != SRM_OK) return s;
  s = tc_set_e_reserve(c, p.e_reserve);
  if (s != SRM_OK) {
    tc_set_m_plan(c, nb, res, st, pf, bx);
    return s;
  }
  if (p.single_pass && !c->fs) TTRY(fused_setup(c));
  if (c->fs) {
    if (p.f_reserve < 0 || p.f_reserve >= c->num_sms) {
      set_error("srm_set_plan: f_reserve must leave SMs to the single pass");
      return SRM_ERR_ARG;
    }
    TTRY(fused_set_reserve(c, p.f_reserve));
    fused_set_pf(c, p.f_prefetch);
    fused_set_hints(c, p.f_l2_hints);
    fused_set_first_stages(c, p.f_first_stages);
    fused_set_lead(c, p.f_lead);
    fused_set_slots(c, p.f_slots);
    if (!p.single_pass) c->p_from_f = false;  // the next E-step streams X^ again
    fused_select(c, p.single_pass != 0);
  }
  drop_graph(c);
  return SRM_OK;
}

// Average milliseconds of `reps` back-to-back launches (after one untimed).
srm_status time_launches(Ctx* c, cudaError_t (*fn)(Ctx*), int reps, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  TCK(fn(c));
  TCK(cudaEventRecord(e0, c->stream));
  for (int r = 0; r < reps; ++r) TCK(fn(c));
  TCK(cudaEventRecord(e1, c->stream));
  TCK(cudaEventSynchronize(e1));
  TCK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= (float)reps;
  return device_status(c);
}

// Milliseconds per EM iteration over `iters` iterations (after two untimed),
// through the same path srm_fit takes.  The log-likelihood trace restarts
// from entry 0 for every candidate.
srm_status time_iterations(Ctx* c, int iters, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  TTRY(flush_pending(c));
  TCK(cudaStreamSynchronize(c->stream));
  c->n_ll = 0;
  TCK(cudaMemsetAsync(c->iter, 0, sizeof(int), c->stream));
  TTRY(run_iterations(c, 2));
  TCK(cudaEventRecord(e0, c->stream));
  TTRY(run_iterations(c, iters));
  TCK(cudaEventRecord(e1, c->stream));
  TCK(cudaEventSynchronize(e1));
  TCK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= (float)iters;
  TTRY(flush_pending(c));
  return device_status(c);
}

std::string signature(const Ctx* c) {
  cudaDeviceProp prop;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, c->device) == cudaSuccess) name = prop.name;
  for (char& ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the voxel counts
  for (int64_t v : c->v)
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  char buf[160];
  snprintf(buf, sizeof buf, "%s/sm%d/N%d/T%d/k%d/v%016llx", name.c_str(), c->num_sms, c->N, c->T, c->k,
           (unsigned long long)h);
  return buf;
}

std::string plan_line(const std::string& sig, const srm_plan& p, double ms) {
  char buf[320];
  snprintf(buf, sizeof buf,
           "%s sp=%d er=%d mst=%d mgb=%d mres=%d mpf=%d mbx=%d fpf=%d fl2=%d fsh=%d fr=%d fld=%d fsl=%d ms=%.6f",
           sig.c_str(), p.single_pass, p.e_reserve, p.m_stages, p.m_gram_bufs, p.m_resident_es, p.m_prefetch,
           p.m_boxes, p.f_prefetch, p.f_l2_hints, p.f_first_stages, p.f_reserve, p.f_lead, p.f_slots, ms);
  return buf;
}

bool parse_line(const std::string& line, const std::string& sig, srm_plan* p, double* ms) {
  if (line.compare(0, sig.size(), sig) != 0 || line.size() <= sig.size() || line[sig.size()] != ' ') return false;
  srm_plan q{};
  double t = 0;
  if (sscanf(line.c_str() + sig.size(),
             " sp=%d er=%d mst=%d mgb=%d mres=%d mpf=%d mbx=%d fpf=%d fl2=%d fsh=%d fr=%d fld=%d fsl=%d ms=%lf",
             &q.single_pass, &q.e_reserve, &q.m_stages, &q.m_gram_bufs, &q.m_resident_es, &q.m_prefetch,
             &q.m_boxes, &q.f_prefetch, &q.f_l2_hints, &q.f_first_stages, &q.f_reserve, &q.f_lead, &q.f_slots,
             &t) != 14)
    return false;
  *p = q;
  *ms = t;
  return true;
}

bool cache_lookup(const char* path, const std::string& sig, srm_plan* p, double* ms) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  while (std::getline(f, line))
    if (parse_line(line, sig, p, ms)) return true;
  return false;
}

srm_status cache_store(const char* path, const std::string& sig, const srm_plan& p, double ms) {
  std::vector<std::string> keep;
  {
    std::ifstream f(path);
    std::string line;
    srm_plan q;
    double t;
    while (f && std::getline(f, line))
      if (!line.empty() && !parse_line(line, sig, &q, &t)) keep.push_back(line);
  }
  keep.push_back(plan_line(sig, p, ms));
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream o(tmp, std::ios::trunc);
    if (!o) {
      set_error(std::string("srm_autotune: cannot write ") + tmp);
      return SRM_ERR_ARG;
    }
    for (const auto& l : keep) o << l << "\n";
    if (!o) {
      set_error(std::string("srm_autotune: write failed on ") + tmp);
      return SRM_ERR_ARG;
    }
  }
  if (rename(tmp.c_str(), path) != 0) {
    set_error(std::string("srm_autotune: cannot rename ") + tmp);
    return SRM_ERR_ARG;
  }
  return SRM_OK;
}

// The context as srm_init leaves it: W0 in A, rho^2 = 1, Sigma_s = I,
// M_i = I, an empty log-likelihood trace, nothing pending.
srm_status restore_initial(Ctx* c, const void* savedA, size_t nA) {
  TTRY(flush_pending(c));
  TCK(cudaStreamSynchronize(c->side));
  TCK(cudaStreamSynchronize(c->side2));
  TCK(cudaMemcpyAsync(c->A, savedA, nA, cudaMemcpyDeviceToDevice, c->stream));
  TCK(launch_init_params(c));
  TCK(launch_phi(c));
  TCK(cudaStreamSynchronize(c->stream));
  c->n_ll = 0;
  c->iters_done = 0;
  c->have_estep = false;
  c->have_es = false;
  c->side_pending = false;
  c->sigma_pending = false;
  c->sig_eig_done = false;
  c->p_from_f = false;
  drop_graph(c);
  c->pending.clear();
  c->ev_next = 0;
  for (int j = 0; j < KK_COUNT; ++j) {
    c->prof_launches[j] = 0;
    c->prof_ms[j] = 0;
  }
  return device_status(c);
}

struct Report {
  std::ostringstream os;
  void add(const char* stage, const srm_plan& p, float ms, const char* unit) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "%-6s sp=%d er=%-3d mst=%d mgb=%d mres=%d mpf=%-2d mbx=%d fpf=%d fl2=%d fsh=%d fr=%-2d fld=%d fsl=%d"
             "  %9.4f %s\n",
             stage, p.single_pass, p.e_reserve, p.m_stages, p.m_gram_bufs, p.m_resident_es, p.m_prefetch,
             p.m_boxes, p.f_prefetch, p.f_l2_hints, p.f_first_stages, p.f_reserve, p.f_lead, p.f_slots, ms, unit);
    os << buf;
  }
};

// The search itself (W0 saved by the caller; the context is restored after).
srm_status search(Ctx* c, int iters, srm_plan* best_out, float* best_ms_out, Report& rep, cudaEvent_t e0,
                  cudaEvent_t e1) {
  const bool fused_ok = fused_supported(c);
  srm_plan base = current_plan(c);
  base.single_pass = 0;
  TTRY(apply_plan(c, base));
  // one real iteration: E[S], A_i and every partial hold values of the data
  TTRY(run_iterations(c, 1));
  TTRY(flush_pending(c));
  TTRY(device_status(c));

  // 1. M-pass plans, launch by launch (the pass is idempotent: same E[S], same A_i)
  std::vector<std::array<int, 5>> mc;
  tc_m_candidates(c, mc);
  float best_m = 1e30f;
  srm_plan bm = base;
  for (const auto& m : mc) {
    TTRY(tc_set_m_plan(c, m[0], m[1], m[2], m[3], m[4]));
    float ms = 0;
    TTRY(time_launches(c, launch_a_tc, 3, e0, e1, &ms));
    srm_plan p = base;
    p.m_gram_bufs = m[0];
    p.m_resident_es = m[1];
    p.m_stages = m[2];
    p.m_prefetch = m[3];
    p.m_boxes = m[4];
    rep.add("mpass", p, ms, "ms/launch");
    if (ms < best_m) {
      best_m = ms;
      bm = p;
    }
  }
  TTRY(apply_plan(c, bm));

  // 2. single-pass prefetch distances, launch by launch
  srm_plan bf = bm;
  bf.single_pass = 1;
  if (fused_ok) {
    TTRY(apply_plan(c, bf));
    float best_f = 1e30f;
    srm_plan bfp = bf;
    // 32 KB stages (every pipeline), then the 16 KB-slot forms (T <= 512),
    // whose rings split the stage memory more finely (on the forrest-1024-like
    // workload the L2 re-reads wanted more than half of it); L2 prefetch never
    // helped the 32 KB form, so the slot forms run without it
    struct FCand {
      int slots, sh, lead, hints, pf;
    };
    std::vector<FCand> cands;
    for (int sh : {1, 2, 3, 4})
      for (int lead : {0, 3})
        for (int hints : {0, 7})
          for (int pf : {0, 1})
            if (sh != 4 || lead == 0)  // the shared ring keeps a lead of one tile by construction
              cands.push_back({0, sh, lead, hints, pf});
    if (fused_fine_supported(c))
      for (int slots : {8, 9})
        for (int sh = 3; sh <= 5; ++sh)
          for (int lead : {0, 3})
            for (int hints : {0, 7}) cands.push_back({slots, sh, lead, hints, 0});
    for (const FCand& fc : cands) {
      fused_set_pf(c, fc.pf);
      fused_set_hints(c, fc.hints);
      fused_set_first_stages(c, fc.sh);
      fused_set_lead(c, fc.lead);
      fused_set_slots(c, fc.slots);
      float ms = 0;
      TTRY(time_launches(c, launch_fpass, 3, e0, e1, &ms));
      srm_plan p = bf;
      p.f_prefetch = fc.pf;
      p.f_l2_hints = fc.hints;
      p.f_first_stages = fc.sh;
      p.f_lead = fc.lead;
      p.f_slots = fc.slots;
      rep.add("fpass", p, ms, "ms/launch");
      if (ms < best_f) {
        best_f = ms;
        bfp = p;
      }
    }
    bf = bfp;
  }

  // 3. E-pass reserves (split-v depths), as whole iterations of the two-pass form
  std::vector<int> reserves = {0, 4, 8, 12, 16, 20, 24, 32, tc_default_e_reserve(c)};
  if (polar_cl_supported(c)) {
    // the clustered polar factors need C SMs per subject beside the pass
    for (int r : {48, 64, 80}) reserves.push_back(r);
  }
  std::sort(reserves.begin(), reserves.end());
  reserves.erase(std::unique(reserves.begin(), reserves.end()), reserves.end());
  float best_it = 1e30f;
  srm_plan best = bm;
  for (int r : reserves) {
    if (r >= c->num_sms) continue;
    srm_plan p = bm;
    p.e_reserve = r;
    TTRY(apply_plan(c, p));
    float ms = 0;
    TTRY(time_iterations(c, iters, e0, e1, &ms));
    rep.add("iter", p, ms, "ms/iteration");
    if (ms < best_it) {
      best_it = ms;
      best = p;
    }
  }

  // 4. the single-pass form with its best pipeline, as whole iterations, for
  // a few SM reserves beside it.  It replaces the two-pass form only when
  // faster by more than the run-to-run noise of these timings (about 1%), so
  // that repeated tunings of one workload agree.
  constexpr float kFormMargin = 0.98f;
  if (fused_ok) {
    const float two_pass_ms = best_it;
    bf.e_reserve = best.e_reserve;  // its first E-step still runs the E-pass
    std::vector<int> fres = {0, 4, 10, bf.f_reserve};
    std::sort(fres.begin(), fres.end());
    fres.erase(std::unique(fres.begin(), fres.end()), fres.end());
    for (int r : fres) {
      srm_plan p = bf;
      p.f_reserve = r;
      TTRY(apply_plan(c, p));
      float ms = 0;
      TTRY(time_iterations(c, iters, e0, e1, &ms));
      rep.add("iter", p, ms, "ms/iteration");
      if (ms < best_it && ms < kFormMargin * two_pass_ms) {
        best_it = ms;
        best = p;
      }
    }
  }
  *best_out = best;
  *best_ms_out = best_it;
  return SRM_OK;
}

}  // namespace
}  // namespace srm

using namespace srm;

extern "C" {

srm_status srm_get_plan(srm_ctx* c, srm_plan* plan) {
  if (!c || !plan) {
    set_error("srm_get_plan: null argument");
    return SRM_ERR_ARG;
  }
  if (!c->batched) {
    set_error("srm_get_plan: the plain FP32 form has no launch plan");
    return SRM_ERR_UNSUPPORTED;
  }
  *plan = current_plan(c);
  return SRM_OK;
}

srm_status srm_set_plan(srm_ctx* c, const srm_plan* plan) {
  if (!c || !plan) {
    set_error("srm_set_plan: null argument");
    return SRM_ERR_ARG;
  }
  if (!c->batched) {
    set_error("srm_set_plan: the plain FP32 form has no launch plan");
    return SRM_ERR_UNSUPPORTED;
  }
  if (c->have_estep || c->shard_partial) {
    set_error("srm_set_plan: an E-step awaits its M-step; change the plan between iterations");
    return SRM_ERR_STATE;
  }
  return apply_plan(c, *plan);
}

srm_status srm_autotune(srm_ctx* c, const char* cache_path, int32_t iters, srm_plan* chosen, double* ms_per_iter,
                        char* report, size_t report_bytes) {
  if (!c) {
    set_error("srm_autotune: null context");
    return SRM_ERR_ARG;
  }
  if (!c->batched) {
    set_error("srm_autotune: the plain FP32 form has no launch plan");
    return SRM_ERR_UNSUPPORTED;
  }
  if (iters < 1) {
    set_error("srm_autotune: iters must be >= 1");
    return SRM_ERR_ARG;
  }
  if (c->n_ll != 0 || c->iters_done != 0 || c->have_estep || c->shard_partial) {
    set_error("srm_autotune: call it right after srm_init, before any E-step");
    return SRM_ERR_STATE;
  }
  if (c->max_iter < iters + 3) {
    set_error("srm_autotune: the log-likelihood trace must hold iters + 3 entries (raise max_iter)");
    return SRM_ERR_ARG;
  }
  if (report && report_bytes) report[0] = '\0';
  const std::string sig = signature(c);
  srm_plan p{};
  double ms = 0;
  if (cache_path && cache_lookup(cache_path, sig, &p, &ms)) {
    if (apply_plan(c, p) == SRM_OK) {
      if (chosen) *chosen = p;
      if (ms_per_iter) *ms_per_iter = ms;
      if (report && report_bytes) snprintf(report, report_bytes, "cached: %s\n", plan_line(sig, p, ms).c_str());
      return SRM_OK;
    }
    // a stale line (e.g. a plan this build cannot run) is tuned afresh
  }
  const size_t nA = (size_t)c->Vpad_tot * c->kld * 2;
  void* savedA = nullptr;
  if (cudaMalloc(&savedA, nA) != cudaSuccess) {
    cudaGetLastError();
    set_error("srm_autotune: no room for the temporary copy of W0");
    return SRM_ERR_NOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  srm_status st = SRM_OK;
  cudaError_t ce = cudaMemcpyAsync(savedA, c->A, nA, cudaMemcpyDeviceToDevice, c->stream);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  const srm_plan before = current_plan(c);
  Report rep;
  float best_ms = 0;
  srm_plan best = before;
  if (ce != cudaSuccess) st = cuda_fail(ce, "srm_autotune: setup");
  if (st == SRM_OK) st = search(c, iters, &best, &best_ms, rep, e0, e1);
  const std::string err = st == SRM_OK ? std::string() : std::string(srm_last_error());
  // the chosen plan (or, after a failure, the plan the context had), then the
  // initial state
  srm_status s2 = apply_plan(c, st == SRM_OK ? best : before);
  srm_status s3 = restore_initial(c, savedA, nA);
  cudaFree(savedA);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != SRM_OK) {
    set_error(err);
    return st;
  }
  if (s2 != SRM_OK) return s2;
  if (s3 != SRM_OK) return s3;
  if (cache_path) TTRY(cache_store(cache_path, sig, best, best_ms));
  if (chosen) *chosen = best;
  if (ms_per_iter) *ms_per_iter = best_ms;
  if (report && report_bytes) {
    const std::string r = rep.os.str() + "chosen: " + plan_line(sig, best, best_ms) + "\n";
    snprintf(report, report_bytes, "%s", r.c_str());
  }
  return SRM_OK;
}

}  // extern "C"
