// api.cu -- the C ABI (include/tsm.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "contract.h"
#include "fft.h"
#include "fields.cuh"
#include "solver.h"

using namespace tsm;

namespace tsm {
const char* last_error();
}

namespace {

int bad(int code, const char* msg) {
  set_error("%s", msg);
  return code;
}

int select_device(Ctx& c) {
  TSM_CUDA(cudaSetDevice(c.device));
  return TSM_OK;
}

// device pointer for a caller buffer: the caller's own (on_device) or a
// workspace staging buffer, optionally filled from host memory
int stage_in(Ctx& c, const char* name, const double* user, size_t bytes, int on_device, const double** dev) {
  if (on_device) {
    *dev = user;
    return TSM_OK;
  }
  void* p = nullptr;
  TSM_TRY(c.buffer(name, bytes, &p));
  TSM_CUDA(cudaMemcpyAsync(p, user, bytes, cudaMemcpyHostToDevice, c.stream));
  *dev = static_cast<const double*>(p);
  return TSM_OK;
}

int stage_out_ptr(Ctx& c, const char* name, double* user, size_t bytes, int on_device, double** dev) {
  if (on_device) {
    *dev = user;
    return TSM_OK;
  }
  void* p = nullptr;
  TSM_TRY(c.buffer(name, bytes, &p));
  *dev = static_cast<double*>(p);
  return TSM_OK;
}

int stage_out_finish(Ctx& c, double* user, const double* dev, size_t bytes, int on_device) {
  if (!on_device && user != nullptr) TSM_CUDA(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, c.stream));
  return TSM_OK;
}

size_t spinor_bytes(const Ctx& c) { return (size_t)c.g.V * 24 * sizeof(double); }

int pack_eo(Ctx& c, int prec, const double* canon, EOField f) {
  return dispatch_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    TSM_TRY(launch_pack<S>(c, 0, canon, f.e));
    return launch_pack<S>(c, 1, canon, f.o);
  });
}

int unpack_eo(Ctx& c, int prec, EOField f, double* canon) {
  return dispatch_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    TSM_TRY(launch_unpack<S>(c, 0, f.e, canon));
    return launch_unpack<S>(c, 1, f.o, canon);
  });
}

int eo_fields(Ctx& c, const std::string& name, int prec, EOField* f, int nrhs = 1) {
  TSM_TRY(c.field(name + "_e", prec, &f->e, nrhs));
  return c.field(name + "_o", prec, &f->o, nrhs);
}

int check_stop(const tm_stop* s) {
  if (s == nullptr) return bad(TSM_ERR_ARG, "null tm_stop");
  if (s->prec < TSM_F64 || s->prec > TSM_F16) return bad(TSM_ERR_ARG, "tm_stop.prec out of range");
  if (s->max_iter < 0 || !(s->rel_tol >= 0.0)) return bad(TSM_ERR_ARG, "tm_stop: max_iter < 0 or rel_tol < 0");
  if (s->precond != 0 && s->precond != 1) return bad(TSM_ERR_ARG, "tm_stop.precond must be 0 or 1");
  if (s->restart < 0) return bad(TSM_ERR_ARG, "tm_stop.restart < 0");
  return TSM_OK;
}

template <class S>
int apply_operator(Ctx& c, int op, int dagger, EOField in, EOField out) {
  const double k = c.lat.kappa, mu = c.lat.mu, k2 = k * k;
  const double m = dagger ? -mu : mu;
  auto zero = [&](PField f) { return launch_convert<S, S>(c, PField{}, f); };
  switch (op) {
    case TM_OP_FULL:
      for (int par = 0; par < 2; ++par) {
        HopArgs<S> h = hop_args<S>(c, par);
        h.in = (par ? in.e : in.o).as<S>();
        h.center = (par ? in.o : in.e).as<S>();
        h.tc = twist_A(k, m);
        h.ac = 1.0;
        h.ah = -k;
        h.out = (par ? out.o : out.e).as<S>();
        TSM_TRY(launch_hop<S>(c, h, dagger, HOP_CENTER, -1));
      }
      return TSM_OK;
    case TM_OP_HOP_EO:
    case TM_OP_HOP_OE: {
      const int par = (op == TM_OP_HOP_EO) ? 0 : 1;
      HopArgs<S> h = hop_args<S>(c, par);
      h.in = (par ? in.e : in.o).as<S>();
      h.out = (par ? out.o : out.e).as<S>();
      TSM_TRY(launch_hop<S>(c, h, dagger, 0, -1));
      return zero(par ? out.e : out.o);
    }
    case TM_OP_SCHUR:
    case TM_OP_NORMAL: {
      PField t, w;
      TSM_TRY(c.field("op_t", S::id, &t));
      TSM_TRY(c.field("op_w", S::id, &w));
      PField src = in.e;
      if (op == TM_OP_NORMAL || !dagger) {
        // Dhat: t = A^-1 H_oe src ; out = A^-1 (A src - kappa^2 H_eo t)
        HopArgs<S> h = hop_args<S>(c, 1);
        h.in = src.as<S>();
        h.out = t.as<S>();
        h.to = twist_Ainv(k, mu);
        TSM_TRY(launch_hop<S>(c, h, 0, 0, -1));
        h = hop_args<S>(c, 0);
        h.in = t.as<S>();
        h.center = src.as<S>();
        h.tc = twist_A(k, mu);
        h.ac = 1.0;
        h.ah = -k2;
        h.to = twist_Ainv(k, mu);
        h.out = (op == TM_OP_NORMAL ? w : out.e).as<S>();
        TSM_TRY(launch_hop<S>(c, h, 0, HOP_CENTER, -1));
        src = (op == TM_OP_NORMAL) ? w : out.e;
      }
      if (op == TM_OP_NORMAL || dagger) {
        // Dhat^dag: u = A^-1(-mu) src ; t = A^-1(-mu) H^dag_oe u ; out = A(-mu) u - kappa^2 H^dag_eo t
        PField u;
        TSM_TRY(c.field("op_u", S::id, &u));
        TSM_TRY(launch_twist<S>(c, twist_Ainv(k, -mu), src, u, nullptr));
        HopArgs<S> h = hop_args<S>(c, 1);
        h.in = u.as<S>();
        h.out = t.as<S>();
        h.to = twist_Ainv(k, -mu);
        TSM_TRY(launch_hop<S>(c, h, 1, 0, -1));
        h = hop_args<S>(c, 0);
        h.in = t.as<S>();
        h.center = u.as<S>();
        h.tc = twist_A(k, -mu);
        h.ac = 1.0;
        h.ah = -k2;
        h.out = out.e.as<S>();
        TSM_TRY(launch_hop<S>(c, h, 1, HOP_CENTER, -1));
      }
      return zero(out.o);
    }
    default:
      return bad(TSM_ERR_ARG, "unknown operator");
  }
}


// ---------------------------------------------------------------- TSM runs
// state of one tsm_loops call: plan, per-source loop buffers and source /
// solution batches, all allocated before any work is recorded (so that the
// recording can also run under stream capture)
struct TsmRun {
  ContractPlan plan;
  NoiseSpec ns{};
  int E = 0, n_hp = 0, n_lp = 0, B = 1;
  int sp_lp = TSM_F32, sp_hp = TSM_F64;
  bool fp64_path = false;
  double2* d_corr = nullptr;
  double2* d_lp = nullptr;
  EOField b_lp, s_lp, b_hp, s_hp;
  bool branch = false;   // LP set recorded as a second graph branch
  EOField b_lp1, s_lp1;  // its source / solution batches
  bool fft = false;      // every spatial momentum: running moments instead of per-source values
  FftProjector fftp;
  ~TsmRun() { fftp.release(); }
};

int prepare_run(Ctx& c, const tsm_params* p, TsmRun* run, bool branch = false) {
  if (!c.has_gauge) return bad(TSM_ERR_NO_GAUGE, "no gauge field loaded");
  if (p->noise != 4 && p->noise != 2) return bad(TSM_ERR_ARG, "noise kind must be 4 or 2");
  if (p->hp_end < p->hp_begin || p->lp_end < p->lp_begin) return bad(TSM_ERR_ARG, "empty-reversed source range");
  if (p->batch < 1) return bad(TSM_ERR_ARG, "batch must be >= 1");
  TSM_TRY(check_stop(&p->hp));
  TSM_TRY(check_stop(&p->lp));
  if (p->estimator < 0 || p->estimator > 2) return bad(TSM_ERR_ARG, "estimator must be 0, 1 or 2");
  if (p->estimator == 2 && c.capturing)
    return bad(TSM_ERR_ARG, "the generalised one-end estimator runs eagerly (tsm_loops), not in a captured graph");
  if (p->deriv_mask < 0 || p->deriv_mask > 15) return bad(TSM_ERR_ARG, "deriv_mask must be in [0, 15]");
  if (p->deriv_mask && p->estimator != 0)
    return bad(TSM_ERR_ARG, "one-derivative insertions use the standard estimator (estimator 0)");
  if (p->all_momenta) {
    if (p->estimator != 0 || p->deriv_mask) return bad(TSM_ERR_ARG, "all_momenta uses the local standard estimator");
    if (c.capturing) return bad(TSM_ERR_ARG, "all_momenta runs eagerly (tsm_loops), not in a captured graph");
    if (p->gammas == nullptr) return bad(TSM_ERR_ARG, "gammas must be non-null");
    TSM_TRY(make_gamma_tab(p->gammas, p->n_gamma, &run->plan.gam));
    run->plan.ng = p->n_gamma;
    run->fft = true;
    run->E = p->n_gamma * c.g.V;
  } else {
    TSM_TRY(run->plan.prepare(c, p->gammas, p->n_gamma, p->moms, p->n_q));
    run->plan.one_end = p->estimator;
    run->plan.deriv_mask = p->deriv_mask;
    run->E = run->plan.entries(c.lat.L[3]);
  }
  run->n_hp = (int)(p->hp_end - p->hp_begin);
  run->n_lp = (int)(p->lp_end - p->lp_begin);
  run->sp_lp = loop_solution_prec(p->lp);
  run->sp_hp = solution_prec(p->hp);
  run->fp64_path = (p->lp.prec == TSM_F64 && p->hp.prec == TSM_F64);
  run->ns = make_noise(p->seed, p->noise);
  run->B = std::min(std::max(p->batch, 1), Ctx::kMaxBatch);
  c.batch_cap = std::max(c.batch_cap, run->B);
  void* vc = nullptr;
  void* vl = nullptr;
  const size_t per = run->fft ? 1 : (size_t)run->E;   // all momenta: no per-source values are kept
  TSM_TRY(c.buffer("tsm_per_corr", (size_t)std::max(run->n_hp, 1) * per * sizeof(double2), &vc));
  TSM_TRY(c.buffer("tsm_per_lp", (size_t)std::max(run->n_lp, 1) * per * sizeof(double2), &vl));
  run->d_corr = static_cast<double2*>(vc);
  run->d_lp = static_cast<double2*>(vl);
  if (run->fft) TSM_TRY(run->fftp.init(c, p->n_gamma, run->fp64_path));
  TSM_TRY(eo_fields(c, "tsm_b_lp", run->sp_lp, &run->b_lp, c.batch_cap));
  TSM_TRY(eo_fields(c, "tsm_s_lp", run->sp_lp, &run->s_lp, c.batch_cap));
  TSM_TRY(eo_fields(c, "tsm_b_hp", run->sp_hp, &run->b_hp, c.batch_cap));
  TSM_TRY(eo_fields(c, "tsm_s_hp", run->sp_hp, &run->s_hp, c.batch_cap));
  TSM_TRY(reserve_solver(c, p->lp, run->sp_lp));
  TSM_TRY(reserve_solver(c, p->hp));
  TSM_TRY(reserve_contract(c));
  run->branch = branch && run->n_hp > 0 && run->n_lp > 0;
  if (run->branch) {
    // the LP-set branch gets its own workspace and reduction slots
    c.ws_prefix = "branch1/";
    int rc = eo_fields(c, "tsm_b_lp", run->sp_lp, &run->b_lp1, c.batch_cap);
    if (rc == TSM_OK) rc = eo_fields(c, "tsm_s_lp", run->sp_lp, &run->s_lp1, c.batch_cap);
    if (rc == TSM_OK) rc = reserve_solver(c, p->lp, run->sp_lp);
    if (rc == TSM_OK) rc = reserve_contract(c);
    c.ws_prefix.clear();
    TSM_TRY(rc);
    if (c.red_branch.partials == nullptr || c.red_branch_cap != c.red_cap) {
      if (c.red_branch.partials) cudaFree(c.red_branch.partials);
      if (c.red_branch.counter) cudaFree(c.red_branch.counter);
      c.red_branch = RedSlot{};
      TSM_CUDA(cudaMalloc(&c.red_branch.partials, Ctx::kMaxBatch * c.red_cap * sizeof(double)));
      TSM_CUDA(cudaMalloc(&c.red_branch.counter, Ctx::kMaxBatch * sizeof(unsigned int)));
      TSM_CUDA(cudaMemset(c.red_branch.counter, 0, Ctx::kMaxBatch * sizeof(unsigned int)));
      c.red_branch.stride = (int)c.red_cap;
      c.red_branch_cap = c.red_cap;
    }
  }
  return TSM_OK;
}

// all work of one TSM estimate, in stream order; eager mode also collects the
// statistics (and verifies HP solutions if asked), capture mode records the
// solves' state ranges for reading after the graph ran
int record_run(Ctx& c, const tsm_params* p, TsmRun& run, tsm_loop_stats* st) {
  const int E = run.E, B = run.B, sp_lp = run.sp_lp, sp_hp = run.sp_hp;
  const NoiseSpec& ns = run.ns;
  *st = tsm_loop_stats{};
  st->lp_max_true_res = -1.0;
  st->hp_max_true_res = (p->verify && !c.capturing) ? 0.0 : -1.0;
  st->n_sources = run.n_hp + run.n_lp;
  // noise of sources j0 .. j0+n-1 into a batch of fields
  auto gen = [&](int prec, uint32_t j0, EOField f, int n) {
    return dispatch_prec(prec, [&](auto tag) {
      using S = decltype(tag);
      TSM_TRY(launch_noise<S>(c, 0, ns, j0, f.e, n));
      return launch_noise<S>(c, 1, ns, j0, f.o, n);
    });
  };
  auto contract_to = [&](uint32_t j, EOField a, int pa, const EOField* b, int pb, double2* out) {
    const ContractPlan& plan = run.plan;
    EOField wa{}, wb{};
    const EOField *pwa = nullptr, *pwb = nullptr;
    if (plan.one_end == CT_GEN_ONE_END) {
      // Eq. 2.6 needs D_W of each solution: one Wilson application per field
      TSM_TRY(eo_fields(c, "gen_wa", pa, &wa));
      TSM_TRY(apply_wilson(c, pa, a, wa));
      pwa = &wa;
      if (b != nullptr) {
        TSM_TRY(eo_fields(c, "gen_wb", pb, &wb));
        TSM_TRY(apply_wilson(c, pb, *b, wb));
        pwb = &wb;
      }
    }
    if (run.fp64_path) return launch_contract<double, F64, F64>(c, plan, ns, j, a, b, out, pwa, pwb);
    if (b == nullptr) pb = pa;
    if (pa == TSM_F64 && pb == TSM_F64) return launch_contract<float, F64, F64>(c, plan, ns, j, a, b, out, pwa, pwb);
    if (pa == TSM_F64 && pb == TSM_F32) return launch_contract<float, F64, F32>(c, plan, ns, j, a, b, out, pwa, pwb);
    if (pa == TSM_F64 && pb == TSM_F16) return launch_contract<float, F64, F16>(c, plan, ns, j, a, b, out, pwa, pwb);
    if (pa == TSM_F32 && pb == TSM_F32) return launch_contract<float, F32, F32>(c, plan, ns, j, a, b, out, pwa, pwb);
    if (pa == TSM_F32 && pb == TSM_F64) return launch_contract<float, F32, F64>(c, plan, ns, j, a, b, out, pwa, pwb);
    if (pa == TSM_F32 && pb == TSM_F16) return launch_contract<float, F32, F16>(c, plan, ns, j, a, b, out, pwa, pwb);
    if (pa == TSM_F16 && pb == TSM_F16) return launch_contract<float, F16, F16>(c, plan, ns, j, a, b, out, pwa, pwb);
    return bad(TSM_ERR_ARG, "no contraction for these field tiers");
  };
  // value of source j for set 0 (HP-set corrections) or 1 (LP set), idx-th of its set
  auto contract = [&](uint32_t j, EOField a, int pa, const EOField* b, int pb, int set, int idx) -> int {
    if (!run.fft) return contract_to(j, a, pa, b, pb, (set ? run.d_lp : run.d_corr) + (size_t)idx * E);
    FftProjector& f = run.fftp;
    const GammaTab& gam = run.plan.gam;
    if (run.fp64_path) return f.accumulate<double, F64, F64>(c, gam, ns, j, a, b, set, idx + 1);
    if (b == nullptr) pb = pa;
    if (pa == TSM_F64 && pb == TSM_F64) return f.accumulate<float, F64, F64>(c, gam, ns, j, a, b, set, idx + 1);
    if (pa == TSM_F64 && pb == TSM_F32) return f.accumulate<float, F64, F32>(c, gam, ns, j, a, b, set, idx + 1);
    if (pa == TSM_F64 && pb == TSM_F16) return f.accumulate<float, F64, F16>(c, gam, ns, j, a, b, set, idx + 1);
    if (pa == TSM_F32 && pb == TSM_F32) return f.accumulate<float, F32, F32>(c, gam, ns, j, a, b, set, idx + 1);
    if (pa == TSM_F32 && pb == TSM_F64) return f.accumulate<float, F32, F64>(c, gam, ns, j, a, b, set, idx + 1);
    if (pa == TSM_F32 && pb == TSM_F16) return f.accumulate<float, F32, F16>(c, gam, ns, j, a, b, set, idx + 1);
    if (pa == TSM_F16 && pb == TSM_F16) return f.accumulate<float, F16, F16>(c, gam, ns, j, a, b, set, idx + 1);
    return bad(TSM_ERR_ARG, "no momentum projection for these field tiers");
  };
  // state slots: fixed in eager mode, one fresh range per solve under capture
  auto slots = [&](int n, std::vector<std::pair<int, int>>& log) {
    if (!c.capturing) return 0;
    const int s0 = c.next_state;
    c.next_state += n;
    log.push_back({s0, n});
    return s0;
  };
  std::vector<SolveResult> r_lp(B), r_hp(B);
  const bool hp_first = !(c.capturing && run.branch);
  if (!hp_first) {
    // graph branch: the LP set runs beside the HP set (the FP64-heavy HP
    // solves and the 16-bit LP solves load different units of the GPU)
    TSM_CUDA(cudaEventRecord(c.fork_ev, c.stream));
    TSM_CUDA(cudaStreamWaitEvent(c.branch_stream, c.fork_ev, 0));
    cudaStream_t main_stream = c.stream;
    const RedSlot main_red = c.red;
    c.stream = c.branch_stream;
    c.red = c.red_branch;
    c.ws_prefix = "branch1/";
    std::vector<SolveResult> r_lp1(B);
    std::swap(r_lp, r_lp1);
    int rc = TSM_OK;
    for (uint32_t j0 = p->lp_begin; j0 < p->lp_end && rc == TSM_OK; j0 += B) {
      const int n = (int)std::min<uint32_t>(B, p->lp_end - j0);
      rc = gen(sp_lp, j0, run.b_lp1, n);
      if (rc == TSM_OK)
        rc = solve_batch(c, p->lp, slots(n, c.cap_lp), n, run.b_lp1, run.s_lp1, r_lp.data(), nullptr, -1, sp_lp);
      for (int r = 0; r < n && rc == TSM_OK; ++r)
        rc = contract(j0 + r, eo_at(run.s_lp1, sp_lp, c.g.Vh, r), sp_lp, nullptr, sp_lp, 1,
                      (int)(j0 + r - p->lp_begin));
    }
    std::swap(r_lp, r_lp1);
    if (rc == TSM_OK && cudaEventRecord(c.join_ev, c.stream) != cudaSuccess) rc = TSM_ERR_CUDA;
    c.stream = main_stream;
    c.red = main_red;
    c.ws_prefix.clear();
    TSM_TRY(rc);
  }
  // HP set: the LP map and the HP solve of every source, then L(s_HP - s_LP)
  for (uint32_t j0 = p->hp_begin; j0 < p->hp_end; j0 += B) {
    const int n = (int)std::min<uint32_t>(B, p->hp_end - j0);
    TSM_TRY(gen(sp_lp, j0, run.b_lp, n));
    TSM_TRY(solve_batch(c, p->lp, slots(n, c.cap_lp), n, run.b_lp, run.s_lp, r_lp.data(), nullptr, -1, sp_lp));
    if (sp_hp != sp_lp) TSM_TRY(gen(sp_hp, j0, run.b_hp, n));
    EOField bh = (sp_hp != sp_lp) ? run.b_hp : run.b_lp;
    // optional warm start of the HP solves from the LP solutions (the LP map
    // itself is untouched, so both sets keep the same LP solver)
    const bool warm = p->hp_warm_start && p->hp.prec == TSM_F32 && p->hp.reliable && !p->hp.precond;
    TSM_TRY(solve_batch(c, p->hp, slots(n, c.cap_hp), n, bh, run.s_hp, r_hp.data(), warm ? &run.s_lp.e : nullptr,
                        sp_lp));
    for (int r = 0; r < n; ++r) {
      if (!c.capturing) {
        if (r_lp[r].status != TSM_OK || r_hp[r].status != TSM_OK) return bad(TSM_ERR_NONFINITE, "NaN/Inf in a solve");
        if (p->verify) {
          double tr = 0.0;
          TSM_TRY(true_residual(c, sp_hp, eo_at(bh, sp_hp, c.g.Vh, r), eo_at(run.s_hp, sp_hp, c.g.Vh, r), &tr));
          st->hp_max_true_res = std::max(st->hp_max_true_res, tr);
        }
        st->lp_iters += r_lp[r].iters;
        st->hp_iters += r_hp[r].iters;
        if (!r_hp[r].converged) st->hp_not_converged++;
      }
      const EOField sl = eo_at(run.s_lp, sp_lp, c.g.Vh, r);
      TSM_TRY(contract(j0 + r, eo_at(run.s_hp, sp_hp, c.g.Vh, r), sp_hp, &sl, sp_lp, 0,
                       (int)(j0 + r - p->hp_begin)));
    }
  }
  // LP set: the same LP map, L(s_LP)
  auto lp_set = [&](EOField bl, EOField sl) -> int {
    for (uint32_t j0 = p->lp_begin; j0 < p->lp_end; j0 += B) {
      const int n = (int)std::min<uint32_t>(B, p->lp_end - j0);
      TSM_TRY(gen(sp_lp, j0, bl, n));
      TSM_TRY(solve_batch(c, p->lp, slots(n, c.cap_lp), n, bl, sl, r_lp.data(), nullptr, -1, sp_lp));
      for (int r = 0; r < n; ++r) {
        if (!c.capturing) {
          if (r_lp[r].status != TSM_OK) return bad(TSM_ERR_NONFINITE, "NaN/Inf in a solve");
          st->lp_iters += r_lp[r].iters;
        }
        TSM_TRY(contract(j0 + r, eo_at(sl, sp_lp, c.g.Vh, r), sp_lp, nullptr, sp_lp, 1,
                         (int)(j0 + r - p->lp_begin)));
      }
    }
    return TSM_OK;
  };
  if (!hp_first) {
    TSM_CUDA(cudaStreamWaitEvent(c.stream, c.join_ev, 0));   // join the LP-set branch
    return TSM_OK;
  }
  return lp_set(run.b_lp, run.s_lp);
}

}  // namespace

extern "C" {

const char* tsm_last_error(void) { return tsm::last_error(); }

const char* tsm_status_str(int s) {
  switch (s) {
    case TSM_OK: return "TSM_OK";
    case TSM_ERR_ARG: return "TSM_ERR_ARG";
    case TSM_ERR_DIMS: return "TSM_ERR_DIMS";
    case TSM_ERR_CUDA: return "TSM_ERR_CUDA";
    case TSM_ERR_NOT_CONVERGED: return "TSM_ERR_NOT_CONVERGED";
    case TSM_ERR_NONFINITE: return "TSM_ERR_NONFINITE";
    case TSM_ERR_TIMEOUT: return "TSM_ERR_TIMEOUT";
    case TSM_ERR_NOT_UNITARY: return "TSM_ERR_NOT_UNITARY";
    case TSM_ERR_NO_GAUGE: return "TSM_ERR_NO_GAUGE";
    case TSM_ERR_TOO_LARGE: return "TSM_ERR_TOO_LARGE";
    default: return "unknown status";
  }
}

int tsm_create(int device, void* cuda_stream, tsm_ctx** out) {
  if (out == nullptr) return bad(TSM_ERR_ARG, "null output handle");
  *out = nullptr;
  int n = 0;
  TSM_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return bad(TSM_ERR_ARG, "device index out of range");
  tsm_ctx* h = new (std::nothrow) tsm_ctx();
  if (h == nullptr) return bad(TSM_ERR_ARG, "out of host memory");
  Ctx& c = h->c;
  c.device = device;
  c.stream = static_cast<cudaStream_t>(cuda_stream);
  int rc = select_device(c);
  if (rc == TSM_OK && cudaMalloc(&c.states, Ctx::kMaxStates * sizeof(CGState)) != cudaSuccess) rc = TSM_ERR_CUDA;
  if (rc == TSM_OK && cudaMallocHost(&c.h_states, Ctx::kMaxStates * sizeof(CGState)) != cudaSuccess)
    rc = TSM_ERR_CUDA;
  if (rc == TSM_OK && cudaMalloc(&c.red.counter, Ctx::kMaxBatch * sizeof(unsigned int)) != cudaSuccess)
    rc = TSM_ERR_CUDA;
  if (rc == TSM_OK && cudaMemset(c.red.counter, 0, Ctx::kMaxBatch * sizeof(unsigned int)) != cudaSuccess)
    rc = TSM_ERR_CUDA;
  if (rc == TSM_OK && cudaMalloc(&c.d_lists, 3 * Ctx::kMaxBatch * sizeof(int)) != cudaSuccess) rc = TSM_ERR_CUDA;
  if (rc == TSM_OK && cudaMallocHost(&c.h_lists, 3 * Ctx::kMaxBatch * sizeof(int)) != cudaSuccess)
    rc = TSM_ERR_CUDA;
  if (rc == TSM_OK && cudaMalloc(&c.d_guard, Ctx::kMaxGuards * sizeof(int)) != cudaSuccess) rc = TSM_ERR_CUDA;
  if (rc == TSM_OK && cudaMemset(c.states, 0, Ctx::kMaxStates * sizeof(CGState)) != cudaSuccess) rc = TSM_ERR_CUDA;
  if (rc != TSM_OK) {
    set_error("tsm_create: device allocation failed");
    c.free_all();
    delete h;
    return rc;
  }
  *out = h;
  return TSM_OK;
}

int tsm_destroy(tsm_ctx* h) {
  if (h == nullptr) return TSM_OK;
  cudaSetDevice(h->c.device);
  h->c.free_all();
  delete h;
  return TSM_OK;
}

int tsm_load_gauge(tsm_ctx* h, const tm_lattice* lat, const double* U, int on_device) {
  if (h == nullptr || lat == nullptr || U == nullptr) return bad(TSM_ERR_ARG, "null argument");
  Ctx& c = h->c;
  TSM_TRY(select_device(c));
  long long V = 1;
  for (int k = 0; k < 4; ++k) {
    if (lat->L[k] < 2 || (lat->L[k] & 1)) return bad(TSM_ERR_DIMS, "every extent must be even and >= 2");
    V *= lat->L[k];
  }
  if (V * 4 >= (1ll << 31)) return bad(TSM_ERR_DIMS, "lattice too large for 32-bit site indexing");
  if (!std::isfinite(lat->kappa) || !std::isfinite(lat->mu)) return bad(TSM_ERR_ARG, "kappa / mu not finite");
  const bool resize = !c.has_gauge || (int)V != c.g.V;
  c.has_gauge = false;
  c.lat = *lat;
  c.g = make_geom(lat->L, lat->t_antiperiodic);
  c.sstride = c.g.Vh;
  c.lstride = c.g.Vh;
  if (resize) {
    TSM_CUDA(cudaStreamSynchronize(c.stream));
    for (auto& kv : c.ws) cudaFree(kv.second.first);
    c.ws.clear();
    for (int k = 0; k < 4; ++k) {
      if (c.links[k]) cudaFree(c.links[k]);
      c.links[k] = nullptr;
    }
    const size_t vh = (size_t)c.g.Vh;
    TSM_CUDA(cudaMalloc(&c.links[TSM_F64], 2 * 4 * F64::LN * vh * sizeof(double2)));
    TSM_CUDA(cudaMalloc(&c.links[TSM_F32], 2 * 4 * F32::LN * vh * sizeof(float4)));
    TSM_CUDA(cudaMalloc(&c.links[TSM_BF16], 2 * 4 * BF16::LN * vh * sizeof(uint2)));
    TSM_CUDA(cudaMalloc(&c.links[TSM_F16], 2 * 4 * F16::LN * vh * sizeof(uint2)));
    if (c.red.partials) cudaFree(c.red.partials);
    c.red_cap = vh / 32 + 64;   // block partials: up to one per 32 sites (link-sharing stencil)
    c.red.stride = (int)c.red_cap;
    TSM_CUDA(cudaMalloc(&c.red.partials, Ctx::kMaxBatch * c.red_cap * sizeof(double)));
    c.batch_cap = 1;
  }
  const double* dU = nullptr;
  TSM_TRY(stage_in(c, "gauge_canon", U, (size_t)V * 4 * 9 * 2 * sizeof(double), on_device, &dU));
  void* dev_max = nullptr;
  TSM_TRY(c.buffer("gauge_maxdev", sizeof(unsigned int), &dev_max));
  TSM_CUDA(cudaMemsetAsync(dev_max, 0, sizeof(unsigned int), c.stream));
  const int nb = (int)((V * 4 + SITE_NT - 1) / SITE_NT);
  pack_links_kernel<<<nb, SITE_NT, 0, c.stream>>>(
      c.g, reinterpret_cast<const double2*>(dU), static_cast<double2*>(c.links[TSM_F64]),
      static_cast<float4*>(c.links[TSM_F32]), static_cast<uint2*>(c.links[TSM_F16]),
      static_cast<uint2*>(c.links[TSM_BF16]), c.lstride, static_cast<unsigned int*>(dev_max));
  c.launches++;
  TSM_TRY(check_launch(c, "pack_links_kernel"));
  unsigned int bits = 0;
  TSM_CUDA(cudaMemcpyAsync(&bits, dev_max, sizeof(bits), cudaMemcpyDeviceToHost, c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  float dev;
  std::memcpy(&dev, &bits, sizeof(dev));
  if (!(dev <= 1e-8f)) {
    set_error("gauge links are not SU(3): max deviation %g", (double)dev);
    return TSM_ERR_NOT_UNITARY;
  }
  c.has_gauge = true;
  return TSM_OK;
}

int tm_dslash(tsm_ctx* h, int prec, int op, int dagger, const double* in, double* out, int on_device) {
  if (h == nullptr || in == nullptr || out == nullptr) return bad(TSM_ERR_ARG, "null argument");
  Ctx& c = h->c;
  if (!c.has_gauge) return bad(TSM_ERR_NO_GAUGE, "no gauge field loaded");
  if (op < TM_OP_FULL || op > TM_OP_NORMAL) return bad(TSM_ERR_ARG, "unknown operator");
  TSM_TRY(select_device(c));
  const size_t bytes = spinor_bytes(c);
  const double* din = nullptr;
  double* dout = nullptr;
  TSM_TRY(stage_in(c, "io_in", in, bytes, on_device, &din));
  TSM_TRY(stage_out_ptr(c, "io_out", out, bytes, on_device, &dout));
  EOField fi, fo;
  TSM_TRY(eo_fields(c, "ds_in", prec, &fi));
  TSM_TRY(eo_fields(c, "ds_out", prec, &fo));
  TSM_TRY(pack_eo(c, prec, din, fi));
  c.prof_this_launch = c.profile;
  c.hop_per_site = true;   // one field: the per-site stencil (no link sharing to exploit)
  int rc = dispatch_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    return apply_operator<S>(c, op, dagger ? 1 : 0, fi, fo);
  });
  c.hop_per_site = false;
  c.prof_this_launch = false;
  TSM_TRY(rc);
  TSM_TRY(unpack_eo(c, prec, fo, dout));
  TSM_TRY(stage_out_finish(c, out, dout, bytes, on_device));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  return c.harvest_events();
}

int tm_solve_batch(tsm_ctx* h, int nrhs, const double* b, double* s, const tm_stop* stop, int on_device, int* iters,
                   double* true_res) {
  if (h == nullptr || b == nullptr || s == nullptr) return bad(TSM_ERR_ARG, "null argument");
  if (nrhs < 0) return bad(TSM_ERR_ARG, "nrhs < 0");
  TSM_TRY(check_stop(stop));
  Ctx& c = h->c;
  if (!c.has_gauge) return bad(TSM_ERR_NO_GAUGE, "no gauge field loaded");
  TSM_TRY(select_device(c));
  const size_t bytes = spinor_bytes(c);
  const int sp = solution_prec(*stop);
  const int width = std::min(std::max(nrhs, 1), Ctx::kMaxBatch);
  c.batch_cap = std::max(c.batch_cap, width);
  EOField fb, fs;
  TSM_TRY(eo_fields(c, "sv_b", sp, &fb, c.batch_cap));
  TSM_TRY(eo_fields(c, "sv_s", sp, &fs, c.batch_cap));
  int worst = TSM_OK;
  std::vector<SolveResult> res(width);
  for (int r0 = 0; r0 < nrhs; r0 += width) {
    const int n = std::min(width, nrhs - r0);
    for (int r = 0; r < n; ++r) {
      const double* db = nullptr;
      TSM_TRY(stage_in(c, "io_in", b + (size_t)(r0 + r) * c.g.V * 24, bytes, on_device, &db));
      TSM_TRY(pack_eo(c, sp, db, eo_at(fb, sp, c.g.Vh, r)));
    }
    TSM_TRY(solve_batch(c, *stop, 0, n, fb, fs, res.data()));
    for (int r = 0; r < n; ++r) {
      const SolveResult& q = res[r];
      if (iters) iters[r0 + r] = q.iters;
      if (true_res) {
        double tr = 0.0;
        TSM_TRY(true_residual(c, sp, eo_at(fb, sp, c.g.Vh, r), eo_at(fs, sp, c.g.Vh, r), &tr));
        true_res[r0 + r] = tr;
      }
      double* ds = nullptr;
      TSM_TRY(stage_out_ptr(c, "io_out", s + (size_t)(r0 + r) * c.g.V * 24, bytes, on_device, &ds));
      TSM_TRY(unpack_eo(c, sp, eo_at(fs, sp, c.g.Vh, r), ds));
      TSM_TRY(stage_out_finish(c, s + (size_t)(r0 + r) * c.g.V * 24, ds, bytes, on_device));
      TSM_CUDA(cudaStreamSynchronize(c.stream));
      if (q.status != TSM_OK) worst = q.status;
      else if (!q.converged && worst == TSM_OK) worst = TSM_ERR_NOT_CONVERGED;
    }
  }
  TSM_TRY(c.harvest_events());
  if (worst != TSM_OK) set_error("at least one solve %s", worst == TSM_ERR_NONFINITE ? "met NaN/Inf" : "did not converge");
  return worst;
}

int tsm_noise(tsm_ctx* h, uint64_t seed, int kind, uint32_t source, double* out, int on_device) {
  if (h == nullptr || out == nullptr) return bad(TSM_ERR_ARG, "null argument");
  if (kind != 4 && kind != 2) return bad(TSM_ERR_ARG, "noise kind must be 4 or 2");
  Ctx& c = h->c;
  if (!c.has_gauge) return bad(TSM_ERR_NO_GAUGE, "no lattice loaded");
  TSM_TRY(select_device(c));
  const size_t bytes = spinor_bytes(c);
  double* dout = nullptr;
  TSM_TRY(stage_out_ptr(c, "io_out", out, bytes, on_device, &dout));
  noise_canon_kernel<<<(c.g.V + SITE_NT - 1) / SITE_NT, SITE_NT, 0, c.stream>>>(c.g.V, make_noise(seed, kind), source,
                                                                                reinterpret_cast<double2*>(dout));
  c.launches++;
  TSM_TRY(check_launch(c, "noise_canon_kernel"));
  TSM_TRY(stage_out_finish(c, out, dout, bytes, on_device));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  return TSM_OK;
}

static int contract_entry(tsm_ctx* h, int one_end, int prec, uint64_t seed, int kind, uint32_t source,
                          const double* s_a, const double* s_b, const int* gammas, int n_gamma, const int* moms,
                          int n_q, double* out, int on_device, int deriv_mask = 0) {
  if (h == nullptr || s_a == nullptr || out == nullptr) return bad(TSM_ERR_ARG, "null argument");
  if (kind != 4 && kind != 2) return bad(TSM_ERR_ARG, "noise kind must be 4 or 2");
  if (prec != TSM_F64 && prec != TSM_F32) return bad(TSM_ERR_ARG, "contraction tier must be TSM_F64 or TSM_F32");
  Ctx& c = h->c;
  if (!c.has_gauge) return bad(TSM_ERR_NO_GAUGE, "no lattice loaded");
  TSM_TRY(select_device(c));
  ContractPlan plan;
  TSM_TRY(plan.prepare(c, gammas, n_gamma, moms, n_q));
  plan.one_end = one_end;
  if (deriv_mask) {
    plan.local = 0;
    plan.deriv_mask = deriv_mask;
  }
  const size_t bytes = spinor_bytes(c);
  EOField fa, fb;
  TSM_TRY(eo_fields(c, "ct_a", TSM_F64, &fa));
  TSM_TRY(eo_fields(c, "ct_b", TSM_F64, &fb));
  const double* da = nullptr;
  TSM_TRY(stage_in(c, "io_in", s_a, bytes, on_device, &da));
  TSM_TRY(pack_eo(c, TSM_F64, da, fa));
  if (s_b) {
    const double* db = nullptr;
    TSM_TRY(stage_in(c, "io_in2", s_b, bytes, on_device, &db));
    TSM_TRY(pack_eo(c, TSM_F64, db, fb));
  }
  const size_t obytes = (size_t)plan.entries(c.lat.L[3]) * sizeof(double2);
  double* dout = nullptr;
  TSM_TRY(stage_out_ptr(c, "io_loops", out, obytes, on_device, &dout));
  const NoiseSpec ns = make_noise(seed, kind);
  EOField wa{}, wb{};
  if (one_end == CT_GEN_ONE_END) {
    TSM_TRY(eo_fields(c, "gen_wa", TSM_F64, &wa));
    TSM_TRY(apply_wilson(c, TSM_F64, fa, wa));
    if (s_b) {
      TSM_TRY(eo_fields(c, "gen_wb", TSM_F64, &wb));
      TSM_TRY(apply_wilson(c, TSM_F64, fb, wb));
    }
  }
  const EOField* pwa = one_end == CT_GEN_ONE_END ? &wa : nullptr;
  const EOField* pwb = (one_end == CT_GEN_ONE_END && s_b) ? &wb : nullptr;
  if (prec == TSM_F64)
    TSM_TRY((launch_contract<double, F64, F64>(c, plan, ns, source, fa, s_b ? &fb : nullptr,
                                               reinterpret_cast<double2*>(dout), pwa, pwb)));
  else
    TSM_TRY((launch_contract<float, F64, F64>(c, plan, ns, source, fa, s_b ? &fb : nullptr,
                                              reinterpret_cast<double2*>(dout), pwa, pwb)));
  TSM_TRY(stage_out_finish(c, out, dout, obytes, on_device));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  return TSM_OK;
}

int tsm_contract(tsm_ctx* h, int prec, uint64_t seed, int kind, uint32_t source, const double* s_a,
                 const double* s_b, const int* gammas, int n_gamma, const int* moms, int n_q, double* out,
                 int on_device) {
  return contract_entry(h, 0, prec, seed, kind, source, s_a, s_b, gammas, n_gamma, moms, n_q, out, on_device);
}

int tsm_contract_one_end(tsm_ctx* h, int prec, const double* s_a, const double* s_b, const int* gammas,
                         int n_gamma, const int* moms, int n_q, double* out, int on_device) {
  return contract_entry(h, CT_ONE_END, prec, 0, 4, 0, s_a, s_b, gammas, n_gamma, moms, n_q, out, on_device);
}

int tsm_contract_gen_one_end(tsm_ctx* h, int prec, const double* s_a, const double* s_b, const int* gammas,
                             int n_gamma, const int* moms, int n_q, double* out, int on_device) {
  return contract_entry(h, CT_GEN_ONE_END, prec, 0, 4, 0, s_a, s_b, gammas, n_gamma, moms, n_q, out, on_device);
}

int tsm_contract_fft(tsm_ctx* h, int prec, uint64_t seed, int kind, uint32_t source, const double* s_a,
                     const double* s_b, const int* gammas, int n_gamma, double* out, int on_device) {
  if (h == nullptr || s_a == nullptr || out == nullptr || gammas == nullptr) return bad(TSM_ERR_ARG, "null argument");
  if (kind != 4 && kind != 2) return bad(TSM_ERR_ARG, "noise kind must be 4 or 2");
  if (prec != TSM_F64 && prec != TSM_F32) return bad(TSM_ERR_ARG, "contraction tier must be TSM_F64 or TSM_F32");
  Ctx& c = h->c;
  if (!c.has_gauge) return bad(TSM_ERR_NO_GAUGE, "no lattice loaded");
  TSM_TRY(select_device(c));
  GammaTab gam{};
  TSM_TRY(make_gamma_tab(gammas, n_gamma, &gam));
  const size_t bytes = spinor_bytes(c);
  EOField fa, fb;
  TSM_TRY(eo_fields(c, "ct_a", TSM_F64, &fa));
  TSM_TRY(eo_fields(c, "ct_b", TSM_F64, &fb));
  const double* da = nullptr;
  TSM_TRY(stage_in(c, "io_in", s_a, bytes, on_device, &da));
  TSM_TRY(pack_eo(c, TSM_F64, da, fa));
  if (s_b) {
    const double* db = nullptr;
    TSM_TRY(stage_in(c, "io_in2", s_b, bytes, on_device, &db));
    TSM_TRY(pack_eo(c, TSM_F64, db, fb));
  }
  FftProjector f;
  int rc = f.init(c, n_gamma, prec == TSM_F64);
  const NoiseSpec ns = make_noise(seed, kind);
  if (rc == TSM_OK) {
    rc = prec == TSM_F64 ? f.transform<double, F64, F64>(c, gam, ns, source, fa, s_b ? &fb : nullptr)
                         : f.transform<float, F64, F64>(c, gam, ns, source, fa, s_b ? &fb : nullptr);
  }
  if (rc == TSM_OK) {
    // widen to complex double in the caller's layout [n_gamma][T][Lz][Ly][Lx]
    const size_t ob = (size_t)f.E * sizeof(double2);
    double* dout = nullptr;
    rc = stage_out_ptr(c, "io_fft", out, ob, on_device, &dout);
    if (rc == TSM_OK) {
      if (prec == TSM_F64) {
        if (cudaMemcpyAsync(dout, f.dens, ob, cudaMemcpyDeviceToDevice, c.stream) != cudaSuccess) rc = TSM_ERR_CUDA;
      } else {
        rc = launch_widen(c, static_cast<const float2*>(f.dens), reinterpret_cast<double2*>(dout), f.E);
      }
    }
    if (rc == TSM_OK) rc = stage_out_finish(c, out, dout, ob, on_device);
    if (rc == TSM_OK && cudaStreamSynchronize(c.stream) != cudaSuccess) rc = TSM_ERR_CUDA;
  }
  f.release();
  return rc;
}

int tsm_contract_deriv(tsm_ctx* h, int prec, uint64_t seed, int kind, uint32_t source, const double* s_a,
                       const double* s_b, const int* gammas, int n_gamma, int deriv_mask, const int* moms, int n_q,
                       double* out, int on_device) {
  if (deriv_mask < 1 || deriv_mask > 15) return bad(TSM_ERR_ARG, "deriv_mask must have bits among 0..3 set");
  return contract_entry(h, CT_STANDARD, prec, seed, kind, source, s_a, s_b, gammas, n_gamma, moms, n_q, out,
                        on_device, deriv_mask);
}

int tsm_loops(tsm_ctx* h, const tsm_params* p, double* loops, double* err, double* lp_mean, double* corr_mean,
              double* per_corr, double* per_lp, int on_device, tsm_loop_stats* stats) {
  if (h == nullptr || p == nullptr) return bad(TSM_ERR_ARG, "null argument");
  Ctx& c = h->c;
  TSM_TRY(select_device(c));
  if (p->all_momenta && (per_corr || per_lp))
    return bad(TSM_ERR_ARG, "all_momenta keeps no per-source values (per_corr / per_lp must be NULL)");
  TsmRun run;
  TSM_TRY(prepare_run(c, p, &run));
  tsm_loop_stats st{};
  TSM_TRY(record_run(c, p, run, &st));
  // Eq. 2.4 combine
  const int E = run.E, n_hp = run.n_hp, n_lp = run.n_lp;
  double *d_est = nullptr, *d_err = nullptr, *d_lpm = nullptr, *d_cm = nullptr;
  const size_t cb = (size_t)E * sizeof(double2), rb = (size_t)E * sizeof(double);
  if (loops) TSM_TRY(stage_out_ptr(c, "out_est", loops, cb, on_device, &d_est));
  if (err) TSM_TRY(stage_out_ptr(c, "out_err", err, rb, on_device, &d_err));
  if (lp_mean) TSM_TRY(stage_out_ptr(c, "out_lpm", lp_mean, cb, on_device, &d_lpm));
  if (corr_mean) TSM_TRY(stage_out_ptr(c, "out_cm", corr_mean, cb, on_device, &d_cm));
  if (run.fft)
    TSM_TRY(run.fftp.finalize(c, n_hp, n_lp, reinterpret_cast<double2*>(d_est), d_err,
                              reinterpret_cast<double2*>(d_lpm), reinterpret_cast<double2*>(d_cm)));
  else
    TSM_TRY(launch_combine(c, run.d_corr, n_hp, run.d_lp, n_lp, E, reinterpret_cast<double2*>(d_est), d_err,
                           reinterpret_cast<double2*>(d_lpm), reinterpret_cast<double2*>(d_cm)));
  if (loops) TSM_TRY(stage_out_finish(c, loops, d_est, cb, on_device));
  if (err) TSM_TRY(stage_out_finish(c, err, d_err, rb, on_device));
  if (lp_mean) TSM_TRY(stage_out_finish(c, lp_mean, d_lpm, cb, on_device));
  if (corr_mean) TSM_TRY(stage_out_finish(c, corr_mean, d_cm, cb, on_device));
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (per_corr && n_hp > 0) TSM_CUDA(cudaMemcpyAsync(per_corr, run.d_corr, (size_t)n_hp * cb, k, c.stream));
  if (per_lp && n_lp > 0) TSM_CUDA(cudaMemcpyAsync(per_lp, run.d_lp, (size_t)n_lp * cb, k, c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  TSM_TRY(c.harvest_events());
  if (stats) *stats = st;
  return TSM_OK;
}

int tsm_loops_graph(tsm_ctx** ctxs, const tsm_params* params, int n, double** loops, double** err,
                    double** per_corr, double** per_lp, tsm_loop_stats* stats) {
  if (ctxs == nullptr || params == nullptr || n < 1) return bad(TSM_ERR_ARG, "null argument or n < 1");
  for (int i = 0; i < n; ++i) {
    if (ctxs[i] == nullptr) return bad(TSM_ERR_ARG, "null context");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return bad(TSM_ERR_ARG, "a context appears twice");
    if (ctxs[i]->c.device != ctxs[0]->c.device) return bad(TSM_ERR_ARG, "contexts on different devices");
  }
  Ctx& c0 = ctxs[0]->c;
  TSM_TRY(select_device(c0));
  std::vector<TsmRun> runs(n);
  for (int i = 0; i < n; ++i) TSM_TRY(prepare_run(ctxs[i]->c, params + i, &runs[i], /*branch=*/true));
  for (int i = 0; i < n; ++i) TSM_CUDA(cudaStreamSynchronize(ctxs[i]->c.stream));
  // private streams for the capture (one branch per context + one for loop bodies)
  // own[0]: origin; per context i: own[1+3i] main branch, own[2+3i] loop
  // bodies, own[3+3i] LP-set branch; evs[n]: fork of the origin, evs[n+1+2i],
  // evs[n+2+2i]: fork / join of the LP-set branch of context i
  std::vector<cudaStream_t> own(3 * n + 1, nullptr);
  std::vector<cudaStream_t> saved(n);
  std::vector<cudaEvent_t> evs(3 * n + 1, nullptr);
  int rc = TSM_OK;
  auto cleanup = [&]() {
    for (int i = 0; i < n; ++i) {
      Ctx& c = ctxs[i]->c;
      if (own[1 + 3 * i]) c.stream = saved[i];
      c.capturing = false;
      c.body_stream = nullptr;
      c.branch_stream = nullptr;
      c.fork_ev = c.join_ev = nullptr;
    }
    for (auto s : own)
      if (s) cudaStreamDestroy(s);
    for (auto e : evs)
      if (e) cudaEventDestroy(e);
  };
  for (size_t k = 0; k < own.size() && rc == TSM_OK; ++k)
    if (cudaStreamCreateWithFlags(&own[k], cudaStreamNonBlocking) != cudaSuccess) rc = TSM_ERR_CUDA;
  for (size_t k = 0; k < evs.size() && rc == TSM_OK; ++k)
    if (cudaEventCreateWithFlags(&evs[k], cudaEventDisableTiming) != cudaSuccess) rc = TSM_ERR_CUDA;
  if (rc != TSM_OK) {
    cleanup();
    return bad(rc, "stream/event creation failed");
  }
  cudaStream_t origin = own[0];
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) rc = TSM_ERR_CUDA;
  if (rc == TSM_OK && cudaEventRecord(evs[n], origin) != cudaSuccess) rc = TSM_ERR_CUDA;
  std::vector<tsm_loop_stats> st(n);
  for (int i = 0; i < n && rc == TSM_OK; ++i) {
    Ctx& c = ctxs[i]->c;
    saved[i] = c.stream;
    c.stream = own[1 + 3 * i];
    c.body_stream = own[2 + 3 * i];
    c.branch_stream = own[3 + 3 * i];
    c.fork_ev = evs[n + 1 + 2 * i];
    c.join_ev = evs[n + 2 + 2 * i];
    c.capturing = true;
    c.next_state = 0;
    c.next_guard = 0;
    c.guard_body_launches.clear();
    c.cap_lp.clear();
    c.cap_hp.clear();
    if (cudaStreamWaitEvent(c.stream, evs[n], 0) != cudaSuccess) rc = TSM_ERR_CUDA;
    if (rc == TSM_OK) rc = record_run(c, params + i, runs[i], &st[i]);
    if (rc == TSM_OK) {
      const int E = runs[i].E;
      rc = launch_combine(c, runs[i].d_corr, runs[i].n_hp, runs[i].d_lp, runs[i].n_lp, E,
                          loops ? reinterpret_cast<double2*>(loops[i]) : nullptr, err ? err[i] : nullptr, nullptr,
                          nullptr);
    }
    const size_t cb = (size_t)runs[i].E * sizeof(double2);
    if (rc == TSM_OK && per_corr && per_corr[i] && runs[i].n_hp > 0 &&
        cudaMemcpyAsync(per_corr[i], runs[i].d_corr, runs[i].n_hp * cb, cudaMemcpyDeviceToDevice, c.stream) !=
            cudaSuccess)
      rc = TSM_ERR_CUDA;
    if (rc == TSM_OK && per_lp && per_lp[i] && runs[i].n_lp > 0 &&
        cudaMemcpyAsync(per_lp[i], runs[i].d_lp, runs[i].n_lp * cb, cudaMemcpyDeviceToDevice, c.stream) !=
            cudaSuccess)
      rc = TSM_ERR_CUDA;
    if (rc == TSM_OK && cudaEventRecord(evs[i], c.stream) != cudaSuccess) rc = TSM_ERR_CUDA;
    if (rc == TSM_OK && cudaStreamWaitEvent(origin, evs[i], 0) != cudaSuccess) rc = TSM_ERR_CUDA;
  }
  const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
  if (rc == TSM_OK && ec != cudaSuccess) {
    set_error("graph capture failed: %s", cudaGetErrorString(ec));
    rc = TSM_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  if (rc == TSM_OK) {
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    if (ei != cudaSuccess) {
      set_error("graph instantiation failed: %s", cudaGetErrorString(ei));
      rc = TSM_ERR_CUDA;
    }
  }
  for (int i = 0; i < n; ++i) {
    ctxs[i]->c.capturing = false;
    ctxs[i]->c.stream = saved[i];
  }
  if (rc == TSM_OK) {
    // launched on the first context's stream; completes before the call returns
    if (cudaGraphLaunch(exec, c0.stream) != cudaSuccess || cudaStreamSynchronize(c0.stream) != cudaSuccess) {
      set_error("graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = TSM_ERR_CUDA;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (rc == TSM_OK) {
    for (int i = 0; i < n; ++i) {
      Ctx& c = ctxs[i]->c;
      const int used = c.next_state;
      if (used > 0 &&
          cudaMemcpy(c.h_states, c.states, used * sizeof(CGState), cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = TSM_ERR_CUDA;
        break;
      }
      // launch count: every while-loop body ran as many rounds as its guard counted
      if (c.next_guard > 0) {
        std::vector<int> rounds(c.next_guard);
        if (cudaMemcpy(rounds.data(), c.d_guard, c.next_guard * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
          rc = TSM_ERR_CUDA;
          break;
        }
        for (int k = 0; k < c.next_guard && k < (int)c.guard_body_launches.size(); ++k)
          if (rounds[k] > 1) c.launches += (long long)c.guard_body_launches[k] * (rounds[k] - 1);
      }
      for (auto& r : c.cap_lp)
        for (int k = 0; k < r.second; ++k) {
          const CGState& q = c.h_states[r.first + k];
          st[i].lp_iters += q.iter;
          if (q.status != 0) rc = TSM_ERR_NONFINITE;
        }
      for (auto& r : c.cap_hp)
        for (int k = 0; k < r.second; ++k) {
          const CGState& q = c.h_states[r.first + k];
          st[i].hp_iters += q.iter;
          if (q.status != 0) rc = TSM_ERR_NONFINITE;
          const bool met = q.rr0 == 0.0 || (q.tol <= 0.0 ? q.iter >= q.max_iter
                                                         : !(std::sqrt(q.rr) >= q.tol * std::sqrt(q.rr0)));
          if (!met) st[i].hp_not_converged++;
        }
      if (stats) stats[i] = st[i];
    }
  }
  cleanup();
  if (rc == TSM_ERR_NONFINITE) set_error("NaN/Inf in a solve");
  return rc;
}

int tsm_combine(tsm_ctx* h, const double* per_corr, int n_hp, const double* per_lp, int n_lp, int n_entries,
                double* loops, double* err, double* lp_mean, double* corr_mean, int on_device) {
  if (h == nullptr || n_hp < 0 || n_lp < 0 || n_entries < 0) return bad(TSM_ERR_ARG, "bad argument");
  if ((n_hp > 0 && per_corr == nullptr) || (n_lp > 0 && per_lp == nullptr)) return bad(TSM_ERR_ARG, "null input");
  Ctx& c = h->c;
  TSM_TRY(select_device(c));
  const size_t cb = (size_t)n_entries * sizeof(double2), rb = (size_t)n_entries * sizeof(double);
  const double *dc = nullptr, *dl = nullptr;
  if (n_hp > 0) TSM_TRY(stage_in(c, "cmb_corr", per_corr, (size_t)n_hp * cb, on_device, &dc));
  if (n_lp > 0) TSM_TRY(stage_in(c, "cmb_lp", per_lp, (size_t)n_lp * cb, on_device, &dl));
  double *d_est = nullptr, *d_err = nullptr, *d_lpm = nullptr, *d_cm = nullptr;
  if (loops) TSM_TRY(stage_out_ptr(c, "out_est", loops, cb, on_device, &d_est));
  if (err) TSM_TRY(stage_out_ptr(c, "out_err", err, rb, on_device, &d_err));
  if (lp_mean) TSM_TRY(stage_out_ptr(c, "out_lpm", lp_mean, cb, on_device, &d_lpm));
  if (corr_mean) TSM_TRY(stage_out_ptr(c, "out_cm", corr_mean, cb, on_device, &d_cm));
  TSM_TRY(launch_combine(c, reinterpret_cast<const double2*>(dc), n_hp, reinterpret_cast<const double2*>(dl), n_lp,
                         n_entries, reinterpret_cast<double2*>(d_est), d_err, reinterpret_cast<double2*>(d_lpm),
                         reinterpret_cast<double2*>(d_cm)));
  if (loops) TSM_TRY(stage_out_finish(c, loops, d_est, cb, on_device));
  if (err) TSM_TRY(stage_out_finish(c, err, d_err, rb, on_device));
  if (lp_mean) TSM_TRY(stage_out_finish(c, lp_mean, d_lpm, cb, on_device));
  if (corr_mean) TSM_TRY(stage_out_finish(c, corr_mean, d_cm, cb, on_device));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  return TSM_OK;
}

int tsm_tune(tsm_ctx* h, const tm_stop* stop, int* best_batch, int* best_tile, int* best_regs, double* times_ms) {
  if (h == nullptr || best_batch == nullptr) return bad(TSM_ERR_ARG, "null argument");
  TSM_TRY(check_stop(stop));
  Ctx& c = h->c;
  if (!c.has_gauge) return bad(TSM_ERR_NO_GAUGE, "no gauge field loaded");
  TSM_TRY(select_device(c));
  char key[160];
  snprintf(key, sizeof(key), "%dx%dx%dx%d/p%d/r%d/t%g/m%d", c.lat.L[0], c.lat.L[1], c.lat.L[2], c.lat.L[3],
           stop->prec, stop->reliable, stop->rel_tol, stop->max_iter);
  const int cand[4] = {8, 16, 32, 64};
  // block shapes of the link-sharing stencil: sources per block x register budget
  constexpr int kShapes = 4;
  const int tiles[kShapes] = {2, 4, 8, 4};
  const int regs[kShapes] = {80, 80, 80, 96};
  // the link-sharing stencil (16-bit tiers; FP32 for its hops without a
  // reduction) has a block shape to choose; FP64 runs one thread per (source, site)
  const bool tiled = stop->prec == TSM_F16 || stop->prec == TSM_BF16 || stop->prec == TSM_F32;
  const int ntile = tiled ? kShapes : 1;
  auto ib = c.tuned_batch.find(key);
  auto it = c.tuned_rpb.find(key);
  if (ib != c.tuned_batch.end() && it != c.tuned_rpb.end() && times_ms == nullptr) {
    const int q = it->second;
    *best_batch = ib->second;
    if (best_tile) *best_tile = tiled ? tiles[q] : 1;
    if (best_regs) *best_regs = tiled ? regs[q] : 0;
    if (tiled) {
      c.tile_rpb[stop->prec] = tiles[q];
      c.tile_regs[stop->prec] = regs[q];
    }
    return TSM_OK;
  }
  const int sp = loop_solution_prec(*stop);   // the solves of the loop estimators
  c.batch_cap = std::max(c.batch_cap, cand[3]);
  EOField fb, fs;
  TSM_TRY(eo_fields(c, "tune_b", sp, &fb, c.batch_cap));
  TSM_TRY(eo_fields(c, "tune_s", sp, &fs, c.batch_cap));
  TSM_TRY(reserve_solver(c, *stop, sp));
  const NoiseSpec ns = make_noise(0x7475ull, 4);   // scratch sources, not part of any estimate
  cudaEvent_t e0, e1;
  TSM_CUDA(cudaEventCreate(&e0));
  TSM_CUDA(cudaEventCreate(&e1));
  std::vector<SolveResult> res(cand[3]);
  double best_t = 1e300;
  int best_w = cand[0], best_q = 1;
  const int saved_rpb = tiled ? c.tile_rpb[stop->prec] : 0, saved_regs = tiled ? c.tile_regs[stop->prec] : 0;
  int rc = TSM_OK;
  for (int k = 0; k < 4 && rc == TSM_OK; ++k) {
    const int w = cand[k];
    rc = dispatch_prec(sp, [&](auto tag) {
      using S = decltype(tag);
      TSM_TRY(launch_noise<S>(c, 0, ns, 0, fb.e, w));
      return launch_noise<S>(c, 1, ns, 0, fb.o, w);
    });
    for (int q = 0; q < ntile && rc == TSM_OK; ++q) {
      if (tiled) {
        c.tile_rpb[stop->prec] = tiles[q];
        c.tile_regs[stop->prec] = regs[q];
      }
      // one untimed solve to settle caches and clocks, then one timed
      rc = solve_batch(c, *stop, 0, w, fb, fs, res.data(), nullptr, -1, sp);
      if (rc != TSM_OK) break;
      if (cudaEventRecord(e0, c.stream) != cudaSuccess) rc = TSM_ERR_CUDA;
      if (rc == TSM_OK) rc = solve_batch(c, *stop, 0, w, fb, fs, res.data(), nullptr, -1, sp);
      if (rc == TSM_OK && cudaEventRecord(e1, c.stream) != cudaSuccess) rc = TSM_ERR_CUDA;
      if (rc == TSM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = TSM_ERR_CUDA;
      float ms = 0.f;
      if (rc == TSM_OK) cudaEventElapsedTime(&ms, e0, e1);
      const double per = ms / w;
      if (times_ms) times_ms[kShapes * k + q] = per;
      if (per < best_t) {
        best_t = per;
        best_w = w;
        best_q = q;
      }
    }
    if (times_ms && !tiled)
      for (int q = 1; q < kShapes; ++q) times_ms[kShapes * k + q] = 0.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TSM_OK) {
    if (tiled) {
      c.tile_rpb[stop->prec] = saved_rpb;
      c.tile_regs[stop->prec] = saved_regs;
    }
    return rc;
  }
  c.tuned_batch[key] = best_w;
  c.tuned_rpb[key] = best_q;
  if (tiled) {
    c.tile_rpb[stop->prec] = tiles[best_q];
    c.tile_regs[stop->prec] = regs[best_q];
  }
  *best_batch = best_w;
  if (best_tile) *best_tile = tiled ? tiles[best_q] : 1;
  if (best_regs) *best_regs = tiled ? regs[best_q] : 0;
  return TSM_OK;
}

int tsm_set_tile(tsm_ctx* h, int prec, int tile_sources, int max_regs) {
  if (h == nullptr) return bad(TSM_ERR_ARG, "null context");
  if (prec != TSM_F16 && prec != TSM_BF16 && prec != TSM_F32)
    return bad(TSM_ERR_ARG, "the FP64 tier has no link-sharing block shape");
  if (tile_sources != 2 && tile_sources != 4 && tile_sources != 8)
    return bad(TSM_ERR_ARG, "sources per block must be 2, 4 or 8");
  if (max_regs != 80 && !(max_regs == 96 && tile_sources == 4))
    return bad(TSM_ERR_ARG, "register budget must be 80, or 96 with 4 sources per block");
  h->c.tile_rpb[prec] = tile_sources;
  h->c.tile_regs[prec] = max_regs;
  return TSM_OK;
}

int tsm_tune_batch(tsm_ctx* h, const tm_stop* stop, int* best, double* times_ms) {
  if (best == nullptr) return bad(TSM_ERR_ARG, "null argument");
  double t[16];
  int tile = 0, regs = 0;
  TSM_TRY(tsm_tune(h, stop, best, &tile, &regs, times_ms ? t : nullptr));
  if (times_ms) {
    // per width: the best over the block shapes
    for (int k = 0; k < 4; ++k) {
      double m = 1e300;
      for (int q = 0; q < 4; ++q)
        if (t[4 * k + q] > 0.0 && t[4 * k + q] < m) m = t[4 * k + q];
      times_ms[k] = m;
    }
  }
  return TSM_OK;
}

int tsm_profile(tsm_ctx* h, int enable) {
  if (h == nullptr) return bad(TSM_ERR_ARG, "null context");
  Ctx& c = h->c;
  TSM_TRY(select_device(c));
  TSM_TRY(c.harvest_events());
  c.profile = enable != 0;
  if (enable) {
    for (int k = 0; k < Ctx::kProfBuckets; ++k) {
      c.prof_ms[k] = 0.0;
      c.prof_cnt[k] = 0;
      c.prof_bytes[k] = 0.0;
    }
  }
  return TSM_OK;
}

int tsm_profile_read(tsm_ctx* h, double ms[16], long long count[16], double bytes[16]) {
  if (h == nullptr) return bad(TSM_ERR_ARG, "null context");
  Ctx& c = h->c;
  TSM_TRY(select_device(c));
  TSM_TRY(c.harvest_events());
  for (int k = 0; k < 16; ++k) {   // the hop buckets (tsm_profile_read_ex: all)
    if (ms) ms[k] = c.prof_ms[k];
    if (count) count[k] = c.prof_cnt[k];
    if (bytes) bytes[k] = c.prof_bytes[k];
  }
  return TSM_OK;
}

int tsm_profile_read_ex(tsm_ctx* h, int n, double* ms, long long* count, double* bytes) {
  if (h == nullptr || n < 0) return bad(TSM_ERR_ARG, "null context or negative bucket count");
  Ctx& c = h->c;
  TSM_TRY(select_device(c));
  TSM_TRY(c.harvest_events());
  for (int k = 0; k < n; ++k) {
    const bool in = k < Ctx::kProfBuckets;
    if (ms) ms[k] = in ? c.prof_ms[k] : 0.0;
    if (count) count[k] = in ? c.prof_cnt[k] : 0;
    if (bytes) bytes[k] = in ? c.prof_bytes[k] : 0.0;
  }
  return TSM_OK;
}

long long tsm_launch_count(tsm_ctx* h) { return h ? h->c.launches : -1; }

}  // extern "C"
