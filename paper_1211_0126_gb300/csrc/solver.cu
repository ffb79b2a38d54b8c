// solver.cu -- CGNR on the even/odd Schur complement of D_tm.
//
// With A = 1 + 2 i kappa mu gamma_5 (site-local) the full system
//   [[A_ee, -kappa H_eo], [-kappa H_oe, A_oo]] s = b
// reduces to Dhat s_e = bhat_e with
//   Dhat   = 1 - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe,
//   bhat_e = A_ee^-1 (b_e + kappa H_eo A_oo^-1 b_o),   s_o = A_oo^-1 (b_o + kappa H_oe s_e),
// and CG runs on Dhat^dag Dhat s_e = Dhat^dag bhat_e from a zero start, where
//   Dhat^dag = 1 - kappa^2 (H^dag)_eo A_oo(-mu)^-1 (H^dag)_oe A_ee(-mu)^-1.
// One iteration is five kernels:
//   K1  t = A^-1(mu) H_oe p
//   K2  q = Dhat p = A^-1(mu) (A(mu) p - kappa^2 H_eo t);  <q, q>;  store w = A^-1(-mu) q
//   K3  t = A^-1(-mu) (H^dag)_oe w
//   K4  v = A(-mu) w - kappa^2 (H^dag)_eo t = Dhat^dag q;  r -= alpha v;  x += alpha p;  <r, r>
//   K5  p = r + beta p
// alpha, beta and the stopping rule are evaluated on the device by the last
// block of K2 / K4; once the rule is met every queued kernel returns at once,
// so the host only polls the state once per chunk of iterations.
#include <cmath>

#include "fields.cuh"
#include "solver.h"

namespace tsm {

int solution_prec(const tm_stop& stop) {
  if (stop.prec == TSM_F64) return TSM_F64;
  if (stop.prec == TSM_F32 && stop.reliable) return TSM_F64;
  return TSM_F32;
}

static int read_state(Ctx& c, int slot, CGState* out) {
  TSM_CUDA(cudaMemcpyAsync(c.h_states + slot, c.states + slot, sizeof(CGState), cudaMemcpyDeviceToHost, c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  *out = c.h_states[slot];
  return c.harvest_events();
}

// r = b - Dhat^dag Dhat x in FP64 (reliable update / true normal residual), <r,r> -> st->rr
static int normal_residual_f64(Ctx& c, PField x, PField b, PField r, CGState* st) {
  const double k = c.lat.kappa, mu = c.lat.mu, k2 = k * k;
  PField t, w;
  TSM_TRY(c.field("rel_t", TSM_F64, &t));
  TSM_TRY(c.field("rel_w", TSM_F64, &w));
  HopArgs<F64> h = hop_args<F64>(c, 1);
  h.in = x.as<F64>();
  h.out = t.as<F64>();
  h.to = twist_Ainv(k, mu);
  TSM_TRY(launch_hop<F64>(c, h, 0, 0, -1));
  h = hop_args<F64>(c, 0);
  h.in = t.as<F64>();
  h.center = x.as<F64>();
  h.tc = twist_A(k, mu);
  h.ac = 1.0;
  h.ah = -k2;
  h.to = twist_Ainv(k, mu);
  h.ts = twist_Ainv(k, -mu);
  h.out = w.as<F64>();
  TSM_TRY(launch_hop<F64>(c, h, 0, HOP_CENTER, -1));
  h = hop_args<F64>(c, 1);
  h.in = w.as<F64>();
  h.out = t.as<F64>();
  h.to = twist_Ainv(k, -mu);
  TSM_TRY(launch_hop<F64>(c, h, 1, 0, -1));
  h = hop_args<F64>(c, 0);
  h.in = t.as<F64>();
  h.center = w.as<F64>();
  h.tc = twist_A(k, -mu);
  h.ac = 1.0;
  h.ah = -k2;
  h.to = twist_scale(-1.0);
  h.base = b.as<F64>();
  h.out = r.as<F64>();
  h.st = st;
  h.post = POST_SETRR;
  return launch_hop<F64>(c, h, 1, HOP_CENTER | HOP_NORM | HOP_BASE, -1);
}

// S: sloppy storage (links, p, t, w); SA: storage of r and x; SP: source /
// solution storage (also used for bhat and the initial Dhat^dag bhat);
// REL: FP32 iterations with an FP64 solution and FP64 residual replacement.
template <class S, class SA, class SP, bool REL>
static int cg_solve(Ctx& c, const tm_stop& stop, int slot, EOField b, EOField s, SolveResult* res) {
  const double k = c.lat.kappa, mu = c.lat.mu, k2 = k * k;
  CGState* st = c.states + slot;
  const int pS = S::id, pA = SA::id, pP = SP::id;
  PField tmp_o, bhat, w0, t0, r0;
  TSM_TRY(c.field("cg_tmp_o", pP, &tmp_o));
  TSM_TRY(c.field("cg_bhat", pP, &bhat));
  TSM_TRY(c.field("cg_w0", pP, &w0));
  TSM_TRY(c.field("cg_t0", pP, &t0));
  TSM_TRY(c.field("cg_r0", pP, &r0));
  // bhat_e = A^-1 (b_e + kappa H_eo A^-1 b_o)
  TSM_TRY(launch_twist<SP>(c, twist_Ainv(k, mu), b.o, tmp_o, nullptr));
  {
    HopArgs<SP> h = hop_args<SP>(c, 0);
    h.in = tmp_o.as<SP>();
    h.center = b.e.as<SP>();
    h.ac = 1.0;
    h.ah = k;
    h.to = twist_Ainv(k, mu);
    h.out = bhat.as<SP>();
    TSM_TRY(launch_hop<SP>(c, h, 0, HOP_CENTER, -1));
  }
  // r0 = Dhat^dag bhat, <r0, r0> initialises the state
  state_init_kernel<<<1, 1, 0, c.stream>>>(st, stop.rel_tol, stop.max_iter);
  c.launches++;
  TSM_TRY(check_launch(c, "state_init_kernel"));
  TSM_TRY(launch_twist<SP>(c, twist_Ainv(k, -mu), bhat, w0, nullptr));
  {
    HopArgs<SP> h = hop_args<SP>(c, 1);
    h.in = w0.as<SP>();
    h.out = t0.as<SP>();
    h.to = twist_Ainv(k, -mu);
    TSM_TRY(launch_hop<SP>(c, h, 1, 0, -1));
    h = hop_args<SP>(c, 0);
    h.in = t0.as<SP>();
    h.center = w0.as<SP>();
    h.tc = twist_A(k, -mu);
    h.ac = 1.0;
    h.ah = -k2;
    h.out = r0.as<SP>();
    h.st = st;
    h.post = POST_INIT;
    TSM_TRY(launch_hop<SP>(c, h, 1, HOP_CENTER | HOP_NORM, -1));
  }
  PField p, t, w, r, x, x64, r64;
  TSM_TRY(c.field("cg_p", pS, &p));
  TSM_TRY(c.field("cg_t", pS, &t));
  TSM_TRY(c.field("cg_w", pS, &w));
  TSM_TRY(c.field("cg_r", pA, &r));
  TSM_TRY(c.field("cg_x", pA, &x));
  TSM_TRY((launch_convert<SP, SA>(c, r0, r)));
  TSM_TRY((launch_convert<SP, S>(c, r0, p)));
  TSM_TRY((launch_convert<SA, SA>(c, PField{}, x)));
  if constexpr (REL) {
    TSM_TRY(c.field("cg_x64", TSM_F64, &x64));
    TSM_TRY(c.field("cg_r64", TSM_F64, &r64));
    TSM_TRY((launch_convert<F64, F64>(c, PField{}, x64)));
  }
  CGState hs{};
  TSM_TRY(read_state(c, slot, &hs));
  const double delta = (stop.reliable_delta > 0.0) ? stop.reliable_delta : 0.1;
  double rr_ref = hs.rr0;
  const int chunk = 8;
  long long launched = 0;   // guards the host loop against a state that stops advancing
  while (!hs.done && hs.status == 0) {
    if (launched > (long long)stop.max_iter + 64) {
      set_error("solver state stopped advancing after %lld iterations", launched);
      return TSM_ERR_CUDA;
    }
    int m = chunk;
    if (stop.max_iter - hs.iter < m) m = stop.max_iter - hs.iter;
    if (m < 1) m = 1;
    launched += m;
    for (int it = 0; it < m; ++it) {
      c.prof_this_launch = c.profile && it == 0;
      HopArgs<S> h = hop_args<S>(c, 1);   // K1
      h.in = p.as<S>();
      h.out = t.as<S>();
      h.to = twist_Ainv(k, mu);
      h.skip = st;
      TSM_TRY(launch_hop<S>(c, h, 0, 0, PK_HOP));
      h = hop_args<S>(c, 0);              // K2
      h.in = t.as<S>();
      h.center = p.as<S>();
      h.tc = twist_A(k, mu);
      h.ac = 1.0;
      h.ah = -k2;
      h.to = twist_Ainv(k, mu);
      h.ts = twist_Ainv(k, -mu);
      h.out = w.as<S>();
      h.skip = st;
      h.st = st;
      h.post = POST_ALPHA;
      TSM_TRY(launch_hop<S>(c, h, 0, HOP_CENTER | HOP_NORM, PK_HOP_XPAY));
      h = hop_args<S>(c, 1);              // K3
      h.in = w.as<S>();
      h.out = t.as<S>();
      h.to = twist_Ainv(k, -mu);
      h.skip = st;
      TSM_TRY(launch_hop<S>(c, h, 1, 0, PK_HOP_DAG));
      CGUpdArgs<S, SA> u{};               // K4
      u.g = c.g;
      u.Ue = c.links_of<S>(0);
      u.Uo = c.links_of<S>(1);
      u.lstride = c.lstride;
      u.t = t.as<S>();
      u.w = w.as<S>();
      u.p = p.as<S>();
      u.r = r.as<SA>();
      u.x = x.as<SA>();
      u.sstride = c.sstride;
      u.kappa2 = k2;
      u.tw = twist_A(k, -mu);
      u.st = st;
      u.red = c.red;
      TSM_TRY((launch_cg_update<S, SA>(c, u)));
      c.prof_this_launch = false;
      TSM_TRY((launch_cg_p<S, SA>(c, r, p, st)));   // K5
    }
    c.prof_this_launch = false;
    TSM_TRY(read_state(c, slot, &hs));
    if (hs.status != 0) break;
    if constexpr (REL) {
      if (hs.done || hs.rr < delta * delta * rr_ref) {
        // reliable update: fold the FP32 increment into the FP64 solution and
        // replace the iterated residual by the true FP64 normal residual
        const int nb = (c.g.Vh + SITE_NT - 1) / SITE_NT;
        accumulate_solution_kernel<<<nb, SITE_NT, 0, c.stream>>>(c.g.Vh, x.as<F32>(), x64.as<F64>(), c.sstride);
        c.launches++;
        TSM_TRY(check_launch(c, "accumulate_solution_kernel"));
        TSM_TRY(normal_residual_f64(c, x64, r0, r64, st));
        TSM_TRY((launch_convert<F64, F32>(c, r64, r)));
        TSM_TRY(read_state(c, slot, &hs));
        rr_ref = hs.rr;
        if (hs.done) {
          const bool met = !(std::sqrt(hs.rr) >= stop.rel_tol * std::sqrt(hs.rr0));
          if (met || hs.iter >= stop.max_iter || hs.status != 0) break;
          state_resume_kernel<<<1, 1, 0, c.stream>>>(st);
          c.launches++;
          TSM_TRY(check_launch(c, "state_resume_kernel"));
          TSM_TRY(read_state(c, slot, &hs));
        }
      }
    }
  }
  // solution: even part from CG, odd part reconstructed
  if constexpr (REL) {
    TSM_TRY((launch_convert<F64, SP>(c, x64, s.e)));
  } else {
    TSM_TRY((launch_convert<SA, SP>(c, x, s.e)));
  }
  {
    HopArgs<SP> h = hop_args<SP>(c, 1);
    h.in = s.e.as<SP>();
    h.center = b.o.as<SP>();
    h.ac = 1.0;
    h.ah = k;
    h.to = twist_Ainv(k, mu);
    h.out = s.o.as<SP>();
    TSM_TRY(launch_hop<SP>(c, h, 0, HOP_CENTER, -1));
  }
  res->iters = hs.iter;
  res->status = hs.status == 0 ? TSM_OK : TSM_ERR_NONFINITE;
  res->rel_res = hs.rr0 > 0 ? std::sqrt(hs.rr / hs.rr0) : 0.0;
  if (hs.rr0 == 0.0) res->converged = 1;
  else if (stop.rel_tol <= 0.0) res->converged = hs.iter >= stop.max_iter;
  else res->converged = !(std::sqrt(hs.rr) >= stop.rel_tol * std::sqrt(hs.rr0));
  return TSM_OK;
}

int solve_source(Ctx& c, const tm_stop& stop, int slot, EOField b, EOField s, SolveResult* res) {
  if (slot < 0 || slot >= Ctx::kMaxStates - 4) return TSM_ERR_ARG;
  switch (stop.prec) {
    case TSM_F64: return cg_solve<F64, F64, F64, false>(c, stop, slot, b, s, res);
    case TSM_F32:
      if (stop.reliable) return cg_solve<F32, F32, F64, true>(c, stop, slot, b, s, res);
      return cg_solve<F32, F32, F32, false>(c, stop, slot, b, s, res);
    case TSM_F16: return cg_solve<F16, F32, F32, false>(c, stop, slot, b, s, res);
    case TSM_BF16: return cg_solve<BF16, F32, F32, false>(c, stop, slot, b, s, res);
    default: set_error("unknown solver tier %d", stop.prec); return TSM_ERR_ARG;
  }
}

int true_residual(Ctx& c, int prec, EOField b, EOField s, double* out) {
  const double k = c.lat.kappa, mu = c.lat.mu;
  EOField b64 = b, s64 = s;
  if (prec != TSM_F64) {
    TSM_TRY(c.field("tr_be", TSM_F64, &b64.e));
    TSM_TRY(c.field("tr_bo", TSM_F64, &b64.o));
    TSM_TRY(c.field("tr_se", TSM_F64, &s64.e));
    TSM_TRY(c.field("tr_so", TSM_F64, &s64.o));
    TSM_TRY((launch_convert<F32, F64>(c, b.e, b64.e)));
    TSM_TRY((launch_convert<F32, F64>(c, b.o, b64.o)));
    TSM_TRY((launch_convert<F32, F64>(c, s.e, s64.e)));
    TSM_TRY((launch_convert<F32, F64>(c, s.o, s64.o)));
  }
  PField tmp;
  TSM_TRY(c.field("tr_tmp", TSM_F64, &tmp));
  CGState* aux = c.states + (Ctx::kMaxStates - 4);
  for (int par = 0; par < 2; ++par) {
    // r_p = b_p - (A s_p - kappa H s_{1-p})
    HopArgs<F64> h = hop_args<F64>(c, par);
    h.in = (par ? s64.e : s64.o).as<F64>();
    h.center = (par ? s64.o : s64.e).as<F64>();
    h.tc = twist_A(k, mu);
    h.ac = 1.0;
    h.ah = -k;
    h.to = twist_scale(-1.0);
    h.base = (par ? b64.o : b64.e).as<F64>();
    h.out = tmp.as<F64>();
    h.st = aux + par;
    h.post = POST_NONE;
    TSM_TRY(launch_hop<F64>(c, h, 0, HOP_CENTER | HOP_NORM | HOP_BASE, -1));
    TSM_TRY(launch_norm<F64>(c, par ? b64.o : b64.e, aux + 2 + par, POST_NONE));
  }
  TSM_CUDA(cudaMemcpyAsync(c.h_states + (Ctx::kMaxStates - 4), aux, 4 * sizeof(CGState), cudaMemcpyDeviceToHost,
                           c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  const CGState* hs = c.h_states + (Ctx::kMaxStates - 4);
  const double nr = hs[0].aux + hs[1].aux, nb = hs[2].aux + hs[3].aux;
  *out = nb > 0 ? std::sqrt(nr / nb) : std::sqrt(nr);
  return TSM_OK;
}

}  // namespace tsm
