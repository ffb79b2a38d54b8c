// solver.cu -- CGNR on the even/odd Schur complement of D_tm, for a batch of
// independent right-hand sides.
//
// With A = 1 + 2 i kappa mu gamma_5 (site-local) the full system
//   [[A_ee, -kappa H_eo], [-kappa H_oe, A_oo]] s = b
// reduces to Dhat s_e = bhat_e with
//   Dhat   = 1 - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe,
//   bhat_e = A_ee^-1 (b_e + kappa H_eo A_oo^-1 b_o),   s_o = A_oo^-1 (b_o + kappa H_oe s_e),
// and CG runs on Dhat^dag Dhat s_e = Dhat^dag bhat_e from a zero start, where
//   Dhat^dag = 1 - kappa^2 (H^dag)_eo A_oo(-mu)^-1 (H^dag)_oe A_ee(-mu)^-1.
// One iteration is five kernels, each over all right-hand sides still iterating:
//   K1  t = A^-1(mu) H_oe p
//   K2  q = Dhat p = A^-1(mu) (A(mu) p - kappa^2 H_eo t);  <q, q>;  store w = A^-1(-mu) q
//   K3  t = A^-1(-mu) (H^dag)_oe w
//   K4  v = A(-mu) w - kappa^2 (H^dag)_eo t = Dhat^dag q;  r -= alpha v;  x += alpha p;  <r, r>
//   K5  p = r + beta p
// alpha, beta and the stopping rule of every right-hand side are evaluated on
// the device by the last block of K2 / K4 for that right-hand side; once its
// rule is met every queued kernel skips it, so its iterates freeze exactly at
// that iteration.  The host polls the states once per chunk of iterations and
// leaves converged right-hand sides out of the following launches.  The
// arithmetic of one right-hand side (including every reduction order) does not
// depend on the others, so a batched solve gives the same bits as a
// single-source one.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <vector>

#include "fields.cuh"
#include "solver.h"
#include "net.h"

namespace tsm {

int solution_prec(const tm_stop& stop) {
  if (stop.prec == TSM_F64) return TSM_F64;
  if (stop.prec == TSM_F32 && stop.reliable) return TSM_F64;
  return TSM_F32;
}

int loop_solution_prec(const tm_stop& stop) {
  if (stop.prec == TSM_F16 && !stop.precond) return TSM_F16;
  return solution_prec(stop);
}

static int read_states(Ctx& c, int s0, int n, std::vector<CGState>& out) {
  TSM_CUDA(cudaMemcpyAsync(c.h_states + s0, c.states + s0, n * sizeof(CGState), cudaMemcpyDeviceToHost, c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  out.assign(c.h_states + s0, c.h_states + s0 + n);
  return c.harvest_events();
}

// copy a host list of right-hand-side indices to device list `which` (0..2)
static int upload_list(Ctx& c, int which, const std::vector<int>& list, const int** dev) {
  int* h = c.h_lists + which * Ctx::kMaxBatch;
  for (size_t k = 0; k < list.size(); ++k) h[k] = list[k];
  int* d = c.d_lists + which * Ctx::kMaxBatch;
  if (!list.empty())
    TSM_CUDA(cudaMemcpyAsync(d, h, list.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  *dev = d;
  return TSM_OK;
}

// Residual replacement of a reliable update, for the listed right-hand sides
// that have one pending (st[rhs].need_rel): the true residual of the Schur
// system bhat - Dhat x is formed in FP64 from the FP64 solution (the only
// place where cancellation makes FP64 necessary), then the normal residual
// r = Dhat^dag (bhat - Dhat x) is applied in FP32 into the iterated residual
// r32, with <r, r> -> st[rhs].rr (POST_SETRR).  Two FP64 and two FP32 hops.
static int normal_residual_mixed(Ctx& c, PField x, PField bhat, PField r32, CGState* st, const int* list, int n) {
  const double k = c.lat.kappa, mu = c.lat.mu, k2 = k * k;
  PField t64, u64, u32, t32;
  TSM_TRY(c.field("rel_t", TSM_F64, &t64, c.batch_cap));
  TSM_TRY(c.field("rel_w", TSM_F64, &u64, c.batch_cap));
  TSM_TRY(c.field("rel_u32", TSM_F32, &u32, c.batch_cap));
  TSM_TRY(c.field("rel_t32", TSM_F32, &t32, c.batch_cap));
  HopArgs<F64> h = hop_args<F64>(c, 1);   // t = A^-1 H_oe x
  h.active = list;
  h.skip = st;
  h.skip_rel = 1;
  h.in = x.as<F64>();
  h.out = t64.as<F64>();
  h.to = twist_Ainv(k, mu);
  TSM_TRY(launch_hop<F64>(c, h, 0, 0, -1, n));
  Twist neg = twist_Ainv(k, mu);           // -A^-1
  for (int q = 0; q < 2; ++q) {
    neg.re[q] = -neg.re[q];
    neg.im[q] = -neg.im[q];
  }
  h = hop_args<F64>(c, 0);                 // u = A^-1(-mu) (bhat - Dhat x)
  h.active = list;
  h.skip = st;
  h.skip_rel = 1;
  h.in = t64.as<F64>();
  h.center = x.as<F64>();
  h.tc = twist_A(k, mu);
  h.ac = 1.0;
  h.ah = -k2;
  h.to = neg;
  h.base = bhat.as<F64>();
  h.ts = twist_Ainv(k, -mu);
  h.out = u64.as<F64>();
  h.st = nullptr;                          // the norm of this variant is not used
  TSM_TRY(launch_hop<F64>(c, h, 0, HOP_CENTER | HOP_NORM | HOP_BASE, -1, n));
  const int blocks = (c.g.Vh + SITE_NT - 1) / SITE_NT;
  rel_narrow_kernel<<<dim3(n, blocks), SITE_NT, 0, c.stream>>>(c.g.Vh, u64.as<F64>(), u32.as<F32>(), c.sstride,
                                                                list, st);
  c.launches++;
  TSM_TRY(check_launch(c, "rel_narrow_kernel"));
  HopArgs<F32> g = hop_args<F32>(c, 1);    // t = A^-1(-mu) H^dag_oe u
  g.active = list;
  g.skip = st;
  g.skip_rel = 1;
  g.in = u32.as<F32>();
  g.out = t32.as<F32>();
  g.to = twist_Ainv(k, -mu);
  TSM_TRY(launch_hop<F32>(c, g, 1, 0, -1, n));
  g = hop_args<F32>(c, 0);                 // r = A(-mu) u - kappa^2 H^dag_eo t
  g.active = list;
  g.skip = st;
  g.skip_rel = 1;
  g.in = t32.as<F32>();
  g.center = u32.as<F32>();
  g.tc = twist_A(k, -mu);
  g.ac = 1.0;
  g.ah = -k2;
  g.out = r32.as<F32>();
  g.st = st;
  g.post = POST_SETRR;
  return launch_hop<F32>(c, g, 1, HOP_CENTER | HOP_NORM, -1, n);
}

// Graph while-loop over one batched solve: the condition starts at 1 (the body
// runs at least once), and while_cond_kernel clears it once no source of the
// batch is iterating (or after a guard of max_iter + 8 rounds).
static __global__ void while_cond_kernel(const CGState* st, int n, cudaGraphConditionalHandle h, int* guard,
                                         int max_rounds) {
  if (threadIdx.x != 0) return;
  bool any = false;
  for (int k = 0; k < n; ++k)
    if (!st[k].done && st[k].status == 0) any = true;
  const int g = ++(*guard);
  if (!any || g >= max_rounds) cudaGraphSetConditional(h, 0);
}

template <class Body>
static int capture_while(Ctx& c, CGState* st, int n, int max_iter, Body&& body) {
  if (c.next_guard >= Ctx::kMaxGuards) {
    set_error("more than %d solves in one captured graph", Ctx::kMaxGuards);
    return TSM_ERR_TOO_LARGE;
  }
  int* guard = c.d_guard + c.next_guard++;
  TSM_CUDA(cudaMemsetAsync(guard, 0, sizeof(int), c.stream));
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  TSM_CUDA(cudaStreamGetCaptureInfo(c.stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) {
    set_error("graph mode without an active stream capture");
    return TSM_ERR_ARG;
  }
  cudaGraphConditionalHandle h;
  TSM_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  TSM_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  TSM_CUDA(cudaStreamUpdateCaptureDependencies(c.stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  TSM_CUDA(cudaStreamBeginCaptureToGraph(c.body_stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  cudaStream_t outer = c.stream;
  c.stream = c.body_stream;
  const long long launches0 = c.launches;
  int rc = body();
  if (rc == TSM_OK) {
    while_cond_kernel<<<1, 32, 0, c.stream>>>(st, n, h, guard, max_iter + 8);
    c.launches++;
    rc = check_launch(c, "while_cond_kernel");
  }
  // the body is counted once here; the graph's caller adds the rounds it ran
  c.guard_body_launches.push_back((int)(c.launches - launches0));
  c.stream = outer;
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c.body_stream, &captured);
  if (rc != TSM_OK) return rc;
  if (e != cudaSuccess) {
    set_error("capture of a while-loop body failed: %s", cudaGetErrorString(e));
    return TSM_ERR_CUDA;
  }
  return TSM_OK;
}

// S: sloppy storage (links, p, t, w); SA: storage of r and x; SP: source /
// solution storage (also used for bhat and the initial Dhat^dag bhat);
// REL: FP32 iterations with an FP64 solution and FP64 residual replacement.
template <class S, class SA, class SP, bool REL>
static int cg_solve(Ctx& c, const tm_stop& stop, int s0, int nrhs, EOField b, EOField s, SolveResult* res,
                    const PField* x0, int x0_prec) {
  const double k = c.lat.kappa, mu = c.lat.mu, k2 = k * k;
  CGState* st = c.states + s0;
  const int pS = S::id, pA = SA::id, pP = SP::id;
  const int nb = c.batch_cap;
  // DIRECT: r and x share the solution's storage tier, so D-hat^dag bhat is
  // written straight into r and x accumulates in the even half of s (no copies)
  constexpr bool DIRECT = !REL && std::is_same<SA, SP>::value;
  PField tmp_o, bhat, w0, t0, r0;
  TSM_TRY(c.field("cg_tmp_o", pP, &tmp_o, nb));
  TSM_TRY(c.field("cg_w0", pP, &w0, nb));
  TSM_TRY(c.field("cg_t0", pP, &t0, nb));
  // bhat_e = A^-1 (b_e + kappa H_eo A^-1 b_o).  Only the reliable updates use
  // bhat itself; otherwise the hop writes w0 = A(-mu)^-1 bhat at once (the two
  // site-local factors multiply to the real 1 / (1 + 4 kappa^2 mu^2))
  TSM_TRY(launch_twist<SP>(c, twist_Ainv(k, mu), b.o, tmp_o, nullptr, nullptr, nrhs));
  if constexpr (REL) TSM_TRY(c.field("cg_bhat", pP, &bhat, nb));
  {
    HopArgs<SP> h = hop_args<SP>(c, 0);
    h.in = tmp_o.as<SP>();
    h.center = b.e.as<SP>();
    h.ac = 1.0;
    h.ah = k;
    h.to = REL ? twist_Ainv(k, mu) : twist_mul(twist_Ainv(k, -mu), twist_Ainv(k, mu));
    h.out = REL ? bhat.as<SP>() : w0.as<SP>();
    TSM_TRY(launch_hop<SP>(c, h, 0, HOP_CENTER, -1, nrhs));
  }
  // r0 = Dhat^dag bhat, <r0, r0> initialises the states
  const double delta = (stop.reliable_delta > 0.0) ? stop.reliable_delta : 0.1;
  state_init_kernel<<<1, Ctx::kMaxBatch, 0, c.stream>>>(st, nrhs, stop.rel_tol, stop.max_iter, REL ? 1 : 0,
                                                         delta * delta);
  c.launches++;
  TSM_TRY(check_launch(c, "state_init_kernel"));
  // r0 is written straight into r when the tiers allow it
  constexpr bool R0_IN_R = DIRECT || REL;
  if constexpr (R0_IN_R) TSM_TRY(c.field("cg_r", pA, &r0, nb));
  else TSM_TRY(c.field("cg_r0", pP, &r0, nb));
  if constexpr (REL) {
    // A(-mu)^-1 bhat in FP64, rounded once to FP32, then Dhat^dag in FP32: the
    // mixed form of the normal residual of every reliable update (x = 0 here)
    PField u32, t32;
    TSM_TRY(c.field("rel_u32", TSM_F32, &u32, nb));
    TSM_TRY(c.field("rel_t32", TSM_F32, &t32, nb));
    TSM_TRY(launch_twist<SP>(c, twist_Ainv(k, -mu), bhat, w0, nullptr, nullptr, nrhs));
    TSM_TRY((launch_convert<SP, F32>(c, w0, u32, nullptr, nrhs)));
    HopArgs<F32> h = hop_args<F32>(c, 1);
    h.in = u32.as<F32>();
    h.out = t32.as<F32>();
    h.to = twist_Ainv(k, -mu);
    TSM_TRY(launch_hop<F32>(c, h, 1, 0, -1, nrhs));
    h = hop_args<F32>(c, 0);
    h.in = t32.as<F32>();
    h.center = u32.as<F32>();
    h.tc = twist_A(k, -mu);
    h.ac = 1.0;
    h.ah = -k2;
    h.out = r0.as<F32>();
    h.st = st;
    h.post = POST_INIT;
    TSM_TRY(launch_hop<F32>(c, h, 1, HOP_CENTER | HOP_NORM, -1, nrhs));
  } else {
    HopArgs<SP> h = hop_args<SP>(c, 1);
    h.in = w0.as<SP>();
    h.out = t0.as<SP>();
    h.to = twist_Ainv(k, -mu);
    TSM_TRY(launch_hop<SP>(c, h, 1, 0, -1, nrhs));
    h = hop_args<SP>(c, 0);
    h.in = t0.as<SP>();
    h.center = w0.as<SP>();
    h.tc = twist_A(k, -mu);
    h.ac = 1.0;
    h.ah = -k2;
    h.out = r0.as<SP>();
    h.st = st;
    h.post = POST_INIT;
    TSM_TRY(launch_hop<SP>(c, h, 1, HOP_CENTER | HOP_NORM, -1, nrhs));
  }
  PField p, t, w, r, x, x64;
  TSM_TRY(c.field("cg_p", pS, &p, nb));
  TSM_TRY(c.field("cg_t", pS, &t, nb));
  TSM_TRY(c.field("cg_w", pS, &w, nb));
  TSM_TRY(c.field("cg_r", pA, &r, nb));
  if constexpr (DIRECT) x = s.e;
  else TSM_TRY(c.field("cg_x", pA, &x, nb));
  if constexpr (R0_IN_R) {
    TSM_TRY((launch_convert<SA, S>(c, r, p, nullptr, nrhs)));
  } else {
    TSM_TRY((launch_convert<SP, SA>(c, r0, r, nullptr, nrhs)));
    TSM_TRY((launch_convert<SP, S>(c, r0, p, nullptr, nrhs)));
  }
  TSM_TRY((launch_convert<SA, SA>(c, PField{}, x, nullptr, nrhs)));
  if constexpr (REL) {
    TSM_TRY(c.field("cg_x64", TSM_F64, &x64, nb));
    if (x0 == nullptr) {
      TSM_TRY((launch_convert<F64, F64>(c, PField{}, x64, nullptr, nrhs)));
    } else {
      // warm start: x = x0, r = Dhat^dag (bhat - Dhat x0) in the reliable
      // update's mixed precision, p = r; a source whose start already meets
      // the stopping rule stops here (rel_finish_kernel)
      if (x0_prec == TSM_F64) TSM_TRY((launch_convert<F64, F64>(c, *x0, x64, nullptr, nrhs)));
      else if (x0_prec == TSM_F16) TSM_TRY((launch_convert<F16, F64>(c, *x0, x64, nullptr, nrhs)));
      else TSM_TRY((launch_convert<F32, F64>(c, *x0, x64, nullptr, nrhs)));
      warm_start_kernel<<<1, Ctx::kMaxBatch, 0, c.stream>>>(st, nrhs);
      c.launches++;
      TSM_TRY(check_launch(c, "warm_start_kernel"));
      TSM_TRY(normal_residual_mixed(c, x64, bhat, r, st, nullptr, nrhs));
      const int blocks = (c.g.Vh + SITE_NT - 1) / SITE_NT;
      restart_direction_kernel<<<dim3(nrhs, blocks), SITE_NT, 0, c.stream>>>(c.g.Vh, r.as<F32>(), p.as<F32>(),
                                                                             c.sstride, nullptr, st);
      c.launches++;
      TSM_TRY(check_launch(c, "restart_direction_kernel"));
      rel_finish_kernel<<<1, Ctx::kMaxBatch, 0, c.stream>>>(st, nullptr, nrhs);
      c.launches++;
      TSM_TRY(check_launch(c, "rel_finish_kernel"));
    }
  }
  // one CG iteration over the listed right-hand sides (n of them), followed,
  // with reliable updates, by the FP64 update of those that asked for one
  auto iteration = [&](const int* dact, int n, bool timed) -> int {
    c.prof_this_launch = c.profile && timed;
    HopArgs<S> h = hop_args<S>(c, 1);   // K1
    h.active = dact;
    h.in = p.as<S>();
    h.out = t.as<S>();
    h.to = twist_Ainv(k, mu);
    h.skip = st;
    TSM_TRY(launch_hop<S>(c, h, 0, 0, PK_HOP, n));
    h = hop_args<S>(c, 0);              // K2
    h.active = dact;
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
    TSM_TRY(launch_hop<S>(c, h, 0, HOP_CENTER | HOP_NORM, PK_HOP_XPAY, n));
    h = hop_args<S>(c, 1);              // K3
    h.active = dact;
    h.in = w.as<S>();
    h.out = t.as<S>();
    h.to = twist_Ainv(k, -mu);
    h.skip = st;
    TSM_TRY(launch_hop<S>(c, h, 1, 0, PK_HOP_DAG, n));
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
    u.active = dact;
    u.st = st;
    u.red = c.red;
    TSM_TRY((launch_cg_update<S, SA>(c, u, n)));
    c.prof_this_launch = false;
    TSM_TRY((launch_cg_p<S, SA>(c, r, p, st, dact, n)));   // K5
    if constexpr (REL) {
      // reliable update (Sleijpen & van der Vorst; Clark et al. for lattice QCD):
      // for every right-hand side whose residual fell by delta since the last
      // update, or that met its stopping rule, fold the FP32 increment into the
      // FP64 solution, replace the iterated residual by the normal residual of
      // the true (FP64) Schur residual and restart the search direction from
      // it; the others return at once from these kernels
      const int blocks = (c.g.Vh + SITE_NT - 1) / SITE_NT;
      accumulate_solution_kernel<<<dim3(n, blocks), SITE_NT, 0, c.stream>>>(c.g.Vh, x.as<F32>(), x64.as<F64>(),
                                                                           c.sstride, dact, st);
      c.launches++;
      TSM_TRY(check_launch(c, "accumulate_solution_kernel"));
      TSM_TRY(normal_residual_mixed(c, x64, bhat, r, st, dact, n));
      restart_direction_kernel<<<dim3(n, blocks), SITE_NT, 0, c.stream>>>(c.g.Vh, r.as<F32>(), p.as<F32>(), c.sstride,
                                                                         dact, st);
      c.launches++;
      TSM_TRY(check_launch(c, "restart_direction_kernel"));
      rel_finish_kernel<<<1, Ctx::kMaxBatch, 0, c.stream>>>(st, dact, n);
      c.launches++;
      TSM_TRY(check_launch(c, "rel_finish_kernel"));
    }
    return TSM_OK;
  };
  std::vector<CGState> hs;
  if (c.capturing) {
    // graph mode: the iterations become a graph while-loop whose condition a
    // device kernel clears once every source has met its stopping rule
    TSM_TRY(capture_while(c, st, nrhs, stop.max_iter, [&]() { return iteration(nullptr, nrhs, false); }));
  } else {
    TSM_TRY(read_states(c, s0, nrhs, hs));
  }
  auto iterating = [&](int i) { return !c.capturing && !hs[i].done && hs[i].status == 0; };
  const int chunk = 8;
  long long launched = 0;   // guards the host loop against states that stop advancing
  for (;;) {
    std::vector<int> act;
    int min_left = stop.max_iter;
    for (int i = 0; i < nrhs; ++i)
      if (iterating(i)) {
        act.push_back(i);
        min_left = std::min(min_left, stop.max_iter - hs[i].iter);
      }
    if (act.empty()) break;
    if (launched > 2 * (long long)stop.max_iter + 64) {
      set_error("solver state stopped advancing after %lld iterations", launched);
      return TSM_ERR_CUDA;
    }
    const int n = (int)act.size();
    const int* dact = nullptr;
    TSM_TRY(upload_list(c, 0, act, &dact));
    int m = chunk;
    // after the first chunk: about as many iterations as the slowest listed
    // source still needs at its convergence rate so far (rr falls by rr / rr0
    // in iter iterations), so that a straggler or two do not drag a chunk of
    // empty iterations behind them; the device still decides every stop
    if (launched > 0 && stop.rel_tol > 0.0) {
      const double goal = stop.rel_tol * stop.rel_tol;   // rr / rr0 at the stopping rule
      int need = 1;
      for (int i : act) {
        const CGState& q = hs[i];
        const double drop = q.rr0 > 0.0 ? q.rr / q.rr0 : 1.0;
        if (q.iter <= 0 || !(drop > 0.0) || !(drop < 1.0)) {
          need = chunk;
          break;
        }
        const double est = q.iter * std::log(goal / drop) / std::log(drop);
        if (est > need) need = est < chunk ? (int)std::ceil(est) : chunk;
      }
      m = need;
    }
    if (min_left < m) m = min_left;
    if (m < 1) m = 1;
    launched += m;
    for (int it = 0; it < m; ++it) TSM_TRY(iteration(dact, n, it == 0));
    TSM_TRY(read_states(c, s0, nrhs, hs));
  }
  // solution: even part from CG, odd part reconstructed
  if constexpr (REL) {
    TSM_TRY((launch_convert<F64, SP>(c, x64, s.e, nullptr, nrhs)));
  } else if constexpr (!DIRECT) {
    TSM_TRY((launch_convert<SA, SP>(c, x, s.e, nullptr, nrhs)));
  }
  {
    HopArgs<SP> h = hop_args<SP>(c, 1);
    h.in = s.e.as<SP>();
    h.center = b.o.as<SP>();
    h.ac = 1.0;
    h.ah = k;
    h.to = twist_Ainv(k, mu);
    h.out = s.o.as<SP>();
    TSM_TRY(launch_hop<SP>(c, h, 0, HOP_CENTER, -1, nrhs));
  }
  if (c.capturing) return TSM_OK;   // results are read from the states after the graph ran
  for (int i = 0; i < nrhs; ++i) {
    const CGState& q = hs[i];
    SolveResult& o = res[i];
    o.iters = q.iter;
    o.status = q.status == 0 ? TSM_OK : TSM_ERR_NONFINITE;
    o.rel_res = q.rr0 > 0 ? std::sqrt(q.rr / q.rr0) : 0.0;
    if (q.rr0 == 0.0) o.converged = 1;
    else if (stop.rel_tol <= 0.0) o.converged = q.iter >= stop.max_iter;
    else o.converged = !(std::sqrt(q.rr) >= stop.rel_tol * std::sqrt(q.rr0));
  }
  return TSM_OK;
}

// allocate every field cg_solve uses for this tier (batch width c.batch_cap),
// so that a later solve makes no allocation (required under stream capture)
int reserve_solver(Ctx& c, const tm_stop& stop, int sol_prec) {
  int pS, pA, pP;
  switch (stop.prec) {
    case TSM_F64: pS = pA = pP = TSM_F64; break;
    case TSM_F32: pS = pA = TSM_F32; pP = stop.reliable ? TSM_F64 : TSM_F32; break;
    default: pS = stop.prec; pA = stop.prec == TSM_F16 ? TSM_F16 : TSM_F32; pP = TSM_F32; break;
  }
  if (stop.prec == TSM_F16 && sol_prec == TSM_F16) pP = TSM_F16;
  const int nb = c.batch_cap;
  PField f;
  for (const char* name : {"cg_tmp_o", "cg_bhat", "cg_w0", "cg_t0", "cg_r0"}) TSM_TRY(c.field(name, pP, &f, nb));
  for (const char* name : {"cg_p", "cg_t", "cg_w"}) TSM_TRY(c.field(name, pS, &f, nb));
  for (const char* name : {"cg_r", "cg_x"}) TSM_TRY(c.field(name, pA, &f, nb));
  if (stop.prec == TSM_F32 && stop.reliable) {
    for (const char* name : {"cg_x64", "rel_t", "rel_w"}) TSM_TRY(c.field(name, TSM_F64, &f, nb));
    for (const char* name : {"rel_u32", "rel_t32"}) TSM_TRY(c.field(name, TSM_F32, &f, nb));
  }
  return TSM_OK;
}

int solve_batch(Ctx& c, const tm_stop& stop, int s0, int nrhs, EOField b, EOField s, SolveResult* res,
                const PField* x0, int x0_prec, int sol_prec) {
  if (sol_prec >= 0 && sol_prec != solution_prec(stop) && !(stop.prec == TSM_F16 && sol_prec == TSM_F16)) {
    set_error("solution storage tier %d not available for solver tier %d", sol_prec, stop.prec);
    return TSM_ERR_ARG;
  }
  if (stop.precond) return fgmres_batch(c, stop, nrhs, b, s, res);
  if (nrhs < 1 || nrhs > c.batch_cap || s0 < 0 || s0 + nrhs > Ctx::kMaxStates - 4) {
    set_error("batch of %d right-hand sides at state %d exceeds the capacity (%d)", nrhs, s0, c.batch_cap);
    return TSM_ERR_TOO_LARGE;
  }
  switch (stop.prec) {
    case TSM_F64: return cg_solve<F64, F64, F64, false>(c, stop, s0, nrhs, b, s, res, nullptr, -1);
    case TSM_F32:
      if (stop.reliable) {
        if (x0 != nullptr && x0_prec != TSM_F16 && x0_prec != TSM_F32 && x0_prec != TSM_F64) {
          set_error("starting guess of tier %d (FP16, FP32 or FP64 expected)", x0_prec);
          return TSM_ERR_ARG;
        }
        return cg_solve<F32, F32, F64, true>(c, stop, s0, nrhs, b, s, res, x0, x0_prec);
      }
      return cg_solve<F32, F32, F32, false>(c, stop, s0, nrhs, b, s, res, nullptr, -1);
    // FP16 tier: r and x in FP16 too (relative storage precision 2^-11, an order
    // below the LP truncation; the memory-bound CG update moves 36 % fewer bytes);
    // source and solution in FP16 too when the caller asks for it
    case TSM_F16:
      if (sol_prec == TSM_F16) return cg_solve<F16, F16, F16, false>(c, stop, s0, nrhs, b, s, res, nullptr, -1);
      return cg_solve<F16, F16, F32, false>(c, stop, s0, nrhs, b, s, res, nullptr, -1);
    case TSM_BF16: return cg_solve<BF16, F32, F32, false>(c, stop, s0, nrhs, b, s, res, nullptr, -1);
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
