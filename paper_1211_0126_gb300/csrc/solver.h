// solver.h -- CG on the normal equations of the even/odd Schur complement.
#pragma once

#include "context.h"

namespace tsm {

struct SolveResult {
  int iters = 0;
  int status = TSM_OK;     // TSM_OK or TSM_ERR_NONFINITE
  int converged = 0;       // stopping rule met (fixed-count rule: max_iter reached)
  double rel_res = 0.0;    // final ||r|| / ||Dhat^dag bhat|| as tracked by the solver
                           // (flexible GMRES: the true ||bhat - Dhat x|| / ||bhat||)
  int fallback = 0;        // flexible GMRES broke down and plain CG produced the solution
};

// Storage tier of a solve's source and solution fields: FP64 for the FP64
// tier and for FP32 with FP64 reliable updates, FP32 otherwise.
int solution_prec(const tm_stop& stop);

// Storage tier of the sources and solutions of the solves inside the loop
// estimators: as solution_prec, except that the FP16 tier (whose iterates x
// and r are FP16 already) keeps its noise source, Schur source and solution in
// FP16 as well, so that its source preparation, odd reconstruction and
// contraction move 16-bit fields through the link-sharing stencil.
int loop_solution_prec(const tm_stop& stop);

// Solve D_tm s_r = b_r for nrhs independent sources at once.  b and s are
// batches of nrhs contiguous even/odd fields of tier sol_prec (-1:
// solution_prec(stop); otherwise solution_prec(stop) or, for the FP16 tier,
// TSM_F16) laid out for c.batch_cap sources; device solver states s0 ..
// s0+nrhs-1 are used; res receives nrhs results.  x0 (optional; FP32 with FP64
// reliable updates only, ignored by the other tiers): a batch of even-site
// starting guesses of storage tier x0_prec (TSM_F16, TSM_F32 or TSM_F64); the
// first iterate's residual is then the true normal residual of b - D x0,
// computed as in a reliable update, and the stopping rule stays relative to
// ||Dhat^dag bhat||.
int solve_batch(Ctx& c, const tm_stop& stop, int s0, int nrhs, EOField b, EOField s, SolveResult* res,
                const PField* x0 = nullptr, int x0_prec = -1, int sol_prec = -1);

// Allocate the solver workspace of a tier for c.batch_cap sources in advance
// (source / solution storage sol_prec as in solve_batch).
int reserve_solver(Ctx& c, const tm_stop& stop, int sol_prec = -1);

// ||b - D_tm s|| / ||b|| in FP64 (fields of tier prec).
int true_residual(Ctx& c, int prec, EOField b, EOField s, double* out);

// hop arguments pre-filled for this context (links of storage S, unit twists)
template <class S>
HopArgs<S> hop_args(const Ctx& c, int p_out) {
  HopArgs<S> a{};
  a.g = c.g;
  a.p_out = p_out;
  a.Uout = c.links_of<S>(p_out);
  a.Uin = c.links_of<S>(1 - p_out);
  a.lstride = c.lstride;
  a.sstride = c.sstride;
  a.ac = 0.0;
  a.ah = 1.0;
  a.tc = twist_one();
  a.to = twist_one();
  a.ts = twist_one();
  a.red = c.red;
  a.post = POST_NONE;
  a.active = nullptr;
  a.skip = nullptr;
  a.st = nullptr;
  return a;
}

}  // namespace tsm
