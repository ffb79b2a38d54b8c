// contract.h -- host interface of the contraction and combine kernels.
#pragma once

#include "context.h"
#include "contract.cuh"

namespace tsm {

struct ContractPlan {
  GammaTab gam{};
  int ng = 0, n_q = 0;
  const double2* phx = nullptr;   // device phase tables [n_q][Lx], [n_q][Ly], [n_q][Lz]
  const double2* phy = nullptr;
  const double2* phz = nullptr;
  const float2* fphx = nullptr;   // the same tables rounded once to FP32 (FP32 contractions)
  const float2* fphy = nullptr;
  const float2* fphz = nullptr;
  int one_end = 0;                // 1: one-end-trick values (Eq. 2.5) with factor -4 i kappa mu;
                                  // 2: generalised one-end trick (Eq. 2.6): 2 s^dag g5 Gamma g5 D_W s
  int local = 1;                  // the local block (standard or one-end values)
  int deriv_mask = 0;             // bit mu: one-derivative insertion block along mu (standard estimator)
  std::vector<CtMoments> passes;  // the momenta of each pass of at most CT_MAXQ, in +-q classes
  int prepare(Ctx& c, const int* gammas, int n_gamma, const int* moms, int n_q);
  int blocks() const {
    int n = local;
    for (int m = 0; m < 4; ++m) n += (deriv_mask >> m) & 1;
    return n;
  }
  // outputs per source: blocks() consecutive [n_gamma][n_q][T] blocks (local
  // first, then one per derivative direction in increasing mu)
  int entries(int T) const { return ng * n_q * T * blocks(); }
};

int make_gamma_tab(const int* gammas, int n, GammaTab* tab);
// group nq momenta (integer n, 3 per momentum) of one pass into +-q classes on an L lattice
int group_momenta(const int* L, const int* moms, int nq, CtMoments* m);
NoiseSpec make_noise(uint64_t seed, int kind);

// out[g][q][t] (device, complex) = sum_t-slice e^{iqx} eta^dag Gamma_g (a - b), or
// with plan.one_end the one-end values f(a) - f(b), f(s) = -4 i kappa mu s^dag g5 Gamma_g s
// (plan.one_end == 2 needs wa = D_W a and, with b, wb = D_W b)
template <class R, class SA, class SB>
int launch_contract(Ctx& c, const ContractPlan& plan, const NoiseSpec& ns, uint32_t source, EOField a,
                    const EOField* b, double2* out, const EOField* wa = nullptr, const EOField* wb = nullptr);

// out = D_W in = in - kappa H in on both parities (fields of tier prec)
int apply_wilson(Ctx& c, int prec, EOField in, EOField out);

// allocate the block-partial buffer of the largest contraction launch
int reserve_contract(Ctx& c);

int launch_combine(Ctx& c, const double2* corr, int n_hp, const double2* lp, int n_lp, int E, double2* est,
                   double* err, double2* lp_mean, double2* corr_mean);

}  // namespace tsm
