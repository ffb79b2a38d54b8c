// fft.h -- loops at every spatial momentum through a batched 3-D FFT per source.
#pragma once

#include <cufft.h>

#include "context.h"
#include "contract.cuh"

namespace tsm {

struct FftProjector {
  int ng = 0;
  bool fp64 = true;
  long long E = 0;                              // n_gamma * V entries
  void* dens = nullptr;                         // per-source densities / transforms [n_gamma][T][Lz][Ly][Lx]
  double2* mean[2] = {nullptr, nullptr};        // running means: [0] HP-set corrections, [1] LP set
  double* m2[2] = {nullptr, nullptr};           // running sums of squared deviations
  cufftHandle plan = 0;
  bool has_plan = false;

  int init(Ctx& c, int n_gamma, bool fp64_arith);
  void release();
  // densities eta^dag Gamma (a - b) of one source, transformed in place
  template <class R, class SA, class SB>
  int transform(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a, const EOField* b);
  // transform, then fold into set `set` as its k-th source (1-based)
  template <class R, class SA, class SB>
  int accumulate(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a, const EOField* b,
                 int set, int k);
  int finalize(Ctx& c, int n_hp, int n_lp, double2* est, double* err, double2* lp_mean, double2* corr_mean);
};

// out[e] = (double) in[e]
int launch_widen(Ctx& c, const float2* in, double2* out, long long n);

}  // namespace tsm
