// fft.h -- loops at every spatial momentum through the library's own 3-D FFT
// per source (in-place mixed-radix passes in shared memory, fft.cu).
#pragma once

#include "context.h"
#include "contract.cuh"

namespace tsm {

constexpr int FFT_MAX_STAGES = 20;
constexpr int FFT_MAX_PRIME = 13;   // largest prime factor of an extent (direct DFT butterfly)

// radices of one axis (product = n); per stage st the block length after it
// m[st] (= block length / radix) and n / (block length) ts[st]
struct FftAxis {
  int n;
  int nst;
  int radix[FFT_MAX_STAGES];
  int m[FFT_MAX_STAGES];
  int ts[FFT_MAX_STAGES];
};

// insertions for the density pass: Gamma_k has one non-zero per row, in
// column row ^ m[k], of value fr + i fi
struct FftGam {
  int n;
  int m[CT_MAXG];
  float fr[CT_MAXG][4], fi[CT_MAXG][4];
};

struct FftPlan {
  FftAxis ax[3];   // x, y, z
  int tw_xy;       // Lx + Ly: twiddle entries of the x and y tables (the z table follows)
};

struct FftProjector {
  int ng = 0;
  bool fp64 = true;
  long long E = 0;                              // n_gamma * V entries
  void* dens = nullptr;                         // per-source densities / transforms [n_gamma][T][Lz][Ly][Lx]
  double2* mean[2] = {nullptr, nullptr};        // running means: [0] HP-set corrections, [1] LP set
  double* m2[2] = {nullptr, nullptr};           // running sums of squared deviations
  // FP32 tier: per-entry sums of d = x - K and |d|^2 over the current batch
  // of up to kFftBatch sources of a set, K = the batch's first value of the
  // entry (shifted sums: no cancellation when |mean| >> spread), merged into
  // the FP64 moments once per batch
  static constexpr int kFftBatch = 32;
  float2* bsum[2] = {nullptr, nullptr};
  float* bsq[2] = {nullptr, nullptr};
  float2* bshift[2] = {nullptr, nullptr};
  int nb[2] = {0, 0};                           // sources in the current batch
  int nmerged[2] = {0, 0};                      // sources already in the FP64 moments
  double2* twd = nullptr;                       // twiddles e^{+2 pi i m / L}: x, y, z tables (FP64)
  int* posd = nullptr;                          // storage position of each frequency: x, y, z tables
  FftPlan plan{};
  int gc = 1;                                   // insertions per xy CTA
  int xy_threads = 512;                         // threads per xy CTA
  int zw = 1;                                   // columns per z CTA
  size_t xy_smem = 0, z_smem = 0;               // dynamic shared memory of the two kernels

  // TSM_ERR_TOO_LARGE when an Lx x Ly plane or an Lz line does not fit in
  // shared memory, or an extent has a prime factor above FFT_MAX_PRIME
  int init(Ctx& c, int n_gamma, bool fp64_arith);
  void release();
  // densities eta^dag Gamma (a - b) of one source, transformed (written to dens)
  template <class R, class SA, class SB>
  int transform(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a, const EOField* b);
  // transform, then fold into set `set` as its k-th source (1-based, in
  // order); the transform itself is not stored.  FP64: Welford update of the
  // FP64 moments per source; FP32: FP32 batch sums, merged into the FP64
  // moments every kFftBatch sources and at finalize
  template <class R, class SA, class SB>
  int accumulate(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a, const EOField* b,
                 int set, int k);
  int finalize(Ctx& c, int n_hp, int n_lp, double2* est, double* err, double2* lp_mean, double2* corr_mean);

 private:
  template <class R, class SA, class SB>
  int xy_pass(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a, const EOField* b);
  template <class R>
  int z_pass(Ctx& c, const void* sink);
  int merge(Ctx& c, int set);
};

// out[e] = (double) in[e]
int launch_widen(Ctx& c, const float2* in, double2* out, long long n);

}  // namespace tsm
