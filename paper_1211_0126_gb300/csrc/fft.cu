// fft.cu -- loops at every spatial momentum: per-site insertion densities,
// one batched 3-D FFT per source (cuFFT, as the paper's Sec. 3 used CUFFT
// for the Fourier transform) and running per-entry means and variances in
// source order (Welford), so that no per-source momentum grid is stored.
//
//   L_j(Gamma, t, n) = sum_{x: x_4 = t} e^{+2 pi i (n_x x / Lx + n_y y / Ly + n_z z / Lz)}
//                      eta_j(x)^dag Gamma (s_a - s_b)(x),
//
// output layout [n_gamma][T][Lz][Ly][Lx] with n_x, n_y, n_z in [0, L).
#include <cufft.h>

#include "contract.h"
#include "fft.h"

namespace tsm {

namespace {

constexpr int FFT_NT = 128;

// per-site densities G_g(x) = eta^dag Gamma_g (a - b) at full-lattice sites of
// one parity (blockIdx.y), written at dens[g][lex] (lexicographic site order)
template <class R, class SA, class SB>
__global__ void __launch_bounds__(FFT_NT) density_kernel(Geom g, NoiseSpec noise, uint32_t source,
                                                         const typename SA::schunk* a0, const typename SA::schunk* a1,
                                                         const typename SB::schunk* b0, const typename SB::schunk* b1,
                                                         int sstride, GammaTab gam, cx<R>* __restrict__ dens) {
  const int ih = blockIdx.x * FFT_NT + threadIdx.x;
  const int parity = blockIdx.y;
  if (ih >= g.Vh) return;
  int c[4];
  site_coords(g, parity, ih, c);
  const uint32_t lex = (uint32_t)(((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0]);
  cx<R> eta[12], s[12];
  noise_site<R>(noise, lex, source, eta);
  cx<typename SA::real> va[12];
  load_spinor<SA>(parity ? a1 : a0, sstride, ih, va);
  if (b0 != nullptr) {
    cx<typename SB::real> vb[12];
    load_spinor<SB>(parity ? b1 : b0, sstride, ih, vb);
    using W = typename SA::real;
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = {(R)(va[k].re - (W)vb[k].re), (R)(va[k].im - (W)vb[k].im)};
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = {(R)va[k].re, (R)va[k].im};
  }
  cx<R> S[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      cx<R> acc = cjmul(eta[3 * x], s[3 * y]);
      acc = acc + cjmul(eta[3 * x + 1], s[3 * y + 1]);
      acc = acc + cjmul(eta[3 * x + 2], s[3 * y + 2]);
      S[x][y] = acc;
    }
  for (int k = 0; k < gam.n; ++k) {
    cx<R> v = {0, 0};
#pragma unroll
    for (int row = 0; row < 4; ++row) {
      const int col = gam.col[k][row];
      cx<R> sv;
      switch (col) {
        case 0: sv = S[row][0]; break;
        case 1: sv = S[row][1]; break;
        case 2: sv = S[row][2]; break;
        default: sv = S[row][3]; break;
      }
      v = v + times_ipow(sv, gam.ph[k][row]);
    }
    dens[(size_t)k * g.V + lex] = v;
  }
}

// running mean and sum of squared deviations of entry e over sources 1..k
template <class R>
__global__ void welford_kernel(const cx<R>* __restrict__ x, int k, double2* __restrict__ mean,
                               double* __restrict__ m2, long long E) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double xr = (double)x[e].re, xi = (double)x[e].im;
  if (k == 1) {
    mean[e] = make_double2(xr, xi);
    m2[e] = 0.0;
    return;
  }
  const double2 m = mean[e];
  const double dr = xr - m.x, di = xi - m.y;
  mean[e] = make_double2(m.x + dr / k, m.y + di / k);
  m2[e] += (dr * dr + di * di) * (double)(k - 1) / (double)k;
}

// Eq. 2.4 from the running moments of the two sets
__global__ void fft_finalize_kernel(const double2* __restrict__ mc, const double* __restrict__ sc, int n_hp,
                                    const double2* __restrict__ ml, const double* __restrict__ sl, int n_lp,
                                    long long E, double2* __restrict__ est, double* __restrict__ err,
                                    double2* __restrict__ lp_mean, double2* __restrict__ corr_mean) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double er = 0.0, ei = 0.0, var = 0.0;
  if (n_hp > 0) {
    er += mc[e].x;
    ei += mc[e].y;
    if (n_hp > 1) var += sc[e] / (n_hp - 1) / n_hp;
  }
  if (n_lp > 0) {
    er += ml[e].x;
    ei += ml[e].y;
    if (n_lp > 1) var += sl[e] / (n_lp - 1) / n_lp;
  }
  if (est) est[e] = make_double2(er, ei);
  if (err) err[e] = sqrt(var);
  if (lp_mean) lp_mean[e] = n_lp > 0 ? ml[e] : make_double2(0.0, 0.0);
  if (corr_mean) corr_mean[e] = n_hp > 0 ? mc[e] : make_double2(0.0, 0.0);
}

__global__ void widen_kernel(const float2* __restrict__ in, double2* __restrict__ out, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = make_double2(in[e].x, in[e].y);
}

int cufft_check(cufftResult r, const char* what) {
  if (r != CUFFT_SUCCESS) {
    set_error("%s failed (cufftResult %d)", what, (int)r);
    return TSM_ERR_CUDA;
  }
  return TSM_OK;
}

}  // namespace

int FftProjector::init(Ctx& c, int ng_, bool dbl) {
  ng = ng_;
  fp64 = dbl;
  E = (long long)ng * c.g.V;
  void* p = nullptr;
  TSM_TRY(c.buffer("fft_dens", (size_t)E * (fp64 ? sizeof(double2) : sizeof(float2)), &p));
  dens = p;
  for (int s = 0; s < 2; ++s) {
    TSM_TRY(c.buffer(s ? "fft_mean_lp" : "fft_mean_corr", (size_t)E * sizeof(double2), &p));
    mean[s] = static_cast<double2*>(p);
    TSM_TRY(c.buffer(s ? "fft_m2_lp" : "fft_m2_corr", (size_t)E * sizeof(double), &p));
    m2[s] = static_cast<double*>(p);
  }
  int n[3] = {c.lat.L[2], c.lat.L[1], c.lat.L[0]};
  const int vs = n[0] * n[1] * n[2];
  TSM_TRY(cufft_check(cufftPlanMany(&plan, 3, n, nullptr, 1, vs, nullptr, 1, vs, fp64 ? CUFFT_Z2Z : CUFFT_C2C,
                                    ng * c.lat.L[3]),
                      "cufftPlanMany"));
  has_plan = true;
  return cufft_check(cufftSetStream(plan, c.stream), "cufftSetStream");
}

void FftProjector::release() {
  if (has_plan) cufftDestroy(plan);
  has_plan = false;
}

template <class R, class SA, class SB>
int FftProjector::transform(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a,
                            const EOField* b) {
  cx<R>* d = static_cast<cx<R>*>(dens);
  density_kernel<R, SA, SB><<<dim3((c.g.Vh + FFT_NT - 1) / FFT_NT, 2), FFT_NT, 0, c.stream>>>(
      c.g, ns, source, a.e.as<SA>(), a.o.as<SA>(), b ? b->e.as<SB>() : nullptr, b ? b->o.as<SB>() : nullptr,
      c.sstride, gam, d);
  c.launches++;
  TSM_TRY(check_launch(c, "density_kernel"));
  if constexpr (sizeof(R) == 8) {
    TSM_TRY(cufft_check(cufftExecZ2Z(plan, reinterpret_cast<cufftDoubleComplex*>(d),
                                     reinterpret_cast<cufftDoubleComplex*>(d), CUFFT_INVERSE),
                        "cufftExecZ2Z"));
  } else {
    TSM_TRY(cufft_check(cufftExecC2C(plan, reinterpret_cast<cufftComplex*>(d), reinterpret_cast<cufftComplex*>(d),
                                     CUFFT_INVERSE),
                        "cufftExecC2C"));
  }
  return TSM_OK;
}

template <class R, class SA, class SB>
int FftProjector::accumulate(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a,
                             const EOField* b, int set, int k) {
  // algorithmic bytes: the fields read, the densities written, one read and
  // one write pass of the transform, the densities read and the running
  // mean (16 B) and sum of squares (8 B) read and written per entry
  const double csz = sizeof(cx<R>);
  TimedLaunch tl(c, PB_FFT,
                 (double)c.g.V * (spinor_site_bytes(SA::id) + (b ? spinor_site_bytes(SB::id) : 0.0)) +
                     (double)E * (csz + 2.0 * csz + csz + 2.0 * 24.0),
                 true);
  TSM_TRY((transform<R, SA, SB>(c, gam, ns, source, a, b)));
  welford_kernel<R><<<(unsigned)((E + 255) / 256), 256, 0, c.stream>>>(static_cast<const cx<R>*>(dens), k, mean[set],
                                                                       m2[set], E);
  c.launches++;
  TSM_TRY(check_launch(c, "welford_kernel"));
  tl.done();
  return TSM_OK;
}

int FftProjector::finalize(Ctx& c, int n_hp, int n_lp, double2* est, double* err, double2* lp_mean,
                           double2* corr_mean) {
  fft_finalize_kernel<<<(unsigned)((E + 255) / 256), 256, 0, c.stream>>>(mean[0], m2[0], n_hp, mean[1], m2[1], n_lp,
                                                                          E, est, err, lp_mean, corr_mean);
  c.launches++;
  return check_launch(c, "fft_finalize_kernel");
}

int launch_widen(Ctx& c, const float2* in, double2* out, long long n) {
  widen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(in, out, n);
  c.launches++;
  return check_launch(c, "widen_kernel");
}

#define TSM_FFT_INST(R, SA, SB)                                                                              \
  template int FftProjector::transform<R, SA, SB>(Ctx&, const GammaTab&, const NoiseSpec&, uint32_t, EOField, \
                                                  const EOField*);                                           \
  template int FftProjector::accumulate<R, SA, SB>(Ctx&, const GammaTab&, const NoiseSpec&, uint32_t, EOField, \
                                                   const EOField*, int, int);
TSM_FFT_INST(double, F64, F64)
TSM_FFT_INST(float, F64, F64)
TSM_FFT_INST(float, F32, F32)
TSM_FFT_INST(float, F64, F32)
TSM_FFT_INST(float, F32, F64)
#undef TSM_FFT_INST

}  // namespace tsm
