// fgmres.cu -- flexible GMRES (Saad 1993) on the even/odd Schur system
// Dhat x = bhat with the learned network as right preconditioner.
//
// A cycle of m steps builds an orthonormal basis v_0 .. v_m of the Krylov-like
// space spanned by Dhat z_j, z_j = net(v_j), with classical Gram-Schmidt
// applied twice (one device reduction for all projections per pass) and FP64
// accumulation of every inner product; the small Hessenberg least-squares
// problem is solved on the host with complex Givens rotations.  The solution
// update x += Z y uses the stored preconditioned vectors, so the
// preconditioner may change from step to step (a network in BF16 is not an
// exact linear map).  Stopping rule: ||bhat - Dhat x|| / ||bhat|| < rel_tol
// (the residual of the system itself, not of the normal equations), or
// max_iter inner steps; rel_tol = 0 gives a fixed step count.  A breakdown
// (NaN/Inf, or a final residual above the starting one) hands the source to
// plain CG on the same tier.
#include <cmath>
#include <complex>
#include <vector>

#include "fields.cuh"
#include "net.h"
#include "solver.h"

namespace tsm {

namespace {

constexpr int FG_NT = 256;
constexpr int FG_BLOCKS = 2 * 152;

// partial inner products <v_i, w> (conj(v) . w) of nv vectors, blockIdx.y = i
__global__ void __launch_bounds__(FG_NT) fg_dot_kernel(const float2* __restrict__ V, size_t vstride,
                                                       const float2* __restrict__ w, long long n,
                                                       double* __restrict__ part) {
  const float2* v = V + (size_t)blockIdx.y * vstride;
  double re = 0.0, im = 0.0;
  for (long long k = (long long)blockIdx.x * FG_NT + threadIdx.x; k < n; k += (long long)gridDim.x * FG_NT) {
    const float2 a = v[k], b = w[k];
    re += (double)a.x * b.x + (double)a.y * b.y;
    im += (double)a.x * b.y - (double)a.y * b.x;
  }
  __shared__ double sh[FG_NT / 32];
  const double sr = block_sum<FG_NT>(re, sh);
  const double si = block_sum<FG_NT>(im, sh);
  if (threadIdx.x == 0) {
    part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 2] = sr;
    part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 2 + 1] = si;
  }
}

// fixed-order sum of the partials of vector blockIdx.x -> out[2 i], out[2 i + 1]
__global__ void __launch_bounds__(FG_NT) fg_sum_kernel(const double* __restrict__ part, int nblk,
                                                       double* __restrict__ out) {
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nblk; b += FG_NT) {
    re += part[((size_t)blockIdx.x * nblk + b) * 2];
    im += part[((size_t)blockIdx.x * nblk + b) * 2 + 1];
  }
  __shared__ double sh[FG_NT / 32];
  const double sr = block_sum<FG_NT>(re, sh);
  const double si = block_sum<FG_NT>(im, sh);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sr;
    out[2 * blockIdx.x + 1] = si;
  }
}

// w += sgn * sum_i coef_i v_i   (coef: nv complex numbers in device memory)
__global__ void __launch_bounds__(FG_NT) fg_axpy_kernel(float2* __restrict__ w, const float2* __restrict__ V,
                                                        size_t vstride, int nv, const double* __restrict__ coef,
                                                        double sgn, long long n) {
  const long long k = (long long)blockIdx.x * FG_NT + threadIdx.x;
  if (k >= n) return;
  double re = w[k].x, im = w[k].y;
  for (int i = 0; i < nv; ++i) {
    const float2 v = V[(size_t)i * vstride + k];
    const double cr = sgn * coef[2 * i], ci = sgn * coef[2 * i + 1];
    re += cr * v.x - ci * v.y;
    im += cr * v.y + ci * v.x;
  }
  w[k] = make_float2((float)re, (float)im);
}

// out = s * in  (out may alias in); s = 0 writes zeros
__global__ void __launch_bounds__(FG_NT) fg_scale_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                         double s, long long n) {
  const long long k = (long long)blockIdx.x * FG_NT + threadIdx.x;
  if (k >= n) return;
  const float2 a = in[k];
  out[k] = make_float2((float)(s * a.x), (float)(s * a.y));
}

// out = a - b
__global__ void __launch_bounds__(FG_NT) fg_sub_kernel(const float2* __restrict__ a, const float2* __restrict__ b,
                                                       float2* __restrict__ out, long long n) {
  const long long k = (long long)blockIdx.x * FG_NT + threadIdx.x;
  if (k >= n) return;
  out[k] = make_float2(a[k].x - b[k].x, a[k].y - b[k].y);
}

using cd = std::complex<double>;

struct Fg {
  Ctx& c;
  long long n;         // complex numbers per even field (12 Vh)
  size_t vstride;      // float2 per field
  double* part = nullptr;
  double* coef = nullptr;    // device: [2 (m + 1)] projections, then norms
  PField t_odd;

  int grid(long long cnt) const { return (int)((cnt + FG_NT - 1) / FG_NT); }

  // dots of w with nv vectors starting at V -> device coef[0 .. 2 nv)
  int dots(const float2* V, int nv, const float2* w, double* out) {
    fg_dot_kernel<<<dim3(FG_BLOCKS, nv), FG_NT, 0, c.stream>>>(V, vstride, w, n, part);
    c.launches++;
    TSM_TRY(check_launch(c, "fg_dot_kernel"));
    fg_sum_kernel<<<nv, FG_NT, 0, c.stream>>>(part, FG_BLOCKS, out);
    c.launches++;
    return check_launch(c, "fg_sum_kernel");
  }
  int axpy(float2* w, const float2* V, int nv, const double* cf, double sgn) {
    fg_axpy_kernel<<<grid(n), FG_NT, 0, c.stream>>>(w, V, vstride, nv, cf, sgn, n);
    c.launches++;
    return check_launch(c, "fg_axpy_kernel");
  }
  int scale(const float2* in, float2* out, double s) {
    fg_scale_kernel<<<grid(n), FG_NT, 0, c.stream>>>(in, out, s, n);
    c.launches++;
    return check_launch(c, "fg_scale_kernel");
  }
  // out = Dhat in = in - kappa^2 A^-1 H_eo A^-1 H_oe in   (FP32 storage)
  int dhat(const PField& in, const PField& out) {
    const double k = c.lat.kappa, mu = c.lat.mu;
    HopArgs<F32> h = hop_args<F32>(c, 1);
    h.in = in.as<F32>();
    h.out = t_odd.as<F32>();
    h.to = twist_Ainv(k, mu);
    TSM_TRY(launch_hop<F32>(c, h, 0, 0, -1));
    h = hop_args<F32>(c, 0);
    h.in = t_odd.as<F32>();
    h.center = in.as<F32>();
    h.tc = twist_A(k, mu);
    h.ac = 1.0;
    h.ah = -k * k;
    h.to = twist_Ainv(k, mu);
    h.out = out.as<F32>();
    return launch_hop<F32>(c, h, 0, HOP_CENTER, -1);
  }
  int read(double* host, const double* dev, int count) {
    TSM_CUDA(cudaMemcpyAsync(host, dev, count * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    TSM_CUDA(cudaStreamSynchronize(c.stream));
    return TSM_OK;
  }
};

inline float2* f2(const PField& f) { return static_cast<float2*>(f.p); }

// complex Givens rotation G = [[cs, sn], [-conj(sn), cs]] with G (a, b)^T = (r, 0)^T
void givens(cd a, cd b, double* cs, cd* sn) {
  const double na = std::abs(a), nb = std::abs(b);
  if (nb == 0.0) {
    *cs = 1.0;
    *sn = 0.0;
    return;
  }
  if (na == 0.0) {
    *cs = 0.0;
    *sn = 1.0;
    return;
  }
  const double rho = std::hypot(na, nb);
  *cs = na / rho;
  *sn = (a / na) * std::conj(b) / rho;
}

}  // namespace

// one source: bhat (even, FP32) -> x (even, FP32)
static int fgmres_one(Fg& F, Net& net, const tm_stop& stop, int m, const PField& bhat, const PField& x,
                      const PField& Vb, const PField& Zb, const PField& w, const PField& r, SolveResult* out) {
  Ctx& c = F.c;
  const size_t fb = field_bytes(TSM_F32, c.g.Vh);
  auto vec = [&](const PField& base, int i) { return field_at(base, TSM_F32, c.g.Vh, i); };
  SolveResult res;
  double h2[2];
  TSM_TRY(F.dots(f2(bhat), 1, f2(bhat), F.coef));
  TSM_TRY(F.read(h2, F.coef, 2));
  const double bnorm = std::sqrt(h2[0]);
  TSM_TRY(F.scale(f2(bhat), f2(x), 0.0));   // x = 0
  if (!(bnorm > 0.0)) {
    res.converged = 1;
    res.status = std::isfinite(bnorm) ? TSM_OK : TSM_ERR_NONFINITE;
    *out = res;
    return TSM_OK;
  }
  const double target = stop.rel_tol * bnorm;
  double beta = bnorm;
  TSM_CUDA(cudaMemcpyAsync(r.p, bhat.p, fb, cudaMemcpyDeviceToDevice, c.stream));
  std::vector<cd> H((size_t)(m + 1) * m), g(m + 1);
  std::vector<double> cs(m);
  std::vector<cd> sn(m);
  std::vector<double> hc(2 * (m + 1));
  int iters = 0;
  bool finite = true;
  for (;;) {
    // new cycle from the residual r (x holds the current solution)
    TSM_TRY(F.scale(f2(r), f2(vec(Vb, 0)), 1.0 / beta));
    std::fill(g.begin(), g.end(), cd(0.0));
    g[0] = beta;
    int j = 0;
    bool done = false;
    for (; j < m; ++j) {
      TSM_TRY(net_apply_even(c, net, vec(Vb, j), vec(Zb, j), 1));
      TSM_TRY(F.dhat(vec(Zb, j), w));
      // classical Gram-Schmidt, twice
      TSM_TRY(F.dots(f2(Vb), j + 1, f2(w), F.coef));
      TSM_TRY(F.axpy(f2(w), f2(Vb), j + 1, F.coef, -1.0));
      TSM_TRY(F.dots(f2(Vb), j + 1, f2(w), F.coef + 2 * (m + 1)));
      TSM_TRY(F.axpy(f2(w), f2(Vb), j + 1, F.coef + 2 * (m + 1), -1.0));
      TSM_TRY(F.dots(f2(w), 1, f2(w), F.coef + 4 * (m + 1)));
      std::vector<double> all(4 * (m + 1) + 2);
      TSM_TRY(F.read(all.data(), F.coef, 4 * (m + 1) + 2));
      const double hn = std::sqrt(all[4 * (m + 1)]);
      for (int i = 0; i <= j; ++i)
        H[(size_t)i * m + j] = cd(all[2 * i] + all[2 * (m + 1) + 2 * i], all[2 * i + 1] + all[2 * (m + 1) + 2 * i + 1]);
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i <= j; ++i) finite = finite && std::isfinite(H[(size_t)i * m + j].real()) &&
                                          std::isfinite(H[(size_t)i * m + j].imag());
      finite = finite && std::isfinite(hn);
      if (!finite) break;
      // earlier rotations on the new column, then a new one
      for (int i = 0; i < j; ++i) {
        const cd a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + cs[i] * b;
      }
      givens(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j], &cs[j], &sn[j]);
      H[(size_t)j * m + j] = cs[j] * H[(size_t)j * m + j] + sn[j] * H[(size_t)(j + 1) * m + j];
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      const double est = std::abs(g[j + 1]);
      if (hn > 0.0) TSM_TRY(F.scale(f2(w), f2(vec(Vb, j + 1)), 1.0 / hn));
      const bool met = stop.rel_tol > 0.0 && est < target;
      if (met || iters >= stop.max_iter || hn == 0.0) {
        ++j;
        done = true;
        break;
      }
    }
    if (!finite) break;
    // y = R^-1 g (upper triangular), x += Z y
    const int k = j;
    std::vector<cd> y(k);
    for (int i = k - 1; i >= 0; --i) {
      cd s = g[i];
      for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    for (int i = 0; i < k; ++i) {
      hc[2 * i] = y[i].real();
      hc[2 * i + 1] = y[i].imag();
      finite = finite && std::isfinite(hc[2 * i]) && std::isfinite(hc[2 * i + 1]);
    }
    if (!finite) break;
    if (k > 0) {
      TSM_CUDA(cudaMemcpyAsync(F.coef, hc.data(), 2 * k * sizeof(double), cudaMemcpyHostToDevice, c.stream));
      TSM_TRY(F.axpy(f2(x), f2(Zb), k, F.coef, 1.0));
    }
    // true residual
    TSM_TRY(F.dhat(x, w));
    fg_sub_kernel<<<F.grid(F.n), FG_NT, 0, c.stream>>>(f2(bhat), f2(w), f2(r), F.n);
    c.launches++;
    TSM_TRY(check_launch(c, "fg_sub_kernel"));
    TSM_TRY(F.dots(f2(r), 1, f2(r), F.coef));
    TSM_TRY(F.read(h2, F.coef, 2));
    beta = std::sqrt(h2[0]);
    finite = finite && std::isfinite(beta);
    if (!finite) break;
    const bool met = stop.rel_tol > 0.0 && beta < target;
    if (met || iters >= stop.max_iter || (done && !(beta > 0.0))) {
      res.converged = stop.rel_tol > 0.0 ? (beta < target) : (iters >= stop.max_iter);
      break;
    }
  }
  res.iters = iters;
  res.rel_res = beta / bnorm;
  res.status = finite ? TSM_OK : TSM_ERR_NONFINITE;
  *out = res;
  return TSM_OK;
}

int fgmres_batch(Ctx& c, const tm_stop& stop, int nrhs, EOField b, EOField s, SolveResult* res) {
  if (c.net == nullptr) {
    set_error("tm_stop.precond is set but no network is attached to the context (tsm_set_precond)");
    return TSM_ERR_ARG;
  }
  if (c.capturing) {
    set_error("flexible GMRES runs eagerly (its Hessenberg problem is solved on the host); not under graph capture");
    return TSM_ERR_ARG;
  }
  if (solution_prec(stop) != TSM_F32) {
    set_error("flexible GMRES needs a tier with FP32 source/solution fields (TSM_F32 without reliable updates, "
              "TSM_BF16, TSM_F16)");
    return TSM_ERR_ARG;
  }
  const int m = stop.restart > 0 ? std::min(stop.restart, 64) : 16;
  const double k = c.lat.kappa, mu = c.lat.mu;
  Fg F{c, 12ll * c.g.Vh, (size_t)6 * c.sstride * 2};
  PField Vb, Zb, w, r, x, bhat, tmp_o;
  TSM_TRY(c.field("fg_V", TSM_F32, &Vb, m + 1));
  TSM_TRY(c.field("fg_Z", TSM_F32, &Zb, m));
  TSM_TRY(c.field("fg_w", TSM_F32, &w));
  TSM_TRY(c.field("fg_r", TSM_F32, &r));
  TSM_TRY(c.field("fg_x", TSM_F32, &x));
  TSM_TRY(c.field("fg_bhat", TSM_F32, &bhat));
  TSM_TRY(c.field("fg_tmp_o", TSM_F32, &tmp_o));
  TSM_TRY(c.field("fg_t_odd", TSM_F32, &F.t_odd));
  void* p = nullptr;
  TSM_TRY(c.buffer("fg_part", (size_t)FG_BLOCKS * (m + 1) * 2 * sizeof(double), &p));
  F.part = static_cast<double*>(p);
  TSM_TRY(c.buffer("fg_coef", (size_t)(4 * (m + 1) + 2) * sizeof(double), &p));
  F.coef = static_cast<double*>(p);
  tm_stop plain = stop;
  plain.precond = 0;
  for (int i = 0; i < nrhs; ++i) {
    const EOField bi = eo_at(b, TSM_F32, c.g.Vh, i), si = eo_at(s, TSM_F32, c.g.Vh, i);
    // bhat_e = A^-1 (b_e + kappa H_eo A^-1 b_o)
    TSM_TRY(launch_twist<F32>(c, twist_Ainv(k, mu), bi.o, tmp_o, nullptr));
    {
      HopArgs<F32> h = hop_args<F32>(c, 0);
      h.in = tmp_o.as<F32>();
      h.center = bi.e.as<F32>();
      h.ac = 1.0;
      h.ah = k;
      h.to = twist_Ainv(k, mu);
      h.out = bhat.as<F32>();
      TSM_TRY(launch_hop<F32>(c, h, 0, HOP_CENTER, -1));
    }
    SolveResult q;
    TSM_TRY(fgmres_one(F, *c.net, stop, m, bhat, x, Vb, Zb, w, r, &q));
    const bool broke = q.status != TSM_OK || !(q.rel_res <= 1.0);
    if (broke) {
      // plain CG on the same tier decides this source
      TSM_TRY(solve_batch(c, plain, 0, 1, bi, si, &q));
      q.fallback = 1;
      res[i] = q;
      continue;
    }
    TSM_CUDA(cudaMemcpyAsync(si.e.p, x.p, field_bytes(TSM_F32, c.g.Vh), cudaMemcpyDeviceToDevice, c.stream));
    // s_o = A^-1 (b_o + kappa H_oe s_e)
    HopArgs<F32> h = hop_args<F32>(c, 1);
    h.in = si.e.as<F32>();
    h.center = bi.o.as<F32>();
    h.ac = 1.0;
    h.ah = k;
    h.to = twist_Ainv(k, mu);
    h.out = si.o.as<F32>();
    TSM_TRY(launch_hop<F32>(c, h, 0, HOP_CENTER, -1));
    res[i] = q;
  }
  return TSM_OK;
}

}  // namespace tsm
