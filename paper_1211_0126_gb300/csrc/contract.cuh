// contract.cuh -- loop contraction with timeslice / momentum reduction, and the
// TSM combine.
//
// Per source j and site x:  S_ab(x) = sum_c conj(eta_a,c(x)) s_b,c(x)  (4x4 in spin),
// Gamma_g trace  G_g(x) = sum_a Gamma_g[a][col_g(a)] S_{a, col_g(a)}  (every
// insertion has one non-zero per row, a power of i), and
// L(g, q, t) = sum_{x: x_4 = t} e^{i q.x} G_g(x).
// The noise is regenerated from the counter generator, never read from memory.
//
// One-end trick (Eq. 2.5, OE = true): S_ab = sum_c conj(s_a,c) s_b,c of the
// solution itself, the trace taken with gamma5 Gamma (rows 2, 3 negated) and
// the result multiplied by f = -4 i kappa mu; with a second field b the value
// is f [s_a^dag g5 Gamma s_a - s_b^dag g5 Gamma s_b], formed without
// cancellation as conj(d) a + conj(b) d with d = a - b.
//
// Generalised one-end trick (Eq. 2.6, MODE 2): S_ab = sum_c conj(s_a,c)
// (D_W s)_b,c with D_W s supplied by the caller, the trace taken with
// gamma5 Gamma gamma5 (rows and columns 2, 3 negated) and the factor 2; with
// a second field, minus the same for s_b.
// Phases come from per-axis FP64 tables built on the host (no device sin/cos).
#pragma once

#include "common.cuh"

namespace tsm {

constexpr int CT_MAXG = 16;
constexpr int CT_MAXQ = 16;

struct GammaTab {
  int n;                       // insertions in use
  int8_t col[CT_MAXG][4];      // column of the non-zero in row a
  int8_t ph[CT_MAXG][4];       // its value i^ph (0: 1, 1: i, 2: -1, 3: -i)
};

template <class SA, class SB>
struct ContractArgs {
  Geom g;
  NoiseSpec noise;
  uint32_t source;
  const typename SA::schunk* a[2];   // even, odd
  const typename SB::schunk* b[2];   // may be null
  const typename SA::schunk* wa[2];  // MODE 2: D_W a
  const typename SB::schunk* wb[2];  // MODE 2: D_W b (when b is given)
  int sstride;
  GammaTab gam;
  int nq;
  const double2* phx;   // [nq][Lx]
  const double2* phy;   // [nq][Ly]
  const double2* phz;   // [nq][Lz]
  double2* partial;     // [T][2][nbx][ng*nq]
  int nbx;
  double fre, fim;      // one-end factor -4 i kappa mu (OE only)
  const float2* fphx;   // phase tables and factor rounded once to FP32 on the host
  const float2* fphy;
  const float2* fphz;
  float ffre, ffim;
};

// e^{i q.x} of momentum q (of this pass) at site c, from the per-axis tables
template <class R, class SA, class SB>
__device__ __forceinline__ cx<R> phase_at(const ContractArgs<SA, SB>& a, int q, const int c[4]) {
  if constexpr (sizeof(R) == 4) {
    const float2 ex = __ldg(a.fphx + q * a.g.L[0] + c[0]);
    const float2 ey = __ldg(a.fphy + q * a.g.L[1] + c[1]);
    const float2 ez = __ldg(a.fphz + q * a.g.L[2] + c[2]);
    return (cx<R>{ex.x, ex.y} * cx<R>{ey.x, ey.y}) * cx<R>{ez.x, ez.y};
  } else {
    const double2 ex = __ldg(a.phx + q * a.g.L[0] + c[0]);
    const double2 ey = __ldg(a.phy + q * a.g.L[1] + c[1]);
    const double2 ez = __ldg(a.phz + q * a.g.L[2] + c[2]);
    return (cx<R>{ex.x, ex.y} * cx<R>{ey.x, ey.y}) * cx<R>{ez.x, ez.y};
  }
}

template <class R>
__device__ __forceinline__ cx<R> times_ipow(cx<R> v, int p) {
  switch (p & 3) {
    case 0: return v;
    case 1: return {-v.im, v.re};
    case 2: return {-v.re, -v.im};
    default: return {v.im, -v.re};
  }
}

// sum over the block's sites of phase(q) x density(g): four interleaved
// accumulators (sites s, s+4, ...) added pairwise at the end, so that the
// dependent FMA chain is a quarter as long; a fixed order
template <int NT, class R, int LD>
__device__ __forceinline__ cx<R> block_phase_sum(const cx<R> (*Ps)[LD], const cx<R> (*Gs)[LD], int q, int gi) {
  cx<R> a0 = {0, 0}, a1 = {0, 0}, a2 = {0, 0}, a3 = {0, 0};
#pragma unroll 4
  for (int s2 = 0; s2 < NT; s2 += 4) {
    a0 = a0 + Ps[s2][q] * Gs[s2][gi];
    a1 = a1 + Ps[s2 + 1][q] * Gs[s2 + 1][gi];
    a2 = a2 + Ps[s2 + 2][q] * Gs[s2 + 2][gi];
    a3 = a3 + Ps[s2 + 3][q] * Gs[s2 + 3][gi];
  }
  return (a0 + a1) + (a2 + a3);
}

template <class R> struct ContractNT { static constexpr int value = 128; };
template <> struct ContractNT<double> { static constexpr int value = 64; };

enum { CT_STANDARD = 0, CT_ONE_END = 1, CT_GEN_ONE_END = 2 };

template <class R, class SA, class SB, int MODE>
__global__ void __launch_bounds__(ContractNT<R>::value) contract_kernel(const ContractArgs<SA, SB> a) {
  constexpr bool OE = MODE == CT_ONE_END;
  constexpr int NT = ContractNT<R>::value;
  __shared__ cx<R> Gs[NT][CT_MAXG + 1];
  __shared__ cx<R> Ps[NT][CT_MAXQ + 1];
  const int t = blockIdx.y, parity = blockIdx.z;
  const int vs2 = a.g.L[0] * a.g.L[1] * a.g.L[2] / 2;
  const int local = blockIdx.x * NT + threadIdx.x;
  const int ng = a.gam.n, nq = a.nq;
  if (local < vs2) {
    const int ih = t * vs2 + local;
    int c[4];
    site_coords(a.g, parity, ih, c);
    cx<R> S[4][4];
    if constexpr (MODE == CT_GEN_ONE_END) {
      cx<typename SA::real> va[12], wa[12];
      load_spinor<SA>(a.a[parity], a.sstride, ih, va);
      load_spinor<SA>(a.wa[parity], a.sstride, ih, wa);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          cx<R> acc = {0, 0};
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
            acc = acc + cjmul(cx<R>{(R)va[3 * x + cc].re, (R)va[3 * x + cc].im},
                              cx<R>{(R)wa[3 * y + cc].re, (R)wa[3 * y + cc].im});
          S[x][y] = acc;
        }
      if (a.b[0] != nullptr) {
        cx<typename SB::real> vb[12], wb[12];
        load_spinor<SB>(a.b[parity], a.sstride, ih, vb);
        load_spinor<SB>(a.wb[parity], a.sstride, ih, wb);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            cx<R> acc = {0, 0};
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
              acc = acc + cjmul(cx<R>{(R)vb[3 * x + cc].re, (R)vb[3 * x + cc].im},
                                cx<R>{(R)wb[3 * y + cc].re, (R)wb[3 * y + cc].im});
            S[x][y] = S[x][y] - acc;
          }
      }
      // gamma5 Gamma gamma5: rows and columns 2, 3 change sign
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
          if ((x >= 2) != (y >= 2)) S[x][y] = (R)(-1) * S[x][y];
    } else if constexpr (!OE) {
      const uint32_t lex = (uint32_t)(((c[3] * a.g.L[2] + c[2]) * a.g.L[1] + c[1]) * a.g.L[0] + c[0]);
      cx<R> eta[12], s[12];
      noise_site<R>(a.noise, lex, a.source, eta);
      {
        cx<typename SA::real> va[12];
        load_spinor<SA>(a.a[parity], a.sstride, ih, va);
        if (a.b[0] != nullptr) {
          cx<typename SB::real> vb[12];
          load_spinor<SB>(a.b[parity], a.sstride, ih, vb);
          using W = typename SA::real;  // subtract in the solution's own precision
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const W re = va[k].re - (W)vb[k].re, im = va[k].im - (W)vb[k].im;
            s[k] = {(R)re, (R)im};
          }
        } else {
#pragma unroll
          for (int k = 0; k < 12; ++k) s[k] = {(R)va[k].re, (R)va[k].im};
        }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          cx<R> acc = cjmul(eta[3 * x], s[3 * y]);
          acc = acc + cjmul(eta[3 * x + 1], s[3 * y + 1]);
          acc = acc + cjmul(eta[3 * x + 2], s[3 * y + 2]);
          S[x][y] = acc;
        }
    } else {
      cx<R> sa[12];
      cx<typename SA::real> va[12];
      load_spinor<SA>(a.a[parity], a.sstride, ih, va);
#pragma unroll
      for (int k = 0; k < 12; ++k) sa[k] = {(R)va[k].re, (R)va[k].im};
      if (a.b[0] != nullptr) {
        cx<typename SB::real> vb[12];
        load_spinor<SB>(a.b[parity], a.sstride, ih, vb);
        using W = typename SA::real;
        cx<R> d[12], sb[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const W re = va[k].re - (W)vb[k].re, im = va[k].im - (W)vb[k].im;
          d[k] = {(R)re, (R)im};
          sb[k] = {(R)vb[k].re, (R)vb[k].im};
        }
        // a^dag X a - b^dag X b = d^dag X a + b^dag X d
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            cx<R> acc = {0, 0};
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
              acc = acc + cjmul(d[3 * x + cc], sa[3 * y + cc]) + cjmul(sb[3 * x + cc], d[3 * y + cc]);
            S[x][y] = acc;
          }
      } else {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            cx<R> acc = cjmul(sa[3 * x], sa[3 * y]);
            acc = acc + cjmul(sa[3 * x + 1], sa[3 * y + 1]);
            acc = acc + cjmul(sa[3 * x + 2], sa[3 * y + 2]);
            S[x][y] = acc;
          }
      }
      // gamma5 Gamma: rows 2 and 3 of Gamma change sign in the chiral basis
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        S[2][y] = (R)(-1) * S[2][y];
        S[3][y] = (R)(-1) * S[3][y];
      }
    }
    for (int k = 0; k < ng; ++k) {
      cx<R> v = {0, 0};
#pragma unroll
      for (int row = 0; row < 4; ++row) {
        const int col = a.gam.col[k][row];
        cx<R> sv;
        switch (col) {   // keep S in registers: no dynamic indexing
          case 0: sv = S[row][0]; break;
          case 1: sv = S[row][1]; break;
          case 2: sv = S[row][2]; break;
          default: sv = S[row][3]; break;
        }
        v = v + times_ipow(sv, a.gam.ph[k][row]);
      }
      if constexpr (MODE != CT_STANDARD)
        v = (sizeof(R) == 4 ? cx<R>{(R)a.ffre, (R)a.ffim} : cx<R>{(R)a.fre, (R)a.fim}) * v;
      Gs[threadIdx.x][k] = v;
    }
    for (int q = 0; q < nq; ++q) Ps[threadIdx.x][q] = phase_at<R>(a, q, c);
  } else {
    for (int k = 0; k < ng; ++k) Gs[threadIdx.x][k] = {0, 0};
    for (int q = 0; q < nq; ++q) Ps[threadIdx.x][q] = {0, 0};
  }
  __syncthreads();
  // one (g, q) output per thread: sum over the block's sites in site order
  const int nout = ng * nq;
  double2* dst = a.partial + ((size_t)(t * 2 + parity) * a.nbx + blockIdx.x) * nout;
  for (int k = threadIdx.x; k < nout; k += NT) {
    const int gi = k % ng, q = k / ng;
    const cx<R> acc = block_phase_sum<NT>(Ps, Gs, q, gi);
    dst[k] = make_double2((double)acc.re, (double)acc.im);
  }
}

// ---------------------------------------------------------------- one-derivative insertions
// Symmetric covariant derivative along mu (reading stated with the oracle):
//   1/4 [eta(x)^dag Gamma (T+ s - T- s)(x) - ((T+ eta - T- eta)(x))^dag Gamma s(x)],
//   T+ f(x) = U_mu(x) f(x+mu), T- f(x) = U_mu(x-mu)^dag f(x-mu), fermion sign on
// hops across t = T-1 <-> 0.  s = a - b when b is given (linear in s).  Noise at
// the neighbours is regenerated like at x.  Links: F64 (three rows) for R =
// double, FP32 two-row with the third row rebuilt for R = float.
template <class R> struct DerivLinks { using type = F32; };
template <> struct DerivLinks<double> { using type = F64; };

template <class SA, class SB, class LS>
struct DerivArgs {
  ContractArgs<SA, SB> base;
  const typename LS::lchunk* U[2];   // links of each parity
  int lstride;
  int mu;
};

template <class R, class SA, class SB>
__device__ __forceinline__ void deriv_field(const ContractArgs<SA, SB>& a, int parity, int ih, cx<R> s[12]) {
  cx<typename SA::real> va[12];
  load_spinor<SA>(a.a[parity], a.sstride, ih, va);
  if (a.b[0] != nullptr) {
    cx<typename SB::real> vb[12];
    load_spinor<SB>(a.b[parity], a.sstride, ih, vb);
    using W = typename SA::real;
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = {(R)(va[k].re - (W)vb[k].re), (R)(va[k].im - (W)vb[k].im)};
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = {(R)va[k].re, (R)va[k].im};
  }
}

// out[s][a] = sign * (U f)_s,a (DAGU: U^dag f), per spin
template <bool DAGU, class R>
__device__ __forceinline__ void colour_mul(const cx<R> u[9], const cx<R> f[12], R sign, cx<R> out[12]) {
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> acc = {0, 0};
#pragma unroll
      for (int b = 0; b < 3; ++b) acc = acc + (DAGU ? cjmul(u[3 * b + a], f[3 * sp + b]) : u[3 * a + b] * f[3 * sp + b]);
      out[3 * sp + a] = sign * acc;
    }
}

template <class R, class SA, class SB, class LS>
__global__ void __launch_bounds__(ContractNT<R>::value) deriv_contract_kernel(const DerivArgs<SA, SB, LS> d) {
  constexpr int NT = ContractNT<R>::value;
  const ContractArgs<SA, SB>& a = d.base;
  __shared__ cx<R> Gs[NT][CT_MAXG + 1];
  __shared__ cx<R> Ps[NT][CT_MAXQ + 1];
  const int t = blockIdx.y, parity = blockIdx.z;
  const int vs2 = a.g.L[0] * a.g.L[1] * a.g.L[2] / 2;
  const int local = blockIdx.x * NT + threadIdx.x;
  const int ng = a.gam.n, nq = a.nq;
  const int mu = d.mu;
  if (local < vs2) {
    const int ih = t * vs2 + local;
    int c[4];
    site_coords(a.g, parity, ih, c);
    const Geom& g = a.g;
    const uint32_t lex = (uint32_t)(((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0]);
    int cf[4] = {c[0], c[1], c[2], c[3]}, cb[4] = {c[0], c[1], c[2], c[3]};
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (m == mu) {
        cf[m] = (c[m] + 1 == g.L[m]) ? 0 : c[m] + 1;
        cb[m] = (c[m] == 0) ? g.L[m] - 1 : c[m] - 1;
      }
    const R sf = (mu == 3 && g.apbc && c[3] == g.L[3] - 1) ? (R)-1 : (R)1;
    const R sb = (mu == 3 && g.apbc && c[3] == 0) ? (R)-1 : (R)1;
    const uint32_t lexf = (uint32_t)(((cf[3] * g.L[2] + cf[2]) * g.L[1] + cf[1]) * g.L[0] + cf[0]);
    const uint32_t lexb = (uint32_t)(((cb[3] * g.L[2] + cb[2]) * g.L[1] + cb[1]) * g.L[0] + cb[0]);
    const int hf = (int)(lexf >> 1), hb = (int)(lexb >> 1);
    cx<R> uf[9], ub[9];
    {
      cx<typename LS::real> r[9];
      load_link<LS>(d.U[parity], d.lstride, mu, ih, r);
      if constexpr (!LS::full_links) third_row(r, r + 6);
#pragma unroll
      for (int k = 0; k < 9; ++k) uf[k] = {(R)r[k].re, (R)r[k].im};
      load_link<LS>(d.U[1 - parity], d.lstride, mu, hb, r);
      if constexpr (!LS::full_links) third_row(r, r + 6);
#pragma unroll
      for (int k = 0; k < 9; ++k) ub[k] = {(R)r[k].re, (R)r[k].im};
    }
    cx<R> eta[12], s[12], ds[12], de[12], tmp[12], f[12];
    noise_site<R>(a.noise, lex, a.source, eta);
    deriv_field<R>(a, parity, ih, s);
    // D s = T+ s - T- s
    deriv_field<R>(a, 1 - parity, hf, f);
    colour_mul<false>(uf, f, sf, ds);
    deriv_field<R>(a, 1 - parity, hb, f);
    colour_mul<true>(ub, f, sb, tmp);
#pragma unroll
    for (int k = 0; k < 12; ++k) ds[k] = ds[k] - tmp[k];
    // D eta = T+ eta - T- eta
    noise_site<R>(a.noise, lexf, a.source, f);
    colour_mul<false>(uf, f, sf, de);
    noise_site<R>(a.noise, lexb, a.source, f);
    colour_mul<true>(ub, f, sb, tmp);
#pragma unroll
    for (int k = 0; k < 12; ++k) de[k] = de[k] - tmp[k];
    cx<R> S[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        cx<R> acc = {0, 0};
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
          acc = acc + cjmul(eta[3 * x + cc], ds[3 * y + cc]) - cjmul(de[3 * x + cc], s[3 * y + cc]);
        S[x][y] = (R)0.25 * acc;
      }
    for (int k = 0; k < ng; ++k) {
      cx<R> v = {0, 0};
#pragma unroll
      for (int row = 0; row < 4; ++row) {
        const int col = a.gam.col[k][row];
        cx<R> sv;
        switch (col) {
          case 0: sv = S[row][0]; break;
          case 1: sv = S[row][1]; break;
          case 2: sv = S[row][2]; break;
          default: sv = S[row][3]; break;
        }
        v = v + times_ipow(sv, a.gam.ph[k][row]);
      }
      Gs[threadIdx.x][k] = v;
    }
    for (int q = 0; q < nq; ++q) Ps[threadIdx.x][q] = phase_at<R>(a, q, c);
  } else {
    for (int k = 0; k < ng; ++k) Gs[threadIdx.x][k] = {0, 0};
    for (int q = 0; q < nq; ++q) Ps[threadIdx.x][q] = {0, 0};
  }
  __syncthreads();
  const int nout = ng * nq;
  double2* dst = a.partial + ((size_t)(t * 2 + parity) * a.nbx + blockIdx.x) * nout;
  for (int k = threadIdx.x; k < nout; k += NT) {
    const int gi = k % ng, q = k / ng;
    const cx<R> acc = block_phase_sum<NT>(Ps, Gs, q, gi);
    dst[k] = make_double2((double)acc.re, (double)acc.im);
  }
}

// sum the block partials of one timeslice in fixed order into the output
// layout [g][q][t] (momenta q0 .. q0+nq-1 of nq_total)
// one warp per output k = t * (ng * nq) + (q * ng + g): lane l adds the
// block partials l, l + 32, ... of both parities, then a fixed shuffle tree
static __global__ void contract_reduce_kernel(const double2* __restrict__ partial, int T, int nbx, int ng, int nq,
                                       int nq_total, int q0, double2* __restrict__ out) {
  const int k = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  const int nout = ng * nq;
  if (k >= nout * T) return;   // the same for the whole warp
  const int t = k / nout, gq = k % nout;
  double re = 0.0, im = 0.0;
  for (int i = lane; i < 2 * nbx; i += 32) {
    const int par = i / nbx, b = i % nbx;
    const double2 v = partial[((size_t)(t * 2 + par) * nbx + b) * nout + gq];
    re += v.x;
    im += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    const int gi = gq % ng, q = gq / ng;
    out[((size_t)gi * nq_total + q0 + q) * T + t] = make_double2(re, im);
  }
}

// Eq. 2.4 per entry: mean of the corrections + mean of the LP set; error from
// the unbiased complex sample variances, two passes in source order.
static __global__ void combine_kernel(const double2* __restrict__ corr, int n_hp, const double2* __restrict__ lp, int n_lp,
                               int E, double2* __restrict__ est, double* __restrict__ err,
                               double2* __restrict__ lp_mean, double2* __restrict__ corr_mean) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double mcr = 0.0, mci = 0.0, mlr = 0.0, mli = 0.0, var = 0.0;
  if (n_hp > 0) {
    for (int j = 0; j < n_hp; ++j) {
      const double2 v = corr[(size_t)j * E + e];
      mcr += v.x;
      mci += v.y;
    }
    mcr /= n_hp;
    mci /= n_hp;
    if (n_hp > 1) {
      double s = 0.0;
      for (int j = 0; j < n_hp; ++j) {
        const double2 v = corr[(size_t)j * E + e];
        const double dr = v.x - mcr, di = v.y - mci;
        s += dr * dr + di * di;
      }
      var += s / (n_hp - 1) / n_hp;
    }
  }
  if (n_lp > 0) {
    for (int j = 0; j < n_lp; ++j) {
      const double2 v = lp[(size_t)j * E + e];
      mlr += v.x;
      mli += v.y;
    }
    mlr /= n_lp;
    mli /= n_lp;
    if (n_lp > 1) {
      double s = 0.0;
      for (int j = 0; j < n_lp; ++j) {
        const double2 v = lp[(size_t)j * E + e];
        const double dr = v.x - mlr, di = v.y - mli;
        s += dr * dr + di * di;
      }
      var += s / (n_lp - 1) / n_lp;
    }
  }
  if (est) est[e] = make_double2(mcr + mlr, mci + mli);
  if (err) err[e] = sqrt(var);
  if (lp_mean) lp_mean[e] = make_double2(mlr, mli);
  if (corr_mean) corr_mean[e] = make_double2(mcr, mci);
}

}  // namespace tsm
