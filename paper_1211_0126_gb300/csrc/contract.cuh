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
constexpr int CT_MAXCH = 2 * CT_MAXQ;   // real weight channels of one pass

struct GammaTab {
  int n;                       // insertions in use
  int8_t col[CT_MAXG][4];      // column of the non-zero in row a
  int8_t ph[CT_MAXG][4];       // its value i^ph (0: 1, 1: i, 2: -1, 3: -i)
  int8_t idx[CT_MAXG];         // which of the 16 chiral-basis insertions (chiral_code)
};

// The 16 insertions in the chiral basis, each a signed permutation whose
// non-zero in row a sits in column a ^ m: code bits 0-1 hold the mask m, bits
// 2 + 2a the power of i of row a's entry.  Order: 1, gamma_1..gamma_4,
// gamma_5, gamma_mu gamma_5 (mu = 1..4), sigma_{mu nu} = i/2 [gamma_mu,
// gamma_nu] for (mu, nu) = (1,2), (1,3), (1,4), (2,3), (2,4), (3,4).  The host
// checks every code against the matrices it builds from the gamma definitions
// before a contraction runs.
constexpr uint64_t kChiralCodes0 = 0x035e020b017f0000ull;   // insertions 0-3, 16 bits each
constexpr uint64_t kChiralCodes1 = 0x0223015702800002ull;   // 4-7
constexpr uint64_t kChiralCodes2 = 0x01dd0088002a0376ull;   // 8-11
constexpr uint64_t kChiralCodes3 = 0x00a0035d02a90281ull;   // 12-15

__host__ __device__ constexpr uint32_t chiral_code(int k) {
  return (uint32_t)(((k < 4 ? kChiralCodes0 : k < 8 ? kChiralCodes1 : k < 12 ? kChiralCodes2 : kChiralCodes3) >>
                     (16 * (k & 3))) & 0xffffu);
}

// The momenta of one pass grouped into classes {q, -q} (components mod L):
// e^{-iqx} = conj(e^{iqx}), so with A = sum_x cos(qx) G(x) and
// B = sum_x sin(qx) G(x) both members follow as A + i B and A - i B from two
// real-weighted sums.  Zero momentum has the single weight 1.
struct CtMoments {
  int ncls;                    // classes
  int nch;                     // real weight channels in use
  int ncp;                     // channels padded to a multiple of 4
  int8_t rep[CT_MAXQ];         // class -> momentum of the pass whose phase table it uses
  int8_t ch[CT_MAXQ];          // class -> its cosine channel (sine: ch + 1 when nz)
  int8_t nz[CT_MAXQ];          // class has a sine channel (non-zero momentum)
  int8_t qch[CT_MAXQ];         // momentum -> cosine channel of its class
  int8_t qsg[CT_MAXQ];         // momentum -> +1 / -1 (the class momentum or its negative), 0: zero momentum
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
  CtMoments mom;
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

// G_k = Tr[Gamma_k S^T] = sum_a Gamma_k[a][a ^ m_k] S[a][a ^ m_k] for all 16
// chiral insertions; the loops unroll, so every column and power of i is a
// constant and each trace is three complex additions
template <class R>
__device__ __forceinline__ void chiral_traces(const cx<R> (&S)[4][4], cx<R> (&G)[16]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t code = chiral_code(k);
    const int m = (int)(code & 3u);
    cx<R> v = times_ipow(S[0][m], (int)(code >> 2));
#pragma unroll
    for (int row = 1; row < 4; ++row) v = v + times_ipow(S[row][row ^ m], (int)(code >> (2 + 2 * row)));
    G[k] = v;
  }
}

template <class R> struct ContractNT { static constexpr int value = 128; };
template <> struct ContractNT<double> { static constexpr int value = 64; };

// Shared memory of a contraction block of NT sites, reused across phases:
//   stage   Gs[NT][CT_GS] complex (the 16 traces of each site) | Ws[ncp][NT + 1] (weights,
//           channel-major: a warp's stores of one channel hit 32 banks)
//   reduce  red[NT][CT_RS] (each thread's tile) | chan[16][CT_CHS] complex (channel sums)
constexpr int CT_GS = 17;            // complex row stride of Gs (16 + 1: no bank conflicts across sites)
constexpr int CT_RS = 36;            // row stride of red (32 + 4, rows stay 16-byte aligned)
constexpr int CT_CHS = CT_MAXCH + 1;
template <class R, int NT>
struct CtSmem {
  static constexpr size_t gs = (size_t)NT * CT_GS * 2 * sizeof(R);
  static constexpr size_t stage = gs + (size_t)(NT + 1) * CT_MAXCH * sizeof(R);
  static constexpr size_t red = (size_t)NT * CT_RS * sizeof(R);
  static constexpr size_t reduce = red + (size_t)CT_MAXG * CT_CHS * 2 * sizeof(R);
  static constexpr size_t bytes = stage > reduce ? stage : reduce;
};

// Stage one site of the block: its 16 traces and its weight channels (cos and
// sin of each momentum class); sites past the end stage zeros.
template <class R, int NT, class SA, class SB>
__device__ __forceinline__ void ct_stage(const ContractArgs<SA, SB>& a, unsigned char* smem, bool valid,
                                         const cx<R> (&S)[4][4], const int c[4]) {
  R* gs = reinterpret_cast<R*>(smem) + (size_t)threadIdx.x * CT_GS * 2;
  R* ws = reinterpret_cast<R*>(smem + CtSmem<R, NT>::gs) + threadIdx.x;   // channel ch at ws[ch * (NT + 1)]
  if (valid) {
    cx<R> G[16];
    chiral_traces(S, G);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      gs[2 * k] = G[k].re;
      gs[2 * k + 1] = G[k].im;
    }
    for (int k = 0; k < a.mom.ncls; ++k) {
      const cx<R> e = phase_at<R>(a, a.mom.rep[k], c);
      const int ch = a.mom.ch[k];
      ws[ch * (NT + 1)] = e.re;
      if (a.mom.nz[k]) ws[(ch + 1) * (NT + 1)] = e.im;
    }
    for (int ch = a.mom.nch; ch < a.mom.ncp; ++ch) ws[ch * (NT + 1)] = (R)0;
  } else {
#pragma unroll
    for (int k = 0; k < 32; ++k) gs[k] = (R)0;
    for (int ch = 0; ch < a.mom.ncp; ++ch) ws[ch * (NT + 1)] = (R)0;
  }
}

template <class R> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void store(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void store(double* p, double a, double b, double c, double d) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
  }
};
template <class R> struct Vec2;
template <> struct Vec2<float> {
  static __device__ __forceinline__ cx<float> load(const float* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return {v.x, v.y};
  }
};
template <> struct Vec2<double> {
  static __device__ __forceinline__ cx<double> load(const double* p) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    return {v.x, v.y};
  }
};

// Reduce the staged block (after a __syncthreads) to its partial sums of every
// requested (insertion, momentum).  Each thread owns a tile of 4 insertions x
// 4 channels (32 accumulators) over a slice of the block's sites (sites
// sl, sl + nsl, ...); the slices are then added in slice order in shared
// memory, and each output is formed from its class's cosine and sine sums
// (times f when MODE applies a factor).  A fixed order throughout.
template <class R, int NT, bool FACTOR, class SA, class SB>
__device__ __forceinline__ void ct_reduce(const ContractArgs<SA, SB>& a, unsigned char* smem, int t, int parity) {
  const int tid = threadIdx.x;
  const int ng = a.gam.n, ncp = a.mom.ncp;
  const int gt_n = (ng + 3) >> 2, ct_n = ncp >> 2, types = gt_n * ct_n;
  const int nsl = NT / types;
  const int type = tid % types, sl = tid / types;
  const bool active = sl < nsl;
  R acc[4][4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[r][u][0] = acc[r][u][1] = (R)0;
  if (active) {
    const R* Gs = reinterpret_cast<const R*>(smem);
    const R* Ws = reinterpret_cast<const R*>(smem + CtSmem<R, NT>::gs);
    const int gt = type % gt_n, ct = type / gt_n;
    int go[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gi = 4 * gt + r;
      go[r] = 2 * (gi < ng ? (int)a.gam.idx[gi] : 0);
    }
    for (int s = sl; s < NT; s += nsl) {
      const R* grow = Gs + (size_t)s * CT_GS * 2;
      cx<R> gv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) gv[r] = Vec2<R>::load(grow + go[r]);
      R w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) w[u] = Ws[(4 * ct + u) * (NT + 1) + s];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[r][u][0] = fma(w[u], gv[r].re, acc[r][u][0]);
          acc[r][u][1] = fma(w[u], gv[r].im, acc[r][u][1]);
        }
    }
  }
  __syncthreads();   // the staged block is consumed
  R* red = reinterpret_cast<R*>(smem);
  R* chan = reinterpret_cast<R*>(smem + CtSmem<R, NT>::red);   // [16][CT_CHS] complex
  if (active) {
    R* row = red + (size_t)tid * CT_RS;   // 16-byte vector stores: no bank conflicts
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int u = 0; u < 4; u += 2)
        Vec4<R>::store(row + (r * 4 + u) * 2, acc[r][u][0], acc[r][u][1], acc[r][u + 1][0], acc[r][u + 1][1]);
  }
  __syncthreads();
  for (int x = tid; x < types * 32; x += NT) {
    const int ty = x >> 5, e = x & 31;
    R sum = (R)0;
    for (int s2 = 0; s2 < nsl; ++s2) sum += red[(size_t)(s2 * types + ty) * CT_RS + e];
    const int gi = 4 * (ty % gt_n) + (e >> 3), ch = 4 * (ty / gt_n) + ((e >> 1) & 3);
    if (gi < ng) chan[(gi * CT_CHS + ch) * 2 + (e & 1)] = sum;
  }
  __syncthreads();
  const int nout = ng * a.nq;
  double2* dst = a.partial + ((size_t)(t * 2 + parity) * a.nbx + blockIdx.x) * nout;
  for (int k = tid; k < nout; k += NT) {
    const int gi = k % ng, q = k / ng;
    const R* cs = chan + (gi * CT_CHS + a.mom.qch[q]) * 2;
    cx<R> v = {cs[0], cs[1]};
    const int sg = a.mom.qsg[q];
    if (sg > 0) v = {cs[0] - cs[3], cs[1] + cs[2]};         // A + i B
    else if (sg < 0) v = {cs[0] + cs[3], cs[1] - cs[2]};    // A - i B
    if constexpr (FACTOR) v = (sizeof(R) == 4 ? cx<R>{(R)a.ffre, (R)a.ffim} : cx<R>{(R)a.fre, (R)a.fim}) * v;
    dst[k] = make_double2((double)v.re, (double)v.im);
  }
}

enum { CT_STANDARD = 0, CT_ONE_END = 1, CT_GEN_ONE_END = 2 };

template <class R, class SA, class SB, int MODE>
__global__ void __launch_bounds__(ContractNT<R>::value) contract_kernel(const ContractArgs<SA, SB> a) {
  constexpr bool OE = MODE == CT_ONE_END;
  constexpr int NT = ContractNT<R>::value;
  __shared__ __align__(16) unsigned char smem[CtSmem<R, NT>::bytes];
  const int t = blockIdx.y, parity = blockIdx.z;
  const int vs2 = a.g.L[0] * a.g.L[1] * a.g.L[2] / 2;
  const int local = blockIdx.x * NT + threadIdx.x;
  const bool valid = local < vs2;
  cx<R> S[4][4];
  int c[4] = {0, 0, 0, 0};
  if (valid) {
    const int ih = t * vs2 + local;
    site_coords(a.g, parity, ih, c);
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
  }
  ct_stage<R, NT>(a, smem, valid, S, c);
  __syncthreads();
  ct_reduce<R, NT, MODE != CT_STANDARD>(a, smem, t, parity);
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
  __shared__ __align__(16) unsigned char smem[CtSmem<R, NT>::bytes];
  const int t = blockIdx.y, parity = blockIdx.z;
  const int vs2 = a.g.L[0] * a.g.L[1] * a.g.L[2] / 2;
  const int local = blockIdx.x * NT + threadIdx.x;
  const bool valid = local < vs2;
  const int mu = d.mu;
  cx<R> S[4][4];
  int c[4] = {0, 0, 0, 0};
  if (valid) {
    const int ih = t * vs2 + local;
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
  }
  ct_stage<R, NT>(a, smem, valid, S, c);
  __syncthreads();
  ct_reduce<R, NT, false>(a, smem, t, parity);
}

// sum the block partials of one timeslice in fixed order into the output
// layout [g][q][t] (momenta q0 .. q0+nq-1 of nq_total).  A block per
// (timeslice, 32 consecutive outputs k = q * ng + g): lane = output, so every
// load of a warp is one contiguous run; warp w adds the partial rows w, w + 8,
// ... (row = parity * nbx + block) in increasing order with four loads in
// flight, then warp 0 adds the eight warp sums in warp order.
constexpr int CT_RED_WARPS = 8;
static __global__ void __launch_bounds__(32 * CT_RED_WARPS)
contract_reduce_kernel(const double2* __restrict__ partial, int T, int nbx, int ng, int nq, int nq_total, int q0,
                       double2* __restrict__ out) {
  __shared__ double2 sh[CT_RED_WARPS][32];
  const int nout = ng * nq, t = blockIdx.y, rows = 2 * nbx;
  const int gq = blockIdx.x * 32 + threadIdx.x, w = threadIdx.y;
  double re = 0.0, im = 0.0;
  if (gq < nout) {
    const double2* col = partial + (size_t)t * rows * nout + gq;
    int i = w;
    for (; i + 3 * CT_RED_WARPS < rows; i += 4 * CT_RED_WARPS) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = col[(size_t)(i + u * CT_RED_WARPS) * nout];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        re += v[u].x;
        im += v[u].y;
      }
    }
    for (; i < rows; i += CT_RED_WARPS) {
      const double2 v = col[(size_t)i * nout];
      re += v.x;
      im += v.y;
    }
  }
  sh[w][threadIdx.x] = make_double2(re, im);
  __syncthreads();
  if (w == 0 && gq < nout) {
#pragma unroll
    for (int u = 1; u < CT_RED_WARPS; ++u) {
      re += sh[u][threadIdx.x].x;
      im += sh[u][threadIdx.x].y;
    }
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
