// fft.cu -- loops at every spatial momentum: per-site insertion densities,
// a 3-D discrete Fourier transform per source written for this library, and
// running per-entry means and variances in source order (Welford), so that no
// per-source momentum grid is stored.  (The paper's Sec. 3 Fourier-transforms
// the loops with a vendor FFT library; here the transform is the library's
// own kernels.)
//
//   L_j(Gamma, t, n) = sum_{x: x_4 = t} e^{+2 pi i (n_x x / Lx + n_y y / Ly + n_z z / Lz)}
//                      eta_j(x)^dag Gamma (s_a - s_b)(x),
//
// output layout [n_gamma][T][Lz][Ly][Lx] with n_x, n_y, n_z in [0, L).
//
// Transform: separable, one axis after the other, each line by an in-place
// mixed-radix decimation-in-frequency FFT in shared memory (Cooley & Tukey
// 1965; Gentleman & Sande 1966): a stage of radix R on blocks of length Ls
// replaces the R inputs j + r Ls / R of a block by their length-R DFT, output
// k multiplied by w_Ls^{j k}, in the same R places, so each place belongs to
// one butterfly and one barrier per stage suffices.  The result is stored in
// digit-reversed order; frequency n sits at pos(n) = sum_s (n_s) N / (R_1 ..
// R_s) with n_s the mixed-radix digits of n, and the writes read it from
// there.  Radices 8, 4, 2 and 3 have register butterflies, 5, 7, 11 and 13 a
// direct DFT of that length.  Twiddles e^{+2 pi i m / N} come from a host
// table evaluated in FP64.  Warps walk the axis of unit stride (along a row
// for x, across lines for y and z), so shared-memory accesses are
// conflict-free apart from the butterfly spread.  Two kernels per source:
//
//   fft_xy_kernel  one CTA per (t, z) plane: the densities of the plane's
//                  Lx * Ly sites for a chunk of insertions go straight into
//                  shared memory, every row is x-transformed and every column
//                  y-transformed there, and the plane is written once.
//   fft_z_kernel   one CTA per (Gamma, t) slice and band of W columns (y, x):
//                  the band's Lz rows are read coalesced, z-transformed in
//                  shared memory, then written back (a single transform) or
//                  folded into the running moments of their entries without
//                  being stored (the TSM over all momenta).
//
// Per source and entry that is one write and one read of the partly
// transformed densities plus the moments' read and write.
#include <algorithm>
#include <cmath>
#include <vector>

#include "contract.h"
#include "fft.h"

namespace tsm {

namespace {

constexpr int FFT_XY_NT = 512;
// resident xy CTAs per SM the kernel is compiled for: two in FP32 (at most 64
// registers; 16 insertions of a 24 x 24 plane take 74 KB of shared memory),
// one in FP64 (the planes take twice the space)
template <class R> struct XYMinBlocks { static constexpr int value = sizeof(R) == 4 ? 2 : 1; };
constexpr int FFT_Z_NT = 256;
constexpr size_t FFT_SMEM_BUDGET = 200 * 1024;   // dynamic shared memory per CTA at most

template <class R> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <class R>
__device__ __forceinline__ cx<R> ld2(const cx<R>* p) {
  const typename Vec2<R>::type v = *reinterpret_cast<const typename Vec2<R>::type*>(p);
  return {v.x, v.y};
}
template <class R>
__device__ __forceinline__ void st2(cx<R>* p, cx<R> v) {
  typename Vec2<R>::type w;
  w.x = v.re;
  w.y = v.im;
  *reinterpret_cast<typename Vec2<R>::type*>(p) = w;
}

// n / d as a multiply-high, exact whenever n * d < 2^32 (m = floor(2^32 / d)
// + 1, computed as floor((2^32 - 1) / d) + 1, which is 2^32 / d for a power of
// two; d = 1: m = 0).  Every quotient below has n * d < 2^24.
struct Div {
  uint32_t d, m;
};
__host__ __device__ __forceinline__ Div make_div(int d) {
  Div r;
  r.d = (uint32_t)d;
  r.m = d <= 1 ? 0u : 0xFFFFFFFFu / (uint32_t)d + 1u;
  return r;
}
__device__ __forceinline__ int divq(int n, Div v) { return v.m ? (int)__umulhi((uint32_t)n, v.m) : n; }

// One in-place DIF stage st of an axis over nlines lines: element k of line l
// sits at buf[(l / lpp) * pstride + (l % lpp) * lstride + k * estride].  With
// Ls the current block length and M = Ls / R, butterfly (block b, j < M) reads
// a_r = x[b Ls + j + r M], writes x[b Ls + j + k M] = w_Ls^{j k} sum_r a_r
// w_R^{r k}.  LF: consecutive threads take consecutive lines (lines of unit
// stride), else consecutive butterflies of one line (elements of unit stride).
template <class R, bool LF>
__device__ __forceinline__ void dif_stage(cx<R>* __restrict__ buf, const FftAxis& ax, int st, int nlines, Div dnl,
                                          Div dlpp, int lstride, int pstride, int estride,
                                          const cx<R>* __restrict__ tw) {
  const int radix = ax.radix[st];
  const Div dM = make_div(ax.m[st]);   // host-checked: m[st] = Ls / R
  const int M = ax.m[st];
  const int Ls = M * radix;
  const int per_line = ax.n / radix;
  const Div dpl = make_div(per_line);
  const int total = nlines * per_line;
  const int ts = ax.ts[st];            // N / Ls: w_Ls^m = w_N^{m ts}; j k ts < N
  const int es = M * estride;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int l, u;
    if (LF) {
      u = divq(w, dnl);
      l = w - u * nlines;
    } else {
      l = divq(w, dpl);
      u = w - l * per_line;
    }
    const int bk = divq(u, dM), j = u - bk * M;
    const int lq = divq(l, dlpp);
    cx<R>* p = buf + lq * pstride + (l - lq * (int)dlpp.d) * lstride + (bk * Ls + j) * estride;
    const int tj = j * ts;
    if (radix == 8) {
      // even and odd halves by 4-point DFTs, joined with w_8^k = e^{i pi k / 4}
      const R r2 = (R)0.70710678118654752440;   // 1 / sqrt(2)
      cx<R> E[4], O[4];
      {
        const cx<R> b0 = p[0], b1 = p[2 * es], b2 = p[4 * es], b3 = p[6 * es];
        const cx<R> s02 = b0 + b2, d02 = b0 - b2, s13 = b1 + b3, d13 = times_i(b1 - b3);
        E[0] = s02 + s13;
        E[1] = d02 + d13;
        E[2] = s02 - s13;
        E[3] = d02 - d13;
      }
      {
        const cx<R> b0 = p[es], b1 = p[3 * es], b2 = p[5 * es], b3 = p[7 * es];
        const cx<R> s02 = b0 + b2, d02 = b0 - b2, s13 = b1 + b3, d13 = times_i(b1 - b3);
        O[0] = s02 + s13;
        O[1] = d02 + d13;
        O[2] = s02 - s13;
        O[3] = d02 - d13;
      }
      O[1] = {r2 * (O[1].re - O[1].im), r2 * (O[1].re + O[1].im)};    // (1 + i) / sqrt 2
      O[2] = times_i(O[2]);                                             // i
      O[3] = {-r2 * (O[3].re + O[3].im), r2 * (O[3].re - O[3].im)};   // (-1 + i) / sqrt 2
      p[0] = E[0] + O[0];
#pragma unroll
      for (int k = 1; k < 4; ++k) p[k * es] = (E[k] + O[k]) * tw[k * tj];
#pragma unroll
      for (int k = 0; k < 4; ++k) p[(k + 4) * es] = (E[k] - O[k]) * tw[(k + 4) * tj];
    } else if (radix == 4) {
      const cx<R> a0 = p[0], a1 = p[es], a2 = p[2 * es], a3 = p[3 * es];
      const cx<R> p02 = a0 + a2, m02 = a0 - a2, p13 = a1 + a3, m13 = times_i(a1 - a3);
      p[0] = p02 + p13;                     // sum_r a_r i^{r k}, k = 0..3
      p[es] = (m02 + m13) * tw[tj];
      p[2 * es] = (p02 - p13) * tw[2 * tj];
      p[3 * es] = (m02 - m13) * tw[3 * tj];
    } else if (radix == 2) {
      const cx<R> a0 = p[0], a1 = p[es];
      p[0] = a0 + a1;
      p[es] = (a0 - a1) * tw[tj];
    } else if (radix == 3) {
      // w_3 = -1/2 + i sqrt(3)/2
      const R h = (R)0.86602540378443864676;
      const cx<R> a0 = p[0], a1 = p[es], a2 = p[2 * es];
      const cx<R> sp = a1 + a2, dm = a1 - a2;
      const cx<R> c = {a0.re - (R)0.5 * sp.re, a0.im - (R)0.5 * sp.im};
      const cx<R> e = times_i(h * dm);
      p[0] = a0 + sp;
      p[es] = (c + e) * tw[tj];
      p[2 * es] = (c - e) * tw[2 * tj];
    } else {
      // other primes (<= FFT_MAX_PRIME): the length-R DFT directly
      cx<R> a[FFT_MAX_PRIME];
      for (int r = 0; r < radix; ++r) a[r] = p[r * es];
      const int nr = per_line;   // w_R^q = w_N^{q N / R}
      for (int k = 0; k < radix; ++k) {
        cx<R> acc = a[0];
        for (int r = 1; r < radix; ++r) acc = acc + a[r] * tw[((r * k) % radix) * nr];
        p[k * es] = k ? acc * tw[k * tj] : acc;
      }
    }
  }
}

// all stages of one axis, in place; every thread of the block calls it
template <class R, bool LF>
__device__ void dif_lines(cx<R>* buf, const FftAxis& ax, int nlines, int lpp, int lstride, int pstride, int estride,
                          const cx<R>* tw) {
  const Div dnl = make_div(nlines), dlpp = make_div(lpp);
  for (int st = 0; st < ax.nst; ++st) {
    dif_stage<R, LF>(buf, ax, st, nlines, dnl, dlpp, lstride, pstride, estride, tw);
    __syncthreads();
  }
}

template <class R>
__device__ __forceinline__ void load_twiddles(const cx<double>* __restrict__ g, const int* __restrict__ gpos, int n,
                                              cx<R>* __restrict__ sh, int* __restrict__ spos) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const cx<double> v = g[i];
    sh[i] = {(R)v.re, (R)v.im};
    spos[i] = gpos[i];
  }
}

// Densities G_g(x) = eta^dag Gamma_g (a - b)(x) of plane (t, z) = blockIdx.x
// for insertions g0 .. g0 + gn - 1 (g0 = blockIdx.y * gc), then their x and y
// transforms; written to dens[g][t][z][y][x] in frequency order.  Every
// insertion of the library's list has one non-zero per row, in column
// row ^ m (chiral basis), so G_g = sum_row f_g,row S[row][row ^ m_g] with
// S[a][b] = sum_colour conj(eta_a) s_b and f = +-1, +-i.
template <class R, class SA, class SB>
__global__ void __launch_bounds__(FFT_XY_NT, XYMinBlocks<R>::value) fft_xy_kernel(
    Geom g, NoiseSpec noise, uint32_t source, const typename SA::schunk* a0, const typename SA::schunk* a1,
    const typename SB::schunk* b0, const typename SB::schunk* b1, int sstride, FftGam gam, FftPlan plan, int gc,
    const cx<double>* __restrict__ twg, const int* __restrict__ posg, cx<R>* __restrict__ dens) {
  extern __shared__ __align__(16) unsigned char fft_smem[];
  const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], T = g.L[3];
  const int P = Lx * Ly;
  const Div dLx = make_div(Lx), dP = make_div(P);
  cx<R>* planes = reinterpret_cast<cx<R>*>(fft_smem);     // gc density planes [k][y][x]
  cx<R>* tw = planes + (size_t)gc * P;                     // x table, then y table
  int* pos = reinterpret_cast<int*>(tw + Lx + Ly);         // x positions, then y positions
  const int t = blockIdx.x / Lz, z = blockIdx.x - t * Lz;
  const int g0 = blockIdx.y * gc;
  const int gn = min(gc, gam.n - g0);
  load_twiddles<R>(twg, posg, Lx + Ly, tw, pos);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const int y = divq(i, dLx), x = i - y * Lx;
    const int lex = ((t * Lz + z) * Ly + y) * Lx + x;
    const int parity = (x + y + z + t) & 1;
    const int ih = lex >> 1;
    cx<R> eta[12], s[12];
    noise_site<R>(noise, (uint32_t)lex, source, eta);
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
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        cx<R> acc = cjmul(eta[3 * r], s[3 * c]);
        acc = acc + cjmul(eta[3 * r + 1], s[3 * c + 1]);
        acc = acc + cjmul(eta[3 * r + 2], s[3 * c + 2]);
        S[r][c] = acc;
      }
    for (int k = 0; k < gn; ++k) {
      const int gi = g0 + k;
      cx<R> d[4];
      switch (gam.m[gi]) {   // the same in every thread
        case 0: d[0] = S[0][0]; d[1] = S[1][1]; d[2] = S[2][2]; d[3] = S[3][3]; break;
        case 1: d[0] = S[0][1]; d[1] = S[1][0]; d[2] = S[2][3]; d[3] = S[3][2]; break;
        case 2: d[0] = S[0][2]; d[1] = S[1][3]; d[2] = S[2][0]; d[3] = S[3][1]; break;
        default: d[0] = S[0][3]; d[1] = S[1][2]; d[2] = S[2][1]; d[3] = S[3][0]; break;
      }
      cx<R> v = {0, 0};
#pragma unroll
      for (int row = 0; row < 4; ++row) {
        const R fr = (R)gam.fr[gi][row], fi = (R)gam.fi[gi][row];
        v = {v.re + fr * d[row].re - fi * d[row].im, v.im + fr * d[row].im + fi * d[row].re};
      }
      planes[k * P + i] = v;
    }
  }
  __syncthreads();
  // rows: gn * Ly lines of Lx elements of unit stride
  dif_lines<R, false>(planes, plan.ax[0], gn * Ly, gn * Ly, Lx, 0, 1, tw);
  // columns: line (k, x) at k P + x, elements Lx apart, consecutive x in a warp
  dif_lines<R, true>(planes, plan.ax[1], gn * Lx, Lx, 1, P, Lx, tw + Lx);
  const int* px = pos;
  const int* py = pos + Lx;
  cx<R>* out = dens + ((size_t)(g0 * T + t) * Lz + z) * P;
  const size_t kstride = (size_t)T * Lz * P;
  for (int e = threadIdx.x; e < gn * P; e += blockDim.x) {
    const int k = divq(e, dP), i = e - k * P;
    const int ny = divq(i, dLx), nx = i - ny * Lx;
    st2(out + k * kstride + i, planes[k * P + py[ny] * Lx + px[nx]]);
  }
}

// What fft_z_kernel does with the transform of each entry.
struct ZSink {
  int mode;              // 0: write back to dens; 1: FP64 running moments; 2: FP32 batch sums
  double inv_k, wk;      // mode 1: 1/k and (k-1)/k of the k-th source (k = 1: assign)
  int first;             // mode 2: first source of the batch (assign instead of add)
  double2* mean;         // mode 1
  double* m2;
  float2* bsum;          // mode 2: sum of d = x - K over the batch
  float* bsq;            // mode 2: sum of |d|^2 over the batch
  float2* bshift;        // mode 2: K, the batch's first value of the entry
};

// z transform of a band of W columns c0 .. c0 + W - 1 (flattened (y, x)) of
// slice (g, t) = blockIdx.y, then the sink per entry.
template <class R>
__global__ void __launch_bounds__(FFT_Z_NT) fft_z_kernel(int P, int Lz, FftAxis axz, int W,
                                                         const cx<double>* __restrict__ twg,
                                                         const int* __restrict__ posg, cx<R>* __restrict__ dens,
                                                         ZSink sink) {
  extern __shared__ __align__(16) unsigned char fft_smem[];
  cx<R>* A = reinterpret_cast<cx<R>*>(fft_smem);   // [Lz][W]
  cx<R>* tw = A + (size_t)Lz * W;
  int* pz = reinterpret_cast<int*>(tw + Lz);
  const int c0 = blockIdx.x * W;
  const int wc = min(W, P - c0);
  const size_t base = (size_t)blockIdx.y * Lz * P + c0;
  const Div dwc = make_div(wc);
  load_twiddles<R>(twg, posg, Lz, tw, pz);
#pragma unroll 4
  for (int e = threadIdx.x; e < Lz * wc; e += blockDim.x) {
    const int z = divq(e, dwc), c = e - z * wc;
    A[z * W + c] = ld2(dens + base + (size_t)z * P + c);
  }
  __syncthreads();
  dif_lines<R, true>(A, axz, wc, wc, 1, 0, W, tw);
#pragma unroll 4
  for (int e = threadIdx.x; e < Lz * wc; e += blockDim.x) {
    const int nz = divq(e, dwc), c = e - nz * wc;
    const size_t idx = base + (size_t)nz * P + c;
    const cx<R> v = A[pz[nz] * W + c];
    if (sink.mode == 0) {
      st2(dens + idx, v);
    } else if (sink.mode == 2) {
      const float2 x = make_float2((float)v.re, (float)v.im);
      if (sink.first) {   // K = x: d = 0
        sink.bshift[idx] = x;
        sink.bsum[idx] = make_float2(0.f, 0.f);
        sink.bsq[idx] = 0.f;
      } else {
        const float2 k = sink.bshift[idx];
        const float dr = x.x - k.x, di = x.y - k.y;
        const float2 o = sink.bsum[idx];
        sink.bsum[idx] = make_float2(o.x + dr, o.y + di);
        sink.bsq[idx] = sink.bsq[idx] + (dr * dr + di * di);
      }
    } else {
      // Welford: mean += d / k, m2 += |d|^2 (k - 1) / k with d = x - mean
      const double xr = (double)v.re, xi = (double)v.im;
      if (sink.inv_k == 1.0) {
        sink.mean[idx] = make_double2(xr, xi);
        sink.m2[idx] = 0.0;
        continue;
      }
      const double2 mu = sink.mean[idx];
      const double dr = xr - mu.x, di = xi - mu.y;
      sink.mean[idx] = make_double2(mu.x + dr * sink.inv_k, mu.y + di * sink.inv_k);
      sink.m2[idx] += (dr * dr + di * di) * sink.wk;
    }
  }
}

// Merge a batch of nb sources (FP32 sums S of d = x - K and Q of |d|^2) into
// the running FP64 moments of the na sources before it (Chan, Golub &
// LeVeque's pairwise update): with the batch mean b = K + S / nb and
// M2_b = Q - |S|^2 / nb, mean += (b - mean) nb / n,
// m2 += M2_b + |b - mean|^2 na nb / n, n = na + nb.
__global__ void fft_merge_kernel(const float2* __restrict__ bsum, const float* __restrict__ bsq,
                                 const float2* __restrict__ bshift, int na, int nb, double2* __restrict__ mean,
                                 double* __restrict__ m2, long long E) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double inv_nb = 1.0 / (double)nb;   // uniform: one division per thread
  const float2 S = bsum[e], K = bshift[e];
  const double sr = (double)S.x * inv_nb, si = (double)S.y * inv_nb;
  const double br = (double)K.x + sr, bi = (double)K.y + si;
  const double m2b = fmax((double)bsq[e] - (sr * sr + si * si) * nb, 0.0);
  if (na == 0) {
    mean[e] = make_double2(br, bi);
    m2[e] = m2b;
    return;
  }
  const double n = (double)(na + nb);
  const double2 mu = mean[e];
  const double dr = br - mu.x, di = bi - mu.y;
  mean[e] = make_double2(mu.x + dr * (nb / n), mu.y + di * (nb / n));
  m2[e] += m2b + (dr * dr + di * di) * ((double)na * nb / n);
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

// radices of a line of length n: one 8 for an odd power of two >= 3, 4s, a 2
// for 2^1, then 3s, then the other primes;
// per stage the sub-block length after it (m) and n / (its block length) (ts)
int factorise_stages(int n, FftAxis* ax);
int factorise(int n, FftAxis* ax) {
  if (factorise_stages(n, ax) != TSM_OK) return TSM_ERR_TOO_LARGE;
  int ls = n;
  for (int st = 0; st < ax->nst; ++st) {
    ax->ts[st] = n / ls;
    ls /= ax->radix[st];
    ax->m[st] = ls;
  }
  return TSM_OK;
}
int factorise_stages(int n, FftAxis* ax) {
  ax->n = n;
  ax->nst = 0;
  int r = n;
  auto take_one = [&](int f) {
    if (ax->nst >= FFT_MAX_STAGES) return false;
    ax->radix[ax->nst++] = f;
    r /= f;
    return true;
  };
  auto take = [&](int f) {
    while (r % f == 0) {
      if (ax->nst >= FFT_MAX_STAGES) return false;
      ax->radix[ax->nst++] = f;
      r /= f;
    }
    return true;
  };
  // powers of two: radix 4 stages, and one radix 8 (odd power >= 3) or 2 (2^1)
  int p2 = 0;
  while ((r >> p2) % 2 == 0) ++p2;
  if (p2 % 2 == 1 && p2 >= 3 && !take_one(8)) return TSM_ERR_TOO_LARGE;
  if (!take(4) || !take(2) || !take(3)) return TSM_ERR_TOO_LARGE;
  for (int f = 5; r > 1 && f <= FFT_MAX_PRIME; f += 2)
    if (!take(f)) return TSM_ERR_TOO_LARGE;
  return r == 1 ? TSM_OK : TSM_ERR_TOO_LARGE;
}

// storage position of frequency n after the in-place DIF stages of ax
int dif_position(const FftAxis& ax, int n) {
  int p = 0, stride = ax.n;
  for (int st = 0; st < ax.nst; ++st) {
    const int r = ax.radix[st];
    stride /= r;
    p += (n % r) * stride;
    n /= r;
  }
  return p;
}

}  // namespace

int FftProjector::init(Ctx& c, int ng_, bool dbl) {
  ng = ng_;
  fp64 = dbl;
  E = (long long)ng * c.g.V;
  const int Lx = c.lat.L[0], Ly = c.lat.L[1], Lz = c.lat.L[2];
  const size_t csz = fp64 ? sizeof(double2) : sizeof(float2);
  for (int a = 0; a < 3; ++a) {
    if (factorise(c.lat.L[a], &plan.ax[a]) != TSM_OK) {
      set_error("all-momenta projection: extent %d has a prime factor above %d", c.lat.L[a], FFT_MAX_PRIME);
      return TSM_ERR_TOO_LARGE;
    }
  }
  plan.tw_xy = Lx + Ly;
  // insertions per xy CTA: gc in-place planes within the budget
  const size_t P = (size_t)Lx * Ly;
  const size_t tab_bytes = (size_t)plan.tw_xy * (csz + sizeof(int));
  const long long fit = (long long)((FFT_SMEM_BUDGET - std::min(FFT_SMEM_BUDGET, tab_bytes)) / (P * csz));
  if (fit < 1) {
    set_error("all-momenta projection: an Lx x Ly = %d x %d plane needs %zu bytes of shared memory "
              "(at most %zu per CTA)", Lx, Ly, P * csz + tab_bytes, FFT_SMEM_BUDGET);
    return TSM_ERR_TOO_LARGE;
  }
  gc = (int)std::min<long long>(fit, ng);
  xy_smem = (size_t)gc * P * csz + tab_bytes;
  // threads of an xy CTA: the plane's sites in equal rounds of at most
  // FFT_XY_NT threads (a 24 x 24 plane: two rounds of 288), whole warps
  {
    const int rounds = (int)((P + FFT_XY_NT - 1) / FFT_XY_NT);
    const int per = (int)((P + rounds - 1) / rounds);
    xy_threads = std::max(64, std::min(FFT_XY_NT, (per + 31) / 32 * 32));
  }
  // z bands: W columns of Lz elements
  zw = 128;
  while (zw > 1 && (size_t)Lz * (csz * (1 + (size_t)zw) + sizeof(int)) > FFT_SMEM_BUDGET) zw /= 2;
  z_smem = (size_t)Lz * (csz * (1 + (size_t)zw) + sizeof(int));
  if (z_smem > FFT_SMEM_BUDGET) {
    set_error("all-momenta projection: Lz = %d too long for a shared-memory line", Lz);
    return TSM_ERR_TOO_LARGE;
  }
  // twiddles e^{+2 pi i m / L}, m < L, and output positions per axis (x, y, z);
  // twiddles evaluated in FP64
  std::vector<double2> tw;
  std::vector<int> pos;
  for (int a = 0; a < 3; ++a) {
    const int n = c.lat.L[a];
    for (int m = 0; m < n; ++m) {
      const double ang = 2.0 * std::acos(-1.0) * (double)m / (double)n;
      tw.push_back(make_double2(std::cos(ang), std::sin(ang)));
      pos.push_back(dif_position(plan.ax[a], m));
    }
  }
  void* p = nullptr;
  TSM_TRY(c.buffer("fft_tw", tw.size() * sizeof(double2), &p));
  twd = static_cast<double2*>(p);
  TSM_TRY(c.buffer("fft_pos", pos.size() * sizeof(int), &p));
  posd = static_cast<int*>(p);
  TSM_CUDA(cudaMemcpyAsync(twd, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
  TSM_CUDA(cudaMemcpyAsync(posd, pos.data(), pos.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));   // the host tables go out of scope
  TSM_TRY(c.buffer("fft_dens", (size_t)E * csz, &p));
  dens = p;
  for (int s = 0; s < 2; ++s) {
    nb[s] = nmerged[s] = 0;
    if (!fp64) {
      TSM_TRY(c.buffer(s ? "fft_bsum_lp" : "fft_bsum_corr", (size_t)E * sizeof(float2), &p));
      bsum[s] = static_cast<float2*>(p);
      TSM_TRY(c.buffer(s ? "fft_bsq_lp" : "fft_bsq_corr", (size_t)E * sizeof(float), &p));
      bsq[s] = static_cast<float*>(p);
      TSM_TRY(c.buffer(s ? "fft_bshift_lp" : "fft_bshift_corr", (size_t)E * sizeof(float2), &p));
      bshift[s] = static_cast<float2*>(p);
    }
    TSM_TRY(c.buffer(s ? "fft_mean_lp" : "fft_mean_corr", (size_t)E * sizeof(double2), &p));
    mean[s] = static_cast<double2*>(p);
    TSM_TRY(c.buffer(s ? "fft_m2_lp" : "fft_m2_corr", (size_t)E * sizeof(double), &p));
    m2[s] = static_cast<double*>(p);
  }
  return TSM_OK;
}

void FftProjector::release() {}

template <class R, class SA, class SB>
int FftProjector::xy_pass(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a,
                          const EOField* b) {
  FftGam fg{};
  fg.n = gam.n;
  for (int k = 0; k < gam.n; ++k) {
    fg.m[k] = gam.col[k][0];
    for (int row = 0; row < 4; ++row) {
      if (gam.col[k][row] != (row ^ fg.m[k])) {
        set_error("all-momenta projection: insertion %d is not of the chiral-basis form", k);
        return TSM_ERR_ARG;
      }
      const int ph = gam.ph[k][row] & 3;   // i^ph
      fg.fr[k][row] = ph == 0 ? 1.f : (ph == 2 ? -1.f : 0.f);
      fg.fi[k][row] = ph == 1 ? 1.f : (ph == 3 ? -1.f : 0.f);
    }
  }
  auto kern = fft_xy_kernel<R, SA, SB>;
  TSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xy_smem));
  const int nch = (ng + gc - 1) / gc;
  kern<<<dim3(c.lat.L[3] * c.lat.L[2], nch), xy_threads, xy_smem, c.stream>>>(
      c.g, ns, source, a.e.as<SA>(), a.o.as<SA>(), b ? b->e.as<SB>() : nullptr, b ? b->o.as<SB>() : nullptr,
      c.sstride, fg, plan, gc, reinterpret_cast<const cx<double>*>(twd), posd, static_cast<cx<R>*>(dens));
  c.launches++;
  return check_launch(c, "fft_xy_kernel");
}

template <class R>
int FftProjector::z_pass(Ctx& c, const void* sink_ptr) {
  const ZSink& sink = *static_cast<const ZSink*>(sink_ptr);
  auto kern = fft_z_kernel<R>;
  TSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)z_smem));
  const int P = c.lat.L[0] * c.lat.L[1];
  const int Lz = c.lat.L[2];
  kern<<<dim3((P + zw - 1) / zw, ng * c.lat.L[3]), FFT_Z_NT, z_smem, c.stream>>>(
      P, Lz, plan.ax[2], zw, reinterpret_cast<const cx<double>*>(twd) + plan.tw_xy, posd + plan.tw_xy,
      static_cast<cx<R>*>(dens), sink);
  c.launches++;
  return check_launch(c, "fft_z_kernel");
}

int FftProjector::merge(Ctx& c, int set) {
  if (nb[set] == 0) return TSM_OK;
  fft_merge_kernel<<<(unsigned)((E + 255) / 256), 256, 0, c.stream>>>(bsum[set], bsq[set], bshift[set], nmerged[set],
                                                                       nb[set], mean[set], m2[set], E);
  c.launches++;
  nmerged[set] += nb[set];
  nb[set] = 0;
  return check_launch(c, "fft_merge_kernel");
}

template <class R, class SA, class SB>
int FftProjector::transform(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a,
                            const EOField* b) {
  TSM_TRY((xy_pass<R, SA, SB>(c, gam, ns, source, a, b)));
  ZSink sink{};
  sink.mode = 0;
  return z_pass<R>(c, &sink);
}

template <class R, class SA, class SB>
int FftProjector::accumulate(Ctx& c, const GammaTab& gam, const NoiseSpec& ns, uint32_t source, EOField a,
                             const EOField* b, int set, int k) {
  // algorithmic bytes: the fields read, the partly transformed densities
  // written and read once, then per entry either the FP64 running mean (16 B)
  // and sum of squares (8 B) read and written, or the FP32 batch sums (12 B)
  // and shift (8 B) written by the batch's first source, the sums read and
  // written and the shift read by the others, plus the batch merge
  const double csz = sizeof(cx<R>);
  const bool batched = sizeof(R) == 4;
  double per_entry = 2.0 * csz;
  if (!batched) per_entry += k > 1 ? 48.0 : 24.0;
  else per_entry += nb[set] > 0 ? 32.0 : 20.0;
  if (batched && nb[set] + 1 == kFftBatch) per_entry += 20.0 + (nmerged[set] > 0 ? 48.0 : 24.0);
  TimedLaunch tl(c, PB_FFT,
                 (double)c.g.V * (spinor_site_bytes(SA::id) + (b ? spinor_site_bytes(SB::id) : 0.0)) +
                     (double)E * per_entry,
                 true);
  TSM_TRY((xy_pass<R, SA, SB>(c, gam, ns, source, a, b)));
  ZSink sink{};
  if (batched) {
    if (k != nmerged[set] + nb[set] + 1) {
      set_error("all-momenta projection: source %d of set %d out of order", k, set);
      return TSM_ERR_ARG;
    }
    sink.mode = 2;
    sink.first = nb[set] == 0;
    sink.bsum = bsum[set];
    sink.bsq = bsq[set];
    sink.bshift = bshift[set];
    TSM_TRY(z_pass<R>(c, &sink));
    if (++nb[set] == kFftBatch) TSM_TRY(merge(c, set));
  } else {
    sink.mode = 1;
    sink.inv_k = 1.0 / (double)k;
    sink.wk = (double)(k - 1) / (double)k;
    sink.mean = mean[set];
    sink.m2 = m2[set];
    TSM_TRY(z_pass<R>(c, &sink));
  }
  tl.done();
  return TSM_OK;
}

int FftProjector::finalize(Ctx& c, int n_hp, int n_lp, double2* est, double* err, double2* lp_mean,
                           double2* corr_mean) {
  TSM_TRY(merge(c, 0));
  TSM_TRY(merge(c, 1));
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
TSM_FFT_INST(float, F64, F16)
TSM_FFT_INST(float, F32, F16)
TSM_FFT_INST(float, F16, F16)
#undef TSM_FFT_INST

}  // namespace tsm
