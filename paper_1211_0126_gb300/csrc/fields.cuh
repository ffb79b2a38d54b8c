// fields.cuh -- site-local kernels: layout conversion between the canonical
// FP64 host format and the even/odd chunked formats, link packing with the
// SU(3) check, noise generation, twist, precision casts and the BLAS-1 pieces
// of the reliable-update step.
#pragma once

#include "common.cuh"

namespace tsm {

constexpr int SITE_NT = 256;

// canonical spinor (24 doubles per lexicographic site) -> parity field in S
template <class S>
__global__ void __launch_bounds__(SITE_NT) pack_spinor_kernel(Geom g, int parity, const double2* __restrict__ canon,
                                                              typename S::schunk* __restrict__ out, int sstride) {
  using R = typename S::real;
  const int ih = blockIdx.x * SITE_NT + threadIdx.x;
  if (ih >= g.Vh) return;
  int c[4];
  site_coords(g, parity, ih, c);
  const int lex = ((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
  cx<R> v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 d = canon[(size_t)lex * 12 + k];
    v[k] = {(R)d.x, (R)d.y};
  }
  store_spinor<S>(out, sstride, ih, v);
}

template <class S>
__global__ void __launch_bounds__(SITE_NT) unpack_spinor_kernel(Geom g, int parity, const typename S::schunk* __restrict__ in,
                                                                int sstride, double2* __restrict__ canon) {
  using R = typename S::real;
  const int ih = blockIdx.x * SITE_NT + threadIdx.x;
  if (ih >= g.Vh) return;
  int c[4];
  site_coords(g, parity, ih, c);
  const int lex = ((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
  cx<R> v[12];
  if (in != nullptr) {
    load_spinor<S>(in, sstride, ih, v);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = {0, 0};
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) canon[(size_t)lex * 12 + k] = make_double2((double)v[k].re, (double)v[k].im);
}

// canonical links [lex][mu][3][3] complex -> parity fields in every precision
// (FP64: 3 rows, others: 2 rows); records the max deviation from SU(3).
static __global__ void __launch_bounds__(SITE_NT) pack_links_kernel(Geom g, const double2* __restrict__ U,
                                                             double2* __restrict__ l64, float4* __restrict__ l32,
                                                             uint2* __restrict__ l16, uint2* __restrict__ lbf,
                                                             int lstride, unsigned int* __restrict__ maxdev) {
  const int tid = blockIdx.x * SITE_NT + threadIdx.x;
  if (tid >= g.V * 4) return;
  const int lex = tid >> 2, mu = tid & 3;
  int rem = lex;
  const int x = rem % g.L[0];
  rem /= g.L[0];
  const int y = rem % g.L[1];
  rem /= g.L[1];
  const int z = rem % g.L[2];
  const int t = rem / g.L[2];
  const int parity = (x + y + z + t) & 1;
  const int ih = lex >> 1;
  const double2* m = U + ((size_t)lex * 4 + mu) * 9;
  cx<double> r[9], w[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) r[k] = {m[k].x, m[k].y};
  third_row(r, w);
  // SU(3) check: unit rows, orthogonal rows, stored row 2 equals the reconstruction
  double dev = fabs(norm2(r[0]) + norm2(r[1]) + norm2(r[2]) - 1.0);
  dev = fmax(dev, fabs(norm2(r[3]) + norm2(r[4]) + norm2(r[5]) - 1.0));
  const cx<double> o = cjmul(r[0], r[3]) + cjmul(r[1], r[4]) + cjmul(r[2], r[5]);
  dev = fmax(dev, sqrt(norm2(o)));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const cx<double> d = cx<double>{m[6 + k].x, m[6 + k].y} - w[k];
    dev = fmax(dev, sqrt(norm2(d)));
  }
  if (!(dev <= 1e30)) dev = 1e30;  // NaN -> huge
  atomicMax(maxdev, __float_as_uint((float)dev));
  const size_t off64 = (size_t)parity * 4 * F64::LN * lstride;
  const size_t off32 = (size_t)parity * 4 * F32::LN * lstride;
  store_link<F64>(l64 + off64, lstride, mu, ih, r);   // all three rows
  cx<float> rf[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) rf[k] = {(float)r[k].re, (float)r[k].im};
  store_link<F32>(l32 + off32, lstride, mu, ih, rf);
  store_link<F16>(l16 + off32, lstride, mu, ih, rf);
  store_link<BF16>(lbf + off32, lstride, mu, ih, rf);
}

// noise sources source0 + rhs -> batch of parity fields in S (eta is exactly
// representable in every tier except the 1/sqrt 2 amplitude, rounded once).
// Grid: x = right-hand side, y = blocks of SITE_NT sites.
template <class S>
__global__ void __launch_bounds__(SITE_NT) noise_kernel(Geom g, int parity, NoiseSpec n, uint32_t source0,
                                                        typename S::schunk* __restrict__ out, int sstride) {
  using R = typename S::real;
  const int rhs = blockIdx.x;
  const int ih = blockIdx.y * SITE_NT + threadIdx.x;
  if (ih >= g.Vh) return;
  int c[4];
  site_coords(g, parity, ih, c);
  const uint32_t lex = (uint32_t)(((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0]);
  cx<R> v[12];
  noise_site<R>(n, lex, source0 + (uint32_t)rhs, v);
  store_spinor<S>(out + rhs_offset<S>(rhs, sstride), sstride, ih, v);
}

// noise source in the canonical layout (for exact comparisons)
static __global__ void __launch_bounds__(SITE_NT) noise_canon_kernel(int V, NoiseSpec n, uint32_t source,
                                                                     double2* __restrict__ out) {
  const int lex = blockIdx.x * SITE_NT + threadIdx.x;
  if (lex >= V) return;
  cx<double> v[12];
  noise_site<double>(n, (uint32_t)lex, source, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) out[(size_t)lex * 12 + k] = make_double2(v[k].re, v[k].im);
}

// out = f * in (site-local chiral twist); a RHS with st[rhs].done is skipped
template <class S>
__global__ void __launch_bounds__(SITE_NT) twist_kernel(int Vh, Twist f, const typename S::schunk* __restrict__ in,
                                                        typename S::schunk* __restrict__ out, int sstride,
                                                        const int* active, const CGState* st) {
  const int rhs = rhs_slot(active);
  if (st != nullptr && st[rhs].done) return;
  const int ih = blockIdx.y * SITE_NT + threadIdx.x;
  if (ih >= Vh) return;
  const size_t off = rhs_offset<S>(rhs, sstride);
  cx<typename S::real> v[12];
  load_spinor<S>(in + off, sstride, ih, v);
  apply_twist(f, v);
  store_spinor<S>(out + off, sstride, ih, v);
}

// out (So) = in (Si), precision cast; in == nullptr writes zero
template <class Si, class So>
__global__ void __launch_bounds__(SITE_NT) convert_kernel(int Vh, const typename Si::schunk* __restrict__ in,
                                                          typename So::schunk* __restrict__ out, int sstride,
                                                          const int* active) {
  const int rhs = rhs_slot(active);
  const int ih = blockIdx.y * SITE_NT + threadIdx.x;
  if (ih >= Vh) return;
  cx<typename Si::real> v[12];
  cx<typename So::real> w[12];
  if (in != nullptr) {
    load_spinor<Si>(in + rhs_offset<Si>(rhs, sstride), sstride, ih, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = {(typename So::real)v[k].re, (typename So::real)v[k].im};
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = {0, 0};
  }
  store_spinor<So>(out + rhs_offset<So>(rhs, sstride), sstride, ih, w);
}

// reliable update, step 1: x64 += y (y in F32), y = 0 -- only for right-hand
// sides with a pending update (st[rhs].need_rel)
static __global__ void __launch_bounds__(SITE_NT) accumulate_solution_kernel(int Vh, float4* __restrict__ y,
                                                                             double2* __restrict__ x, int sstride,
                                                                             const int* active, const CGState* st) {
  const int rhs = rhs_slot(active);
  if (!st[rhs].need_rel) return;
  const int ih = blockIdx.y * SITE_NT + threadIdx.x;
  if (ih >= Vh) return;
  y += rhs_offset<F32>(rhs, sstride);
  x += rhs_offset<F64>(rhs, sstride);
  cx<float> yv[12];
  cx<double> xv[12];
  load_spinor<F32>(y, sstride, ih, yv);
  load_spinor<F64>(x, sstride, ih, xv);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    xv[k] = xv[k] + cx<double>{(double)yv[k].re, (double)yv[k].im};
    yv[k] = {0.f, 0.f};
  }
  store_spinor<F64>(x, sstride, ih, xv);
  store_spinor<F32>(y, sstride, ih, yv);
}

// FP64 -> FP32 copy of a field for the right-hand sides with a reliable
// update pending (the others return at once)
static __global__ void __launch_bounds__(SITE_NT) rel_narrow_kernel(int Vh, const double2* __restrict__ in,
                                                                    float4* __restrict__ out, int sstride,
                                                                    const int* active, const CGState* st) {
  const int rhs = rhs_slot(active);
  if (!st[rhs].need_rel) return;
  const int ih = blockIdx.y * SITE_NT + threadIdx.x;
  if (ih >= Vh) return;
  cx<double> v[12];
  cx<float> w[12];
  load_spinor<F64>(in + rhs_offset<F64>(rhs, sstride), sstride, ih, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) w[k] = {(float)v[k].re, (float)v[k].im};
  store_spinor<F32>(out + rhs_offset<F32>(rhs, sstride), sstride, ih, w);
}

// after a residual replacement the search direction restarts from the new
// residual, p = r: after many FP32 iterations the iterated residual can lie
// orders of magnitude below the true one, and the old direction would no
// longer be conjugate to the replaced residual
static __global__ void __launch_bounds__(SITE_NT) restart_direction_kernel(int Vh, const float4* __restrict__ r,
                                                                           float4* __restrict__ p, int sstride,
                                                                           const int* active, const CGState* st) {
  const int rhs = rhs_slot(active);
  if (!st[rhs].need_rel) return;
  const int ih = blockIdx.y * SITE_NT + threadIdx.x;
  if (ih >= Vh) return;
  cx<float> w[12];
  load_spinor<F32>(r + rhs_offset<F32>(rhs, sstride), sstride, ih, w);
  store_spinor<F32>(p + rhs_offset<F32>(rhs, sstride), sstride, ih, w);
}

// closes the reliable updates of one iteration: clears need_rel and, where the
// iterated residual had met the stopping rule, lets the true FP64 residual
// decide between stopping and iterating on
static __global__ void rel_finish_kernel(CGState* st, const int* active, int n) {
  const int k = threadIdx.x + blockIdx.x * blockDim.x;
  if (k >= n) return;
  CGState& s = st[active != nullptr ? active[k] : k];
  if (!s.need_rel) return;
  s.need_rel = 0;
  if (s.final_check) {
    s.final_check = 0;
    if (s.status != 0 || s.iter >= s.max_iter || rule_met(&s, s.rr)) s.done = 1;
  }
}

// a warm-started solve asks every iterating source for a residual replacement
// before its first iteration; final_check lets rel_finish_kernel stop a source
// whose starting guess already meets the rule
static __global__ void warm_start_kernel(CGState* st, int n) {
  const int k = threadIdx.x + blockIdx.x * blockDim.x;
  if (k >= n) return;
  CGState& s = st[k];
  if (s.done || s.status != 0) return;
  s.need_rel = 1;
  s.final_check = 1;
}

// <v, v> per right-hand side with post action (deterministic two-stage sum)
template <class S>
__global__ void __launch_bounds__(SITE_NT) norm_kernel(int Vh, const typename S::schunk* __restrict__ v, int sstride,
                                                       RedSlot red, const int* active, CGState* st, int post) {
  const int rhs = rhs_slot(active);
  const int ih = blockIdx.y * SITE_NT + threadIdx.x;
  double part = 0.0;
  if (ih < Vh) {
    cx<typename S::real> w[12];
    load_spinor<S>(v + rhs_offset<S>(rhs, sstride), sstride, ih, w);
    typename S::real s = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) s += norm2(w[k]);
    part = (double)s;
  }
  double total;
  if (grid_sum<SITE_NT>(part, red, rhs, &total) && threadIdx.x == 0) post_action(st + rhs, post, total);
}

// states 0 .. n-1: fresh solve
static __global__ void state_init_kernel(CGState* st, int n, double tol, int max_iter, int rel, double delta2) {
  const int k = threadIdx.x + blockIdx.x * blockDim.x;
  if (k >= n) return;
  CGState& s = st[k];
  s.tol = tol;
  s.max_iter = max_iter;
  s.iter = 0;
  s.done = 0;
  s.status = 0;
  s.rel = rel;
  s.need_rel = 0;
  s.final_check = 0;
  s.delta2 = delta2;
  s.rr = s.rr0 = s.pAp = s.alpha = s.beta = s.aux = s.rr_ref = 0.0;
  s.alpha_f = s.beta_f = 0.0f;
}

}  // namespace tsm
