// dslash.cuh -- the half-lattice Wilson hopping stencil with twisted-mass
// epilogues, and the fused CG-update kernel.
//
// H_{p <- 1-p} psi (x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                               + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
// evaluated for the sites x of one parity p; the adjoint stencil H^dag swaps
// the two projectors.  Each hop projects the neighbour spinor onto two spin
// components (the (1 +- gamma_mu) projectors have rank 2 in the chiral basis),
// multiplies by the two-row-reconstructed SU(3) link and rebuilds the lower
// spin components from the upper ones.  Hops crossing t = T-1 <-> 0 are
// multiplied by -1 for an antiperiodic fermion field.
#pragma once

#include "common.cuh"

namespace tsm {

// ------------------------------------------------------------- projectors
// (1 + s gamma_mu) psi = [h ; M_mu^s h] with h = psi_up - s (i sigma_mu) psi_dn
// (k = x, y, z) or h = psi_up + s psi_dn (t).  i sigma_1 v = (i v1, i v0),
// i sigma_2 v = (v1, -v0), i sigma_3 v = (i v0, -i v1).
template <int MU, int SG, class R>
__device__ __forceinline__ void project(const cx<R> v[12], cx<R> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<R> p0 = v[c], p1 = v[3 + c], p2 = v[6 + c], p3 = v[9 + c];
    if constexpr (MU == 0) {
      h[c] = (SG > 0) ? p0 - times_i(p3) : p0 + times_i(p3);
      h[3 + c] = (SG > 0) ? p1 - times_i(p2) : p1 + times_i(p2);
    } else if constexpr (MU == 1) {
      h[c] = (SG > 0) ? p0 - p3 : p0 + p3;
      h[3 + c] = (SG > 0) ? p1 + p2 : p1 - p2;
    } else if constexpr (MU == 2) {
      h[c] = (SG > 0) ? p0 - times_i(p2) : p0 + times_i(p2);
      h[3 + c] = (SG > 0) ? p1 + times_i(p3) : p1 - times_i(p3);
    } else {
      h[c] = (SG > 0) ? p0 + p2 : p0 - p2;
      h[3 + c] = (SG > 0) ? p1 + p3 : p1 - p3;
    }
  }
}

// FP16 storage: the same projection on the stored words in packed f16x2
// arithmetic (one rounding of a sum of two stored values, below the storage
// rounding of the LP tier), then widened: 6 packed adds and 12 conversions
// instead of 24 conversions and 12 FP32 adds.  A word holds (re, im) with the
// real part in the low half; i v = (-im, re) and -i v = (im, -re) are a swap
// and a sign flip.
__device__ __forceinline__ uint32_t h2_add(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t h2_sub(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t h2_mul_i(uint32_t a) { return __byte_perm(a, 0u, 0x1032) ^ 0x00008000u; }
__device__ __forceinline__ uint32_t h2_mul_mi(uint32_t a) { return __byte_perm(a, 0u, 0x1032) ^ 0x80000000u; }

template <int MU, int SG>
__device__ __forceinline__ void project_f16(const uint32_t v[12], cx<float> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const uint32_t p0 = v[c], p1 = v[3 + c], p2 = v[6 + c], p3 = v[9 + c];
    uint32_t h0, h1;
    if constexpr (MU == 0) {
      h0 = (SG > 0) ? h2_add(p0, h2_mul_mi(p3)) : h2_add(p0, h2_mul_i(p3));
      h1 = (SG > 0) ? h2_add(p1, h2_mul_mi(p2)) : h2_add(p1, h2_mul_i(p2));
    } else if constexpr (MU == 1) {
      h0 = (SG > 0) ? h2_sub(p0, p3) : h2_add(p0, p3);
      h1 = (SG > 0) ? h2_add(p1, p2) : h2_sub(p1, p2);
    } else if constexpr (MU == 2) {
      h0 = (SG > 0) ? h2_add(p0, h2_mul_mi(p2)) : h2_add(p0, h2_mul_i(p2));
      h1 = (SG > 0) ? h2_add(p1, h2_mul_i(p3)) : h2_add(p1, h2_mul_mi(p3));
    } else {
      h0 = (SG > 0) ? h2_add(p0, p2) : h2_sub(p0, p2);
      h1 = (SG > 0) ? h2_add(p1, p3) : h2_sub(p1, p3);
    }
    h[c] = Pack16<F16>::unpack(h0);
    h[3 + c] = Pack16<F16>::unpack(h1);
  }
}

// the projected half spinor of the neighbour at index n
template <class S, int MU, int SG>
__device__ __forceinline__ void load_projected(const typename S::schunk* __restrict__ in, int sstride, int n,
                                               cx<typename S::real> h[6]) {
  if constexpr (S::id == F16::id) {
    uint32_t v[12];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint4 u = in[j * sstride + n];
      v[4 * j] = u.x;
      v[4 * j + 1] = u.y;
      v[4 * j + 2] = u.z;
      v[4 * j + 3] = u.w;
    }
    project_f16<MU, SG>(v, h);
  } else {
    cx<typename S::real> v[12];
    load_spinor<S>(in, sstride, n, v);
    project<MU, SG>(v, h);
  }
}

// acc += (1 + s gamma_mu)-reconstruction of the link-multiplied half spinor u
// (FIRST: acc = ..., the site's first hop, instead of adding to zeros)
template <int MU, int SG, bool FIRST, class R>
__device__ __forceinline__ void accumulate(cx<R> acc[12], const cx<R> u[6]) {
  auto put = [&](int k, cx<R> v) { acc[k] = FIRST ? v : acc[k] + v; };
  auto neg = [](cx<R> v) { return cx<R>{-v.re, -v.im}; };
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<R> u0 = u[c], u1 = u[3 + c];
    put(c, u0);
    put(3 + c, u1);
    if constexpr (MU == 0) {        // lower = s i sigma_1 h = s (i h1, i h0)
      put(6 + c, (SG > 0) ? times_i(u1) : neg(times_i(u1)));
      put(9 + c, (SG > 0) ? times_i(u0) : neg(times_i(u0)));
    } else if constexpr (MU == 1) { // lower = s (h1, -h0)
      put(6 + c, (SG > 0) ? u1 : neg(u1));
      put(9 + c, (SG > 0) ? neg(u0) : u0);
    } else if constexpr (MU == 2) { // lower = s (i h0, -i h1)
      put(6 + c, (SG > 0) ? times_i(u0) : neg(times_i(u0)));
      put(9 + c, (SG > 0) ? neg(times_i(u1)) : times_i(u1));
    } else {                        // lower = s h
      put(6 + c, (SG > 0) ? u0 : neg(u0));
      put(9 + c, (SG > 0) ? u1 : neg(u1));
    }
  }
}

// u = U h (dag = false) or U^dag h (dag = true) on both spin components of h;
// r holds the three rows of U (r[6..8] = row 2)
template <bool DAGU, class R>
__device__ __forceinline__ void su3_mul(const cx<R> r[9], const cx<R> h[6], cx<R> u[6]) {
  const cx<R>* w = r + 6;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const cx<R> a = h[3 * s], b = h[3 * s + 1], c = h[3 * s + 2];
    if constexpr (!DAGU) {
      u[3 * s + 0] = r[0] * a + r[1] * b + r[2] * c;
      u[3 * s + 1] = r[3] * a + r[4] * b + r[5] * c;
      u[3 * s + 2] = w[0] * a + w[1] * b + w[2] * c;
    } else {
      u[3 * s + 0] = cjmul(r[0], a) + cjmul(r[3], b) + cjmul(w[0], c);
      u[3 * s + 1] = cjmul(r[1], a) + cjmul(r[4], b) + cjmul(w[1], c);
      u[3 * s + 2] = cjmul(r[2], a) + cjmul(r[5], b) + cjmul(w[2], c);
    }
  }
}

// One direction of the stencil at output site (c, ih) of parity p.
// links(h, nb, r) fills r[0..8] with the three rows of the link of hop h
// (2 MU forward at x, 2 MU + 1 backward at x - mu, neighbour index nb).
template <class S, int DAG, int MU, class Links>
__device__ __forceinline__ void hop_dir(const Geom& g, const int c[4], const typename S::schunk* __restrict__ in,
                                        int sstride, Links&& links, cx<typename S::real> acc[12]) {
  using R = typename S::real;
  constexpr int SF = DAG ? +1 : -1;   // forward hop: (1 + SF gamma_mu)
  constexpr int SB = -SF;             // backward hop
  cx<R> h[6], u[6], r[9];
  // forward neighbour x + mu
  {
    int x = c[0], y = c[1], z = c[2], t = c[3];
    if constexpr (MU == 0) x = (x + 1 == g.L[0]) ? 0 : x + 1;
    if constexpr (MU == 1) y = (y + 1 == g.L[1]) ? 0 : y + 1;
    if constexpr (MU == 2) z = (z + 1 == g.L[2]) ? 0 : z + 1;
    if constexpr (MU == 3) t = (t + 1 == g.L[3]) ? 0 : t + 1;
    const int nf = half_index(g, x, y, z, t);
    load_projected<S, MU, SF>(in, sstride, nf, h);
    if constexpr (MU == 3) {
      if (g.apbc && c[3] == g.L[3] - 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = (R)(-1) * h[k];
      }
    }
    links(2 * MU, -1, r);
    su3_mul<false>(r, h, u);
    accumulate<MU, SF, MU == 0>(acc, u);   // the site's first hop assigns
  }
  // backward neighbour x - mu
  {
    int x = c[0], y = c[1], z = c[2], t = c[3];
    if constexpr (MU == 0) x = (x == 0) ? g.L[0] - 1 : x - 1;
    if constexpr (MU == 1) y = (y == 0) ? g.L[1] - 1 : y - 1;
    if constexpr (MU == 2) z = (z == 0) ? g.L[2] - 1 : z - 1;
    if constexpr (MU == 3) t = (t == 0) ? g.L[3] - 1 : t - 1;
    const int nb = half_index(g, x, y, z, t);
    load_projected<S, MU, SB>(in, sstride, nb, h);
    if constexpr (MU == 3) {
      if (g.apbc && c[3] == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = (R)(-1) * h[k];
      }
    }
    links(2 * MU + 1, nb, r);
    su3_mul<true>(r, h, u);
    accumulate<MU, SB, false>(acc, u);
  }
}

// the link of hop h from global memory: 2 MU forward at the output site ih
// (links of the output parity), 2 MU + 1 backward at the neighbour nb
template <class S>
struct GlobalLinks {
  const typename S::lchunk* __restrict__ Uout;
  const typename S::lchunk* __restrict__ Uin;
  int lstride, ih;
  __device__ __forceinline__ void operator()(int h, int nb, cx<typename S::real> r[9]) const {
    load_link<S>((h & 1) ? Uin : Uout, lstride, h >> 1, (h & 1) ? nb : ih, r);
    if constexpr (!S::full_links) third_row(r, r + 6);
  }
};

template <class S, int DAG, class Links>
__device__ __forceinline__ void hop_site_with(const Geom& g, const int c[4], const typename S::schunk* __restrict__ in,
                                              int sstride, Links&& links, cx<typename S::real> acc[12]) {
  hop_dir<S, DAG, 0>(g, c, in, sstride, links, acc);   // assigns acc
  hop_dir<S, DAG, 1>(g, c, in, sstride, links, acc);
  hop_dir<S, DAG, 2>(g, c, in, sstride, links, acc);
  hop_dir<S, DAG, 3>(g, c, in, sstride, links, acc);
}

template <class S, int DAG>
__device__ __forceinline__ void hop_site(const Geom& g, int ih, const int c[4],
                                         const typename S::lchunk* __restrict__ Uout,
                                         const typename S::lchunk* __restrict__ Uin, int lstride,
                                         const typename S::schunk* __restrict__ in, int sstride,
                                         cx<typename S::real> acc[12]) {
  hop_site_with<S, DAG>(g, c, in, sstride, GlobalLinks<S>{Uout, Uin, lstride, ih}, acc);
}

// ------------------------------------------------------------- generic hop kernel
// out(x) = ts * q,  q = base(x) + to * (ac * tc * center(x) + ah * H psi (x))
// with optional <q, q> reduction.  MODE bits select center / base / norm.
// Grid: blockIdx.x = right-hand side (through an optional active list),
// blockIdx.y = block of HOP_NT output sites.  in / center / base / out are
// batches of contiguous parity fields, one per right-hand side; the links are
// shared by all of them (their reuse across right-hand sides comes from L2,
// since consecutive blocks in launch order handle the same sites).
enum { HOP_CENTER = 1, HOP_NORM = 2, HOP_BASE = 4 };

template <class S>
struct HopArgs {
  Geom g;
  int p_out;                               // parity of the output sites
  const typename S::lchunk* Uout;          // links of parity p_out
  const typename S::lchunk* Uin;           // links of parity 1 - p_out
  int lstride;
  const typename S::schunk* in;            // parity 1 - p_out
  const typename S::schunk* center;        // parity p_out (HOP_CENTER)
  const typename S::schunk* base;          // parity p_out (HOP_BASE)
  typename S::schunk* out;                 // parity p_out
  int sstride;
  double ac, ah;
  Twist tc, to, ts;
  const int* active;                       // optional list of right-hand sides
  const CGState* skip;                     // optional: a RHS returns at once when skip[rhs].done
  int skip_rel;                            // 1: instead, return unless skip[rhs].need_rel
  CGState* st;                             // states receiving the HOP_NORM post action
  RedSlot red;                             // HOP_NORM
  int post;                                // PostOp for HOP_NORM
  TwistF fto_ah, fto_tc_ac, fts;           // FP32 kernels: to * ah, to * tc * ac and ts, formed in
                                           // FP64 on the host and rounded once (set by launch_hop)
};

constexpr int HOP_NT = 128;

// Blocks per SM the stencil kernels are compiled for: the 32- and 16-bit tiers
// are bound by FP32 issue and memory latency together, and six resident blocks
// (at most 80 registers, a few spilled words) beat five with no spills; the
// FP64 tier keeps the compiler's choice.
template <class S> struct HopMinBlocks { static constexpr int value = 6; };
template <> struct HopMinBlocks<F64> { static constexpr int value = 1; };

// epilogue of one output site of one right-hand side, acc = H psi on entry:
// out = ts q, q = base + to (ac tc center + ah acc); returns <q, q> (HOP_NORM)
template <class S, int MODE>
__device__ __forceinline__ typename S::real hop_epilogue(const HopArgs<S>& a, size_t off, int ih,
                                                         cx<typename S::real> acc[12]) {
  using R = typename S::real;
  constexpr bool FP32 = sizeof(R) == 4;
  R part = 0;
  if constexpr (FP32) {
    // q = (to ah) acc + (to tc ac) center with the combined factors
    apply_twist(a.fto_ah, acc);
    if constexpr (MODE & HOP_CENTER) {
      cx<R> v[12];
      load_spinor<S>(a.center + off, a.sstride, ih, v);
      apply_twist(a.fto_tc_ac, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = acc[k] + v[k];
    }
  } else {
    const R ah = (R)a.ah;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = ah * acc[k];
    if constexpr (MODE & HOP_CENTER) {
      cx<R> v[12];
      load_spinor<S>(a.center + off, a.sstride, ih, v);
      apply_twist(a.tc, v);
      const R ac = (R)a.ac;
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = acc[k] + ac * v[k];
    }
    apply_twist(a.to, acc);
  }
  if constexpr (MODE & HOP_BASE) {
    cx<R> v[12];
    load_spinor<S>(a.base + off, a.sstride, ih, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = acc[k] + v[k];
  }
  if constexpr (MODE & HOP_NORM) {
    R s = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) s += norm2(acc[k]);
    part = s;
  }
  if constexpr (FP32) apply_twist(a.fts, acc);
  else apply_twist(a.ts, acc);
  store_spinor<S>(a.out + off, a.sstride, ih, acc);
  return part;
}

template <class S, int DAG, int MODE>
__global__ void __launch_bounds__(HOP_NT, HopMinBlocks<S>::value) hop_kernel(const HopArgs<S> a) {
  using R = typename S::real;
  const int rhs = rhs_slot(a.active);
  if (a.skip != nullptr && (a.skip_rel ? !a.skip[rhs].need_rel : a.skip[rhs].done)) return;
  const size_t off = rhs_offset<S>(rhs, a.sstride);
  const int ih = blockIdx.y * HOP_NT + threadIdx.x;
  R part = 0;   // FP32 kernels: FP32 up to the warp sums
  if (ih < a.g.Vh) {
    int c[4];
    site_coords(a.g, a.p_out, ih, c);
    cx<R> acc[12];
    hop_site<S, DAG>(a.g, ih, c, a.Uout, a.Uin, a.lstride, a.in + off, a.sstride, acc);
    part = hop_epilogue<S, MODE>(a, off, ih, acc);
  }
  if constexpr (MODE & HOP_NORM) {
    double total;
    if (grid_sum<HOP_NT>(part, a.red, rhs, &total) && threadIdx.x == 0 && a.st != nullptr)
      post_action(a.st + rhs, a.post, total);
  }
}

// ------------------------------------------------------------- fused CG update
// For even output sites:  v = A(-mu) w - kappa^2 (H^dag)_eo t  (= Dhat^dag Dhat p),
// r -= alpha v,  x += alpha p,  <r, r> -> post POST_RR (beta, iteration, stop).
// Sloppy storage S for w, t, p and links; SA for r and x.  Batched like hop_kernel.
template <class S, class SA>
struct CGUpdArgs {
  Geom g;
  const typename S::lchunk* Ue;
  const typename S::lchunk* Uo;
  int lstride;
  const typename S::schunk* t;     // odd
  const typename S::schunk* w;     // even
  const typename S::schunk* p;     // even
  typename SA::schunk* r;          // even
  typename SA::schunk* x;          // even
  int sstride;
  double kappa2;
  Twist tw;                         // A(-mu)
  float fkappa2;                    // kappa2 and tw rounded on the host (set by launch_cg_update)
  TwistF ftw;
  const int* active;
  CGState* st;
  RedSlot red;
};

// epilogue of one even site of one right-hand side: acc = (H^dag)_eo t on
// entry; v = A(-mu) w - kappa^2 acc, r -= alpha v, x += alpha p; returns <r, r>.
// w, p, r and x are read at index li of chunk stride ls from ws, ps, rs, xs
// (the fields themselves, or their copies in shared memory); r and x are
// written to the fields.
template <class S, class SA>
__device__ __forceinline__ typename SA::real cg_update_epilogue(const CGUpdArgs<S, SA>& a, const CGState* st,
                                                                size_t offa, int ih, cx<typename S::real> acc[12],
                                                                const typename S::schunk* ws,
                                                                const typename S::schunk* ps,
                                                                const typename SA::schunk* rs,
                                                                const typename SA::schunk* xs, int ls, int li) {
  using R = typename S::real;
  using RA = typename SA::real;
  cx<R> v[12];
  load_spinor<S>(ws, ls, li, v);
  constexpr bool FP32 = sizeof(R) == 4;
  if constexpr (FP32) apply_twist(a.ftw, v);
  else apply_twist(a.tw, v);
  const R k2 = FP32 ? (R)a.fkappa2 : (R)a.kappa2;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = v[k] - k2 * acc[k];
  const RA alpha = sizeof(RA) == 4 ? (RA)st->alpha_f : (RA)st->alpha;
  cx<RA> rv[12], xv[12];
  load_spinor<SA>(rs, ls, li, rv);
  load_spinor<SA>(xs, ls, li, xv);
  load_spinor<S>(ps, ls, li, v);
  RA s = 0;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    rv[k] = rv[k] - alpha * cx<RA>{(RA)acc[k].re, (RA)acc[k].im};
    xv[k] = xv[k] + alpha * cx<RA>{(RA)v[k].re, (RA)v[k].im};
    s += norm2(rv[k]);
  }
  store_spinor<SA>(a.r + offa, a.sstride, ih, rv);
  store_spinor<SA>(a.x + offa, a.sstride, ih, xv);
  return s;
}

// The FP16 tier (S = SA = F16): the four site-local streams of the epilogue
// (w, p, r, x: twelve 16-byte chunks per thread) are copied into shared
// memory with cp.async when the thread starts, so that their latency hides
// behind the hop instead of following it.
template <class S, class SA> struct UpdPrefetch {
  static constexpr bool value = S::id == F16::id && SA::id == F16::id;
};

__device__ __forceinline__ void copy16_async(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void copy16_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// groups of HOP_NT sites per block of the fused CG update: 4 for the FP16
// tier (485 against 515 us per 32-source launch), 1 for FP32 (2 groups
// measured 409 against 362 us)
template <class S, class SA> struct UpdGroups { static constexpr int value = UpdPrefetch<S, SA>::value ? 4 : 1; };

template <class S, class SA>
__global__ void __launch_bounds__(HOP_NT, HopMinBlocks<S>::value) cg_update_kernel(const CGUpdArgs<S, SA> a) {
  using R = typename S::real;
  constexpr bool PF = UpdPrefetch<S, SA>::value;
  constexpr int NCH = PF ? 3 : 1;   // 16-byte chunks per 16-bit spinor
  __shared__ uint4 pf[PF ? 4 * NCH : 1][PF ? HOP_NT : 1];
  const int rhs = rhs_slot(a.active);
  CGState* st = a.st + rhs;
  if (st->done) return;
  const size_t off = rhs_offset<S>(rhs, a.sstride), offa = rhs_offset<SA>(rhs, a.sstride);
  typename SA::real part = 0;
  // a block walks UpdGroups consecutive groups of HOP_NT sites, so that its
  // grid-sum step (fence, ticket) is paid once per group run
  constexpr int G = UpdGroups<S, SA>::value;
#pragma unroll 1
  for (int grp = 0; grp < G; ++grp) {
    const int ih = (blockIdx.y * G + grp) * HOP_NT + threadIdx.x;
    if (ih >= a.g.Vh) break;
    if constexpr (PF) {
      const uint4* src[4] = {reinterpret_cast<const uint4*>(a.w + off), reinterpret_cast<const uint4*>(a.p + off),
                             reinterpret_cast<const uint4*>(a.r + offa), reinterpret_cast<const uint4*>(a.x + offa)};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) copy16_async(&pf[q * NCH + ch][threadIdx.x], src[q] + ch * a.sstride + ih);
    }
    int c[4];
    site_coords(a.g, 0, ih, c);
    cx<R> acc[12];
    hop_site<S, 1>(a.g, ih, c, a.Ue, a.Uo, a.lstride, a.t + off, a.sstride, acc);
    if constexpr (PF) {
      copy16_wait_all();   // this thread's own copies: no block barrier needed
      part += cg_update_epilogue<S, SA>(a, st, offa, ih, acc, reinterpret_cast<const typename S::schunk*>(pf[0]),
                                        reinterpret_cast<const typename S::schunk*>(pf[NCH]),
                                        reinterpret_cast<const typename SA::schunk*>(pf[2 * NCH]),
                                        reinterpret_cast<const typename SA::schunk*>(pf[3 * NCH]), HOP_NT, threadIdx.x);
    } else {
      part += cg_update_epilogue<S, SA>(a, st, offa, ih, acc, a.w + off, a.p + off, a.r + offa, a.x + offa,
                                        a.sstride, ih);
    }
  }
  double total;
  if (grid_sum<HOP_NT>(part, a.red, rhs, &total) && threadIdx.x == 0) post_action(st, POST_RR, total);
}

// ------------------------------------------------------------- link-sharing stencil
// The 16-bit tiers' hop kernels (K1-K3 of their CG): blocks of LT_SITES
// consecutive output sites x up to RPB right-hand sides (threadIdx.x =
// site, threadIdx.y = right-hand side of the block, one warp each; RPB = 2, 4
// or 8, chosen per tier by the autotuner, LT_RHS by default).  The
// block's 8 x LT_SITES links are read, widened to FP32 and completed with row
// 2 once, kept in shared memory, and read from there by every right-hand side
// of the block: 5 shared loads per link and source instead of 3 global loads,
// 12 conversions and the 24-FMA row rebuild.  Per-link and per-site
// arithmetic does not depend on how many right-hand sides share a block, nor
// do the reductions (a warp per right-hand side and block, then a fixed
// virtual-lane order over the blocks), so batched and single-source results
// agree bit for bit.
constexpr int LT_SITES = 32;
constexpr int LT_RHS = 4;   // default right-hand sides per block

// resident blocks per SM the tile kernels are compiled for: 768 threads at
// the default register budget of 80 per thread (the per-site stencil's budget
// at six blocks of 128), or 640 threads at 96 registers (REGS = 96: fewer
// spills, fewer resident warps; the autotuner chooses)
constexpr int LT_REGS = 80;   // default register budget of the tile kernels
template <int RPB, int REGS> struct TileMinBlocks { static constexpr int value = (REGS == 96 ? 20 : 24) / RPB; };

// groups of LT_SITES sites a link-tile block walks: 4 for the hops with a
// norm (fewer block partials and grid-sum steps), 1 otherwise
template <int MODE> struct LtGroups { static constexpr int value = (MODE & HOP_NORM) ? 4 : 1; };

struct LinkTile {
  float4 v[8][5][LT_SITES];   // [hop 2 mu + backward][pair of complex][site]: rows 0..2, then a zero
};

template <class S>
__device__ __forceinline__ void stage_link(const typename S::lchunk* __restrict__ U, int lstride, int dir, int site,
                                           float4* dst) {
  cx<float> r[9];
  load_link<S>(U, lstride, dir, site, r);
  if constexpr (!S::full_links) third_row(r, r + 6);
#pragma unroll
  for (int k = 0; k < 4; ++k) dst[k * LT_SITES] = make_float4(r[2 * k].re, r[2 * k].im, r[2 * k + 1].re, r[2 * k + 1].im);
  dst[4 * LT_SITES] = make_float4(r[8].re, r[8].im, 0.f, 0.f);
}

__device__ __forceinline__ int backward_index(const Geom& g, const int c[4], int mu) {
  int x = c[0], y = c[1], z = c[2], t = c[3];
  if (mu == 0) x = (x == 0) ? g.L[0] - 1 : x - 1;
  else if (mu == 1) y = (y == 0) ? g.L[1] - 1 : y - 1;
  else if (mu == 2) z = (z == 0) ? g.L[2] - 1 : z - 1;
  else t = (t == 0) ? g.L[3] - 1 : t - 1;
  return half_index(g, x, y, z, t);
}

// the block's links: thread (site, w) stages directions w, w + blockDim.y, ...
template <class S>
__device__ __forceinline__ void stage_tile(const Geom& g, int ih, const int c[4],
                                           const typename S::lchunk* __restrict__ Uout,
                                           const typename S::lchunk* __restrict__ Uin, int lstride, LinkTile& T) {
  if (ih >= g.Vh) return;
  const int s = threadIdx.x;
  for (int mu = threadIdx.y; mu < 4; mu += blockDim.y) {
    stage_link<S>(Uout, lstride, mu, ih, &T.v[2 * mu][0][s]);
    stage_link<S>(Uin, lstride, mu, backward_index(g, c, mu), &T.v[2 * mu + 1][0][s]);
  }
}

struct TileLinks {
  const LinkTile& t;
  int s;
  __device__ __forceinline__ void operator()(int h, int, cx<float> r[9]) const {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float4 q = t.v[h][k][s];
      r[2 * k] = {q.x, q.y};
      if (k < 4) r[2 * k + 1] = {q.z, q.w};
    }
  }
};

// per-right-hand-side sums of a link-sharing launch (grid.y = site blocks):
// the block partial of a right-hand side is its warp's sum; the last block of
// a right-hand side adds the partials over LT_VLANES virtual lanes (virtual
// lane v: blocks v, v + LT_VLANES, ... in order), then the virtual lanes'
// sums in a fixed tree.  The threads of the block share the virtual lanes
// out, so the order is the same whatever the block's width.
constexpr int LT_VLANES = 128;

template <int RPB>
__device__ __forceinline__ void tile_grid_sum(float part, int rhs, RedSlot slot, CGState* st, int post) {
  __shared__ int last_rhs[RPB];
  __shared__ double vsum[LT_VLANES];
  const int w = threadIdx.y, lane = threadIdx.x, nthr = LT_SITES * blockDim.y, tid = w * LT_SITES + lane;
  float v = part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) {
    int last = -1;
    if (rhs >= 0) {
      slot.partials[(size_t)rhs * slot.stride + blockIdx.y] = (double)v;
      __threadfence();
      const unsigned int ticket = atomicAdd(slot.counter + rhs, 1u);
      if (ticket == gridDim.y - 1) last = rhs;
    }
    last_rhs[w] = last;
  }
  __syncthreads();
  for (int j = 0; j < (int)blockDim.y; ++j) {
    const int r = last_rhs[j];   // the same in every thread
    if (r < 0) continue;
    __threadfence();
    const double* partials = slot.partials + (size_t)r * slot.stride;
    for (int vl = tid; vl < LT_VLANES; vl += nthr) vsum[vl] = strided_sum_ordered(partials, vl, (int)gridDim.y, LT_VLANES);
    __syncthreads();
    if (w == 0) {
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < LT_VLANES / 32; ++q) acc += vsum[lane + 32 * q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        if (st != nullptr) post_action(st + r, post, acc);
        slot.counter[r] = 0u;
      }
    }
    __syncthreads();
  }
}

// right-hand side of thread (site, w) from the launch's list, -1 past it
__device__ __forceinline__ int tile_rhs(const int* active, int nrhs) {
  const int k = blockIdx.x * blockDim.y + threadIdx.y;
  if (k >= nrhs) return -1;
  return active != nullptr ? active[k] : k;
}

template <class S, int DAG, int MODE, int RPB, int REGS>
__global__ void __launch_bounds__(LT_SITES * RPB, (TileMinBlocks<RPB, REGS>::value))
    hop_tile_kernel(const HopArgs<S> a, int nrhs) {
  __shared__ LinkTile tile;
  using R = typename S::real;
  int rhs = tile_rhs(a.active, nrhs);
  if (rhs >= 0 && a.skip != nullptr && (a.skip_rel ? !a.skip[rhs].need_rel : a.skip[rhs].done)) rhs = -1;
  if (!__syncthreads_or(rhs >= 0)) return;   // every right-hand side of the block is idle
  // a reducing block walks LT_GROUPS<MODE> consecutive groups of 32 sites, so
  // that its grid-sum step (fence, ticket, barrier) is paid once per group run
  R part = 0;
#pragma unroll 1
  for (int grp = 0; grp < LtGroups<MODE>::value; ++grp) {
    const int ih = (blockIdx.y * LtGroups<MODE>::value + grp) * LT_SITES + threadIdx.x;
    int c[4] = {0, 0, 0, 0};
    if (ih < a.g.Vh) site_coords(a.g, a.p_out, ih, c);
    if (grp > 0) __syncthreads();   // the previous group's links are consumed
    stage_tile<S>(a.g, ih, c, a.Uout, a.Uin, a.lstride, tile);
    __syncthreads();
    if (rhs >= 0 && ih < a.g.Vh) {
      const size_t off = rhs_offset<S>(rhs, a.sstride);
      cx<R> acc[12];
      hop_site_with<S, DAG>(a.g, c, a.in + off, a.sstride, TileLinks{tile, (int)threadIdx.x}, acc);
      part += hop_epilogue<S, MODE>(a, off, ih, acc);
    }
  }
  if constexpr (MODE & HOP_NORM) tile_grid_sum<RPB>(part, rhs, a.red, a.st, a.post);
}

// p = r + beta p   (grid: x = right-hand side, y = blocks of 256 sites)
template <class S, class SA>
__global__ void __launch_bounds__(256) cg_p_kernel(const typename SA::schunk* __restrict__ r,
                                                   typename S::schunk* __restrict__ p, int sstride, int Vh,
                                                   const int* active, const CGState* st) {
  const int rhs = rhs_slot(active);
  if (st[rhs].done) return;
  const int ih = blockIdx.y * blockDim.x + threadIdx.x;
  if (ih >= Vh) return;
  using R = typename S::real;
  using RA = typename SA::real;
  r += rhs_offset<SA>(rhs, sstride);
  p += rhs_offset<S>(rhs, sstride);
  const RA beta = sizeof(RA) == 4 ? (RA)st[rhs].beta_f : (RA)st[rhs].beta;
  cx<RA> rv[12];
  cx<R> pv[12];
  load_spinor<SA>(r, sstride, ih, rv);
  load_spinor<S>(p, sstride, ih, pv);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    cx<RA> q = rv[k] + beta * cx<RA>{(RA)pv[k].re, (RA)pv[k].im};
    pv[k] = {(R)q.re, (R)q.im};
  }
  store_spinor<S>(p, sstride, ih, pv);
}

}  // namespace tsm
