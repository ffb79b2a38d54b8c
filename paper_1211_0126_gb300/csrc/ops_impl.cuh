// ops_impl.cuh -- definitions of the launch helpers declared in context.h.
// Included by ops_f64.cu / ops_f32.cu / ops_f16.cu, each of which
// instantiates them for its storage types (parallel compilation).
#pragma once

#include "context.h"
#include "fields.cuh"

namespace tsm {

inline int blocks_for(int n, int nt) { return (n + nt - 1) / nt; }

template <class S>
static int hop_kind_of(int dag, int mode) {
  if (dag) return PK_HOP_DAG;
  return (mode & HOP_CENTER) ? PK_HOP_XPAY : PK_HOP;
}


template <class S>
int launch_hop(Ctx& c, const HopArgs<S>& a0, int dag, int mode, int prof_kind, int nrhs) {
  const int nb = blocks_for(a0.g.Vh, HOP_NT);
  if (nb == 0 || nrhs == 0) return TSM_OK;
  HopArgs<S> a = a0;
  a.fts = to_float(a.ts);
  {
    Twist toah, totc;
    for (int q = 0; q < 2; ++q) {
      toah.re[q] = a.to.re[q] * a.ah;
      toah.im[q] = a.to.im[q] * a.ah;
      totc.re[q] = (a.to.re[q] * a.tc.re[q] - a.to.im[q] * a.tc.im[q]) * a.ac;
      totc.im[q] = (a.to.re[q] * a.tc.im[q] + a.to.im[q] * a.tc.re[q]) * a.ac;
    }
    a.fto_ah = to_float(toah);
    a.fto_tc_ac = to_float(totc);
  }
  const int kind = prof_kind >= 0 ? prof_kind : hop_kind_of<S>(dag, mode);
  const double sb = spinor_site_bytes(S::id), lb = link_site_bytes(S::id);
  // links once per launch (shared by the right-hand sides), spinor streams per RHS
  const double bytes = (double)a.g.Vh *
      (lb + nrhs * sb * (2 + ((mode & HOP_CENTER) ? 1 : 0) + ((mode & HOP_BASE) ? 1 : 0)));
  TimedLaunch tl(c, 4 * S::id + kind, bytes);
  // 16-bit tiers: link-sharing blocks of LT_SITES sites x up to RPB sources
  // (RPB = c.tile_rpb, 2, 4 or 8, and for 4 a register budget of 80 or 96,
  // from the autotuner; every solve, whatever its
  // batch width, so that a source's iterates do not depend on its batch); the
  // FP32 tier the same for the hops without a reduction (its reducing hop K2
  // measured slower in tiles; per-site arithmetic, and so every result, is the
  // same in both kernels); FP64, and single-source operator applications
  // outside the solvers (c.hop_per_site): one thread per (source, site),
  // blocks of HOP_NT sites
  constexpr bool TILE16 = S::id == F16::id || S::id == BF16::id;
  constexpr bool TILE32 = S::id == F32::id;
  // (FP32: only with several sources to share the links; a single field runs
  // faster one thread per site, with the same bits)
  const bool tile = TILE16 ? !(c.hop_per_site && nrhs == 1) : (TILE32 && !(mode & HOP_NORM) && nrhs >= 2);
  const int RPB = c.tile_rpb[S::id];
  const bool wide = RPB == 4 && c.tile_regs[S::id] == 96;   // 96-register variant (4 sources only)
  const int rpb = nrhs < RPB ? nrhs : RPB;
  const int tile_sites = LT_SITES * ((mode & HOP_NORM) ? LtGroups<HOP_NORM>::value : LtGroups<0>::value);
  const dim3 grid = tile ? dim3((nrhs + rpb - 1) / rpb, blocks_for(a.g.Vh, tile_sites)) : dim3(nrhs, nb);
  const dim3 block = tile ? dim3(LT_SITES, rpb) : dim3(HOP_NT);
#define TSM_HOP_CASE(D, M)                                                                        \
  if (dag == (D) && mode == (M)) {                                                                \
    if (tile) {                                                                                   \
      if constexpr (TILE16 || (TILE32 && !((M) & HOP_NORM))) {                                    \
        if (RPB == 2) hop_tile_kernel<S, (D), (M), 2, 80><<<grid, block, 0, c.stream>>>(a, nrhs); \
        else if (RPB == 8) hop_tile_kernel<S, (D), (M), 8, 80><<<grid, block, 0, c.stream>>>(a, nrhs); \
        else if (wide) hop_tile_kernel<S, (D), (M), 4, 96><<<grid, block, 0, c.stream>>>(a, nrhs); \
        else hop_tile_kernel<S, (D), (M), 4, 80><<<grid, block, 0, c.stream>>>(a, nrhs);          \
      }                                                                                           \
    } else {                                                                                      \
      hop_kernel<S, (D), (M)><<<grid, block, 0, c.stream>>>(a);                                   \
    }                                                                                             \
  }
  TSM_HOP_CASE(0, 0)
  else TSM_HOP_CASE(0, HOP_CENTER)
  else TSM_HOP_CASE(0, HOP_CENTER | HOP_NORM)
  else TSM_HOP_CASE(0, HOP_CENTER | HOP_NORM | HOP_BASE)
  else TSM_HOP_CASE(1, 0)
  else TSM_HOP_CASE(1, HOP_CENTER)
  else TSM_HOP_CASE(1, HOP_CENTER | HOP_NORM)
  else TSM_HOP_CASE(1, HOP_CENTER | HOP_NORM | HOP_BASE)
  else {
    set_error("hop kernel variant dag=%d mode=%d not built", dag, mode);
    return TSM_ERR_ARG;
  }
#undef TSM_HOP_CASE
  tl.done();
  c.launches++;
  return check_launch(c, "hop_kernel");
}

template <class S, class SA>
int launch_cg_update(Ctx& c, const CGUpdArgs<S, SA>& a0, int nrhs) {
  const int nb = blocks_for(a0.g.Vh, HOP_NT);
  if (nb == 0 || nrhs == 0) return TSM_OK;
  CGUpdArgs<S, SA> a = a0;
  a.fkappa2 = (float)a.kappa2;
  a.ftw = to_float(a.tw);
  const double sb = spinor_site_bytes(S::id), lb = link_site_bytes(S::id), sa = spinor_site_bytes(SA::id);
  TimedLaunch tl(c, 4 * S::id + PK_HOP_UPDATE, (double)a.g.Vh * (lb + nrhs * (3 * sb + 4 * sa)));
  // one thread per (source, site) for every tier: the update is memory-bound,
  // and link sharing measured slower here (534 against 511 us per launch)
  cg_update_kernel<S, SA><<<dim3(nrhs, blocks_for(a.g.Vh, HOP_NT * UpdGroups<S, SA>::value)), HOP_NT, 0, c.stream>>>(a);
  tl.done();
  c.launches++;
  return check_launch(c, "cg_update_kernel");
}

template <class S, class SA>
int launch_cg_p(Ctx& c, const PField& r, const PField& p, CGState* st, const int* active, int nrhs) {
  const int nb = blocks_for(c.g.Vh, SITE_NT);
  if (nb == 0 || nrhs == 0) return TSM_OK;
  cg_p_kernel<S, SA><<<dim3(nrhs, nb), SITE_NT, 0, c.stream>>>(r.as<SA>(), p.as<S>(), c.sstride, c.g.Vh, active, st);
  c.launches++;
  return check_launch(c, "cg_p_kernel");
}

template <class S>
int launch_pack(Ctx& c, int parity, const double* canon, const PField& out) {
  const int nb = blocks_for(c.g.Vh, SITE_NT);
  pack_spinor_kernel<S><<<nb, SITE_NT, 0, c.stream>>>(c.g, parity, reinterpret_cast<const double2*>(canon),
                                                      out.as<S>(), c.sstride);
  c.launches++;
  return check_launch(c, "pack_spinor_kernel");
}

template <class S>
int launch_unpack(Ctx& c, int parity, const PField& in, double* canon) {
  const int nb = blocks_for(c.g.Vh, SITE_NT);
  unpack_spinor_kernel<S><<<nb, SITE_NT, 0, c.stream>>>(c.g, parity, in.as<S>(), c.sstride,
                                                        reinterpret_cast<double2*>(canon));
  c.launches++;
  return check_launch(c, "unpack_spinor_kernel");
}

template <class S>
int launch_noise(Ctx& c, int parity, const NoiseSpec& n, uint32_t source0, const PField& out, int nrhs) {
  const int nb = blocks_for(c.g.Vh, SITE_NT);
  noise_kernel<S><<<dim3(nrhs, nb), SITE_NT, 0, c.stream>>>(c.g, parity, n, source0, out.as<S>(), c.sstride);
  c.launches++;
  return check_launch(c, "noise_kernel");
}

template <class S>
int launch_twist(Ctx& c, const Twist& f, const PField& in, const PField& out, const CGState* st,
                 const int* active, int nrhs) {
  const int nb = blocks_for(c.g.Vh, SITE_NT);
  if (nrhs == 0) return TSM_OK;
  twist_kernel<S><<<dim3(nrhs, nb), SITE_NT, 0, c.stream>>>(c.g.Vh, f, in.as<S>(), out.as<S>(), c.sstride, active,
                                                            st);
  c.launches++;
  return check_launch(c, "twist_kernel");
}

template <class S>
int launch_norm(Ctx& c, const PField& v, CGState* st, int post, const int* active, int nrhs) {
  const int nb = blocks_for(c.g.Vh, SITE_NT);
  if (nrhs == 0) return TSM_OK;
  norm_kernel<S><<<dim3(nrhs, nb), SITE_NT, 0, c.stream>>>(c.g.Vh, v.as<S>(), c.sstride, c.red, active, st, post);
  c.launches++;
  return check_launch(c, "norm_kernel");
}

template <class Si, class So>
int launch_convert(Ctx& c, const PField& in, const PField& out, const int* active, int nrhs) {
  const int nb = blocks_for(c.g.Vh, SITE_NT);
  if (nrhs == 0) return TSM_OK;
  convert_kernel<Si, So><<<dim3(nrhs, nb), SITE_NT, 0, c.stream>>>(c.g.Vh, in.as<Si>(), out.as<So>(), c.sstride,
                                                                   active);
  c.launches++;
  return check_launch(c, "convert_kernel");
}

}  // namespace tsm

#define TSM_INSTANTIATE_STORAGE(S)                                                                    \
  template int tsm::launch_hop<S>(Ctx&, const HopArgs<S>&, int, int, int, int);                      \
  template int tsm::launch_pack<S>(Ctx&, int, const double*, const PField&);                         \
  template int tsm::launch_unpack<S>(Ctx&, int, const PField&, double*);                             \
  template int tsm::launch_noise<S>(Ctx&, int, const NoiseSpec&, uint32_t, const PField&, int);      \
  template int tsm::launch_twist<S>(Ctx&, const Twist&, const PField&, const PField&, const CGState*, \
                                    const int*, int);                                                \
  template int tsm::launch_norm<S>(Ctx&, const PField&, CGState*, int, const int*, int);

#define TSM_INSTANTIATE_PAIR(S, SA)                                                    \
  template int tsm::launch_cg_update<S, SA>(Ctx&, const CGUpdArgs<S, SA>&, int);      \
  template int tsm::launch_cg_p<S, SA>(Ctx&, const PField&, const PField&, CGState*, const int*, int);

#define TSM_INSTANTIATE_CONVERT(Si, So) \
  template int tsm::launch_convert<Si, So>(Ctx&, const PField&, const PField&, const int*, int);
