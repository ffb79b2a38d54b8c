// contract.cu -- host side of the loop contraction: insertion tables, phase
// tables, launches of the contraction / reduction / combine kernels.
#include <cmath>
#include <complex>

#include "contract.h"

namespace tsm {

// The 16 insertions in the chiral basis, reduced to (column, power of i) per
// row.  Built here from the gamma matrices themselves:
// gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0, 1], [1, 0]].
static void build_insertions(std::complex<double> G[16][4][4]) {
  using C = std::complex<double>;
  const C I(0.0, 1.0);
  C sig[3][2][2] = {{{0.0, 1.0}, {1.0, 0.0}}, {{0.0, -I}, {I, 0.0}}, {{1.0, 0.0}, {0.0, -1.0}}};
  C g[4][4][4] = {};
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        g[k][a][2 + b] = -I * sig[k][a][b];
        g[k][2 + a][b] = I * sig[k][a][b];
      }
  for (int a = 0; a < 2; ++a) {
    g[3][a][2 + a] = 1.0;
    g[3][2 + a][a] = 1.0;
  }
  auto mul = [](const C A[4][4], const C B[4][4], C out[4][4]) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        C s = 0.0;
        for (int k = 0; k < 4; ++k) s += A[i][k] * B[k][j];
        out[i][j] = s;
      }
  };
  C g5[4][4], t1[4][4], t2[4][4];
  mul(g[0], g[1], t1);
  mul(t1, g[2], t2);
  mul(t2, g[3], g5);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) G[0][i][j] = (i == j) ? 1.0 : 0.0;
  for (int m = 0; m < 4; ++m)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) G[1 + m][i][j] = g[m][i][j];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) G[5][i][j] = g5[i][j];
  for (int m = 0; m < 4; ++m) mul(g[m], g5, G[6 + m]);
  const int pairs[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  for (int k = 0; k < 6; ++k) {
    C ab[4][4], ba[4][4];
    mul(g[pairs[k][0]], g[pairs[k][1]], ab);
    mul(g[pairs[k][1]], g[pairs[k][0]], ba);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) G[10 + k][i][j] = 0.5 * I * (ab[i][j] - ba[i][j]);
  }
}

int make_gamma_tab(const int* gammas, int n, GammaTab* tab) {
  if (n < 1 || n > CT_MAXG) {
    set_error("n_gamma must be in [1, %d]", CT_MAXG);
    return TSM_ERR_ARG;
  }
  std::complex<double> G[16][4][4];
  build_insertions(G);
  tab->n = n;
  for (int k = 0; k < n; ++k) {
    const int gi = gammas[k];
    if (gi < 0 || gi > 15) {
      set_error("gamma index %d out of [0, 16)", gi);
      return TSM_ERR_ARG;
    }
    for (int row = 0; row < 4; ++row) {
      int found = 0;
      for (int col = 0; col < 4; ++col) {
        const std::complex<double> v = G[gi][row][col];
        if (std::abs(v) < 1e-12) continue;
        int ph;
        if (std::abs(v - 1.0) < 1e-12) ph = 0;
        else if (std::abs(v - std::complex<double>(0, 1)) < 1e-12) ph = 1;
        else if (std::abs(v + 1.0) < 1e-12) ph = 2;
        else if (std::abs(v - std::complex<double>(0, -1)) < 1e-12) ph = 3;
        else {
          set_error("insertion %d is not a signed permutation", gi);
          return TSM_ERR_ARG;
        }
        tab->col[k][row] = (int8_t)col;
        tab->ph[k][row] = (int8_t)ph;
        ++found;
      }
      if (found != 1) {
        set_error("insertion %d row %d has %d non-zeros", gi, row, found);
        return TSM_ERR_ARG;
      }
    }
    // the contraction kernels take the insertion from its compiled code
    const uint32_t code = chiral_code(gi);
    for (int row = 0; row < 4; ++row)
      if (tab->col[k][row] != (int)(row ^ (code & 3u)) || tab->ph[k][row] != (int)((code >> (2 + 2 * row)) & 3u)) {
        set_error("insertion %d: compiled chiral code disagrees with the gamma matrices", gi);
        return TSM_ERR_ARG;
      }
    tab->idx[k] = (int8_t)gi;
  }
  return TSM_OK;
}

int group_momenta(const int* L, const int* moms, int nq, CtMoments* m) {
  if (nq < 1 || nq > CT_MAXQ) {
    set_error("a contraction pass takes 1 to %d momenta", CT_MAXQ);
    return TSM_ERR_ARG;
  }
  *m = CtMoments{};
  int key[CT_MAXQ][3], neg[CT_MAXQ][3];
  for (int q = 0; q < nq; ++q)
    for (int ax = 0; ax < 3; ++ax) {
      int k = moms[3 * q + ax] % L[ax];
      if (k < 0) k += L[ax];
      key[q][ax] = k;
      neg[q][ax] = (L[ax] - k) % L[ax];
    }
  auto same = [](const int* x, const int* y) { return x[0] == y[0] && x[1] == y[1] && x[2] == y[2]; };
  for (int q = 0; q < nq; ++q) {
    int cls = -1, sg = 0;
    for (int j = 0; j < m->ncls && cls < 0; ++j)
      if (same(key[q], key[m->rep[j]])) cls = j, sg = 1;
    for (int j = 0; j < m->ncls && cls < 0; ++j)
      if (same(neg[q], key[m->rep[j]])) cls = j, sg = -1;
    if (cls < 0) {
      cls = m->ncls++;
      m->rep[cls] = (int8_t)q;
      m->nz[cls] = (int8_t)!(key[q][0] == 0 && key[q][1] == 0 && key[q][2] == 0);
      m->ch[cls] = (int8_t)m->nch;
      m->nch += 1 + m->nz[cls];
      sg = 1;
    }
    m->qch[q] = m->ch[cls];
    m->qsg[q] = (int8_t)(m->nz[cls] ? sg : 0);
  }
  m->ncp = (m->nch + 3) & ~3;
  return TSM_OK;
}

int ContractPlan::prepare(Ctx& c, const int* gammas, int n_gamma, const int* moms, int n_q_) {
  if (moms == nullptr || gammas == nullptr || n_q_ < 1) {
    set_error("gammas / moms must be non-null, n_q >= 1");
    return TSM_ERR_ARG;
  }
  TSM_TRY(make_gamma_tab(gammas, n_gamma, &gam));
  n_q = n_q_;
  ng = n_gamma;
  const int* L = c.lat.L;
  passes.clear();
  for (int q0 = 0; q0 < n_q; q0 += CT_MAXQ) {
    CtMoments m{};
    TSM_TRY(group_momenta(L, moms + 3 * q0, std::min(CT_MAXQ, n_q - q0), &m));
    passes.push_back(m);
  }
  std::vector<double2> tab((size_t)n_q * (L[0] + L[1] + L[2]));
  const double twopi = 2.0 * std::acos(-1.0);
  size_t off = 0;
  for (int ax = 0; ax < 3; ++ax)
    for (int q = 0; q < n_q; ++q)
      for (int x = 0; x < L[ax]; ++x) {
        // reduce n*x mod L exactly in integers before the angle is formed
        long long nx = (long long)moms[3 * q + ax] * x;
        nx %= L[ax];
        if (nx < 0) nx += L[ax];
        const double ang = twopi * (double)nx / (double)L[ax];
        tab[off++] = make_double2(std::cos(ang), std::sin(ang));
      }
  void* dev = nullptr;
  TSM_TRY(c.buffer("phase_tab", tab.size() * sizeof(double2), &dev));
  TSM_CUDA(cudaMemcpyAsync(dev, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  phx = static_cast<double2*>(dev);
  phy = phx + (size_t)n_q * L[0];
  phz = phy + (size_t)n_q * L[1];
  std::vector<float2> ftab(tab.size());
  for (size_t k = 0; k < tab.size(); ++k) ftab[k] = make_float2((float)tab[k].x, (float)tab[k].y);
  void* fdev = nullptr;
  TSM_TRY(c.buffer("phase_tab_f32", ftab.size() * sizeof(float2), &fdev));
  TSM_CUDA(cudaMemcpyAsync(fdev, ftab.data(), ftab.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream));
  TSM_CUDA(cudaStreamSynchronize(c.stream));
  fphx = static_cast<float2*>(fdev);
  fphy = fphx + (size_t)n_q * L[0];
  fphz = fphy + (size_t)n_q * L[1];
  return TSM_OK;
}

template <class R, class SA, class SB>
int launch_contract(Ctx& c, const ContractPlan& plan, const NoiseSpec& ns, uint32_t source, EOField a,
                    const EOField* b, double2* out, const EOField* wa, const EOField* wb) {
  if (plan.one_end == CT_GEN_ONE_END && (wa == nullptr || (b != nullptr && wb == nullptr))) {
    set_error("generalised one-end contraction needs D_W of its fields");
    return TSM_ERR_ARG;
  }
  constexpr int NT = ContractNT<R>::value;
  const int vs2 = c.lat.L[0] * c.lat.L[1] * c.lat.L[2] / 2;
  const int T = c.lat.L[3];
  const int nbx = (vs2 + NT - 1) / NT;
  const size_t block = (size_t)plan.ng * plan.n_q * T;   // one [n_gamma][n_q][T] output block
  // one kernel + fixed-order reduction per chunk of at most CT_MAXQ momenta
  // algorithmic bytes per site of a pass: the fields it reads (noise is regenerated)
  const double sa = spinor_site_bytes(SA::id), sbb = spinor_site_bytes(SB::id);
  const double fields = sa + (b ? sbb : 0.0) + (wa ? sa : 0.0) + (wb ? sbb : 0.0);
  auto passes = [&](double2* dst, int kind, double site_bytes, auto&& launch) -> int {
    for (int q0 = 0; q0 < plan.n_q; q0 += CT_MAXQ) {
      const int nq = std::min(CT_MAXQ, plan.n_q - q0);
      const int nout = plan.ng * nq;
      // + block partials written and read back, + the output block
      TimedLaunch tl(c, kind,
                     (double)c.g.V * site_bytes + (double)T * 2 * nbx * nout * 32.0 + (double)nout * T * 16.0, true);
      void* part = nullptr;
      TSM_TRY(c.buffer("contract_partial", (size_t)T * 2 * nbx * CT_MAXG * CT_MAXQ * sizeof(double2), &part));
      ContractArgs<SA, SB> args{};
      args.g = c.g;
      args.noise = ns;
      args.source = source;
      args.a[0] = a.e.as<SA>();
      args.a[1] = a.o.as<SA>();
      args.b[0] = b ? b->e.as<SB>() : nullptr;
      args.b[1] = b ? b->o.as<SB>() : nullptr;
      args.sstride = c.sstride;
      args.gam = plan.gam;
      args.mom = plan.passes[q0 / CT_MAXQ];
      args.nq = nq;
      args.phx = plan.phx + (size_t)q0 * c.lat.L[0];
      args.phy = plan.phy + (size_t)q0 * c.lat.L[1];
      args.phz = plan.phz + (size_t)q0 * c.lat.L[2];
      args.fphx = plan.fphx + (size_t)q0 * c.lat.L[0];
      args.fphy = plan.fphy + (size_t)q0 * c.lat.L[1];
      args.fphz = plan.fphz + (size_t)q0 * c.lat.L[2];
      args.partial = static_cast<double2*>(part);
      args.nbx = nbx;
      args.wa[0] = wa ? wa->e.as<SA>() : nullptr;
      args.wa[1] = wa ? wa->o.as<SA>() : nullptr;
      args.wb[0] = wb ? wb->e.as<SB>() : nullptr;
      args.wb[1] = wb ? wb->o.as<SB>() : nullptr;
      args.fre = plan.one_end == CT_GEN_ONE_END ? 2.0 : 0.0;
      args.fim = plan.one_end == CT_ONE_END ? -4.0 * c.lat.kappa * c.lat.mu : 0.0;
      args.ffre = (float)args.fre;
      args.ffim = (float)args.fim;
      launch(args, dim3(nbx, T, 2));
      c.launches++;
      TSM_TRY(check_launch(c, "contract_kernel"));
      const dim3 rgrid((unsigned)((nout + 31) / 32), (unsigned)T), rblock(32, CT_RED_WARPS);
      contract_reduce_kernel<<<rgrid, rblock, 0, c.stream>>>(static_cast<double2*>(part), T, nbx, plan.ng, nq,
                                                             plan.n_q, q0, dst);
      c.launches++;
      TSM_TRY(check_launch(c, "contract_reduce_kernel"));
      tl.done();
    }
    return TSM_OK;
  };
  double2* dst = out;
  if (plan.local) {
    TSM_TRY(passes(dst, PB_CONTRACT, fields, [&](const ContractArgs<SA, SB>& args, dim3 grid) {
      if (plan.one_end == CT_ONE_END) contract_kernel<R, SA, SB, CT_ONE_END><<<grid, NT, 0, c.stream>>>(args);
      else if (plan.one_end == CT_GEN_ONE_END)
        contract_kernel<R, SA, SB, CT_GEN_ONE_END><<<grid, NT, 0, c.stream>>>(args);
      else contract_kernel<R, SA, SB, CT_STANDARD><<<grid, NT, 0, c.stream>>>(args);
    }));
    dst += block;
  }
  using LS = typename DerivLinks<R>::type;
  for (int mu = 0; mu < 4; ++mu) {
    if (!((plan.deriv_mask >> mu) & 1)) continue;
    // the direction's forward and backward link of every site on top of the fields
    TSM_TRY(passes(dst, PB_DERIV, fields + link_site_bytes(LS::id) / 4.0, [&](const ContractArgs<SA, SB>& args,
                                                                             dim3 grid) {
      DerivArgs<SA, SB, LS> d{};
      d.base = args;
      d.U[0] = c.links_of<LS>(0);
      d.U[1] = c.links_of<LS>(1);
      d.lstride = c.lstride;
      d.mu = mu;
      deriv_contract_kernel<R, SA, SB, LS><<<grid, NT, 0, c.stream>>>(d);
    }));
    dst += block;
  }
  return TSM_OK;
}

template int launch_contract<double, F64, F64>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                               const EOField*, double2*, const EOField*, const EOField*);
template int launch_contract<float, F64, F64>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                              const EOField*, double2*, const EOField*, const EOField*);
template int launch_contract<float, F32, F32>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                              const EOField*, double2*, const EOField*, const EOField*);
template int launch_contract<float, F64, F32>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                              const EOField*, double2*, const EOField*, const EOField*);
template int launch_contract<double, F64, F32>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                               const EOField*, double2*, const EOField*, const EOField*);
template int launch_contract<float, F32, F64>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                              const EOField*, double2*, const EOField*, const EOField*);
template int launch_contract<float, F64, F16>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                              const EOField*, double2*, const EOField*, const EOField*);
template int launch_contract<float, F32, F16>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                              const EOField*, double2*, const EOField*, const EOField*);
template int launch_contract<float, F16, F16>(Ctx&, const ContractPlan&, const NoiseSpec&, uint32_t, EOField,
                                              const EOField*, double2*, const EOField*, const EOField*);

int apply_wilson(Ctx& c, int prec, EOField in, EOField out) {
  // one field: the one-thread-per-site stencil (link tiles pay only when
  // several sources share them)
  const bool per_site = c.hop_per_site;
  c.hop_per_site = true;
  const int rc = dispatch_prec(prec, [&](auto tag) -> int {
    using S = decltype(tag);
    // both parities: links, neighbour field, centre field, output
    TimedLaunch tl(c, PB_WILSON, (double)c.g.V * (link_site_bytes(S::id) + 3.0 * spinor_site_bytes(S::id)), true);
    for (int par = 0; par < 2; ++par) {
      HopArgs<S> h{};
      h.g = c.g;
      h.p_out = par;
      h.Uout = c.links_of<S>(par);
      h.Uin = c.links_of<S>(1 - par);
      h.lstride = c.lstride;
      h.sstride = c.sstride;
      h.in = (par ? in.e : in.o).as<S>();
      h.center = (par ? in.o : in.e).as<S>();
      h.out = (par ? out.o : out.e).as<S>();
      h.ac = 1.0;
      h.ah = -c.lat.kappa;
      h.tc = twist_one();
      h.to = twist_one();
      h.ts = twist_one();
      h.red = c.red;
      h.post = POST_NONE;
      TSM_TRY(launch_hop<S>(c, h, 0, HOP_CENTER, -1));
    }
    tl.done();
    return (int)TSM_OK;
  });
  c.hop_per_site = per_site;
  return rc;
}

int reserve_contract(Ctx& c) {
  constexpr int NT = ContractNT<double>::value;   // the smaller block: the most partials
  const int vs2 = c.lat.L[0] * c.lat.L[1] * c.lat.L[2] / 2;
  const int nbx = (vs2 + NT - 1) / NT;
  void* part = nullptr;
  return c.buffer("contract_partial", (size_t)c.lat.L[3] * 2 * nbx * CT_MAXG * CT_MAXQ * sizeof(double2), &part);
}

int launch_combine(Ctx& c, const double2* corr, int n_hp, const double2* lp, int n_lp, int E, double2* est,
                   double* err, double2* lp_mean, double2* corr_mean) {
  if (E <= 0) return TSM_OK;
  combine_kernel<<<(E + 127) / 128, 128, 0, c.stream>>>(corr, n_hp, lp, n_lp, E, est, err, lp_mean, corr_mean);
  c.launches++;
  return check_launch(c, "combine_kernel");
}

NoiseSpec make_noise(uint64_t seed, int kind) {
  NoiseSpec n{};
  n.k0 = (uint32_t)(seed & 0xffffffffull);
  n.k1 = (uint32_t)(seed >> 32);
  n.kind = kind;
  n.amp = (kind == 4) ? 1.0 / std::sqrt(2.0) : 1.0;
  n.famp = (float)n.amp;
  return n;
}

}  // namespace tsm
