"""Loop contraction, exact loops and the TSM combine (oracle; test infrastructure).

Loop of one source (Sec. 2.3: (1/N) sum_r <eta_r^dag X s_r> ~ Tr(M^-1 X); all
timeslices come out at once, Sec. 4):

    L_j(Gamma, t, q) = sum_{x : x_4 = t} exp(i q.x) eta_j(x)^dag Gamma s_j(x),
    q = 2 pi (n_x / Lx, n_y / Ly, n_z / Lz),  x in [0, L).

Exact loop from a dense inverse (what the estimator converges to, Eq. 2.2):

    L(Gamma, t, q) = sum_{x : x_4 = t} exp(i q.x) tr_{spin,colour}[Gamma D^-1(x, x)].

TSM estimator (Sec. 2.2, Eq. 2.4).  Reading of the index sets: the HP set is
j = 0..N_HP-1 and the LP set j = N_HP..N_HP+N_LP-1, disjoint (the printed LP
sum runs over N_LP + 1 terms, read as an off-by-one; the text after Eq. 2.4
counts N_HP + N_LP low-precision inversions).

    L_TSM = (1/N_HP) sum_{j in HP} [L_j(s_HP) - L_j(s_LP)] + (1/N_LP) sum_{j in LP} L_j(s_LP)

Error (reading; the paper gives none): sigma^2 = Var_corr / N_HP + Var_LP / N_LP
with Var the unbiased sample variance of the complex per-source values,
Var = sum |X_j - mean|^2 / (N - 1).

One-end trick (Sec. 2.3, Eq. 2.5) for the isovector loop u - d of twisted
mass, D_u = D_tm(+mu), D_d = D_tm(-mu) = gamma5 D_u^dag gamma5.  Since
D_u - D_d = 4 i kappa mu gamma5 in this normalisation,

    D_u^-1 - D_d^-1 = -4 i kappa mu D_u^-1 D_u^-dag gamma5,

so with s = D_u^-1 eta and E[eta eta^dag] = 1,

    Tr[P Gamma (D_u^-1 - D_d^-1)] = -4 i kappa mu E[s^dag gamma5 P Gamma s]

(P: the diagonal timeslice / phase projector, which commutes with gamma5).
The per-source value is L^1_j(Gamma, t, q) = -4 i kappa mu
sum_{x: x_4 = t} e^{iq.x} s_j(x)^dag gamma5 Gamma s_j(x); it is quadratic in s,
so the TSM correction is L^1(s_HP) - L^1(s_LP).  The paper writes the same
identity for M = D / (2 kappa) in physical units (-2 i mu a M_d^-1 gamma5
M_u^-1); the factor and sign here are those of D_tm itself, fixed by the
dense-matrix pins in tests.

Generalised one-end trick (Eq. 2.6) for the isoscalar loop u + d: with the
Wilson operator D_W = 1 - kappa H, D_u + D_d = 2 D_W, hence
D_u^-1 + D_d^-1 = 2 D_d^-1 D_W D_u^-1 = 2 gamma5 D_u^-dag gamma5 D_W D_u^-1,
and because D_u D_u^dag = gamma5 D_u^dag D_u gamma5 for twisted mass,

    Tr[P Gamma (D_u^-1 + D_d^-1)] = 2 E[s^dag gamma5 P Gamma gamma5 D_W s].

Per-source value L^2_j = 2 sum_{x: x_4 = t} e^{iq.x} s_j(x)^dag gamma5 Gamma
gamma5 (D_W s_j)(x): one extra application of the Wilson hop per source; no
mu suppression, so it is noisier than Eq. 2.5 (as the paper notes).

One-derivative insertions (the paper tunes the TSM on i psibar gamma_3 D_3 psi,
Sec. 3, without defining D; reading: the symmetric covariant derivative
D<->_mu = (D->_mu - D<-_mu) / 2 with D->_mu psi(x) = [U_mu(x) psi(x+mu) -
U_mu(x-mu)^dag psi(x-mu)] / 2, the fermion boundary sign on hops across
t = T-1 <-> 0, the operator and its phase at x):

    O_{Gamma mu}(x) = 1/4 [psibar(x) Gamma U_mu(x) psi(x+mu) - psibar(x) Gamma U_mu(x-mu)^dag psi(x-mu)
                          - psibar(x+mu) U_mu(x)^dag Gamma psi(x) + psibar(x-mu) U_mu(x-mu) Gamma psi(x)]

whose loop (same trace convention as the local loops) is estimated per source by
1/4 [eta(x)^dag Gamma (T+ s - T- s)(x) - ((T+ eta - T- eta)(x))^dag Gamma s(x)],
T+ f(x) = U_mu(x) f(x+mu), T- f(x) = U_mu(x-mu)^dag f(x-mu) (signs included).
"""
import numpy as np

from .gamma import gamma_list
from . import dirac, philox, ptnet, solver


def phases(dims, moms):
    """exp(i q.x) on the full lattice for each momentum n in moms: [n_q, T, Z, Y, X]."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                             np.arange(lx), indexing='ij')
    out = []
    for n in moms:
        arg = 2 * np.pi * (n[0] * x / lx + n[1] * y / ly + n[2] * z / lz)
        out.append(np.exp(1j * arg))
    return np.array(out)


def local_loops(eta, s, dims, gammas, moms):
    """L(Gamma, t, q) for one source: [n_gamma, n_q, T] complex."""
    G = gamma_list()[list(gammas)]
    # eta^dag Gamma s at each site, colour summed
    dens = np.einsum('tzyxac,gab,tzyxbc->gtzyx', np.conj(eta), G, s)
    ph = phases(dims, moms)
    return np.einsum('qtzyx,gtzyx->gqt', ph, dens)


def one_end_loops(s, dims, kappa, mu, gammas, moms):
    """One-end-trick value of one source s = D_u^-1 eta: [n_gamma, n_q, T] complex."""
    G = gamma_list()[list(gammas)]
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    G5 = np.einsum('ab,gbc->gac', g5, G)              # gamma5 Gamma
    dens = np.einsum('tzyxac,gab,tzyxbc->gtzyx', np.conj(s), G5, s)
    ph = phases(dims, moms)
    return -4j * kappa * mu * np.einsum('qtzyx,gtzyx->gqt', ph, dens)


def gen_one_end_loops(U, s, dims, kappa, gammas, moms, antiperiodic_t=True):
    """Generalised one-end-trick value of one source s = D_u^-1 eta (Eq. 2.6)."""
    G = gamma_list()[list(gammas)]
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    Y = np.einsum('ab,gbc,cd->gad', g5, G, g5)           # gamma5 Gamma gamma5
    dw = s - kappa * dirac.hop(U, s, dims, antiperiodic_t)   # D_W s
    dens = np.einsum('tzyxac,gab,tzyxbc->gtzyx', np.conj(s), Y, dw)
    ph = phases(dims, moms)
    return 2.0 * np.einsum('qtzyx,gtzyx->gqt', ph, dens)


def fft_loops(eta, s, dims, gammas):
    """Local loops of one source at every spatial momentum, [n_gamma, T, Lz, Ly, Lx]:
    index (n_z, n_y, n_x) holds q = 2 pi n / L with the phase e^{+i q.x} (numpy's
    inverse FFT has that sign and a 1/N factor, undone here)."""
    lx, ly, lz, lt = dims
    G = gamma_list()[list(gammas)]
    dens = np.einsum('tzyxac,gab,tzyxbc->gtzyx', np.conj(eta), G, s)
    return np.fft.ifftn(dens, axes=(2, 3, 4)) * (lx * ly * lz)


def deriv_loops(U, eta, s, dims, gammas, mus, moms, antiperiodic_t=True):
    """Per-source one-derivative loops: [n_gamma, n_mu, n_q, T] complex."""
    G = gamma_list()[list(gammas)]
    ph = phases(dims, moms)
    out = []
    for mu in mus:
        ts = (ptnet.transport(U, s, dims, 2 * mu + 1, antiperiodic_t)
              - ptnet.transport(U, s, dims, 2 * mu + 2, antiperiodic_t))
        te = (ptnet.transport(U, eta, dims, 2 * mu + 1, antiperiodic_t)
              - ptnet.transport(U, eta, dims, 2 * mu + 2, antiperiodic_t))
        dens = 0.25 * (np.einsum('tzyxac,gab,tzyxbc->gtzyx', np.conj(eta), G, ts)
                       - np.einsum('tzyxac,gab,tzyxbc->gtzyx', np.conj(te), G, s))
        out.append(np.einsum('qtzyx,gtzyx->gqt', ph, dens))
    return np.transpose(np.array(out), (1, 0, 2, 3))


def exact_deriv_loops(U, Dinv, dims, gammas, mus, moms, antiperiodic_t=True):
    """One-derivative loops from a dense inverse, term by term from the operator's
    definition: sum_{x in t} e^{iqx} Tr[A_{Gamma mu}(x) D^-1] with the four
    site-pair blocks of A (index 12*site + 3*spin + colour)."""
    lx, ly, lz, lt = dims
    vol = lx * ly * lz * lt
    B = Dinv.reshape(vol, 4, 3, vol, 4, 3)
    G = gamma_list()[list(gammas)]
    ph = phases(dims, moms)
    out = np.zeros((len(gammas), len(mus), len(moms), lt), dtype=np.complex128)

    def site(c):
        return ((c[3] * lz + c[2]) * ly + c[1]) * lx + c[0]

    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    c = [x, y, z, t]
                    i = site(c)
                    for k, mu in enumerate(mus):
                        cf, cb = list(c), list(c)
                        cf[mu] = (c[mu] + 1) % dims[mu]
                        cb[mu] = (c[mu] - 1) % dims[mu]
                        sf = -1.0 if (mu == 3 and antiperiodic_t and c[3] == lt - 1) else 1.0
                        sb = -1.0 if (mu == 3 and antiperiodic_t and c[3] == 0) else 1.0
                        f, b = site(cf), site(cb)
                        uf = U[t, z, y, x, mu]                                      # U_mu(x)
                        ub = U[cb[3], cb[2], cb[1], cb[0], mu]                       # U_mu(x - mu)
                        for gi in range(len(gammas)):
                            g = G[gi]
                            # tr[(Gamma x M) D^-1(z, y)] = sum g_{ss'} M_{ab} D^-1_{(z s' b), (y s a)}
                            t1 = np.einsum('rs,ab,sbra->', g, uf, B[f, :, :, i, :, :]) * sf
                            t2 = np.einsum('rs,ab,sbra->', g, ub.conj().T, B[b, :, :, i, :, :]) * sb
                            t3 = np.einsum('rs,ab,sbra->', g, uf.conj().T, B[i, :, :, f, :, :]) * sf
                            t4 = np.einsum('rs,ab,sbra->', g, ub, B[i, :, :, b, :, :]) * sb
                            val = 0.25 * (t1 - t2 - t3 + t4)
                            out[gi, k, :, t] += ph[:, t, z, y, x] * val
    return out


def exact_loops(Dinv, dims, gammas, moms):
    """L(Gamma, t, q) from a dense inverse (index 12*site + 3*spin + colour)."""
    lx, ly, lz, lt = dims
    vol = lx * ly * lz * lt
    blocks = Dinv.reshape(vol, 4, 3, vol, 4, 3)
    diag = blocks[np.arange(vol), :, :, np.arange(vol), :, :]  # [V, 4, 3, 4, 3]
    diag_spin = np.einsum('vacbc->vab', diag)                   # colour trace
    G = gamma_list()[list(gammas)]
    tr = np.einsum('gba,vab->gv', G, diag_spin).reshape(len(gammas), lt, lz, ly, lx)
    ph = phases(dims, moms)
    return np.einsum('qtzyx,gtzyx->gqt', ph, tr)


def tsm_combine(corr, lp):
    """Eq. 2.4 from per-source loops.

    corr: [N_HP, ...] values L_j(s_HP) - L_j(s_LP) over the HP set
    lp:   [N_LP, ...] values L_j(s_LP) over the LP set
    Returns (estimate, sigma).
    """
    corr = np.asarray(corr)
    lp = np.asarray(lp)
    n_hp, n_lp = corr.shape[0], lp.shape[0]
    est = np.zeros(lp.shape[1:], dtype=np.complex128)
    var = np.zeros(lp.shape[1:], dtype=np.float64)
    if n_hp > 0:
        m = corr.mean(axis=0)
        est += m
        if n_hp > 1:
            var += (np.abs(corr - m) ** 2).sum(axis=0) / (n_hp - 1) / n_hp
    if n_lp > 0:
        m = lp.mean(axis=0)
        est += m
        if n_lp > 1:
            var += (np.abs(lp - m) ** 2).sum(axis=0) / (n_lp - 1) / n_lp
    return est, np.sqrt(var)


def tsm_loops(U, dims, kappa, mu, seed, noise_kind, n_hp, n_lp, hp_stop, lp_stop,
              gammas, moms, antiperiodic_t=True, estimator='standard', deriv_mus=()):
    """The whole TSM estimate, source by source, in the order of Eq. 2.4.

    hp_stop / lp_stop = (rel_tol, max_iter).  Source j uses eta_j from
    oracle.philox.noise(seed, j, ...).  estimator: 'standard' (eta^dag Gamma s,
    loops of D_u^-1), 'one_end' (Eq. 2.5, loops of D_u^-1 - D_d^-1) or
    'gen_one_end' (Eq. 2.6, loops of D_u^-1 + D_d^-1).
    deriv_mus (standard estimator only): directions of one-derivative blocks
    appended after the local block, per-source layout [1 + n_mu][n_gamma][n_q][T].
    Returns a dict with the estimate, its error, the LP-only mean over the LP
    set, the mean correction, the per-source loops and iteration counts.
    """
    if estimator == 'one_end':
        def value(eta, s):
            return one_end_loops(s, dims, kappa, mu, gammas, moms)
    elif estimator == 'gen_one_end':
        def value(eta, s):
            return gen_one_end_loops(U, s, dims, kappa, gammas, moms, antiperiodic_t)
    elif deriv_mus:
        def value(eta, s):
            loc = local_loops(eta, s, dims, gammas, moms)
            der = deriv_loops(U, eta, s, dims, gammas, deriv_mus, moms, antiperiodic_t)
            return np.concatenate([loc[None], np.transpose(der, (1, 0, 2, 3))])
    else:
        def value(eta, s):
            return local_loops(eta, s, dims, gammas, moms)
    corr, lp_vals, hp_iters, lp_iters = [], [], [], []
    for j in range(n_hp + n_lp):
        eta = philox.noise(seed, j, dims, noise_kind)
        s_lp, it_lp, _, _ = solver.solve_full(U, eta, dims, kappa, mu, lp_stop[0], lp_stop[1],
                                              antiperiodic_t)
        lp_iters.append(it_lp)
        l_lp = value(eta, s_lp)
        if j < n_hp:
            s_hp, it_hp, _, _ = solver.solve_full(U, eta, dims, kappa, mu, hp_stop[0], hp_stop[1],
                                                  antiperiodic_t)
            hp_iters.append(it_hp)
            corr.append(value(eta, s_hp) - l_lp)
        else:
            lp_vals.append(l_lp)
    shape = (len(gammas), len(moms), dims[3])
    if deriv_mus and estimator == 'standard':
        shape = (1 + len(deriv_mus),) + shape
    corr = np.array(corr).reshape((n_hp,) + shape)
    lp_vals = np.array(lp_vals).reshape((n_lp,) + shape)
    est, err = tsm_combine(corr, lp_vals)
    return {
        'loops': est, 'err': err,
        'lp_mean': lp_vals.mean(axis=0) if n_lp else np.zeros(shape, np.complex128),
        'corr_mean': corr.mean(axis=0) if n_hp else np.zeros(shape, np.complex128),
        'corr': corr, 'lp': lp_vals, 'hp_iters': hp_iters, 'lp_iters': lp_iters,
    }
