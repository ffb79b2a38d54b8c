/*
 * tsm.h -- C ABI of the GB300 truncated-solver-method (TSM) loop library.
 *
 * The library computes disconnected fermion loops with the truncated solver
 * method of Alexandrou et al., "Evaluation of disconnected contributions using
 * GPUs" (LATTICE 2012):
 *
 *   - Z4 / Z2 noise sources with the moments of Sec. 2.1, Eq. (2.1), generated
 *     on the fly from a counter-based generator (Sec. 3: no propagators stored);
 *   - inversions of the twisted-mass operator
 *         D_tm = 1 - kappa H + 2 i kappa mu gamma_5,
 *         (H psi)(x) = sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *                             + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)]
 *     (the twisted-mass regularisation of Sec. 2.2), by CG on the normal
 *     equations of the even/odd Schur complement, truncated (LP) or run to high
 *     precision (HP) (Sec. 2.2);
 *   - loops L_j(Gamma, t, q) = sum_{x: x_4 = t} e^{i q.x} eta_j(x)^dag Gamma s_j(x)
 *     (Sec. 2.3, first estimator; all insertion times at once, Sec. 4);
 *   - the TSM estimate of Sec. 2.2, Eq. (2.4): LP mean over the LP set plus the
 *     HP - LP correction over the HP set.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: L = {Lx, Ly, Lz, T}, every extent even and >= 2.  Site index
 *   i = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) mod 2, even = 0.
 * Gamma basis: Euclidean chiral, gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *   gamma_4 = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1).
 * Insertion list: 0: 1, 1-4: gamma_1..gamma_4, 5: gamma_5, 6-9: gamma_mu gamma_5,
 *   10-15: sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] for
 *   (mu nu) = 12, 13, 14, 23, 24, 34.
 * Canonical host formats (complex = two doubles, re then im):
 *   gauge  U[T][Z][Y][X][mu][a][b]    mu = 0:x, 1:y, 2:z, 3:t; every link SU(3)
 *   spinor psi[T][Z][Y][X][spin][colour]   (24 doubles per site)
 *   loops  L[n_gamma][n_q][T] complex
 * Momenta: integer triples n, q = 2 pi (n_x / Lx, n_y / Ly, n_z / Lz).
 * Noise: source j, seed s -> Philox4x32-10 (Salmon et al., SC'11), key
 *   (s mod 2^32, s >> 32), counter (i, j, 0, 0); word 0 bit 2a (2a+1) set makes
 *   the real (imaginary) part of component a = 3*spin + colour negative.
 *   Z4 entries (+-1 +- i)/sqrt 2, Z2 entries +-1 (bit 2a).  The noise of
 *   source j does not depend on batching or on how sources are split.
 * Memory: the caller owns every pointer it passes.  With on_device = 0 the
 *   pointers are host memory and the library copies in and out; with
 *   on_device = 1 they are device pointers on the context's device.  The
 *   context owns its own device workspace (allocated on first use, freed by
 *   tsm_destroy).
 * Streams: every call is ordered on the stream given to tsm_create and has
 *   completed when the call returns.
 * Errors: every call returns a tsm_status; none throws across the ABI.
 *   tsm_last_error() gives a one-line message for the last failure on the
 *   calling thread.
 */
#ifndef TSM_H
#define TSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsm_ctx tsm_ctx;

typedef enum {
  TSM_OK = 0,
  TSM_ERR_ARG = -1,            /* null pointer, bad enum, bad count */
  TSM_ERR_DIMS = -2,           /* an extent odd or < 2, or lattice too large */
  TSM_ERR_CUDA = -3,           /* a CUDA runtime call failed */
  TSM_ERR_NOT_CONVERGED = -4,  /* a solve hit max_iter above its tolerance (outputs still written) */
  TSM_ERR_NONFINITE = -5,      /* NaN/Inf met in a reduction */
  TSM_ERR_TIMEOUT = -6,        /* a bounded device wait ran out */
  TSM_ERR_NOT_UNITARY = -7,    /* gauge links not SU(3) to 1e-8 (2-row storage needs SU(3)) */
  TSM_ERR_NO_GAUGE = -8,       /* no gauge field loaded */
  TSM_ERR_TOO_LARGE = -9       /* request above a fixed internal capacity */
} tsm_status;

/* Storage / arithmetic tier.
 *   TSM_F64  FP64 storage and arithmetic (the plain FP64 path).
 *   TSM_F32  FP32 storage and arithmetic; in solves optionally with FP64
 *            reliable updates (tm_stop.reliable).
 *   TSM_BF16, TSM_F16  16-bit storage of links and Krylov/operator vectors,
 *            FP32 arithmetic.  TSM_F16 keeps the CG residual and iterate in
 *            FP16 as well (relative precision 2^-11, below the truncation of
 *            an LP solve); TSM_BF16 keeps them in FP32.  Sources and solutions
 *            are exchanged in FP32 for both through tm_solve_batch; inside
 *            tsm_loops / tsm_loops_graph the TSM_F16 tier also keeps its noise
 *            source, Schur source and solution in FP16 (the solution is FP16
 *            already as the CG iterate; the source's rounding is part of the LP
 *            map, which both source sets share). */
typedef enum { TSM_F64 = 0, TSM_F32 = 1, TSM_BF16 = 2, TSM_F16 = 3 } tsm_prec;

typedef struct {
  int L[4];            /* Lx, Ly, Lz, T */
  double kappa;        /* hopping parameter */
  double mu;           /* twisted mass (sign selects the flavour: +mu = u) */
  int t_antiperiodic;  /* 1: fermion field antiperiodic in t (hops across t = T-1 <-> 0 get -1) */
} tm_lattice;

/* Stopping rule of one solve (Sec. 2.2 truncates a solve either at a loose
 * residual or at a fixed iteration count; both are offered).  The solve is CG
 * on Dhat^dag Dhat x = Dhat^dag bhat with zero start; it stops after the first
 * iteration k with ||r_k|| / ||Dhat^dag bhat|| < rel_tol (not squared), or
 * after max_iter iterations.  rel_tol = 0 gives a fixed iteration count.
 *
 * precond = 1 replaces CG by flexible GMRES on Dhat x = bhat with the
 * learned network attached to the context (tsm_set_precond) as right
 * preconditioner (the paper has no such solver: this is the project's
 * learned LP path).  Its rule is ||bhat - Dhat x|| / ||bhat|| < rel_tol (the
 * residual of the Schur system itself, a different norm from CG's) or
 * max_iter inner steps (each = one network application and one Dhat), with
 * restarts every `restart` steps (0 -> 16, at most 64).  Its vectors are
 * FP32 (tiers TSM_F32 without reliable updates, TSM_BF16, TSM_F16 only); a
 * breakdown hands the source to plain CG of the same tier.  Eager only: not
 * under tsm_loops_graph. */
typedef struct {
  double rel_tol;
  int max_iter;
  int prec;            /* tsm_prec */
  int reliable;        /* TSM_F32 only: FP64 solution and FP64 residual recomputation
                          whenever ||r|| fell by reliable_delta since the last one */
  double reliable_delta; /* 0 -> 0.1 */
  int precond;         /* 0: CG (default); 1: flexible GMRES with the learned preconditioner */
  int restart;         /* flexible GMRES cycle length (0 -> 16) */
} tm_stop;

/* Per-call statistics of tsm_loops. */
typedef struct {
  int n_sources;            /* HP + LP sources processed */
  long long lp_iters;       /* summed CG iterations of LP solves (HP set + LP set) */
  long long hp_iters;       /* summed CG iterations of HP solves */
  int hp_not_converged;     /* HP solves that hit max_iter */
  double hp_max_true_res;   /* max over HP solves of ||eta - D s|| / ||eta|| */
  double lp_max_true_res;   /* max over LP solves of the same */
} tsm_loop_stats;

/* Operators of tm_dslash. */
enum {
  TM_OP_FULL = 0,      /* out = D_tm in  (dagger: D_tm^dag in); full lattice */
  TM_OP_HOP_EO = 1,    /* out_e = H_eo in_o, out_o = 0  (dagger: (H^dag)_eo) */
  TM_OP_HOP_OE = 2,    /* out_o = H_oe in_e, out_e = 0  (dagger: (H^dag)_oe) */
  TM_OP_SCHUR = 3,     /* out_e = Dhat in_e, out_o = 0  (dagger: Dhat^dag);
                          Dhat = 1 - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe,
                          A = 1 + 2 i kappa mu gamma_5 */
  TM_OP_NORMAL = 4     /* out_e = Dhat^dag Dhat in_e, out_o = 0 */
};

/* Create a context on CUDA device `device`, ordering all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the handle. */
int tsm_create(int device, void* cuda_stream, tsm_ctx** out);

/* Free the context and all device memory it owns.  NULL is accepted. */
int tsm_destroy(tsm_ctx* ctx);

/* Load the gauge field: canonical FP64 links (host or device), converted to the
 * library's even/odd storage: FP64 all three rows, FP32, FP16 and BF16 rows 0
 * and 1 (12 reals; row 2 = conj(row0 x row1) is rebuilt in the stencil).
 * Checks every link for SU(3) (unitary rows, row 3 = conj(row1 x row2)) to
 * 1e-8 and returns TSM_ERR_NOT_UNITARY otherwise; extents must be even >= 2.
 * The boundary sign is applied inside the operator, never folded into links. */
int tsm_load_gauge(tsm_ctx* ctx, const tm_lattice* lat, const double* U, int on_device);

/* Apply an operator (TM_OP_*) to one canonical spinor, with links and vectors
 * stored in tier `prec` (input rounded to that tier on entry, output written
 * in FP64).  Sites the operator does not produce are written as zero. */
int tm_dslash(tsm_ctx* ctx, int prec, int op, int dagger,
              const double* in, double* out, int on_device);

/* Solve D_tm s_r = b_r for nrhs canonical right-hand sides (b and s each
 * nrhs * 24 * V doubles, source r at offset r * 24 * V) by even/odd reduction,
 * CG on the Schur complement normal equations (tier stop->prec) and odd-site
 * reconstruction.  iters[r] (may be NULL) receives the CG iteration count and
 * true_res[r] (may be NULL) ||b_r - D_tm s_r|| / ||b_r|| computed in FP64.
 * Returns TSM_ERR_NOT_CONVERGED if any solve hit max_iter above rel_tol (the
 * solutions are still written). */
int tm_solve_batch(tsm_ctx* ctx, int nrhs, const double* b, double* s,
                   const tm_stop* stop, int on_device, int* iters, double* true_res);

/* Write the canonical noise source eta_j (24 * V doubles) for seed, kind
 * (4 = Z4, 2 = Z2) and source index j, exactly as the solvers see it. */
int tsm_noise(tsm_ctx* ctx, uint64_t seed, int kind, uint32_t source,
              double* out, int on_device);

/* Contract one canonical solution with its regenerated noise source:
 * out[g][q][t] = sum_{x: x_4 = t} e^{i q.x} eta_j(x)^dag Gamma_g (s_a - s_b)(x),
 * s_b may be NULL (treated as zero).  gammas: n_gamma indices in [0, 16);
 * moms: n_q integer triples.  prec TSM_F64 contracts in FP64, TSM_F32 in FP32
 * per site with FP64 sums over blocks and sites. */
int tsm_contract(tsm_ctx* ctx, int prec, uint64_t seed, int kind, uint32_t source,
                 const double* s_a, const double* s_b,
                 const int* gammas, int n_gamma, const int* moms, int n_q,
                 double* out, int on_device);

/* One-end-trick value (Sec. 2.3, Eq. 2.5) of one canonical solution
 * s = D_u^-1 eta of the loaded (+mu) operator, for the isovector loop u - d:
 *   out[g][q][t] = -4 i kappa mu sum_{x: x_4 = t} e^{i q.x}
 *                  [s_a^dag gamma5 Gamma_g s_a - s_b^dag gamma5 Gamma_g s_b](x)
 * (s_b may be NULL), from D_u^-1 - D_d^-1 = -4 i kappa mu D_u^-1 D_u^-dag gamma5
 * for D_tm = 1 - kappa H + 2 i kappa mu gamma5 (the paper states it for
 * M = D / (2 kappa)).  Its noise average is Tr[P Gamma (D_u^-1 - D_d^-1)].
 * Layouts, tiers and errors as tsm_contract. */
int tsm_contract_one_end(tsm_ctx* ctx, int prec, const double* s_a, const double* s_b,
                         const int* gammas, int n_gamma, const int* moms, int n_q,
                         double* out, int on_device);

/* Generalised one-end-trick value (Sec. 2.3, Eq. 2.6) of one canonical
 * solution s = D_u^-1 eta, for the isoscalar loop u + d:
 *   out[g][q][t] = 2 sum_{x: x_4 = t} e^{i q.x}
 *                  [s_a^dag gamma5 Gamma_g gamma5 (D_W s_a) - (same for s_b)](x)
 * with the Wilson operator D_W = 1 - kappa H (applied by the library), from
 * D_u + D_d = 2 D_W and D_u D_u^dag = gamma5 D_u^dag D_u gamma5.  Its noise
 * average is Tr[P Gamma (D_u^-1 + D_d^-1)].  Layouts, tiers, errors as
 * tsm_contract. */
int tsm_contract_gen_one_end(tsm_ctx* ctx, int prec, const double* s_a, const double* s_b,
                             const int* gammas, int n_gamma, const int* moms, int n_q,
                             double* out, int on_device);

/* Local loops of one canonical solution at every spatial momentum (the paper
 * Fourier-transforms the loops, Sec. 3):
 *   out[g][t][n_z][n_y][n_x] = sum_{x: x_4 = t} e^{+2 pi i (n_x x/Lx + n_y y/Ly + n_z z/Lz)}
 *                              eta_j(x)^dag Gamma_g (s_a - s_b)(x),  n_i in [0, L_i)
 * (momentum -n is index L - n).  Per-site densities and the transform in FP64
 * or FP32 (prec): the library's own mixed-radix FFT, the x and y axes of each
 * (t, z) plane in one shared-memory pass and the z axis in a second.  Even
 * extents whose prime factors are at most 13; TSM_ERR_TOO_LARGE otherwise or
 * if an Lx x Ly plane of the tier's complex type does not fit in 200 KB of
 * shared memory (FP64: Lx * Ly <= 12800).  Host or device pointers per
 * on_device; errors as tsm_contract. */
int tsm_contract_fft(tsm_ctx* ctx, int prec, uint64_t seed, int kind, uint32_t source,
                     const double* s_a, const double* s_b, const int* gammas, int n_gamma,
                     double* out, int on_device);

/* One-derivative insertions of one canonical solution with its regenerated
 * noise source (the paper's TSM tuning operator i psibar gamma_3 D_3 psi,
 * Sec. 3; D is not defined there -- reading: the symmetric covariant
 * derivative D<->_mu = (D->_mu - D<-_mu) / 2, operator and phase at x):
 *   out[k][g][q][t] = 1/4 sum_{x: x_4 = t} e^{i q.x} [eta(x)^dag Gamma_g (T+ s - T- s)(x)
 *                                                   - ((T+ eta - T- eta)(x))^dag Gamma_g s(x)]
 * for the k-th set bit mu of deriv_mask (1..15), T+ f(x) = U_mu(x) f(x+mu),
 * T- f(x) = U_mu(x-mu)^dag f(x-mu), the fermion sign on hops across
 * t = T-1 <-> 0, s = s_a - s_b (s_b may be NULL).  Tiers and errors as
 * tsm_contract. */
int tsm_contract_deriv(tsm_ctx* ctx, int prec, uint64_t seed, int kind, uint32_t source,
                       const double* s_a, const double* s_b, const int* gammas, int n_gamma,
                       int deriv_mask, const int* moms, int n_q, double* out, int on_device);

/* TSM parameters (Sec. 2.2, Eq. 2.4).  Sources hp_begin .. hp_end-1 form this
 * call's part of the HP set and lp_begin .. lp_end-1 its part of the LP set;
 * a single process passes hp = [0, N_HP) and lp = [N_HP, N_HP + N_LP). */
typedef struct {
  uint64_t seed;
  int noise;                /* 4 = Z4, 2 = Z2 */
  uint32_t hp_begin, hp_end;
  uint32_t lp_begin, lp_end;
  tm_stop hp;               /* stopping rule / tier of the HP solves */
  tm_stop lp;               /* stopping rule / tier of the LP solves (same map for both sets) */
  int batch;                /* sources solved together (>= 1; 1 = single-RHS kernels) */
  const int* gammas; int n_gamma;
  const int* moms; int n_q; /* host pointers */
  int verify;               /* 1: recompute every HP solution's true residual in FP64
                               (tsm_loop_stats.hp_max_true_res; 2 extra FP64 hops per HP source) */
  int estimator;            /* 0: eta^dag Gamma s, loops of D_u^-1 (Sec. 2.3 first estimator);
                               1: one-end trick, loops of D_u^-1 - D_d^-1 (Eq. 2.5, see
                               tsm_contract_one_end);
                               2: generalised one-end trick, loops of D_u^-1 + D_d^-1
                               (Eq. 2.6, see tsm_contract_gen_one_end; one Wilson
                               application per solution; not in tsm_loops_graph).
                               For 1 and 2 the TSM correction is f(s_HP) - f(s_LP) of
                               the quadratic per-source value */
  int deriv_mask;           /* estimator 0 only: bit mu (0..3) adds the one-derivative
                               insertion block along mu (see tsm_contract_deriv) after
                               the local block in every output and per-source array */
  int all_momenta;          /* 1 (estimator 0, no derivatives, eager only): every spatial
                               momentum through the library's 3-D FFT per source (see
                               tsm_contract_fft; same size limit); moms / n_q are ignored,
                               outputs are
                               [n_gamma][T][Lz][Ly][Lx], per_corr / per_lp must be NULL
                               (means and variances are accumulated in source order) */
  int hp_warm_start;        /* 1: each HP solve of tier FP32 with FP64 reliable updates starts
                               from its source's LP solution (the LP map is unchanged, so the
                               estimate stays unbiased; the HP solution still meets hp.rel_tol);
                               ignored for the other HP tiers.  0: zero start */
} tsm_params;

/* Run the TSM over this call's source ranges.  Outputs (host or device per
 * on_device; any may be NULL):
 *   loops     [n_gamma][n_q][T] complex   the estimate of Eq. 2.4
 *   err       [n_gamma][n_q][T] double    sigma = sqrt(Var_corr / N_HP + Var_LP / N_LP)
 *   lp_mean   [n_gamma][n_q][T] complex   LP-only mean over the LP set (biased)
 *   corr_mean [n_gamma][n_q][T] complex   mean HP - LP correction over the HP set
 *   per_corr  [hp_end-hp_begin][n_gamma][n_q][T] complex  per-source L(s_HP - s_LP)
 *   per_lp    [lp_end-lp_begin][n_gamma][n_q][T] complex  per-source L(s_LP)
 * With deriv_mask set, every [n_gamma][n_q][T] shape above becomes
 * [1 + popcount(deriv_mask)][n_gamma][n_q][T] (local block first).
 * stats (host, may be NULL) receives iteration counts and residuals.
 * Var is the unbiased complex sample variance sum |X_j - mean|^2 / (N - 1),
 * evaluated in two passes in source order (bit-reproducible). */
int tsm_loops(tsm_ctx* ctx, const tsm_params* p,
              double* loops, double* err, double* lp_mean, double* corr_mean,
              double* per_corr, double* per_lp, int on_device, tsm_loop_stats* stats);

/* Run the TSM of n contexts -- typically lattices of different volumes, all
 * on one device -- as ONE captured CUDA graph.  Every batched CG solve becomes
 * a graph while-loop whose condition a device kernel clears once each of its
 * sources has met its stopping rule (no host round trip inside the graph);
 * converged sources are skipped by the remaining iterations; the contexts'
 * work forms parallel branches of the graph.  params[i] applies to ctxs[i]
 * (verify is ignored).  Outputs are DEVICE pointers (arrays of n; the array
 * itself or any entry may be NULL): loops[i], err[i], per_corr[i], per_lp[i]
 * as in tsm_loops; stats (host, n entries, may be NULL) receives iteration
 * counts.  The graph runs on ctxs[0]'s stream and has completed on return.
 * Results are bit-identical to tsm_loops with the same parameters. */
int tsm_loops_graph(tsm_ctx** ctxs, const tsm_params* params, int n, double** loops, double** err,
                    double** per_corr, double** per_lp, tsm_loop_stats* stats);

/* Autotuner of the multi-RHS batch width: for the loaded lattice and the
 * stopping rule / tier `stop`, times one batched solve of noise sources (a
 * scratch seed; nothing else is changed) for every width in {8, 16, 32, 64}
 * and writes the width with the lowest time per source to *best.  Results
 * are cached per context, lattice and tier.  times_ms (may be NULL) receives
 * the 4 measured times per source in milliseconds. */
int tsm_tune_batch(tsm_ctx* ctx, const tm_stop* stop, int* best, double* times_ms);

/* Autotuner of the whole multi-RHS launch shape: the batch width as above
 * and, for the 16-bit tiers and FP32, the block shape of their link-sharing
 * stencil (blocks of 32 sites x 2, 4 or 8 sources, one warp per source; the
 * block's links are widened once and shared; FP32 uses it for its hops
 * without a reduction), the 4-source blocks compiled for either 80 or 96
 * registers per thread (768 or 640 resident threads per SM).  Times one
 * batched solve of scratch noise sources per (width, block shape) pair and
 * keeps the pair with the lowest time per source: *best_batch, *best_tile
 * (may be NULL; 1 for tiers without that stencil), *best_regs (may be NULL;
 * 0 for tiers without it).  The block shape is then used by every later solve
 * of that tier on this context; the results do not depend on it (per-site
 * arithmetic and reduction order are independent of the block shape).  Cached
 * per context, lattice and stopping rule.  times_ms (may be NULL): 16 entries,
 * [width k][shape q] = ms per source for widths {8, 16, 32, 64} and shapes
 * {2 sources / 80 registers, 4 / 80, 8 / 80, 4 / 96} (0 where a shape does not
 * apply).  tsm_tune_batch runs the same search and reports, per width, the best
 * time over the shapes. */
int tsm_tune(tsm_ctx* ctx, const tm_stop* stop, int* best_batch, int* best_tile, int* best_regs, double* times_ms);

/* Set the block shape of the link-sharing stencil of tier prec (TSM_F16,
 * TSM_BF16 or TSM_F32) for this context's later solves, as tsm_tune does:
 * tile_sources 2, 4 or 8 sources per block, max_regs 80 (or 96 with 4
 * sources); 4 and 80 by default.  TSM_ERR_ARG for other tiers or values. */
int tsm_set_tile(tsm_ctx* ctx, int prec, int tile_sources, int max_regs);


/* Tensor-core GEMM of the learned preconditioner's channel mixing (the dense
 * contraction of the parallel-transport layers; the paper has no network --
 * this is the project's learned LP preconditioner):
 *   C[M][N] (FP32) = A[M][K] (BF16) * B[N][K]^T (BF16)  (+ C when beta = 1),
 * all row-major DEVICE pointers, K % 8 == 0, computed with tcgen05.mma
 * (accumulator in tensor memory), ordered on cuda_stream and completed on
 * return.  TSM_ERR_TIMEOUT if a bounded tensor-core wait ran out. */
int tsm_umma_gemm(const void* A, const void* B, float* C, int M, int N, int K, int beta, void* cuda_stream);

/* The same GEMM with leading dimensions (elements; lda, ldb >= K and
 * multiples of 8, ldc >= N) and split-K: with splits > 1 the K range is cut
 * into at most `splits` chunks of a multiple of 64 columns and chunk z writes
 * its partial product to C + z * M * ldc (the caller sums the partials);
 * *used_splits (may be NULL) receives the number of partials written.
 * TSM_ERR_ARG for bad sizes, TSM_ERR_TIMEOUT as above. */
int tsm_umma_gemm_ex(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M, int N, int K,
                     int beta, int splits, int* used_splits, void* cuda_stream);

/* Fault injection for tests of the bounded tensor-core waits (the paper has
 * no counterpart).  withhold = 1: the following TMA-fed tensor-core GEMM
 * launches of this process (tsm_umma_gemm*, the network's layers) issue no
 * operand copies and give their stage waits a limit of 4096 polls instead of
 * 2^26, so the MMA thread's first wait -- on a stage nothing fills -- runs
 * out; nothing is in flight, every CTA frees its tensor memory and returns,
 * and the call reports TSM_ERR_TIMEOUT with the context still usable.
 * Launches whose operands the TMA cannot address (base not 16-byte aligned)
 * run normally.  withhold = 0 restores normal operation.  Returns TSM_OK. */
int tsm_umma_inject_timeout(int withhold);

/* ---- learned LP preconditioner (the paper has no network; this is the
 * project's extension of the LP solves of Sec. 2.2: because the HP - LP
 * correction of Eq. 2.4 removes any LP bias, it may change the variance per
 * unit cost only, never the expectation, provided HP-set and LP-set sources
 * see the same LP solver, which tsm_loops guarantees).
 *
 * Network: n_layers parallel-transport layers, C_0 = C_L = 1 channel (a
 * spinor field), C_l complex channels in between.  Layer l maps psi (C_in
 * channels) to
 *   y_{c'}(x)_{s'a} = sum_{p=0..8} sum_{c,s} W[c'*4+s'][(p*C_in+c)*4+s] (T_p psi_c)(x)_{sa}
 * with T_0 = 1, T_{2mu+1} psi(x) = U_mu(x) psi(x+mu), T_{2mu+2} psi(x) =
 * U_mu(x-mu)^dag psi(x-mu) (time-boundary sign as in D_tm): gauge covariant,
 * linear, no activation.  W is complex [4 C_out][36 C_in] (host: interleaved
 * re, im doubles).  The transports run in FP32 (FP32 links of the context),
 * the channel mixing as BF16 x BF16 -> FP32 tensor-core GEMMs.  Gradients use
 * G = dL/dRe + i dL/dIm of a real loss L. */
typedef struct tsm_net tsm_net;

/* Create a network on `device` with channels[0 .. n_layers] (first and last
 * 1, others in [1, 64]); weights start near the identity map (channel c'
 * copies channel c' mod C_in on path 0, the last layer averages) plus complex
 * Gaussian noise of standard deviation init_scale / sqrt(36 C_in) from a
 * seeded splitmix64 stream. */
int tsm_net_create(int device, int n_layers, const int* channels, uint64_t seed, double init_scale,
                   tsm_net** out);
int tsm_net_destroy(tsm_net* net);
/* Host copies of one layer's complex weights [4 C_out][36 C_in]. */
int tsm_net_set_weights(tsm_net* net, int layer, const double* W);
int tsm_net_get_weights(tsm_net* net, int layer, double* W);
/* y = net(x) for nb samples on ctx's gauge field; x [nb][C_0][V][4][3],
 * y [nb][C_L][V][4][3] complex (canonical site order), host or device. */
int tsm_net_forward(tsm_net* net, tsm_ctx* ctx, int nb, const double* x, double* y, int on_device);
/* Given the output gradient gy (layout of y), the input gradient gx (layout
 * of x; may be NULL) and the weight gradients gw (all layers' [4 C_out][36 C_in]
 * complex arrays one after another; may be NULL).  Host pointers. */
int tsm_net_gradient(tsm_net* net, tsm_ctx* ctx, int nb, const double* x, const double* gy, double* gx,
                     double* gw);
/* Make n training pairs (r, Dhat^-1 r) on ctx's gauge field: r = Z4 noise of
 * `seed` (sources 0 .. n-1) on the even sites, Dhat^-1 r by batched FP32 CG
 * (stop: TSM_F32, no reliable updates).  *group receives the pair group id.
 * The pairs stay in device memory (2 x 96 V bytes each) until the network is
 * destroyed; the context must outlive the network's use of them. */
int tsm_net_add_pairs(tsm_net* net, tsm_ctx* ctx, int n, uint64_t seed, const tm_stop* stop, int* group);
/* Make training pairs from the method's own solves: for the Z4 noise sources
 * eta_j of `seed` (j = 0 .. n_sources-1, as tsm_loops draws them) the converged
 * solution x* of Dhat x = bhat_j (stop: TSM_F32, no reliable updates) and the
 * CGNR iterates x_k after k = iters[q] >= 0 iterations from zero (the first
 * k iterations of the same solve; k = 0: x_0 = 0, the pair (Dhat x*, x*)
 * of the source itself) give n_sources * n_iters pairs
 *   t = x* - x_k,   r = Dhat t   (= bhat - Dhat x_k up to x*'s tolerance):
 * the Krylov residuals of those solves with their exact targets Dhat^-1 r.
 * Pairs are stored batch by batch (batches of up to 64 consecutive
 * sources): in the batch of m sources starting at j0, the pair of source j
 * and iteration count iters[q] has index j0 * n_iters + q * m + (j - j0).
 * TSM_ERR_ARG if an iterate equals x* (k too large).  The pairs stay in
 * device memory until the network is destroyed. */
int tsm_net_add_solve_pairs(tsm_net* net, tsm_ctx* ctx, int n_sources, uint64_t seed, const int* iters, int n_iters,
                            const tm_stop* stop, int* group);
/* Host copies of pair `index` of `group`: r and t as canonical spinors
 * (24 V doubles each; odd sites zero). */
int tsm_net_get_pair(tsm_net* net, int group, int index, double* r, double* t);
/* Adam (lr; betas 0.9, 0.999) on the mean over a minibatch of the relative
 * loss |net(r) - t|^2 / |t|^2 over even sites; step k uses groups[k mod
 * n_groups] and `batch` consecutive pairs of it.  loss (may be NULL) receives
 * the minibatch mean loss of every step. */
int tsm_net_train(tsm_net* net, const int* groups, int n_groups, int steps, int batch, double lr, double* loss);
/* Mean relative loss over all pairs of a group, without training. */
int tsm_net_loss(tsm_net* net, int group, double* loss);
/* Attach (net) or detach (NULL) the preconditioner used by solves with
 * tm_stop.precond = 1 on this context.  Not owned by the context. */
int tsm_set_precond(tsm_ctx* ctx, tsm_net* net);

/* Combine per-source loops gathered from several processes into the estimate
 * of Eq. 2.4.  Runs the same device kernel, in the same summation order, as
 * the final step of tsm_loops, so any split of the source ranges gives
 * bit-identical results.  per_corr: n_hp x n_entries complex, per_lp:
 * n_lp x n_entries complex (host or device per on_device); outputs as in
 * tsm_loops, each n_entries long, any may be NULL. */
int tsm_combine(tsm_ctx* ctx, const double* per_corr, int n_hp, const double* per_lp, int n_lp,
                int n_entries, double* loops, double* err, double* lp_mean, double* corr_mean,
                int on_device);

/* Instrumentation.  tsm_profile(ctx, 1) starts recording CUDA-event times of
 * hop-kernel launches on the context's stream (in CG solves: the hop kernels
 * of the first iteration of every chunk of 8 iterations); tsm_profile_read
 * returns, per bucket b = 4 * tier + kind (tier: tsm_prec; kind 0 plain hop
 * K1, 1 hop + xpay/norm K2, 2 adjoint hop K3, 3 adjoint hop + CG update K4),
 * the summed milliseconds, launch count and algorithmic bytes (links once per
 * launch, spinor streams once per right-hand side).  Arrays hold 16 entries.
 * tsm_launch_count returns the number of library kernels launched so far. */
int tsm_profile(tsm_ctx* ctx, int enable);
int tsm_profile_read(tsm_ctx* ctx, double ms[16], long long count[16], double bytes[16]);
/* All buckets: the 16 hop buckets above, then 16 local contraction passes
 * (kernel + fixed-order reduction, any estimator; bytes = fields read + block
 * partials + output), 17 derivative-insertion passes (+ the direction's two
 * links per site), 18 all-momenta FFT projections (fields, densities, one
 * read and one write pass of the transform, running moments), 19 Wilson
 * applications of the generalised one-end estimator (both parities).  These
 * are timed on every launch while instrumentation is on.  n: length of the
 * caller's arrays (entries past the library's buckets read 0; any may be NULL). */
int tsm_profile_read_ex(tsm_ctx* ctx, int n, double* ms, long long* count, double* bytes);
long long tsm_launch_count(tsm_ctx* ctx);

/* Measured arithmetic peak of CUDA device `device` (instrumentation: the
 * denominator of the FP32 and FP64 arithmetic rooflines).  A register-resident
 * kernel runs 8 independent FMA chains per thread on every resident thread of
 * every SM; *tflops receives 2 flop per FMA over the best of three timed
 * launches (after a warm-up).  prec: TSM_F32 or TSM_F64.  Allocates a small
 * device buffer and its own stream; the calling thread's current device is
 * restored on return. */
int tsm_measure_fma_peak(int device, int prec, double* tflops);

/* Contraction for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc where they need a contraction -- code running under
 * a memory manager that owns the whole device, paths where cudaMalloc's
 * implicit synchronisation and latency are not acceptable, or callers that
 * hold no tsm_ctx.  It computes the same loops as tsm_contract with TSM_F64
 * and s_b = NULL, allocates nothing, and needs no context:
 *   s_dev    device pointer, canonical spinor (24 * V doubles) of one source
 *   out_dev  device pointer, [n_gamma][n_q][T] complex (written)
 *   gammas, moms  host arrays as for tsm_contract; 1 <= n_gamma <= 16,
 *            1 <= n_q <= 16, Lx + Ly + Lz <= 3072
 *   cuda_stream   cudaStream_t the work is ordered on (NULL = legacy stream);
 *            the call returns once the work is queued, and runs on the
 *            current CUDA device.
 * Scratch: a fixed 1 MiB device array compiled into the library (one per
 * device, held until the library is unloaded) stores the phase tables and the
 * block partial sums; requests that need more return TSM_ERR_TOO_LARGE.  Each
 * call looks up that array's device address on the current device
 * (cudaGetSymbolAddress, no allocation; TSM_ERR_CUDA if it fails); the first
 * call on a device also loads the library's device code there -- make that
 * first call before any stream capture.  Every call shares the array: calls
 * whose work overlaps on the GPU race and must be serialised by the caller.
 * Nothing in the array needs clearing: each call writes every entry it reads. */
int tsm_contract_noalloc(const tm_lattice* lat, uint64_t seed, int kind, uint32_t source,
                         const double* s_dev, const int* gammas, int n_gamma, const int* moms, int n_q,
                         double* out_dev, void* cuda_stream);

/* One-line message for the last failed call on this thread ("" if none). */
const char* tsm_last_error(void);
/* Name of a status code. */
const char* tsm_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* TSM_H */
