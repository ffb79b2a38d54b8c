"""One captured CUDA graph over three lattices (tsm_loops_graph).

Each lattice has its own context; every batched CG solve runs as a graph
while-loop (device-side stopping rule, converged sources skipped) and the
three lattices are parallel branches of one graph.  The results must be
bit-identical to the eager tsm_loops of each context with the same
parameters (same kernels, same per-source arithmetic and reduction order).
"""
import numpy as np
import pytest

from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

KAPPA, MU = 0.1245, 0.005
LATTICES = [(4, 4, 4, 4), (6, 4, 4, 6), (8, 4, 4, 8)]
GAM = list(range(16))
MOMS = S.default_momenta(7)


@pytest.mark.parametrize("tier", ["mixed", "fp64"])
def test_graph_over_three_lattices_bit_identical(libtsm, tier):
    import torch
    if tier == "mixed":
        hp = tsm.stop(1e-10, 3000, tsm.TSM_F32, reliable=True, reliable_delta=1e-3)
        lp = tsm.stop(5e-3, 60, tsm.TSM_F16)
    else:
        hp = tsm.stop(1e-12, 3000, tsm.TSM_F64)
        lp = tsm.stop(1e-2, 60, tsm.TSM_F64)
    n_hp, n_lp, batch = 4, 21, 8
    ctxs = [tsm.Context(0) for _ in LATTICES]
    try:
        eager, plist, outs = [], [], []
        for k, (ctx, dims) in enumerate(zip(ctxs, LATTICES)):
            ctx.load_gauge(S.gauge_field(dims, 0.25, 40 + k), dims, KAPPA, MU)
            eager.append(ctx.loops(500 + k, 4, n_hp, n_lp, hp, lp, GAM, MOMS, per_source=True, batch=batch,
                                   verify=False))
            plist.append(tsm.params(500 + k, 4, (0, n_hp), (n_hp, n_hp + n_lp), hp, lp, GAM, MOMS,
                                    batch=batch))
            shape = (len(GAM), len(MOMS), dims[3])
            outs.append({
                "loops": torch.zeros(shape, dtype=torch.complex128, device="cuda"),
                "err": torch.zeros(shape, dtype=torch.float64, device="cuda"),
                "per_corr": torch.zeros((n_hp,) + shape, dtype=torch.complex128, device="cuda"),
                "per_lp": torch.zeros((n_lp,) + shape, dtype=torch.complex128, device="cuda"),
            })
        stats = tsm.tsm_loops_graph([c.h for c in ctxs], plist,
                                    loops=[o["loops"] for o in outs], err=[o["err"] for o in outs],
                                    per_corr=[o["per_corr"] for o in outs], per_lp=[o["per_lp"] for o in outs])
        torch.cuda.synchronize()
        for k in range(len(LATTICES)):
            for key in ("loops", "err", "per_corr", "per_lp"):
                got = outs[k][key].cpu().numpy()
                assert np.array_equal(got, eager[k][key]), (k, key)
            assert stats[k].lp_iters == eager[k]["stats"]["lp_iters"]
            assert stats[k].hp_iters == eager[k]["stats"]["hp_iters"]
            assert stats[k].hp_not_converged == 0
        # the graph can be built and run again (fresh seeds) on the same contexts
        plist2 = [tsm.params(900 + k, 4, (0, n_hp), (n_hp, n_hp + n_lp), hp, lp, GAM, MOMS, batch=batch)
                  for k in range(len(LATTICES))]
        tsm.tsm_loops_graph([c.h for c in ctxs], plist2, loops=[o["loops"] for o in outs])
        torch.cuda.synchronize()
        ref = ctxs[1].loops(901, 4, n_hp, n_lp, hp, lp, GAM, MOMS, batch=batch, verify=False)
        assert np.array_equal(outs[1]["loops"].cpu().numpy(), ref["loops"])
    finally:
        for c in ctxs:
            c.close()


def test_autotuner_and_config_sizes_graph_matches_eager(libtsm):
    """The three lattices of the batching workload (8^3x16, 12^3x24, 16^3x32,
    links eps = 0.25, kappa = 0.1245, mu = 0.005, BF16 LP at 1e-2, FP32+FP64
    HP at 1e-10) with autotuned batch widths: one graph equals the eager runs
    bit for bit (fewer sources than the benchmark to keep the test short)."""
    import torch
    lattices = [(8, 8, 8, 16), (12, 12, 12, 24), (16, 16, 16, 32)]
    hp = tsm.stop(1e-10, 3000, tsm.TSM_F32, reliable=True, reliable_delta=1e-3)
    lp = tsm.stop(1e-2, 200, tsm.TSM_BF16)
    n_hp, n_lp = 4, 40
    ctxs = [tsm.Context(0) for _ in lattices]
    try:
        plist, outs, eager = [], [], []
        for k, (ctx, dims) in enumerate(zip(ctxs, lattices)):
            ctx.load_gauge(S.gauge_field(dims, 0.25, 60 + k), dims, KAPPA, MU)
            best, times = tsm.tsm_tune_batch(ctx.h, lp)
            assert best in (8, 16, 32, 64) and np.all(times > 0)
            assert times[[8, 16, 32, 64].index(best)] == times.min()
            eager.append(ctx.loops(700 + k, 4, n_hp, n_lp, hp, lp, GAM, MOMS, per_source=True, batch=best,
                                   verify=False))
            plist.append(tsm.params(700 + k, 4, (0, n_hp), (n_hp, n_hp + n_lp), hp, lp, GAM, MOMS, batch=best))
            outs.append(torch.zeros((n_lp, len(GAM), len(MOMS), dims[3]), dtype=torch.complex128, device="cuda"))
        tsm.tsm_loops_graph([c.h for c in ctxs], plist, per_lp=outs)
        torch.cuda.synchronize()
        for k in range(len(lattices)):
            assert np.array_equal(outs[k].cpu().numpy(), eager[k]["per_lp"]), k
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("prec", [tsm.TSM_F16, tsm.TSM_BF16])
def test_tuned_launch_shape_bit_identical(libtsm, prec):
    """tsm_tune picks the batch width and the block shape of the link-sharing
    stencil (2, 4 or 8 sources per block; 80 or 96 registers per thread for 4);
    whatever it picks, the TSM results are bit-identical to the default shape
    (batch 32, 4 sources per block, 80 registers): the per-site arithmetic and
    every reduction order are independent of both."""
    dims = (8, 8, 8, 16)
    hp = tsm.stop(1e-10, 3000, tsm.TSM_F32, reliable=True, reliable_delta=1e-3)
    lp = tsm.stop(5e-3, 60, prec)
    with tsm.Context(0) as ref, tsm.Context(0) as tuned:
        for c in (ref, tuned):
            c.load_gauge(S.gauge_field(dims, 0.25, 71), dims, KAPPA, MU)
        best, tile, regs, times = tsm.tsm_tune(tuned.h, lp)
        print("tuned: batch %d, %d sources per block, %d registers; ms per source:\n%s" % (best, tile, regs, times))
        assert best in (8, 16, 32, 64) and (tile, regs) in tsm.TILE_SHAPES
        assert times.min() > 0
        assert times[[8, 16, 32, 64].index(best), tsm.TILE_SHAPES.index((tile, regs))] == times.min()
        want = ref.loops(5, 4, 3, 29, hp, lp, GAM, MOMS, per_source=True, batch=32, verify=False)
        for b in (best, 32, 7):   # the tuned block shape with several batch widths
            got = tuned.loops(5, 4, 3, 29, hp, lp, GAM, MOMS, per_source=True, batch=b, verify=False)
            for k in ("loops", "err", "per_corr", "per_lp"):
                assert np.array_equal(got[k], want[k]), (b, k)
        # each of the other block shapes, forced, gives the same bits
        # too, for the LP tier and for the FP32 iterations of the HP solves
        for t, r in ((2, 80), (8, 80), (4, 96)):
            tsm.tsm_set_tile(tuned.h, prec, t, r)
            tsm.tsm_set_tile(tuned.h, tsm.TSM_F32, t, r)
            got = tuned.loops(5, 4, 3, 29, hp, lp, GAM, MOMS, per_source=True, batch=32, verify=False)
            assert np.array_equal(got["per_lp"], want["per_lp"]), t
            assert np.array_equal(got["per_corr"], want["per_corr"]), t
