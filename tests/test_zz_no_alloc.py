"""The contraction entry point that allocates nothing (tsm_contract_noalloc).

It serves callers that cannot allocate device memory where they need a
contraction (a foreign allocator owns the device, cudaMalloc's implicit
synchronisation is not acceptable, or there is no library context).  The GPU
test calls it through the C ABI three times in a row -- each call with other
arguments, so stale scratch contents would show -- and compares each result
with the existing tsm_contract (FP64) and with the oracle's local loops at the
tolerance of the other FP64 contraction tests.  The third call runs on a
16x16x20x8 lattice with 16 Gammas x 13 momenta (208 outputs per timeslice):
the scratch limit then lowers the number of blocks per timeslice to 38, so
every block sums two chunks of sites and holds two outputs per thread, and
the reduction adds 38 block partials.  The file name makes pytest collect it
last.
"""
import numpy as np
import pytest

from oracle import loops as oloops
from oracle import philox
from paper_1211_0126_gb300 import synthetic as S
from paper_1211_0126_gb300 import tsm


def test_rejects_requests_beyond_the_scratch_limit(libtsm):
    lat = tsm.lattice((4, 4, 4, 4), 0.124, 0.01)
    g = (np.arange(16, dtype=np.int32))
    m = np.zeros((17, 3), dtype=np.int32)
    dummy = np.zeros(1, dtype=np.float64)
    import ctypes
    p = ctypes.c_void_p(dummy.ctypes.data)
    rc = libtsm.tsm_contract_noalloc(ctypes.byref(lat), 1, 4, 0, p, ctypes.c_void_p(g.ctypes.data), 16,
                                     ctypes.c_void_p(m.ctypes.data), 17, p, None)
    assert rc == -9 and b"n_q" in libtsm.tsm_last_error()
    big = tsm.lattice((2048, 1024, 2, 2), 0.124, 0.01)
    rc = libtsm.tsm_contract_noalloc(ctypes.byref(big), 1, 4, 0, p, ctypes.c_void_p(g.ctypes.data), 16,
                                     ctypes.c_void_p(m.ctypes.data), 4, p, None)
    assert rc == -9
    odd = tsm.lattice((3, 4, 4, 4), 0.124, 0.01)
    rc = libtsm.tsm_contract_noalloc(ctypes.byref(odd), 1, 4, 0, p, ctypes.c_void_p(g.ctypes.data), 16,
                                     ctypes.c_void_p(m.ctypes.data), 4, p, None)
    assert rc == -2


@pytest.mark.gpu
def test_noalloc_contraction_matches_tsm_contract_and_oracle(ctx):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    calls = [
        ((6, 4, 4, 8), 2024, 4, 3, list(range(16)), S.default_momenta(7)),
        ((6, 4, 4, 8), 7, 2, 11, [5, 0, 12], S.default_momenta(13)),
        ((16, 16, 20, 8), 31, 4, 5, list(range(16)), S.default_momenta(13)),
    ]
    for k, (dims, seed, kind, source, gam, moms) in enumerate(calls):
        lat = tsm.lattice(dims, 0.124, 0.01)
        ctx.load_gauge(S.gauge_field(dims, 0.0, 0), dims, 0.124, 0.01)
        s = S.random_spinor(dims, 100 + k)
        want = ctx.contract(seed, source, s, gam, moms, kind=kind, prec=tsm.TSM_F64)
        ref = oloops.local_loops(philox.noise(seed, source, dims, kind), s, dims, gam, moms)
        s_dev = torch.from_numpy(s).to("cuda")
        out = torch.full((len(gam), len(moms), dims[3]), complex("nan"), dtype=torch.complex128, device="cuda")
        tsm.tsm_contract_noalloc(lat, seed, kind, source, s_dev, gam, moms, out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), k
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max(), k
