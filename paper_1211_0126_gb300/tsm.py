"""Python binding of libtsm (include/tsm.h): argument marshalling only.

Every entry point of the C ABI has a function of the same name here
(``tsm_create``, ``tsm_load_gauge``, ``tm_dslash``, ``tm_solve_batch``,
``tsm_noise``, ``tsm_contract``, ``tsm_loops``, ``tsm_combine``, ...).  Arrays
are either numpy arrays in host memory (copied in/out by the library) or torch
CUDA tensors (passed as device pointers).  All arithmetic runs in the CUDA
library; if the library has not been built this module raises at import of
the library, it never falls back to another implementation.

Array layouts (complex128 numpy arrays, or torch complex128 / float64 tensors):
    gauge  [T, Z, Y, X, 4, 3, 3]
    spinor [T, Z, Y, X, 4, 3]        (batches: leading axis)
    loops  [n_gamma, n_q, T]
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtsm.so")

TSM_F64, TSM_F32, TSM_BF16, TSM_F16 = 0, 1, 2, 3
TM_OP_FULL, TM_OP_HOP_EO, TM_OP_HOP_OE, TM_OP_SCHUR, TM_OP_NORMAL = 0, 1, 2, 3, 4
STATUS = {0: "TSM_OK", -1: "TSM_ERR_ARG", -2: "TSM_ERR_DIMS", -3: "TSM_ERR_CUDA",
          -4: "TSM_ERR_NOT_CONVERGED", -5: "TSM_ERR_NONFINITE", -6: "TSM_ERR_TIMEOUT",
          -7: "TSM_ERR_NOT_UNITARY", -8: "TSM_ERR_NO_GAUGE", -9: "TSM_ERR_TOO_LARGE"}
TSM_ERR_NOT_CONVERGED = -4


class TmLattice(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("kappa", ctypes.c_double), ("mu", ctypes.c_double),
                ("t_antiperiodic", ctypes.c_int)]


class TmStop(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("prec", ctypes.c_int),
                ("reliable", ctypes.c_int), ("reliable_delta", ctypes.c_double), ("precond", ctypes.c_int),
                ("restart", ctypes.c_int)]


class TsmLoopStats(ctypes.Structure):
    _fields_ = [("n_sources", ctypes.c_int), ("lp_iters", ctypes.c_longlong), ("hp_iters", ctypes.c_longlong),
                ("hp_not_converged", ctypes.c_int), ("hp_max_true_res", ctypes.c_double),
                ("lp_max_true_res", ctypes.c_double)]


class TsmParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("noise", ctypes.c_int),
                ("hp_begin", ctypes.c_uint32), ("hp_end", ctypes.c_uint32),
                ("lp_begin", ctypes.c_uint32), ("lp_end", ctypes.c_uint32),
                ("hp", TmStop), ("lp", TmStop), ("batch", ctypes.c_int),
                ("gammas", ctypes.POINTER(ctypes.c_int)), ("n_gamma", ctypes.c_int),
                ("moms", ctypes.POINTER(ctypes.c_int)), ("n_q", ctypes.c_int), ("verify", ctypes.c_int),
                ("estimator", ctypes.c_int), ("deriv_mask", ctypes.c_int), ("all_momenta", ctypes.c_int),
                ("hp_warm_start", ctypes.c_int)]


# exported symbol -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "tsm_create": (ctypes.c_int, [ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "tsm_destroy": (ctypes.c_int, [_P]),
    "tsm_load_gauge": (ctypes.c_int, [_P, ctypes.POINTER(TmLattice), _P, ctypes.c_int]),
    "tm_dslash": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int]),
    "tm_solve_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.POINTER(TmStop), ctypes.c_int,
                                      _P, _P]),
    "tsm_noise": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, _P, ctypes.c_int]),
    "tsm_contract": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, _P, _P,
                                    _P, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int]),
    "tsm_contract_one_end": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, ctypes.c_int, _P,
                                            ctypes.c_int]),
    "tsm_contract_gen_one_end": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, ctypes.c_int,
                                                _P, ctypes.c_int]),
    "tsm_contract_fft": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, _P, _P, _P,
                                        ctypes.c_int, _P, ctypes.c_int]),
    "tsm_contract_deriv": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, _P, _P,
                                          _P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int]),
    "tsm_loops": (ctypes.c_int, [_P, ctypes.POINTER(TsmParams), _P, _P, _P, _P, _P, _P, ctypes.c_int,
                                 ctypes.POINTER(TsmLoopStats)]),
    "tsm_combine": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                   ctypes.c_int]),
    "tsm_contract_noalloc": (ctypes.c_int, [ctypes.POINTER(TmLattice), ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_uint32, _P, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    "tsm_loops_graph": (ctypes.c_int, [_P, ctypes.POINTER(TsmParams), ctypes.c_int, _P, _P, _P, _P,
                                       ctypes.POINTER(TsmLoopStats)]),
    "tsm_tune_batch": (ctypes.c_int, [_P, ctypes.POINTER(TmStop), ctypes.POINTER(ctypes.c_int), _P]),
    "tsm_tune": (ctypes.c_int, [_P, ctypes.POINTER(TmStop), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _P]),
    "tsm_set_tile": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "tsm_umma_gemm": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "tsm_umma_inject_timeout": (ctypes.c_int, [ctypes.c_int]),
    "tsm_measure_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "tsm_umma_gemm_ex": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), _P]),
    "tsm_net_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.c_uint64, ctypes.c_double,
                                      ctypes.POINTER(_P)]),
    "tsm_net_destroy": (ctypes.c_int, [_P]),
    "tsm_net_set_weights": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "tsm_net_get_weights": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "tsm_net_forward": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.c_int]),
    "tsm_net_gradient": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, _P]),
    "tsm_net_add_pairs": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(TmStop),
                                         ctypes.POINTER(ctypes.c_int)]),
    "tsm_net_add_solve_pairs": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_uint64, _P, ctypes.c_int,
                                               ctypes.POINTER(TmStop), ctypes.POINTER(ctypes.c_int)]),
    "tsm_net_get_pair": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "tsm_net_train": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P]),
    "tsm_net_loss": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "tsm_set_precond": (ctypes.c_int, [_P, _P]),
    "tsm_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "tsm_profile_read": (ctypes.c_int, [_P, _P, _P, _P]),
    "tsm_profile_read_ex": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "tsm_launch_count": (ctypes.c_longlong, [_P]),
    "tsm_last_error": (ctypes.c_char_p, []),
    "tsm_status_str": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def _preload_cudart():
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        for name in ("libcudart.so.13", "libcudart.so"):
            p = os.path.join(d, name)
            if os.path.exists(p):
                try:
                    ctypes.CDLL(p, mode=ctypes.RTLD_GLOBAL)
                    return
                except OSError:
                    pass


def library():
    """Load libtsm.so (built in-tree by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libtsm.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                           "g.build()\"` first" % LIB_PATH)
    try:
        lib = ctypes.CDLL(LIB_PATH)
    except OSError:
        _preload_cudart()
        lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TsmError(RuntimeError):
    def __init__(self, status, where):
        msg = library().tsm_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), msg))
        self.status = status


def _check(status, where, allow=()):
    if status != 0 and status not in allow:
        raise TsmError(status, where)
    return status


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, writable=False):
    """(pointer, on_device) of a numpy array or torch tensor, checked for layout."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("torch tensor must be contiguous")
        if a.dtype not in (__import__("torch").complex128, __import__("torch").float64):
            raise ValueError("torch tensor must be complex128 or float64")
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    if not isinstance(a, np.ndarray):
        raise TypeError("expected a numpy array or torch tensor")
    if a.dtype not in (np.complex128, np.float64) or not a.flags.c_contiguous:
        raise ValueError("numpy array must be C-contiguous complex128/float64")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    return ctypes.c_void_p(a.ctypes.data), 0


def _same_side(*flags):
    fl = [f for f in flags if f is not None]
    if fl and any(f != fl[0] for f in fl):
        raise ValueError("mix of host and device arrays in one call")
    return fl[0] if fl else 0


# ------------------------------------------------------------ C-ABI names
def tsm_create(device=0, stream=None):
    """Create a context; `stream` is a cudaStream_t as int (e.g. torch's cuda_stream) or None."""
    h = ctypes.c_void_p()
    _check(library().tsm_create(int(device), ctypes.c_void_p(stream or 0), ctypes.byref(h)), "tsm_create")
    return h


def tsm_destroy(h):
    _check(library().tsm_destroy(h), "tsm_destroy")


def lattice(dims, kappa, mu, antiperiodic_t=True):
    lat = TmLattice()
    for k in range(4):
        lat.L[k] = int(dims[k])
    lat.kappa = float(kappa)
    lat.mu = float(mu)
    lat.t_antiperiodic = 1 if antiperiodic_t else 0
    return lat


def stop(rel_tol, max_iter, prec=TSM_F64, reliable=False, reliable_delta=0.0, precond=False, restart=0):
    return TmStop(float(rel_tol), int(max_iter), int(prec), 1 if reliable else 0, float(reliable_delta),
                  1 if precond else 0, int(restart))


def tsm_load_gauge(h, lat, U):
    p, dev = _ptr(U)
    return _check(library().tsm_load_gauge(h, ctypes.byref(lat), p, dev), "tsm_load_gauge")


def tm_dslash(h, prec, op, dagger, psi, out):
    pi, di = _ptr(psi)
    po, do = _ptr(out, True)
    return _check(library().tm_dslash(h, int(prec), int(op), int(dagger), pi, po, _same_side(di, do)),
                  "tm_dslash")


def tm_solve_batch(h, b, s, stp, nrhs=1, allow_not_converged=True):
    """Solve D_tm s = b for nrhs stacked sources; returns (status, iters, true_res)."""
    pb, db = _ptr(b)
    ps, ds = _ptr(s, True)
    iters = np.zeros(nrhs, dtype=np.int32)
    tres = np.zeros(nrhs, dtype=np.float64)
    st = library().tm_solve_batch(h, int(nrhs), pb, ps, ctypes.byref(stp), _same_side(db, ds),
                                  ctypes.c_void_p(iters.ctypes.data), ctypes.c_void_p(tres.ctypes.data))
    _check(st, "tm_solve_batch", allow=(TSM_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return st, iters, tres


def tsm_noise(h, seed, kind, source, out):
    po, do = _ptr(out, True)
    return _check(library().tsm_noise(h, ctypes.c_uint64(seed), int(kind), ctypes.c_uint32(source), po, do),
                  "tsm_noise")


def _int_array(vals, name):
    arr = np.ascontiguousarray(np.asarray(vals, dtype=np.int32).reshape(-1))
    return arr, ctypes.c_void_p(arr.ctypes.data)


def tsm_contract(h, prec, seed, kind, source, s_a, s_b, gammas, moms, out):
    g, gp = _int_array(gammas, "gammas")
    m, mp = _int_array(moms, "moms")
    pa, da = _ptr(s_a)
    pb, db = _ptr(s_b)
    po, do = _ptr(out, True)
    return _check(library().tsm_contract(h, int(prec), ctypes.c_uint64(seed), int(kind), ctypes.c_uint32(source),
                                         pa, pb, gp, len(g), mp, len(m) // 3, po, _same_side(da, db, do)),
                  "tsm_contract")


def tsm_contract_one_end(h, prec, s_a, s_b, gammas, moms, out):
    g, gp = _int_array(gammas, "gammas")
    m, mp = _int_array(moms, "moms")
    pa, da = _ptr(s_a)
    pb, db = _ptr(s_b)
    po, do = _ptr(out, True)
    return _check(library().tsm_contract_one_end(h, int(prec), pa, pb, gp, len(g), mp, len(m) // 3, po,
                                                 _same_side(da, db, do)), "tsm_contract_one_end")


def tsm_contract_gen_one_end(h, prec, s_a, s_b, gammas, moms, out):
    g, gp = _int_array(gammas, "gammas")
    m, mp = _int_array(moms, "moms")
    pa, da = _ptr(s_a)
    pb, db = _ptr(s_b)
    po, do = _ptr(out, True)
    return _check(library().tsm_contract_gen_one_end(h, int(prec), pa, pb, gp, len(g), mp, len(m) // 3, po,
                                                     _same_side(da, db, do)), "tsm_contract_gen_one_end")


def tsm_contract_fft(h, prec, seed, kind, source, s_a, s_b, gammas, out):
    g, gp = _int_array(gammas, "gammas")
    pa, da = _ptr(s_a)
    pb, db = _ptr(s_b)
    po, do = _ptr(out, True)
    return _check(library().tsm_contract_fft(h, int(prec), ctypes.c_uint64(seed), int(kind), ctypes.c_uint32(source),
                                             pa, pb, gp, len(g), po, _same_side(da, db, do)), "tsm_contract_fft")


def tsm_contract_deriv(h, prec, seed, kind, source, s_a, s_b, gammas, deriv_mask, moms, out):
    g, gp = _int_array(gammas, "gammas")
    m, mp = _int_array(moms, "moms")
    pa, da = _ptr(s_a)
    pb, db = _ptr(s_b)
    po, do = _ptr(out, True)
    return _check(library().tsm_contract_deriv(h, int(prec), ctypes.c_uint64(seed), int(kind), ctypes.c_uint32(source),
                                               pa, pb, gp, len(g), int(deriv_mask), mp, len(m) // 3, po,
                                               _same_side(da, db, do)), "tsm_contract_deriv")


def tsm_contract_noalloc(lat, seed, kind, source, s_dev, gammas, moms, out_dev, stream=None):
    """Contraction that allocates nothing (for callers that cannot allocate
    device memory); s_dev and out_dev are torch CUDA tensors (complex128).
    Queued on `stream` (cudaStream_t as int, None = legacy stream)."""
    g, gp = _int_array(gammas, "gammas")
    m, mp = _int_array(moms, "moms")
    ps, ds = _ptr(s_dev)
    po, do = _ptr(out_dev, True)
    if ds != 1 or do != 1:
        raise ValueError("tsm_contract_noalloc takes device tensors")
    return _check(library().tsm_contract_noalloc(ctypes.byref(lat), ctypes.c_uint64(seed), int(kind),
                                                 ctypes.c_uint32(source), ps, gp, len(g), mp, len(m) // 3, po,
                                                 ctypes.c_void_p(stream or 0)), "tsm_contract_noalloc")


def params(seed, noise, hp_range, lp_range, hp_stop, lp_stop, gammas, moms, batch=1, verify=False,
           estimator=0, deriv_mask=0, all_momenta=False, hp_warm_start=False):
    """TsmParams; keeps the integer arrays alive on the returned object."""
    p = TsmParams()
    p.seed = int(seed)
    p.noise = int(noise)
    p.hp_begin, p.hp_end = int(hp_range[0]), int(hp_range[1])
    p.lp_begin, p.lp_end = int(lp_range[0]), int(lp_range[1])
    p.hp = hp_stop
    p.lp = lp_stop
    p.batch = int(batch)
    g = np.ascontiguousarray(np.asarray(gammas, dtype=np.int32).reshape(-1))
    m = np.ascontiguousarray(np.asarray(moms, dtype=np.int32).reshape(-1))
    p._keep = (g, m)
    p.gammas = g.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    p.n_gamma = len(g)
    p.moms = m.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    p.n_q = len(m) // 3
    p.verify = 1 if verify else 0
    p.estimator = int(estimator)
    p.deriv_mask = int(deriv_mask)
    p.all_momenta = 1 if all_momenta else 0
    p.hp_warm_start = 1 if hp_warm_start else 0
    return p


def tsm_loops(h, p, loops=None, err=None, lp_mean=None, corr_mean=None, per_corr=None, per_lp=None):
    ptrs = [_ptr(a, True) for a in (loops, err, lp_mean, corr_mean, per_corr, per_lp)]
    dev = _same_side(*[d for _, d in ptrs])
    stats = TsmLoopStats()
    _check(library().tsm_loops(h, ctypes.byref(p), *[q for q, _ in ptrs], dev, ctypes.byref(stats)), "tsm_loops")
    return stats


def tsm_loops_graph(handles, plist, loops=None, err=None, per_corr=None, per_lp=None):
    """One CUDA graph over several contexts; outputs are lists of torch CUDA
    tensors (or None) per context.  Returns the list of TsmLoopStats."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value for h in handles])
    ps = (TsmParams * n)(*plist)

    def ptr_array(arrs):
        if arrs is None:
            return None
        vals = []
        for a in arrs:
            if a is None:
                vals.append(None)
                continue
            p, dev = _ptr(a, True)
            if dev != 1:
                raise ValueError("tsm_loops_graph outputs must be device tensors")
            vals.append(p.value)
        return (ctypes.c_void_p * n)(*vals)

    stats = (TsmLoopStats * n)()
    _check(library().tsm_loops_graph(hs, ps, n, ptr_array(loops), ptr_array(err), ptr_array(per_corr),
                                     ptr_array(per_lp), stats), "tsm_loops_graph")
    return list(stats)


def tsm_combine(h, per_corr, per_lp, n_entries, loops=None, err=None, lp_mean=None, corr_mean=None):
    n_hp = 0 if per_corr is None else per_corr.shape[0]
    n_lp = 0 if per_lp is None else per_lp.shape[0]
    ins = [_ptr(per_corr), _ptr(per_lp)]
    outs = [_ptr(a, True) for a in (loops, err, lp_mean, corr_mean)]
    dev = _same_side(*[d for _, d in ins + outs])
    return _check(library().tsm_combine(h, ins[0][0], n_hp, ins[1][0], n_lp, int(n_entries),
                                        *[q for q, _ in outs], dev), "tsm_combine")


def tsm_tune_batch(h, stp):
    """Autotuned multi-RHS batch width for the loaded lattice and tier:
    returns (best width, per-source ms for widths 8, 16, 32, 64)."""
    best = ctypes.c_int(0)
    times = np.zeros(4)
    _check(library().tsm_tune_batch(h, ctypes.byref(stp), ctypes.byref(best), ctypes.c_void_p(times.ctypes.data)),
           "tsm_tune_batch")
    return best.value, times


# block shapes the autotuner tries: (sources per block, registers per thread)
TILE_SHAPES = ((2, 80), (4, 80), (8, 80), (4, 96))


def tsm_tune(h, stp):
    """Autotuned launch shape for the loaded lattice and tier: returns (best
    batch width, best sources per link-sharing block, its register budget,
    per-source ms [4][4] for widths 8, 16, 32, 64 x the block shapes of
    TILE_SHAPES)."""
    best = ctypes.c_int(0)
    tile = ctypes.c_int(0)
    regs = ctypes.c_int(0)
    times = np.zeros(16)
    _check(library().tsm_tune(h, ctypes.byref(stp), ctypes.byref(best), ctypes.byref(tile), ctypes.byref(regs),
                              ctypes.c_void_p(times.ctypes.data)), "tsm_tune")
    return best.value, tile.value, regs.value, times.reshape(4, 4)


def tsm_set_tile(h, prec, tile_sources, max_regs=80):
    return _check(library().tsm_set_tile(h, int(prec), int(tile_sources), int(max_regs)), "tsm_set_tile")


def tsm_umma_gemm(A, B, C, beta=0, stream=None):
    """C = A @ B^T (+ C) on the tensor cores: A (M, K), B (N, K) torch bfloat16
    CUDA tensors, C (M, N) torch float32 CUDA tensor."""
    import torch
    for t, dt in ((A, torch.bfloat16), (B, torch.bfloat16), (C, torch.float32)):
        if not (t.is_cuda and t.is_contiguous() and t.dtype == dt):
            raise ValueError("tsm_umma_gemm wants contiguous CUDA tensors (bf16, bf16, fp32)")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or tuple(C.shape) != (M, N):
        raise ValueError("shape mismatch")
    return _check(library().tsm_umma_gemm(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                          ctypes.c_void_p(C.data_ptr()), M, N, K, int(beta),
                                          ctypes.c_void_p(stream or 0)), "tsm_umma_gemm")


def tsm_net_create(channels, seed=0, init_scale=0.1, device=0):
    """Network with channels[0..L] (first and last 1); returns its handle."""
    ch = np.ascontiguousarray(channels, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(library().tsm_net_create(int(device), len(ch) - 1, ctypes.c_void_p(ch.ctypes.data),
                                    ctypes.c_uint64(seed), float(init_scale), ctypes.byref(h)), "tsm_net_create")
    return h


def tsm_net_destroy(n):
    _check(library().tsm_net_destroy(n), "tsm_net_destroy")


def tsm_net_set_weights(n, layer, W):
    W = np.ascontiguousarray(W, dtype=np.complex128)
    _check(library().tsm_net_set_weights(n, int(layer), ctypes.c_void_p(W.ctypes.data)), "tsm_net_set_weights")


def tsm_net_get_weights(n, layer, shape):
    W = np.zeros(shape, dtype=np.complex128)
    _check(library().tsm_net_get_weights(n, int(layer), ctypes.c_void_p(W.ctypes.data)), "tsm_net_get_weights")
    return W


def tsm_net_forward(n, h, nb, x, y):
    px, dx = _ptr(x)
    py, dy = _ptr(y, True)
    _check(library().tsm_net_forward(n, h, int(nb), px, py, _same_side(dx, dy)), "tsm_net_forward")


def tsm_net_gradient(n, h, nb, x, gy, gx, gw):
    px, _ = _ptr(x)
    pg, _ = _ptr(gy)
    pgx, _ = _ptr(gx, True)
    pgw, _ = _ptr(gw, True)
    _check(library().tsm_net_gradient(n, h, int(nb), px, pg, pgx, pgw), "tsm_net_gradient")


def tsm_net_add_solve_pairs(n, h, n_sources, seed, iters, stp):
    it = np.ascontiguousarray(np.asarray(iters, dtype=np.int32))
    g = ctypes.c_int(-1)
    _check(library().tsm_net_add_solve_pairs(n, h, int(n_sources), ctypes.c_uint64(seed),
                                             ctypes.c_void_p(it.ctypes.data), len(it), ctypes.byref(stp),
                                             ctypes.byref(g)), "tsm_net_add_solve_pairs")
    return g.value


def tsm_net_get_pair(n, group, index, r, t):
    _check(library().tsm_net_get_pair(n, int(group), int(index), ctypes.c_void_p(r.ctypes.data),
                                      ctypes.c_void_p(t.ctypes.data)), "tsm_net_get_pair")


def tsm_net_add_pairs(n, h, count, seed, stp):
    g = ctypes.c_int(-1)
    _check(library().tsm_net_add_pairs(n, h, int(count), ctypes.c_uint64(seed), ctypes.byref(stp), ctypes.byref(g)),
           "tsm_net_add_pairs")
    return g.value


def tsm_net_train(n, groups, steps, batch, lr):
    gr = np.ascontiguousarray(groups, dtype=np.int32)
    loss = np.zeros(max(int(steps), 1))
    _check(library().tsm_net_train(n, ctypes.c_void_p(gr.ctypes.data), len(gr), int(steps), int(batch), float(lr),
                                   ctypes.c_void_p(loss.ctypes.data)), "tsm_net_train")
    return loss[:int(steps)]


def tsm_net_loss(n, group):
    v = ctypes.c_double(0.0)
    _check(library().tsm_net_loss(n, int(group), ctypes.byref(v)), "tsm_net_loss")
    return v.value


def tsm_set_precond(h, n):
    _check(library().tsm_set_precond(h, n), "tsm_set_precond")


def tsm_measure_fma_peak(device, prec):
    """Measured FMA peak of the device in TFLOP/s (prec TSM_F32 or TSM_F64)."""
    v = ctypes.c_double(0.0)
    _check(library().tsm_measure_fma_peak(int(device), int(prec), ctypes.byref(v)), "tsm_measure_fma_peak")
    return v.value


def tsm_umma_inject_timeout(withhold):
    return _check(library().tsm_umma_inject_timeout(1 if withhold else 0), "tsm_umma_inject_timeout")


def tsm_umma_gemm_ex(A, B, C, splits=1, beta=0, stream=None):
    """Split-K form: A (M, K) and B (N, K) bfloat16 (row strides may exceed K),
    C (splits, M, N) float32 receives the partial products; returns the number
    of partials written."""
    import torch
    for t, dt in ((A, torch.bfloat16), (B, torch.bfloat16), (C, torch.float32)):
        if not (t.is_cuda and t.dtype == dt and t.stride(-1) == 1):
            raise ValueError("tsm_umma_gemm_ex wants CUDA tensors (bf16, bf16, fp32) with unit inner stride")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or tuple(C.shape[-2:]) != (M, N) or not C.is_contiguous():
        raise ValueError("shape mismatch")
    used = ctypes.c_int(0)
    _check(library().tsm_umma_gemm_ex(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                                      B.stride(0), ctypes.c_void_p(C.data_ptr()), N, M, N, K, int(beta),
                                      int(splits), ctypes.byref(used), ctypes.c_void_p(stream or 0)),
           "tsm_umma_gemm_ex")
    return used.value


def tsm_profile(h, enable):
    return _check(library().tsm_profile(h, 1 if enable else 0), "tsm_profile")


def tsm_profile_read(h):
    ms = np.zeros(16)
    cnt = np.zeros(16, dtype=np.int64)
    by = np.zeros(16)
    _check(library().tsm_profile_read(h, ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(cnt.ctypes.data),
                                      ctypes.c_void_p(by.ctypes.data)), "tsm_profile_read")
    return ms, cnt, by


# profile buckets after the 16 hop buckets (tsm_profile_read_ex)
PB_CONTRACT, PB_DERIV, PB_FFT, PB_WILSON = 16, 17, 18, 19


def tsm_profile_read_ex(h, n=24):
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    by = np.zeros(n)
    _check(library().tsm_profile_read_ex(h, int(n), ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(cnt.ctypes.data),
                                         ctypes.c_void_p(by.ctypes.data)), "tsm_profile_read_ex")
    return ms, cnt, by


def tsm_launch_count(h):
    return int(library().tsm_launch_count(h))


# ------------------------------------------------------------ convenience
class Context:
    """Owning wrapper around a tsm_ctx handle with numpy-returning helpers."""

    def __init__(self, device=0, stream=None):
        self.h = tsm_create(device, stream)
        self.dims = None

    def close(self):
        if self.h is not None:
            tsm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_gauge(self, U, dims, kappa, mu, antiperiodic_t=True):
        self.dims = tuple(int(d) for d in dims)
        self.lat = lattice(dims, kappa, mu, antiperiodic_t)
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
        tsm_load_gauge(self.h, self.lat, U)

    def _spinor_shape(self):
        lx, ly, lz, lt = self.dims
        return (lt, lz, ly, lx, 4, 3)

    def dslash(self, psi, op=TM_OP_FULL, dagger=False, prec=TSM_F64):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.zeros(self._spinor_shape(), dtype=np.complex128)
        tm_dslash(self.h, prec, op, dagger, psi, out)
        return out

    def solve(self, b, stp):
        b = np.ascontiguousarray(b, dtype=np.complex128)
        nrhs = 1 if b.ndim == 6 else b.shape[0]
        s = np.zeros_like(b)
        st, iters, tres = tm_solve_batch(self.h, b, s, stp, nrhs)
        return s, iters, tres, st

    def noise(self, seed, source, kind=4):
        out = np.zeros(self._spinor_shape(), dtype=np.complex128)
        tsm_noise(self.h, seed, kind, source, out)
        return out

    def contract(self, seed, source, s_a, gammas, moms, s_b=None, kind=4, prec=TSM_F64):
        s_a = np.ascontiguousarray(s_a, dtype=np.complex128)
        if s_b is not None:
            s_b = np.ascontiguousarray(s_b, dtype=np.complex128)
        out = np.zeros((len(gammas), len(moms), self.dims[3]), dtype=np.complex128)
        tsm_contract(self.h, prec, seed, kind, source, s_a, s_b, gammas, moms, out)
        return out

    def loops(self, seed, noise, n_hp, n_lp, hp_stop, lp_stop, gammas, moms, hp_range=None, lp_range=None,
              per_source=False, batch=1, verify=True, estimator=0, deriv_mask=0, all_momenta=False,
              hp_warm_start=False):
        hp_range = hp_range or (0, n_hp)
        lp_range = lp_range or (n_hp, n_hp + n_lp)
        if all_momenta:
            moms = [(0, 0, 0)]
        p = params(seed, noise, hp_range, lp_range, hp_stop, lp_stop, gammas, moms, batch, verify, estimator,
                   deriv_mask, all_momenta, hp_warm_start)
        shape = (len(gammas), len(moms), self.dims[3])
        if deriv_mask:
            shape = (1 + bin(int(deriv_mask)).count("1"),) + shape
        if all_momenta:
            lx, ly, lz, lt = self.dims
            shape = (len(gammas), lt, lz, ly, lx)
        out = {k: np.zeros(shape, dtype=np.complex128) for k in ("loops", "lp_mean", "corr_mean")}
        out["err"] = np.zeros(shape, dtype=np.float64)
        pc = pl = None
        if per_source:
            pc = np.zeros((hp_range[1] - hp_range[0],) + shape, dtype=np.complex128)
            pl = np.zeros((lp_range[1] - lp_range[0],) + shape, dtype=np.complex128)
        stats = tsm_loops(self.h, p, out["loops"], out["err"], out["lp_mean"], out["corr_mean"], pc, pl)
        out["stats"] = {f: getattr(stats, f) for f, _ in TsmLoopStats._fields_}
        if per_source:
            out["per_corr"], out["per_lp"] = pc, pl
        return out

    def contract_one_end(self, s_a, gammas, moms, s_b=None, prec=TSM_F64):
        s_a = np.ascontiguousarray(s_a, dtype=np.complex128)
        if s_b is not None:
            s_b = np.ascontiguousarray(s_b, dtype=np.complex128)
        out = np.zeros((len(gammas), len(moms), self.dims[3]), dtype=np.complex128)
        tsm_contract_one_end(self.h, prec, s_a, s_b, gammas, moms, out)
        return out

    def contract_gen_one_end(self, s_a, gammas, moms, s_b=None, prec=TSM_F64):
        s_a = np.ascontiguousarray(s_a, dtype=np.complex128)
        if s_b is not None:
            s_b = np.ascontiguousarray(s_b, dtype=np.complex128)
        out = np.zeros((len(gammas), len(moms), self.dims[3]), dtype=np.complex128)
        tsm_contract_gen_one_end(self.h, prec, s_a, s_b, gammas, moms, out)
        return out

    def contract_fft(self, seed, source, s_a, gammas, s_b=None, kind=4, prec=TSM_F64):
        """[n_gamma][T][Lz][Ly][Lx] local loops of one source at every spatial momentum."""
        s_a = np.ascontiguousarray(s_a, dtype=np.complex128)
        if s_b is not None:
            s_b = np.ascontiguousarray(s_b, dtype=np.complex128)
        lx, ly, lz, lt = self.dims
        out = np.zeros((len(gammas), lt, lz, ly, lx), dtype=np.complex128)
        tsm_contract_fft(self.h, prec, seed, kind, source, s_a, s_b, gammas, out)
        return out

    def contract_deriv(self, seed, source, s_a, gammas, deriv_mask, moms, s_b=None, kind=4, prec=TSM_F64):
        """[n_dirs][n_gamma][n_q][T] one-derivative loops of one source."""
        s_a = np.ascontiguousarray(s_a, dtype=np.complex128)
        if s_b is not None:
            s_b = np.ascontiguousarray(s_b, dtype=np.complex128)
        nd = bin(int(deriv_mask)).count("1")
        out = np.zeros((nd, len(gammas), len(moms), self.dims[3]), dtype=np.complex128)
        tsm_contract_deriv(self.h, prec, seed, kind, source, s_a, s_b, gammas, deriv_mask, moms, out)
        return out

    def combine(self, per_corr, per_lp):
        ref = per_corr if per_corr is not None and per_corr.shape[0] else per_lp
        shape = ref.shape[1:]
        n = int(np.prod(shape))
        out = {k: np.zeros(shape, dtype=np.complex128) for k in ("loops", "lp_mean", "corr_mean")}
        out["err"] = np.zeros(shape, dtype=np.float64)
        pc = None if per_corr is None else np.ascontiguousarray(per_corr)
        pl = None if per_lp is None else np.ascontiguousarray(per_lp)
        tsm_combine(self.h, pc, pl, n, out["loops"], out["err"], out["lp_mean"], out["corr_mean"])
        return out

    def profile(self, enable=True):
        tsm_profile(self.h, enable)

    def profile_read(self):
        return tsm_profile_read(self.h)

    def profile_read_ex(self, n=24):
        return tsm_profile_read_ex(self.h, n)

    def launch_count(self):
        return tsm_launch_count(self.h)

    def set_precond(self, net):
        tsm_set_precond(self.h, None if net is None else net.h)


class Network:
    """Owning wrapper around a tsm_net (the learned LP preconditioner)."""

    def __init__(self, channels, seed=0, init_scale=0.1, device=0):
        self.channels = [int(c) for c in channels]
        self.h = tsm_net_create(self.channels, seed, init_scale, device)

    def close(self):
        if self.h is not None:
            tsm_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, layer):
        return (4 * self.channels[layer + 1], 36 * self.channels[layer])

    def set_weights(self, layer, W):
        tsm_net_set_weights(self.h, layer, W)

    def get_weights(self, layer):
        return tsm_net_get_weights(self.h, layer, self.shape(layer))

    def forward(self, ctx, x):
        """x [nb, C0, T, Z, Y, X, 4, 3] complex -> [nb, CL, ...]."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.zeros((x.shape[0], self.channels[-1]) + x.shape[2:], dtype=np.complex128)
        tsm_net_forward(self.h, ctx.h, x.shape[0], x, y)
        return y

    def gradient(self, ctx, x, gy):
        """(gx, [gW per layer]) for output gradient gy (G = dL/dRe + i dL/dIm)."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        gy = np.ascontiguousarray(gy, dtype=np.complex128)
        gx = np.zeros_like(x)
        sizes = [int(np.prod(self.shape(l))) for l in range(len(self.channels) - 1)]
        gw = np.zeros(sum(sizes), dtype=np.complex128)
        tsm_net_gradient(self.h, ctx.h, x.shape[0], x, gy, gx, gw)
        out, off = [], 0
        for l, sz in enumerate(sizes):
            out.append(gw[off:off + sz].reshape(self.shape(l)))
            off += sz
        return gx, out

    def add_pairs(self, ctx, count, seed, stp):
        return tsm_net_add_pairs(self.h, ctx.h, count, seed, stp)

    def add_solve_pairs(self, ctx, n_sources, seed, iters, stp):
        """Pairs (r = Dhat t, t = x* - x_k) from the CGNR iterates x_k (k in
        iters) of solves of the noise sources 0 .. n_sources-1 of seed."""
        return tsm_net_add_solve_pairs(self.h, ctx.h, n_sources, seed, iters, stp)

    def get_pair(self, group, index, spinor_shape):
        r = np.zeros(spinor_shape, dtype=np.complex128)
        t = np.zeros(spinor_shape, dtype=np.complex128)
        tsm_net_get_pair(self.h, group, index, r, t)
        return r, t

    def train(self, groups, steps, batch, lr):
        return tsm_net_train(self.h, groups, steps, batch, lr)

    def loss(self, group):
        return tsm_net_loss(self.h, group)
