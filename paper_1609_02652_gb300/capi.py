"""Thin ctypes binding of the C-ABI in include/pfmp.h.

Functions keep the C names and argument order; device buffers are passed as integer
addresses (e.g. ``tensor.data_ptr()``), host arrays as numpy arrays.  A non-zero status
raises ``PfmpError`` with the library's message.  Nothing here computes: every step of
the method runs in the CUDA library.  Importing this module without the built library
raises ``ImportError`` -- there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpfmp.so")

PFMP_OK = 0
PFMP_E_INVALID = 1
PFMP_E_NOMEM = 2
PFMP_E_CUDA = 3
PFMP_E_NOT_CONVERGED = 4
PFMP_E_TIMEOUT = 5
PFMP_E_NAN = 6
PFMP_E_UNSUPPORTED = 7
PFMP_F64 = 0
PFMP_F32 = 1
PFMP_DF = 2
PFMP_H16 = 3
PFMP_HOST = 0
PFMP_DEVICE = 1
PFMP_KERNEL_HOP_F32 = 0
PFMP_KERNEL_HOP_F64 = 1
PFMP_KERNEL_HOP_DF = 2
PFMP_KERNEL_HOP_H16 = 3
PFMP_KERNEL_CG_F32 = 4
PFMP_SOLVER_CG64 = 0
PFMP_SOLVER_CG_MIXED = 1
PFMP_SOLVER_CG_HALF = 2


class PfmpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pfmp status {status}: {msg}")
        self.status = status


class SolverParams(C.Structure):
    _fields_ = [("method", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("delta", C.c_double),
                ("check_every", C.c_int), ("restart", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("reliable_updates", C.c_int), ("true_rel_res", C.c_double),
                ("k_apply", C.c_int64), ("status", C.c_int)]


class ActionParams(C.Structure):
    _fields_ = [("beta", C.c_double), ("kappa", C.c_double), ("kappa_h", C.c_double), ("csw", C.c_double),
                ("n", C.c_int), ("mu", C.c_double), ("nu", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int)]


PFMP_MAX_TERMS = 8
PFMP_MAX_KAPPA = 4
PFMP_KIND_GAUGE, PFMP_KIND_DET, PFMP_KIND_FILTER, PFMP_KIND_FILTERCORR, PFMP_KIND_RATIO, PFMP_KIND_INV = range(6)
PFMP_TERM_GAUGE, PFMP_TERM_DET, PFMP_TERM_POLY, PFMP_TERM_POLYCORR, PFMP_TERM_HASEN = range(5)
(PFMP_SCHEME_1PF, PFMP_SCHEME_2PF, PFMP_SCHEME_1MP, PFMP_SCHEME_2MP, PFMP_SCHEME_PFMP, PFMP_SCHEME_2PF1MP,
 PFMP_SCHEME_1PF2MP) = range(7)


class Term(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_int), ("b", C.c_int), ("p1", C.c_int), ("p2", C.c_int)]


class ActionDef(C.Structure):
    _fields_ = [("beta", C.c_double), ("csw", C.c_double), ("nkappa", C.c_int),
                ("kappa", C.c_double * PFMP_MAX_KAPPA), ("nterms", C.c_int), ("term", Term * PFMP_MAX_TERMS),
                ("mu", C.c_double), ("nu", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int),
                ("solver", C.c_int), ("force_prec", C.c_int), ("md_tol", C.c_double)]


class CostInfo(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("p_acc", "p_acc_err", "nmat", "nmat_err", "cost", "cost_err", "exp_mdh",
                                          "exp_mdh_err")]


class TrajInfo(C.Structure):
    _fields_ = [("H0", C.c_double), ("H1", C.c_double), ("dH", C.c_double), ("accepted", C.c_int),
                ("S0", C.c_double * PFMP_MAX_TERMS), ("S1", C.c_double * PFMP_MAX_TERMS),
                ("plaquette", C.c_double), ("k_apply", C.c_int64), ("force_evals", C.c_int),
                ("k_apply_term", C.c_int64 * PFMP_MAX_TERMS), ("nforce", C.c_int * PFMP_MAX_TERMS),
                ("fmax", C.c_double * PFMP_MAX_TERMS), ("favg", C.c_double * PFMP_MAX_TERMS),
                ("ms_force", C.c_double * PFMP_MAX_TERMS), ("ms_update", C.c_double), ("ms_total", C.c_double)]

P = C.c_void_p
I = C.c_int
D = C.c_double
DP = C.POINTER(C.c_double)

# name: (restype, argtypes)
SIGNATURES = {
    "pfmp_strerror": (C.c_char_p, [I]),
    "pfmp_last_error": (C.c_char_p, []),
    "pfmp_version": (I, []),
    "pfmp_launch_count": (C.c_int64, []),
    "pfmp_ctx_create": (I, [C.POINTER(P), C.POINTER(I), I, P]),
    "pfmp_ctx_destroy": (I, [P]),
    "pfmp_ctx_set_stream": (I, [P, P]),
    "pfmp_half_volume": (C.c_int64, [P]),
    "pfmp_spinor_bytes": (C.c_int64, [P, I]),
    "pfmp_gauge_set": (I, [P, P, I]),
    "pfmp_gauge_get": (I, [P, P, I]),
    "pfmp_gauge_from_algebra": (I, [P, P, D, I]),
    "pfmp_plaquette": (I, [P, DP]),
    "pfmp_spinor_pack": (I, [P, P, I, P, I, I]),
    "pfmp_spinor_unpack": (I, [P, P, I, P, I, I]),
    "pfmp_op_create": (I, [P, D, D, C.POINTER(P)]),
    "pfmp_op_update": (I, [P]),
    "pfmp_op_destroy": (I, [P]),
    "pfmp_op_logdet": (I, [P, DP]),
    "pfmp_op_set_split": (I, [P, I, I]),
    "pfmp_op_get_split": (I, [P, I, C.POINTER(I)]),
    "pfmp_op_set_block": (I, [P, I]),
    "pfmp_dslash": (I, [P, I, P, P, I, I]),
    "pfmp_clover_apply": (I, [P, I, P, P, I, I]),
    "pfmp_mhat": (I, [P, I, P, P, I]),
    "pfmp_mhat_noalloc": (I, [P, I, P, P, I]),
    "pfmp_kop": (I, [P, I, P, P, DP]),
    "pfmp_true_residual": (I, [P, I, P, P, P, DP]),
    "pfmp_norm2": (I, [P, I, P, DP]),
    "pfmp_cdot": (I, [P, I, P, P, DP]),
    "pfmp_axpy": (I, [P, I, D, D, P, P]),
    "pfmp_convert": (I, [P, P, I, P, I]),
    "pfmp_solve": (I, [P, C.POINTER(SolverParams), P, P, C.POINTER(SolveInfo)]),
    "pfmp_solve_host": (I, [P, C.POINTER(SolverParams), P, P, C.POINTER(SolveInfo)]),
    "pfmp_solve_multishift": (I, [P, I, DP, DP, C.POINTER(P), P, D, I, C.POINTER(SolveInfo)]),
    "pfmp_poly_roots": (I, [I, D, D, DP, DP, DP]),
    "pfmp_poly_apply": (I, [P, I, D, D, I, P, P]),
    "pfmp_action_create": (I, [P, C.POINTER(ActionParams), C.POINTER(P)]),
    "pfmp_action_scheme": (I, [I, I, I, C.POINTER(ActionDef)]),
    "pfmp_spectrum": (I, [P, I, P, DP, DP, DP, DP, C.POINTER(I)]),
    "pfmp_balance_steps": (I, [I, DP, I, C.POINTER(I)]),
    "pfmp_md": (I, [P, I, DP, I, DP, C.POINTER(I), P, I]),
    "pfmp_cost": (I, [I, C.POINTER(I), DP, DP, D, C.POINTER(CostInfo)]),
    "pfmp_action_create_def": (I, [P, C.POINTER(ActionDef), C.POINTER(P)]),
    "pfmp_action_counts": (I, [P, C.POINTER(I), C.POINTER(I)]),
    "pfmp_action_destroy": (I, [P]),
    "pfmp_action_refresh": (I, [P]),
    "pfmp_action_heatbath": (I, [P, P, I]),
    "pfmp_action_get_phi": (I, [P, I, P, I]),
    "pfmp_action_set_phi": (I, [P, I, P, I]),
    "pfmp_action_eval": (I, [P, DP]),
    "pfmp_action_force": (I, [P, I, P, I]),
    "pfmp_schedule_2mn": (I, [I, D, D, DP, DP]),
    "pfmp_schedule_merge": (I, [I, C.POINTER(I), DP, DP, I, DP, DP, C.POINTER(I)]),
    "pfmp_trajectory": (I, [P, I, DP, I, DP, C.POINTER(I), P, P, I, D, C.POINTER(TrajInfo)]),
    "pfmp_batch_create": (I, [I, C.POINTER(P), C.POINTER(I), C.POINTER(P)]),
    "pfmp_batch_destroy": (I, [P]),
    "pfmp_batch_tune": (I, [P, I, C.POINTER(I), DP]),
    "pfmp_batch_solve": (I, [P, C.POINTER(SolverParams), C.POINTER(P), C.POINTER(P), C.POINTER(SolveInfo)]),
    "pfmp_batch_barrier_check": (I, [P, I, I, C.c_double]),
    "pfmp_nn_create": (I, [P, I, C.POINTER(I), I, C.POINTER(P)]),
    "pfmp_nn_destroy": (I, [P]),
    "pfmp_nn_num_weights": (C.c_int64, [P]),
    "pfmp_nn_set_weights": (I, [P, DP]),
    "pfmp_nn_get_weights": (I, [P, DP]),
    "pfmp_nn_apply": (I, [P, I, P, P]),
    "pfmp_nn_set_tensor_cores": (I, [P, I]),
    "pfmp_nn_loss_grad": (I, [P, P, I, P, P, DP, DP]),
    "pfmp_nn_train": (I, [P, P, I, I, C.POINTER(P), C.POINTER(P), I, I, D, DP]),
    "pfmp_solve_fgcr": (I, [P, P, C.POINTER(SolverParams), P, P, C.POINTER(SolveInfo)]),
    "pfmp_profile_begin": (I, [P]),
    "pfmp_profile_end": (I, [P, I, C.POINTER(C.c_int64), DP, DP]),
    "pfmp_fma_rate": (I, [P, I, DP]),
    "pfmp_solve_multishift_prec": (I, [P, I, I, DP, DP, C.POINTER(P), P, D, I, C.POINTER(SolveInfo)]),
}

_lib = None


def lib():
    """Load libpfmp.so (built in-tree by paper_1609_02652_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1609_02652_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != PFMP_OK:
        L = lib()
        msg = L.pfmp_last_error().decode() or L.pfmp_strerror(status).decode()
        raise PfmpError(status, msg)
    return status


def _ptr(x):
    """Address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    raise TypeError(type(x))


# ---------------------------------------------------------------- same-name wrappers
def pfmp_ctx_create(dims, bc_t=-1, stream=None):
    h = P()
    d = (I * 4)(*dims)
    check(lib().pfmp_ctx_create(C.byref(h), d, int(bc_t), stream))
    return h


def pfmp_ctx_destroy(ctx):
    check(lib().pfmp_ctx_destroy(ctx))


def pfmp_ctx_set_stream(ctx, stream):
    check(lib().pfmp_ctx_set_stream(ctx, stream))


def pfmp_half_volume(ctx):
    return int(lib().pfmp_half_volume(ctx))


def pfmp_spinor_bytes(ctx, prec):
    return int(lib().pfmp_spinor_bytes(ctx, prec))


def pfmp_gauge_set(ctx, U, where):
    check(lib().pfmp_gauge_set(ctx, _ptr(U), where))


def pfmp_gauge_get(ctx, U, where):
    check(lib().pfmp_gauge_get(ctx, _ptr(U), where))


def pfmp_gauge_from_algebra(ctx, h, eps, where):
    check(lib().pfmp_gauge_from_algebra(ctx, _ptr(h), float(eps), where))


def pfmp_plaquette(ctx):
    v = C.c_double()
    check(lib().pfmp_plaquette(ctx, C.byref(v)))
    return v.value


def pfmp_spinor_pack(ctx, dst, prec, src, where, parity):
    check(lib().pfmp_spinor_pack(ctx, _ptr(dst), prec, _ptr(src), where, parity))


def pfmp_spinor_unpack(ctx, dst, where, src, prec, parity):
    check(lib().pfmp_spinor_unpack(ctx, _ptr(dst), where, _ptr(src), prec, parity))


def pfmp_op_create(ctx, kappa, csw):
    h = P()
    check(lib().pfmp_op_create(ctx, float(kappa), float(csw), C.byref(h)))
    return h


def pfmp_op_update(op):
    check(lib().pfmp_op_update(op))


def pfmp_op_destroy(op):
    check(lib().pfmp_op_destroy(op))


def pfmp_op_logdet(op):
    v = C.c_double()
    check(lib().pfmp_op_logdet(op, C.byref(v)))
    return v.value


def pfmp_op_set_split(op, prec, ns):
    check(lib().pfmp_op_set_split(op, prec, ns))


def pfmp_op_set_block(op, threads):
    check(lib().pfmp_op_set_block(op, threads))


def pfmp_op_get_split(op, prec):
    v = I()
    check(lib().pfmp_op_get_split(op, prec, C.byref(v)))
    return v.value


def pfmp_dslash(op, prec, out, inp, out_parity, dagger=0):
    check(lib().pfmp_dslash(op, prec, _ptr(out), _ptr(inp), out_parity, dagger))


def pfmp_clover_apply(op, prec, out, inp, parity, inverse):
    check(lib().pfmp_clover_apply(op, prec, _ptr(out), _ptr(inp), parity, inverse))


def pfmp_mhat(op, prec, out, inp, dagger=0):
    check(lib().pfmp_mhat(op, prec, _ptr(out), _ptr(inp), dagger))


def pfmp_mhat_noalloc(op, prec, out, inp, dagger=0):
    check(lib().pfmp_mhat_noalloc(op, prec, _ptr(out), _ptr(inp), dagger))


def pfmp_kop(op, prec, out, inp, want_norm=False):
    v = C.c_double()
    check(lib().pfmp_kop(op, prec, _ptr(out), _ptr(inp), C.byref(v) if want_norm else None))
    return v.value if want_norm else None


def pfmp_true_residual(op, arith, r, x, b):
    v = C.c_double()
    check(lib().pfmp_true_residual(op, arith, _ptr(r), _ptr(x), _ptr(b), C.byref(v)))
    return v.value


def pfmp_norm2(ctx, prec, x):
    v = C.c_double()
    check(lib().pfmp_norm2(ctx, prec, _ptr(x), C.byref(v)))
    return v.value


def pfmp_cdot(ctx, prec, x, y):
    v = (C.c_double * 2)()
    check(lib().pfmp_cdot(ctx, prec, _ptr(x), _ptr(y), v))
    return complex(v[0], v[1])


def pfmp_axpy(ctx, prec, a, x, y):
    a = complex(a)
    check(lib().pfmp_axpy(ctx, prec, a.real, a.imag, _ptr(x), _ptr(y)))


def pfmp_convert(ctx, dst, dst_prec, src, src_prec):
    check(lib().pfmp_convert(ctx, _ptr(dst), dst_prec, _ptr(src), src_prec))


def pfmp_solve(op, params, x, b, raise_on_error=True):
    info = SolveInfo()
    st = lib().pfmp_solve(op, C.byref(params), _ptr(x), _ptr(b), C.byref(info))
    if raise_on_error:
        check(st)
    return info


def pfmp_solve_host(op, params, x_host, b_host, raise_on_error=True):
    info = SolveInfo()
    st = lib().pfmp_solve_host(op, C.byref(params), _ptr(x_host), _ptr(b_host), C.byref(info))
    if raise_on_error:
        check(st)
    return info


def pfmp_fma_rate(ctx, prec):
    v = C.c_double()
    check(lib().pfmp_fma_rate(ctx, int(prec), C.byref(v)))
    return v.value


def pfmp_profile_begin(ctx):
    check(lib().pfmp_profile_begin(ctx))


def pfmp_profile_end(ctx, kernel_class):
    n, ms, by = C.c_int64(), C.c_double(), C.c_double()
    check(lib().pfmp_profile_end(ctx, kernel_class, C.byref(n), C.byref(ms), C.byref(by)))
    return n.value, ms.value, by.value


def pfmp_launch_count():
    return int(lib().pfmp_launch_count())


def _dp(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(DP)


def pfmp_solve_multishift_prec(op, prec, sigmas, xs, b, tol, max_iter):
    sig = np.asarray(sigmas, dtype=np.complex128)
    re, pre = _dp(sig.real)
    im, pim = _dp(sig.imag)
    arr = (P * len(xs))(*[_ptr(x) for x in xs])
    info = SolveInfo()
    check(lib().pfmp_solve_multishift_prec(op, int(prec), len(xs), pre, pim, arr, _ptr(b), float(tol), int(max_iter),
                                           C.byref(info)))
    return info


def pfmp_solve_multishift(op, sigmas, xs, b, tol, max_iter, want_info=True):
    sig = np.asarray(sigmas, dtype=np.complex128)
    re, pre = _dp(sig.real)
    im, pim = _dp(sig.imag)
    arr = (P * len(xs))(*[_ptr(x) for x in xs])
    info = SolveInfo()
    check(lib().pfmp_solve_multishift(op, len(xs), pre, pim, arr, _ptr(b), float(tol), int(max_iter),
                                      C.byref(info) if want_info else None))
    return info


def pfmp_poly_roots(n, mu, nu):
    zr = np.zeros(n)
    zi = np.zeros(n)
    an = C.c_double()
    check(lib().pfmp_poly_roots(n, mu, nu, zr.ctypes.data_as(DP), zi.ctypes.data_as(DP), C.byref(an)))
    return zr + 1j * zi, an.value


def pfmp_poly_apply(op, n, mu, nu, which, out, inp):
    check(lib().pfmp_poly_apply(op, n, mu, nu, which, _ptr(out), _ptr(inp)))


def pfmp_action_create(ctx, params):
    h = P()
    check(lib().pfmp_action_create(ctx, C.byref(params), C.byref(h)))
    return h


def pfmp_spectrum(op, nsteps, v0):
    """Returns (lmin, lmax, alpha, beta) of nsteps Lanczos steps on K from v0."""
    lo, hi, k = C.c_double(), C.c_double(), I()
    a = np.zeros(nsteps)
    b = np.zeros(nsteps)
    check(lib().pfmp_spectrum(op, nsteps, _ptr(v0), C.byref(lo), C.byref(hi), a.ctypes.data_as(DP),
                              b.ctypes.data_as(DP), C.byref(k)))
    return lo.value, hi.value, a[:k.value].copy(), b[:k.value].copy()


def pfmp_md(a, T, S_levels, term_level, mom, where=PFMP_HOST):
    """MD alone; mom (host float64 array or device address) is overwritten."""
    T, pT = _dp(T)
    S, pS = _dp(np.asarray(S_levels).reshape(-1))
    tl = (I * len(term_level))(*term_level)
    check(lib().pfmp_md(a, len(T), pT, np.asarray(S_levels).shape[0], pS, tl, _ptr(mom), where))


def pfmp_balance_steps(fmax, n_coarse):
    f, pf = _dp(np.asarray(fmax, dtype=np.float64))
    n = (I * len(f))()
    check(lib().pfmp_balance_steps(len(f), pf, n_coarse, n))
    return list(n)


def pfmp_cost(accepted, nmat, dH, tau_int=12.5):
    acc = (I * len(accepted))(*[int(bool(a)) for a in accepted])
    nm, pn = _dp(np.asarray(nmat, dtype=np.float64))
    dh, pd = _dp(np.asarray(dH, dtype=np.float64))
    info = CostInfo()
    check(lib().pfmp_cost(len(acc), acc, pn, pd, float(tau_int), C.byref(info)))
    return info


def pfmp_action_scheme(scheme, p1, p2, d):
    check(lib().pfmp_action_scheme(scheme, p1, p2, C.byref(d)))
    return d


def pfmp_action_create_def(ctx, d):
    h = P()
    check(lib().pfmp_action_create_def(ctx, C.byref(d), C.byref(h)))
    return h


def pfmp_action_counts(a):
    nt, npf = I(), I()
    check(lib().pfmp_action_counts(a, C.byref(nt), C.byref(npf)))
    return nt.value, npf.value


def pfmp_action_destroy(a):
    check(lib().pfmp_action_destroy(a))


def pfmp_action_refresh(a):
    check(lib().pfmp_action_refresh(a))


def pfmp_action_heatbath(a, xi, where=PFMP_HOST):
    check(lib().pfmp_action_heatbath(a, _ptr(xi), where))


def pfmp_action_get_phi(a, i, out, where=PFMP_HOST):
    check(lib().pfmp_action_get_phi(a, i, _ptr(out), where))


def pfmp_action_set_phi(a, i, phi, where=PFMP_HOST):
    check(lib().pfmp_action_set_phi(a, i, _ptr(phi), where))


def pfmp_action_eval(a):
    S = (C.c_double * PFMP_MAX_TERMS)()
    check(lib().pfmp_action_eval(a, S))
    return np.array(S[:pfmp_action_counts(a)[0]])


def pfmp_action_force(a, term, out, where=PFMP_HOST):
    check(lib().pfmp_action_force(a, term, _ptr(out), where))


def pfmp_schedule_2mn(n, tau, lam):
    T = np.zeros(2 * n + 1)
    S = np.zeros(2 * n + 1)
    check(lib().pfmp_schedule_2mn(n, tau, lam, T.ctypes.data_as(DP), S.ctypes.data_as(DP)))
    return T, S


def pfmp_schedule_merge(schemes, cap=4096):
    lens = (I * len(schemes))(*[len(T) for T, _ in schemes])
    T, pT = _dp(np.concatenate([np.asarray(T, float) for T, _ in schemes]))
    S, pS = _dp(np.concatenate([np.asarray(S, float) for _, S in schemes]))
    Tout = np.zeros(cap)
    Sout = np.zeros((len(schemes), cap))
    m = I()
    check(lib().pfmp_schedule_merge(len(schemes), lens, pT, pS, cap, Tout.ctypes.data_as(DP),
                                    Sout.ctypes.data_as(DP), C.byref(m)))
    return Tout[:m.value].copy(), Sout[:, :m.value].copy()


def pfmp_trajectory(a, T, S_levels, term_level, mom, xi, u, where=PFMP_HOST):
    T, pT = _dp(T)
    S, pS = _dp(np.asarray(S_levels).reshape(-1))
    tl = (I * len(term_level))(*term_level)
    info = TrajInfo()
    check(lib().pfmp_trajectory(a, len(T), pT, np.asarray(S_levels).shape[0], pS, tl, _ptr(mom), _ptr(xi), where,
                                float(u), C.byref(info)))
    return info


def pfmp_batch_create(ops, nrhs):
    h = P()
    arr = (P * len(ops))(*[o.value if isinstance(o, P) else o for o in ops])
    nr = (I * len(nrhs))(*nrhs)
    check(lib().pfmp_batch_create(len(ops), arr, nr, C.byref(h)))
    return h


def pfmp_batch_destroy(b):
    check(lib().pfmp_batch_destroy(b))


def pfmp_batch_tune(b, chunk=8):
    blk, ms = I(), C.c_double()
    check(lib().pfmp_batch_tune(b, chunk, C.byref(blk), C.byref(ms)))
    return blk.value, ms.value


def pfmp_batch_solve(b, params, xs, bs, raise_on_error=True):
    n = len(xs)
    xa = (P * n)(*[_ptr(v) for v in xs])
    ba = (P * n)(*[_ptr(v) for v in bs])
    infos = (SolveInfo * n)()
    st = lib().pfmp_batch_solve(b, C.byref(params), xa, ba, infos)
    if raise_on_error:
        check(st)
    return list(infos)


def pfmp_batch_barrier_check(b, rounds, missing, limit_s):
    """Status of `rounds` grid barriers with `missing` more blocks expected than launched
    (PFMP_OK, or PFMP_E_TIMEOUT once every wait ran out); returned, not raised."""
    return lib().pfmp_batch_barrier_check(b, rounds, missing, float(limit_s))


def pfmp_nn_create(ctx, channels, prec=PFMP_F32):
    h = P()
    ch = (I * len(channels))(*channels)
    check(lib().pfmp_nn_create(ctx, len(channels) - 1, ch, prec, C.byref(h)))
    return h


def pfmp_nn_destroy(nn):
    check(lib().pfmp_nn_destroy(nn))


def pfmp_nn_num_weights(nn):
    return int(lib().pfmp_nn_num_weights(nn))


def pfmp_nn_set_weights(nn, weights):
    """weights: list of complex arrays W[9][c_out][c_in][4][4] (one per layer)."""
    flat = np.concatenate([np.ascontiguousarray(w, dtype=np.complex128).reshape(-1) for w in weights])
    a = np.ascontiguousarray(flat.view(np.float64))
    check(lib().pfmp_nn_set_weights(nn, a.ctypes.data_as(DP)))


def _unflatten(nn_shapes, flat):
    out, off = [], 0
    for shp in nn_shapes:
        n = int(np.prod(shp))
        out.append(flat[off:off + n].reshape(shp))
        off += n
    return out


def pfmp_nn_get_weights(nn, shapes):
    n = pfmp_nn_num_weights(nn)
    a = np.zeros(2 * n)
    check(lib().pfmp_nn_get_weights(nn, a.ctypes.data_as(DP)))
    return _unflatten(shapes, a.view(np.complex128))


def pfmp_nn_apply(nn, prec, out, inp):
    check(lib().pfmp_nn_apply(nn, prec, _ptr(out), _ptr(inp)))


def pfmp_nn_set_tensor_cores(nn, on):
    check(lib().pfmp_nn_set_tensor_cores(nn, int(on)))


PFMP_NN_LOSS_SOLUTION = 0
PFMP_NN_LOSS_RESIDUAL = 1


def pfmp_nn_loss_grad(nn, b, x, shapes=None, op=None, kind=PFMP_NN_LOSS_SOLUTION):
    loss = C.c_double()
    if shapes is None:
        check(lib().pfmp_nn_loss_grad(nn, op, kind, _ptr(b), _ptr(x), C.byref(loss), None))
        return loss.value, None
    n = pfmp_nn_num_weights(nn)
    a = np.zeros(2 * n)
    check(lib().pfmp_nn_loss_grad(nn, op, kind, _ptr(b), _ptr(x), C.byref(loss), a.ctypes.data_as(DP)))
    return loss.value, _unflatten(shapes, a.view(np.complex128))


def pfmp_nn_train(nn, bs, xs, steps, batch, lr, op=None, kind=PFMP_NN_LOSS_SOLUTION):
    n = len(bs)
    ba = (P * n)(*[_ptr(v) for v in bs])
    xa = (P * n)(*[_ptr(v) for v in xs])
    loss = C.c_double()
    check(lib().pfmp_nn_train(nn, op, kind, n, ba, xa, steps, batch, lr, C.byref(loss)))
    return loss.value


def pfmp_solve_fgcr(op, nn, params, x, b, raise_on_error=True):
    info = SolveInfo()
    st = lib().pfmp_solve_fgcr(op, nn, C.byref(params), _ptr(x), _ptr(b), C.byref(info))
    if raise_on_error:
        check(st)
    return info
