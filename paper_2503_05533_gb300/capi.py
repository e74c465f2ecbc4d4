"""Thin Python binding of libmlmc (include/libmlmc.h) via ctypes.

Functions carry the C names and only marshal arguments: tensors become device
pointers (``tensor.data_ptr()``), ``stream=None`` becomes PyTorch's current CUDA
stream, and a non-OK status raises :class:`MlmcError` with the library's
message.  Every computation happens in the CUDA library; if ``libmlmc.so`` is
missing the import of this module's functions fails loudly.
"""
import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int32, c_int64, c_uint64, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmlmc.so")

MLMC_MAX_LEVELS = 16

# mlmc_status
MLMC_OK, MLMC_E_ARG, MLMC_E_NOMEM, MLMC_E_CUDA, MLMC_E_NOCONV, MLMC_E_NONFINITE, MLMC_E_TIMEOUT, \
    MLMC_E_UNSUPPORTED = range(8)
STATUS_NAMES = ["MLMC_OK", "MLMC_E_ARG", "MLMC_E_NOMEM", "MLMC_E_CUDA", "MLMC_E_NOCONV", "MLMC_E_NONFINITE",
                "MLMC_E_TIMEOUT", "MLMC_E_UNSUPPORTED"]
# mlmc_prec
MLMC_FP64, MLMC_FP32, MLMC_BF16S, MLMC_FP16S, MLMC_FP64TC, MLMC_FP8S = range(6)
# mlmc_solver
MLMC_CG, MLMC_MINRES, MLMC_CHOLESKY = range(3)
MLMC_PC_JACOBI, MLMC_PC_MG = range(2)
# mlmc_form
MLMC_FORM_MIXED, MLMC_FORM_FP64_ADAPTIVE, MLMC_FORM_FP64_FIXED = range(3)
# flags
MLMC_F_CONVERGED, MLMC_F_MAXIT, MLMC_F_STAGNATED, MLMC_F_NONFINITE, MLMC_F_TIMEOUT = 1, 2, 4, 8, 16


class mlmc_field(ctypes.Structure):
    _fields_ = [("kind", c_int), ("K", c_int), ("sigma2", c_double), ("corr_len", c_double), ("q", c_double)]


class mlmc_problem(ctypes.Structure):
    _fields_ = [("n0", c_int), ("m", c_int), ("L_max", c_int), ("field", mlmc_field), ("qoi", c_int),
                ("box", c_double * 4), ("f", c_double), ("seed", c_uint64)]


class mlmc_acc(ctypes.Structure):
    _fields_ = [("n", c_int64), ("mean", c_double), ("m2", c_double), ("sum", c_double), ("sum_c", c_double),
                ("sumsq", c_double), ("sumsq_c", c_double)]


class mlmc_options(ctypes.Structure):
    _fields_ = [("tol", c_double), ("L_start", c_int), ("N_init", c_int), ("kp", c_double),
                ("alpha1", c_double), ("alpha2", c_double), ("beta1", c_double), ("beta2", c_double),
                ("alpha", c_double), ("gamma", c_double), ("r", c_double), ("form", c_int),
                ("fixed_delta", c_double), ("force_prec", c_int), ("solver", c_int), ("max_iters", c_int),
                ("max_rounds", c_int), ("fixed_N", POINTER(c_int64)), ("contrast", c_double),
                ("mixed_field", c_int), ("prec_rule", c_int), ("chol_table", c_int), ("resume", c_void_p),
                ("log_path", c_char_p)]


class mlmc_result(ctypes.Structure):
    _fields_ = [("estimate", c_double), ("rmse", c_double), ("var_est", c_double), ("L", c_int),
                ("rounds", c_int), ("bias_failed", c_int), ("flags_or", c_int32),
                ("N", c_int64 * MLMC_MAX_LEVELS), ("Yhat", c_double * MLMC_MAX_LEVELS),
                ("s2", c_double * MLMC_MAX_LEVELS), ("delta", c_double * MLMC_MAX_LEVELS),
                ("prec", c_int32 * MLMC_MAX_LEVELS), ("inner_iters", c_int64 * MLMC_MAX_LEVELS),
                ("dofs", c_int64 * MLMC_MAX_LEVELS), ("acc", mlmc_acc * MLMC_MAX_LEVELS), ("seconds", c_double),
                ("fp64_retries", c_int64 * MLMC_MAX_LEVELS), ("contrast", c_double * MLMC_MAX_LEVELS),
                ("a_min", c_double * MLMC_MAX_LEVELS), ("a_max", c_double * MLMC_MAX_LEVELS)]


class mlmc_profile(ctypes.Structure):
    _fields_ = [("solve_launches", c_int64), ("solve_ms", c_double), ("solve_bytes", c_double),
                ("inner_iters", c_int64), ("unknown_iters", c_int64), ("kl_launches", c_int64),
                ("kl_ms", c_double), ("kl_bytes", c_double), ("kl_flops", c_double),
                ("h2d_bytes", c_int64), ("d2h_bytes", c_int64), ("solve_busy_ms", c_double),
                ("solve_flops", c_double), ("chol_bits", c_double)]


class mlmc_tune_entry(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_char * 192), ("prec", c_int), ("solver", c_int), ("precond", c_int),
                ("med_items", c_int), ("ring", c_int), ("nu", c_int), ("mg_min", c_int), ("mg_coarse", c_int),
                ("mg_omega", c_double), ("mg_smem", c_int), ("theta", c_double), ("tau_min", c_double),
                ("best_ms", c_double), ("default_ms", c_double), ("trials", c_int)]


SAMPLER_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_int, c_int64, c_int, POINTER(c_double), POINTER(c_double))

# name -> (restype, argtypes)
_SIGS = {
    "mlmc_create": (c_int, [POINTER(mlmc_problem), c_int, POINTER(c_void_p)]),
    "mlmc_destroy": (None, [c_void_p]),
    "mlmc_last_error": (c_char_p, [c_void_p]),
    "mlmc_version": (c_char_p, []),
    "mlmc_launch_count": (c_int64, []),
    "mlmc_sample_fields": (c_int, [c_void_p, c_int, c_uint64, c_int, c_void_p, c_void_p, c_int64, c_int, c_void_p]),
    "mlmc_synthesize_fields": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int64, c_int, c_void_p]),
    "mlmc_apply_operator": (c_int, [c_int, c_int, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_int,
                                    c_void_p]),
    "mlmc_level_solve": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_int64, c_int, c_int, c_double, c_int,
                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "mlmc_sync": (c_int, [c_void_p, c_void_p]),
    "mlmc_level_solve_noalloc": (c_int, [c_int, c_int, c_int, c_void_p, c_int, c_int, c_int, c_double, c_int,
                                         c_int, POINTER(c_double), c_double, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p]),
    "mlmc_level_stats": (c_int, [c_void_p, c_int, c_void_p, c_void_p, POINTER(mlmc_acc), c_void_p]),
    "mlmc_acc_merge": (None, [POINTER(mlmc_acc), POINTER(mlmc_acc)]),
    "mlmc_adapt_precision": (c_int, [c_int, POINTER(c_double), c_double, c_double, c_double, c_double, c_double,
                                     c_double, POINTER(c_double), POINTER(c_int)]),
    "mlmc_default_options": (None, [POINTER(mlmc_options)]),
    "mlmc_estimate": (c_int, [c_void_p, POINTER(mlmc_options), POINTER(mlmc_result)]),
    "mlmc_estimate_host": (c_int, [c_int, c_int, c_int, POINTER(mlmc_options), SAMPLER_FN, c_void_p,
                                   POINTER(mlmc_result)]),
    "mlmc_adjoint_grad": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_double, c_int, c_void_p, c_void_p,
                                  c_void_p]),
    "mlmc_set_wait_timeout": (c_int, [c_void_p, c_double]),
    "mlmc_set_autotune": (c_int, [c_void_p, c_int]),
    "mlmc_set_sample_ahead": (c_int, [c_void_p, c_int]),
    "mlmc_set_cholesky_precision": (c_int, [c_void_p, c_int, c_int]),
    "mlmc_autotune_count": (c_int, [c_void_p]),
    "mlmc_autotune_entry": (c_int, [c_void_p, c_int, c_void_p]),
    "mlmc_debug_set_wait_extra": (c_int, [c_void_p, c_int]),
    "mlmc_debug_set_solve_ring": (c_int, [c_void_p, c_int]),
    "mlmc_debug_fail_allocation": (c_int, [c_int64]),
    "mlmc_set_seed": (c_int, [c_void_p, c_uint64]),
    "mlmc_set_mg_coarsest": (c_int, [c_void_p, c_int]),
    "mlmc_set_full_multigrid": (c_int, [c_void_p, c_int]),
    "mlmc_debug_set_medium_items": (c_int, [c_void_p, c_int]),
    "mlmc_set_precond": (c_int, [c_void_p, c_int, c_int, c_int, c_double]),
    "mlmc_set_inner_tolerance": (c_int, [c_void_p, c_double, c_double]),
    "mlmc_profile_enable": (c_int, [c_void_p, c_int]),
    "mlmc_profile_get": (c_int, [c_void_p, c_void_p]),
    "mlmc_profile_reset": (c_int, [c_void_p]),
}

_lib = None


class MlmcError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, msg))


def lib():
    """The loaded libmlmc.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmlmc.so is not built (expected at %s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status, ctx=None):
    if status != MLMC_OK:
        msg = lib().mlmc_last_error(ctx)
        raise MlmcError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
def make_problem(n0=16, m=2, L_max=4, kind=0, K=64, sigma2=1.0, corr_len=0.3, q=2.0, qoi=0,
                 box=(0.0, 1.0, 0.0, 1.0), f=1.0, seed=0):
    p = mlmc_problem()
    p.n0, p.m, p.L_max = n0, m, L_max
    p.field = mlmc_field(kind, K, sigma2, corr_len, q)
    p.qoi = qoi
    p.box = (c_double * 4)(*box)
    p.f = f
    p.seed = seed
    return p


def mlmc_create(problem, device=0):
    h = c_void_p()
    st = lib().mlmc_create(byref(problem), device, byref(h))
    _check(st, None)
    return h


def mlmc_destroy(ctx):
    lib().mlmc_destroy(ctx)


def mlmc_set_seed(ctx, seed):
    _check(lib().mlmc_set_seed(ctx, seed), ctx)


def mlmc_set_mg_coarsest(ctx, min_cells):
    _check(lib().mlmc_set_mg_coarsest(ctx, min_cells), ctx)


def mlmc_set_full_multigrid(ctx, on=True):
    _check(lib().mlmc_set_full_multigrid(ctx, 1 if on else 0), ctx)


def mlmc_last_error(ctx=None):
    msg = lib().mlmc_last_error(ctx)
    return msg.decode() if msg else ""


def mlmc_version():
    return lib().mlmc_version().decode()


def mlmc_launch_count():
    return lib().mlmc_launch_count()


def mlmc_set_cholesky_precision(ctx, u, u_r):
    _check(lib().mlmc_set_cholesky_precision(ctx, u, u_r), ctx)


def mlmc_set_autotune(ctx, on=True):
    _check(lib().mlmc_set_autotune(ctx, 1 if on else 0), ctx)


def mlmc_set_sample_ahead(ctx, on=True):
    _check(lib().mlmc_set_sample_ahead(ctx, 1 if on else 0), ctx)


def mlmc_autotune_count(ctx):
    return lib().mlmc_autotune_count(ctx)


def mlmc_autotune_entry(ctx, i):
    e = mlmc_tune_entry()
    _check(lib().mlmc_autotune_entry(ctx, i, byref(e)), ctx)
    d = {name: getattr(e, name) for name, _ in mlmc_tune_entry._fields_}
    d["shape"] = e.shape.decode()
    return d


def mlmc_set_wait_timeout(ctx, seconds):
    _check(lib().mlmc_set_wait_timeout(ctx, seconds), ctx)


def mlmc_profile_enable(ctx, on=True):
    _check(lib().mlmc_profile_enable(ctx, 1 if on else 0), ctx)


def mlmc_profile_get(ctx):
    p = mlmc_profile()
    _check(lib().mlmc_profile_get(ctx, byref(p)), ctx)
    return {name: getattr(p, name) for name, _ in mlmc_profile._fields_}


def mlmc_profile_reset(ctx):
    _check(lib().mlmc_profile_reset(ctx), ctx)


def mlmc_debug_set_wait_extra(ctx, extra):
    _check(lib().mlmc_debug_set_wait_extra(ctx, extra), ctx)


def mlmc_set_precond(ctx, pc, nu=0, coarse_sweeps=0, omega=0.0):
    _check(lib().mlmc_set_precond(ctx, pc, nu, coarse_sweeps, omega), ctx)


def mlmc_set_inner_tolerance(ctx, theta=0.0, tau_min=0.0):
    _check(lib().mlmc_set_inner_tolerance(ctx, theta, tau_min), ctx)


def mlmc_debug_set_solve_ring(ctx, ring):
    _check(lib().mlmc_debug_set_solve_ring(ctx, ring), ctx)


def mlmc_debug_fail_allocation(after):
    """Make the (after+1)-th next device allocation of the library fail once (-1 disarms)."""
    _check(lib().mlmc_debug_fail_allocation(after))


def set_resume(opts, res):
    """Continue an estimate from the checkpoint `res` (an mlmc_result; None clears)."""
    opts._resume_ref = res
    opts.resume = ctypes.addressof(res) if res is not None else None


def set_log_path(opts, path):
    """Append one JSON line per Alg. 4.1 round to `path` (None turns logging off)."""
    opts._log_ref = path.encode() if path is not None else None
    opts.log_path = opts._log_ref


def save_result(res, path):
    """Write an mlmc_result (a checkpoint for mlmc_options.resume) to a file, as its raw bytes."""
    with open(path, "wb") as f:
        f.write(bytes(res))


def load_result(path):
    """Read a checkpoint written by save_result."""
    with open(path, "rb") as f:
        data = f.read()
    if len(data) != ctypes.sizeof(mlmc_result):
        raise ValueError("not an mlmc_result of this library version: %d bytes" % len(data))
    return mlmc_result.from_buffer_copy(data)


def mlmc_debug_set_medium_items(ctx, items):
    _check(lib().mlmc_debug_set_medium_items(ctx, items), ctx)


def mlmc_sample_fields(ctx, level, first, S, xi, a, field_prec, stream=None, a_ld=0):
    _check(lib().mlmc_sample_fields(ctx, level, first, S, _ptr(xi), _ptr(a), a_ld, field_prec, _stream(stream)),
           ctx)


def mlmc_synthesize_fields(ctx, level, S, xi, a, field_prec, stream=None, a_ld=0):
    _check(lib().mlmc_synthesize_fields(ctx, level, S, _ptr(xi), _ptr(a), a_ld, field_prec, _stream(stream)), ctx)


def mlmc_apply_operator(n, S, a, a_prec, a_n, op_prec, x, y, vec_prec, stream=None):
    _check(lib().mlmc_apply_operator(n, S, _ptr(a), a_prec, a_n, op_prec, _ptr(x), _ptr(y), vec_prec,
                                     _stream(stream)))


def mlmc_level_solve(ctx, n, S, a, a_prec, a_n, prec, solver, delta, max_iters, u, Q, iters=None, relres=None,
                     flags=None, stream=None, a_ld=0):
    _check(lib().mlmc_level_solve(ctx, n, S, _ptr(a), a_prec, a_n, a_ld, prec, solver, delta, max_iters, _ptr(u),
                                  _ptr(Q), _ptr(iters), _ptr(relres), _ptr(flags), _stream(stream)), ctx)


def mlmc_sync(ctx, stream=None):
    """Wait for the context's work on `stream`; raises on a bounded wait that ran out."""
    _check(lib().mlmc_sync(ctx, _stream(stream)), ctx)


def mlmc_level_solve_noalloc(device, n, S, a, a_prec, a_n, prec, delta, max_iters, qoi, box, f, Q, iters=None,
                             relres=None, flags=None, stream=None):
    """Allocation-free solve (no context, scratch in the library's static device array)."""
    bx = (c_double * 4)(*(box if box is not None else (0.0, 1.0, 0.0, 1.0)))
    _check(lib().mlmc_level_solve_noalloc(device, n, S, _ptr(a), a_prec, a_n, prec, delta, max_iters, qoi, bx, f,
                                          _ptr(Q), _ptr(iters), _ptr(relres), _ptr(flags), _stream(stream)))


def mlmc_level_stats(ctx, S, Qf, Qc, acc=None, stream=None):
    acc = acc if acc is not None else mlmc_acc()
    _check(lib().mlmc_level_stats(ctx, S, _ptr(Qf), _ptr(Qc), byref(acc), _stream(stream)), ctx)
    return acc


def mlmc_acc_merge(into, other):
    lib().mlmc_acc_merge(byref(into), byref(other))
    return into


def mlmc_adapt_precision(h, kp=0.05, alpha1=2.0, alpha2=1.0, beta1=4.0, beta2=2.0, contrast=1.0):
    L = len(h) - 1
    hh = (c_double * (L + 1))(*h)
    d = (c_double * (L + 1))()
    p = (c_int * (L + 1))()
    _check(lib().mlmc_adapt_precision(L, hh, kp, alpha1, alpha2, beta1, beta2, contrast, d, p))
    return list(d), list(p)


def mlmc_default_options():
    o = mlmc_options()
    lib().mlmc_default_options(byref(o))
    return o


def mlmc_estimate(ctx, opts):
    res = mlmc_result()
    _check(lib().mlmc_estimate(ctx, byref(opts), byref(res)), ctx)
    return res


def mlmc_estimate_host(m, L_max, n0, opts, sampler):
    """sampler(level, first, count, delta_list) -> sequence of count floats."""

    def cb(user, level, first, count, delta, Y):
        try:
            vals = sampler(level, first, count, delta)
            for i in range(count):
                Y[i] = float(vals[i])
            return 0
        except Exception:  # propagated as MLMC_E_ARG
            return 1

    fn = SAMPLER_FN(cb)
    res = mlmc_result()
    _check(lib().mlmc_estimate_host(m, L_max, n0, byref(opts), fn, None, byref(res)))
    return res


def mlmc_adjoint_grad(ctx, level, S, xi, prec, delta, max_iters, Q, dQdxi, stream=None):
    _check(lib().mlmc_adjoint_grad(ctx, level, S, _ptr(xi), prec, delta, max_iters, _ptr(Q), _ptr(dQdxi),
                                   _stream(stream)), ctx)


def result_dict(res):
    """Plain-Python view of an mlmc_result."""
    L = res.L
    return {
        "estimate": res.estimate, "rmse": res.rmse, "var_est": res.var_est, "L": L, "rounds": res.rounds,
        "bias_failed": bool(res.bias_failed), "flags_or": res.flags_or,
        "N": list(res.N[:L + 1]), "Yhat": list(res.Yhat[:L + 1]), "s2": list(res.s2[:L + 1]),
        "delta": list(res.delta[:L + 1]), "prec": list(res.prec[:L + 1]),
        "inner_iters": list(res.inner_iters[:L + 1]), "dofs": list(res.dofs[:L + 1]), "seconds": res.seconds,
        "fp64_retries": list(res.fp64_retries[:L + 1]), "contrast": list(res.contrast[:L + 1]),
    }
