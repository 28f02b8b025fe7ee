"""Thin Python binding of the C ABI in include/sisdc.h (argument marshalling only).

Every entry point has the C name.  Device arrays are passed as torch CUDA
float64 tensors (or raw integer addresses); all arithmetic runs in the CUDA
library.  A missing library raises instead of falling back to anything.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsisdc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sisdc.h")

c_int, c_double, c_ll, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p

# sisdc_alloc_fn / sisdc_release_fn of include/sisdc.h
ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, ctypes.c_size_t, c_void_p, c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, c_void_p, ctypes.c_size_t, c_void_p, c_void_p)

SISDC_OK, SISDC_E_ARG, SISDC_E_CUDA, SISDC_E_NOCONV = 0, -1, -2, -3
SISDC_E_TIMEOUT, SISDC_E_NONFINITE, SISDC_E_OOM, SISDC_E_STATE = -4, -5, -6, -7
STATUS_NAMES = {0: "SISDC_OK", -1: "SISDC_E_ARG", -2: "SISDC_E_CUDA", -3: "SISDC_E_NOCONV",
                -4: "SISDC_E_TIMEOUT", -5: "SISDC_E_NONFINITE", -6: "SISDC_E_OOM", -7: "SISDC_E_STATE"}
SISDC_RADAU_RIGHT, SISDC_LOBATTO = 0, 1
SISDC_PDE_CONVDIFF, SISDC_PDE_BURGERS, SISDC_PDE_EULER, SISDC_PDE_NS = 0, 1, 2, 3
SISDC_FP64, SISDC_MIXED = 0, 1
SISDC_START_SPREAD, SISDC_START_PREDICTOR, SISDC_START_CASCADE, SISDC_START_FMG1 = 0, 1, 2, 3
T_INTERP, T_PROJECT, T_RESTRICT, T_PROJECT_SPACE = 0, 1, 2, 3


class sisdc_level_desc(ctypes.Structure):
    _fields_ = [("dim", c_int), ("nel", c_int * 2), ("P", c_int), ("M", c_int), ("nodes", c_int),
                ("lo", c_double * 2), ("hi", c_double * 2)]


class sisdc_problem(ctypes.Structure):
    _fields_ = [("pde", c_int), ("ncomp", c_int), ("nu", c_double), ("gamma", c_double),
                ("adv", c_double * 2), ("precision", c_int), ("si_stages", c_int),
                ("cg_rtol", c_double), ("cg_maxit", c_int), ("Nc", c_int), ("use_graph", c_int),
                ("mu", c_double), ("Pr", c_double), ("rho_ref", c_double), ("projection", c_int),
                ("fmg_cycles", c_int), ("form", c_int), ("mixed_levels", c_int),
                ("nu_tilde", c_double)]


class sisdc_stats(ctypes.Structure):
    _fields_ = [("cg_solves", c_ll), ("cg_iters", c_ll), ("cg_max_iters", c_ll), ("cg_noconv", c_ll),
                ("ir_steps", c_ll), ("sweeps", c_ll * 8), ("launches", c_ll)]


class sisdc_ens_instance(ctypes.Structure):
    _fields_ = [("nel", c_int * 2), ("P", c_int), ("nu", c_double), ("adv", c_double * 2), ("dt", c_double)]


class sisdc_ens_opts(ctypes.Structure):
    _fields_ = [("M", c_int), ("Mc", c_int), ("nodes", c_int), ("precision", c_int), ("si_stages", c_int),
                ("cg_rtol", c_double), ("cg_maxit", c_int), ("Nc", c_int), ("ncycles", c_int), ("start", c_int),
                ("post_sweep", c_int), ("use_graph", c_int), ("mixed_levels", c_int)]


class sisdc_stab_opts(ctypes.Structure):
    _fields_ = [("nlevels", c_int), ("M", c_int * 4), ("nodes", c_int), ("si_stages", c_int), ("ncycles", c_int),
                ("start", c_int), ("post_sweep", c_int), ("Nc", c_int), ("fmg_cycles", c_int)]


class SisdcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def header_symbols():
    """Entry points declared in include/sisdc.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:sisdc_status|void|int|const char\*)\s+(sisdc_\w+)\s*\(",
                                 text, flags=re.M)))


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsisdc.so is not built (run paper_2504_18526_gb300/build.py); "
                           "there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "sisdc_create": (c_int, [P(sisdc_problem), c_void_p, P(c_void_p)]),
        "sisdc_destroy": (None, [c_void_p]),
        "sisdc_create_level": (c_int, [c_void_p, P(sisdc_level_desc), P(c_void_p)]),
        "sisdc_set_allocator": (c_int, [c_void_p, ALLOC_FN, RELEASE_FN, c_void_p]),
        "sisdc_set_av": (c_int, [c_void_p, c_double, c_double, c_int]),
        "sisdc_level_info": (c_int, [c_void_p, P(c_int), P(c_ll), P(c_int)]),
        "sisdc_level_coords": (c_int, [c_void_p, c_void_p, c_void_p]),
        "sisdc_level_tables": (c_int, [c_void_p] + [c_void_p] * 5),
        "sisdc_apply_conv": (c_int, [c_void_p, c_void_p, c_void_p]),
        "sisdc_apply_lap": (c_int, [c_void_p, c_void_p, c_void_p]),
        "sisdc_apply_f": (c_int, [c_void_p, c_void_p, c_void_p]),
        "sisdc_solve": (c_int, [c_void_p, c_double, c_void_p, c_void_p, P(c_int)]),
        "sisdc_solve_fds": (c_int, [c_void_p, c_double, c_void_p, c_void_p, P(c_int)]),
        "sisdc_predict": (c_int, [c_void_p, c_void_p, c_void_p, c_double]),
        "sisdc_sweep": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int]),
        "sisdc_residual": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_void_p]),
        "sisdc_transfer": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
        "sisdc_vcycle": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int]),
        "sisdc_step": (c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_int, c_int]),
        "sisdc_sync": (c_int, [c_void_p]),
        "sisdc_get_stats": (c_int, [c_void_p, P(sisdc_stats)]),
        "sisdc_reset_stats": (c_int, [c_void_p]),
        "sisdc_last_error": (ctypes.c_char_p, [c_void_p]),
        "sisdc_set_kernel_timing": (c_int, [c_void_p, c_int, c_int]),
        "sisdc_norms": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "sisdc_mlp_create": (c_int, [c_void_p, c_int, ctypes.c_ulonglong, c_int, P(c_void_p)]),
        "sisdc_mlp_destroy": (None, [c_void_p]),
        "sisdc_mlp_info": (c_int, [c_void_p, P(c_int), P(c_int), P(c_int), P(c_ll)]),
        "sisdc_mlp_params": (c_int, [c_void_p, c_void_p, c_void_p]),
        "sisdc_mlp_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_double, P(c_double), c_void_p]),
        "sisdc_mlp_train": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_double, P(c_double)]),
        "sisdc_mlp_apply": (c_int, [c_void_p, c_void_p, c_double, c_void_p, c_int]),
        "sisdc_mlp_last_error": (ctypes.c_char_p, [c_void_p]),
        "sisdc_mlp_set_tc": (c_int, [c_void_p, c_int]),
        "sisdc_mlp_sync": (c_int, [c_void_p]),
        "sisdc_set_solve_log": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int]),
        "sisdc_get_solve_log_count": (c_int, [c_void_p, P(c_int)]),
        "sisdc_set_learned": (c_int, [c_void_p, c_int, c_void_p]),
        "sisdc_solve_learned": (c_int, [c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_int, P(c_int)]),
        "sisdc_solve_noalloc": (c_int, [P(sisdc_level_desc), c_int, c_double, c_void_p, c_void_p, c_double,
                                        c_int, c_void_p, P(c_int), ctypes.c_char_p, c_int]),
        "sisdc_get_kernel_timing": (c_int, [c_void_p, P(c_double), P(c_ll), P(c_ll), P(c_ll), P(c_ll)]),
        "sisdc_autotune": (c_int, [c_void_p, c_void_p, c_double, c_int, c_void_p]),
        "sisdc_stability": (c_int, [P(sisdc_stab_opts), c_void_p, c_void_p, c_ll, c_void_p]),
        "sisdc_convert": (c_int, [c_int, c_void_p, c_ll, c_void_p, c_void_p]),
        "sisdc_barrier_selftest": (c_int, [c_int, c_int, c_double, c_void_p]),
        "sisdc_level_config": (c_int, [c_void_p, P(c_int), P(c_int), P(c_int)]),
        "sisdc_ens_create": (c_int, [P(sisdc_ens_instance), c_int, P(sisdc_ens_opts), c_void_p, P(c_void_p)]),
        "sisdc_ens_destroy": (None, [c_void_p]),
        "sisdc_ens_layout": (c_int, [c_void_p, c_void_p, P(c_ll)]),
        "sisdc_ens_step": (c_int, [c_void_p, c_void_p, c_int]),
        "sisdc_ens_autotune": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
        "sisdc_ens_config": (c_int, [c_void_p, c_void_p]),
        "sisdc_ens_num_groups": (c_int, [c_void_p]),
        "sisdc_ens_set_tiles": (c_int, [c_void_p, c_int, c_int, c_int, c_int]),
        "sisdc_ens_sync": (c_int, [c_void_p]),
        "sisdc_ens_get_stats": (c_int, [c_void_p, P(sisdc_stats), c_void_p]),
        "sisdc_ens_reset_stats": (c_int, [c_void_p]),
        "sisdc_ens_last_error": (ctypes.c_char_p, [c_void_p]),
        "sisdc_ens_coords": (c_int, [c_void_p, c_void_p, c_void_p]),
        "sisdc_ens_set_kernel_timing": (c_int, [c_void_p, c_int]),
        "sisdc_ens_get_kernel_timing": (c_int, [c_void_p, c_void_p, c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Device address of a torch tensor (float64, contiguous) or an int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if x.dtype.is_floating_point and x.element_size() != 8:
        raise TypeError("expected float64 storage")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _hptr(a):
    """Host address of a numpy float64 array."""
    if a is None:
        return None
    return a.ctypes.data


_LEVEL_CTX = {}


def _check(st, ctx=None, lv=None):
    if st != SISDC_OK:
        ctx = ctx if ctx else _LEVEL_CTX.get(lv)
        msg = load().sisdc_last_error(ctx).decode() if ctx else ""
        raise SisdcError(st, msg)


# ---- entry points (same names as the C ABI) ------------------------------------
def sisdc_create(prob, stream=0):
    out = c_void_p()
    _check(load().sisdc_create(ctypes.byref(prob), c_void_p(stream), ctypes.byref(out)))
    return out.value


def sisdc_destroy(ctx):
    load().sisdc_destroy(ctx)


class TorchAllocator:
    """sisdc_set_allocator callbacks backed by PyTorch's caching allocator, so
    that the level work arrays are part of torch's memory pool.  Keep the
    object alive as long as the context (Context does)."""

    def __init__(self):
        import torch
        self._torch = torch
        self.live = {}

        def _alloc(nbytes, stream, user):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            except Exception:
                return None
            self.live[ptr] = int(nbytes)
            return ptr

        def _release(ptr, nbytes, stream, user):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(_alloc)
        self.release = RELEASE_FN(_release)


def sisdc_set_allocator(ctx, allocator=None):
    """Install an allocator object with .alloc/.release ctypes callbacks
    (e.g. TorchAllocator()), or restore cudaMalloc with None."""
    if allocator is None:
        _check(load().sisdc_set_allocator(ctx, ALLOC_FN(), RELEASE_FN(), None), ctx)
    else:
        _check(load().sisdc_set_allocator(ctx, allocator.alloc, allocator.release, None), ctx)


def sisdc_set_av(ctx, d_s, c_s, comp=0):
    """Persson-Peraire artificial viscosity in f (before the first level)."""
    _check(load().sisdc_set_av(ctx, float(d_s), float(c_s), int(comp)), ctx)


def sisdc_create_level(ctx, desc):
    out = c_void_p()
    _check(load().sisdc_create_level(ctx, ctypes.byref(desc), ctypes.byref(out)), ctx)
    _LEVEL_CTX[out.value] = ctx
    return out.value


def sisdc_level_info(lv):
    nc, n, m = c_int(), c_ll(), c_int()
    _check(load().sisdc_level_info(lv, ctypes.byref(nc), ctypes.byref(n), ctypes.byref(m)))
    return nc.value, n.value, m.value


def sisdc_level_coords(lv, hx, hy=None):
    _check(load().sisdc_level_coords(lv, _hptr(hx), _hptr(hy)))


def sisdc_level_tables(lv, tau=None, wnn=None, gll=None, w=None, D=None):
    _check(load().sisdc_level_tables(lv, _hptr(tau), _hptr(wnn), _hptr(gll), _hptr(w), _hptr(D)))


def sisdc_apply_conv(lv, u, c):
    _check(load().sisdc_apply_conv(lv, _ptr(u), _ptr(c)), lv=lv)


def sisdc_apply_lap(lv, u, Lu):
    _check(load().sisdc_apply_lap(lv, _ptr(u), _ptr(Lu)), lv=lv)


def sisdc_apply_f(lv, u, f):
    _check(load().sisdc_apply_f(lv, _ptr(u), _ptr(f)), lv=lv)


def sisdc_solve(lv, c, rhs, x, want_iters=False):
    it = c_int()
    _check(load().sisdc_solve(lv, c, _ptr(rhs), _ptr(x), ctypes.byref(it) if want_iters else None),
           lv=lv)
    return it.value if want_iters else None


def sisdc_solve_fds(lv, c, rhs, x, want_iters=False):
    it = c_int()
    _check(load().sisdc_solve_fds(lv, c, _ptr(rhs), _ptr(x), ctypes.byref(it) if want_iters else None),
           lv=lv)
    return it.value if want_iters else None


def sisdc_solve_noalloc(desc, ncomp, c, rhs, x, rtol, maxit, stream=0):
    """Solve without any allocation (static scratch); returns the iteration count."""
    it = c_int()
    buf = ctypes.create_string_buffer(256)
    st = load().sisdc_solve_noalloc(ctypes.byref(desc), ncomp, c, _ptr(rhs), _ptr(x), rtol, maxit,
                                    c_void_p(stream), ctypes.byref(it), buf, 256)
    if st != SISDC_OK:
        raise SisdcError(st, buf.value.decode())
    return it.value


def sisdc_predict(lv, u0, U, dt):
    _check(load().sisdc_predict(lv, _ptr(u0), _ptr(U), dt), lv=lv)


def sisdc_sweep(lv, u0, U, g, dt, nsweeps):
    _check(load().sisdc_sweep(lv, _ptr(u0), _ptr(U), _ptr(g), dt, nsweeps), lv=lv)


def sisdc_residual(lv, u0, U, g, dt, r):
    _check(load().sisdc_residual(lv, _ptr(u0), _ptr(U), _ptr(g), dt, _ptr(r)), lv=lv)


def sisdc_transfer(fine, coarse, op, src, dst):
    _check(load().sisdc_transfer(fine, coarse, op, _ptr(src), _ptr(dst)), lv=fine)


def sisdc_vcycle(ctx, u0, U, dt, Nc):
    _check(load().sisdc_vcycle(ctx, _ptr(u0), _ptr(U), dt, Nc), ctx)


def sisdc_step(ctx, u, t, dt, ncycles, start, post_sweep):
    _check(load().sisdc_step(ctx, _ptr(u), t, dt, ncycles, start, 1 if post_sweep else 0), ctx)


def sisdc_norms(lv, u, ref=None):
    """(l2[ncomp], mass[ncomp], maxabs[ncomp]) of u (or of u - ref)."""
    import numpy as np
    nc = sisdc_level_info(lv)[0]
    l2, mass, mx = np.zeros(nc), np.zeros(nc), np.zeros(nc)
    _check(load().sisdc_norms(lv, _ptr(u), _ptr(ref), _hptr(l2), _hptr(mass), _hptr(mx)), lv=lv)
    return l2, mass, mx


def _mcheck(st, mlp):
    if st != SISDC_OK:
        raise SisdcError(st, load().sisdc_mlp_last_error(mlp).decode() if mlp else "")


def sisdc_mlp_create(lv, hidden, seed=0, bf16=1):
    out = c_void_p()
    _check(load().sisdc_mlp_create(lv, hidden, seed, bf16, ctypes.byref(out)), lv=lv)
    return out.value


def sisdc_mlp_destroy(mlp):
    load().sisdc_mlp_destroy(mlp)


def sisdc_mlp_info(mlp):
    a, b, c, d = c_int(), c_int(), c_int(), c_ll()
    _mcheck(load().sisdc_mlp_info(mlp, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), mlp)
    return a.value, b.value, c.value, d.value


def sisdc_mlp_params(mlp, get=None, set_=None):
    _mcheck(load().sisdc_mlp_params(mlp, None if get is None else get.ctypes.data,
                                    None if set_ is None else set_.ctypes.data), mlp)


def sisdc_mlp_loss_grad(mlp, r, dx, c, grad=None):
    l = c_double()
    _mcheck(load().sisdc_mlp_loss_grad(mlp, _ptr(r), _ptr(dx), c, ctypes.byref(l),
                                       None if grad is None else grad.ctypes.data), mlp)
    return l.value


def sisdc_mlp_train(mlp, r, dx, cs, nsolves, epochs, lr):
    import numpy as np
    cs = np.ascontiguousarray(cs, dtype=np.float64)
    l = c_double()
    _mcheck(load().sisdc_mlp_train(mlp, _ptr(r), _ptr(dx), cs.ctypes.data, nsolves, epochs, lr, ctypes.byref(l)),
            mlp)
    return l.value


def sisdc_mlp_apply(mlp, r, c, z, add=False):
    _mcheck(load().sisdc_mlp_apply(mlp, _ptr(r), c, _ptr(z), 1 if add else 0), mlp)


def sisdc_mlp_set_tc(mlp, enable):
    _mcheck(load().sisdc_mlp_set_tc(mlp, 1 if enable else 0), mlp)


def sisdc_mlp_sync(mlp):
    _mcheck(load().sisdc_mlp_sync(mlp), mlp)


def sisdc_set_solve_log(ctx, level, r=None, dx=None, cs=None, capacity=0):
    _check(load().sisdc_set_solve_log(ctx, level, _ptr(r), _ptr(dx), _ptr(cs), capacity), ctx)


def sisdc_set_learned(ctx, level, mlp=None):
    _check(load().sisdc_set_learned(ctx, level, mlp), ctx)


def sisdc_get_solve_log_count(ctx):
    n = c_int()
    _check(load().sisdc_get_solve_log_count(ctx, ctypes.byref(n)), ctx)
    return n.value


def sisdc_solve_learned(lv, mlp, c, rhs, x, mode):
    it = c_int()
    _check(load().sisdc_solve_learned(lv, mlp, c, _ptr(rhs), _ptr(x), mode, ctypes.byref(it)), lv=lv)
    return it.value


def sisdc_sync(ctx):
    _check(load().sisdc_sync(ctx), ctx)


def sisdc_get_stats(ctx):
    s = sisdc_stats()
    _check(load().sisdc_get_stats(ctx, ctypes.byref(s)), ctx)
    return {"cg_solves": s.cg_solves, "cg_iters": s.cg_iters, "cg_max_iters": s.cg_max_iters,
            "cg_noconv": s.cg_noconv, "ir_steps": s.ir_steps, "sweeps": list(s.sweeps),
            "launches": s.launches}


def sisdc_reset_stats(ctx):
    _check(load().sisdc_reset_stats(ctx), ctx)


def sisdc_autotune(ctx, u, dt, nlevels, reps=2):
    """Returns the chosen (elements per tile, blocks, threads per block) per level."""
    import numpy as np
    cfg = np.zeros(3 * nlevels, dtype=np.int32)
    _check(load().sisdc_autotune(ctx, _ptr(u), dt, reps, cfg.ctypes.data), ctx)
    return cfg.reshape(nlevels, 3)


def sisdc_stability(z, Ms, nodes="radau_right", stages=2, ncycles=1, start="predictor", post_sweep=True, Nc=2,
                    fmg_cycles=1, stream=0):
    """R(z) of one SI-MLSDC step on the Dahlquist problem for a complex torch
    tensor z (on the GPU); returns a complex128 tensor."""
    import torch
    o = sisdc_stab_opts()
    o.nlevels = len(Ms)
    for k, M in enumerate(Ms):
        o.M[k] = M
    o.nodes, o.si_stages, o.ncycles = NODE_IDS[nodes], stages, ncycles
    o.start, o.post_sweep, o.Nc, o.fmg_cycles = START_IDS[start], 1 if post_sweep else 0, Nc, fmg_cycles
    zr = torch.view_as_real(z.to(torch.complex128).contiguous()).contiguous()
    R = torch.empty_like(zr)
    st = load().sisdc_stability(ctypes.byref(o), zr.data_ptr(), R.data_ptr(), zr.shape[0], c_void_p(stream))
    if st != SISDC_OK:
        raise SisdcError(st, "sisdc_stability")
    return torch.view_as_complex(R)


def sisdc_convert(kind, x, stream=0):
    """The mixed-precision kernels' integer-pipe format conversions applied to
    a CUDA tensor x: kind 0 float64 -> float32, 1 float32 -> float64, 2
    float64 -> [n, 2] float32 double-single pairs, 3 [n, 2] float32 pairs ->
    float64."""
    import torch
    x = x.contiguous()
    n = x.shape[0]
    out_shape, out_dtype = {0: ((n,), torch.float32), 1: ((n,), torch.float64),
                            2: ((n, 2), torch.float32), 3: ((n,), torch.float64)}[kind]
    out = torch.empty(out_shape, dtype=out_dtype, device=x.device)
    st = load().sisdc_convert(kind, x.data_ptr(), n, out.data_ptr(), c_void_p(stream))
    if st != SISDC_OK:
        raise SisdcError(st, "sisdc_convert")
    return out


def sisdc_level_config(lv):
    e, g, b = c_int(), c_int(), c_int()
    _check(load().sisdc_level_config(lv, ctypes.byref(e), ctypes.byref(g), ctypes.byref(b)), lv=lv)
    return e.value, g.value, b.value


def sisdc_set_kernel_timing(ctx, enable, level=-1):
    _check(load().sisdc_set_kernel_timing(ctx, 1 if enable else 0, level), ctx)


def sisdc_get_kernel_timing(ctx):
    ms, n, it, nxi, ds = c_double(), c_ll(), c_ll(), c_ll(), c_ll()
    _check(load().sisdc_get_kernel_timing(ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(it),
                                          ctypes.byref(nxi), ctypes.byref(ds)), ctx)
    return {"ms": ms.value, "launches": n.value, "iters": it.value, "nodes_x_iters": nxi.value,
            "dof_sweeps": ds.value}


def sisdc_last_error(ctx):
    return load().sisdc_last_error(ctx).decode()


# ---- batched ensemble ------------------------------------------------------------
def _echeck(st, ens):
    if st != SISDC_OK:
        raise SisdcError(st, load().sisdc_ens_last_error(ens).decode() if ens else "")


def sisdc_ens_create(instances, opts, stream=0):
    arr = (sisdc_ens_instance * len(instances))(*instances)
    out = c_void_p()
    _echeck(load().sisdc_ens_create(arr, len(instances), ctypes.byref(opts), c_void_p(stream), ctypes.byref(out)),
            None)
    return out.value


def sisdc_ens_destroy(ens):
    load().sisdc_ens_destroy(ens)


def sisdc_ens_layout(ens, n):
    import numpy as np
    off = np.zeros(n, dtype=np.int64)
    tot = c_ll()
    _echeck(load().sisdc_ens_layout(ens, off.ctypes.data, ctypes.byref(tot)), ens)
    return off, tot.value


def sisdc_ens_coords(ens, hx, hy=None):
    _echeck(load().sisdc_ens_coords(ens, _hptr(hx), _hptr(hy) if hy is not None else None), ens)


def sisdc_ens_set_kernel_timing(ens, enable):
    _echeck(load().sisdc_ens_set_kernel_timing(ens, 1 if enable else 0), ens)


def sisdc_ens_get_kernel_timing(ens):
    """Per group (increasing degree): summed fine correction-launch ms and launch counts."""
    import numpy as np
    ng = sisdc_ens_num_groups(ens)
    ms = np.zeros(ng)
    cnt = np.zeros(ng, dtype=np.int64)
    _echeck(load().sisdc_ens_get_kernel_timing(ens, ms.ctypes.data, cnt.ctypes.data), ens)
    return ms, cnt


def sisdc_ens_step(ens, u, nsteps=1):
    _echeck(load().sisdc_ens_step(ens, _ptr(u), nsteps), ens)


def sisdc_ens_num_groups(ens):
    return load().sisdc_ens_num_groups(ens)


def sisdc_ens_config(ens):
    import numpy as np
    cfg = np.zeros(8 * sisdc_ens_num_groups(ens), dtype=np.int32)
    _echeck(load().sisdc_ens_config(ens, cfg.ctypes.data), ens)
    return cfg.reshape(-1, 4)


def sisdc_ens_autotune(ens, u, nsweeps=1):
    import numpy as np
    cfg = np.zeros(8 * sisdc_ens_num_groups(ens), dtype=np.int32)
    _echeck(load().sisdc_ens_autotune(ens, _ptr(u), nsweeps, cfg.ctypes.data), ens)
    return cfg.reshape(-1, 4)


def sisdc_ens_set_tiles(ens, group, fine, epb, grid):
    _echeck(load().sisdc_ens_set_tiles(ens, group, 1 if fine else 0, epb, grid), ens)


def sisdc_ens_sync(ens):
    _echeck(load().sisdc_ens_sync(ens), ens)


def sisdc_ens_get_stats(ens, n=0):
    import numpy as np
    s = sisdc_stats()
    it = np.zeros(max(n, 1), dtype=np.int64)
    _echeck(load().sisdc_ens_get_stats(ens, ctypes.byref(s), it.ctypes.data if n else None), ens)
    out = {"cg_solves": s.cg_solves, "cg_iters": s.cg_iters, "cg_max_iters": s.cg_max_iters,
           "cg_noconv": s.cg_noconv, "ir_steps": s.ir_steps, "sweeps": list(s.sweeps[:2]),
           "launches": s.launches}
    if n:
        out["inst_iters"] = it
    return out


def sisdc_ens_reset_stats(ens):
    _echeck(load().sisdc_ens_reset_stats(ens), ens)


def sisdc_ens_last_error(ens):
    return load().sisdc_ens_last_error(ens).decode()


def make_ens_instance(d):
    s = sisdc_ens_instance()
    s.nel[0], s.nel[1] = d["nel"]
    s.P = d["P"]
    s.nu = d["nu"]
    s.adv[0], s.adv[1] = d["adv"]
    s.dt = d["dt"]
    return s


def make_ens_opts(M=5, Mc=3, nodes="radau_right", precision=SISDC_FP64, si_stages=2, cg_rtol=1e-12,
                  cg_maxit=1000, Nc=2, ncycles=3, start="cascade", post_sweep=1, use_graph=0, mixed_levels=0):
    o = sisdc_ens_opts()
    o.M, o.Mc, o.nodes, o.precision, o.si_stages = M, Mc, NODE_IDS[nodes], precision, si_stages
    o.cg_rtol, o.cg_maxit, o.Nc, o.ncycles = cg_rtol, cg_maxit, Nc, ncycles
    o.start, o.post_sweep, o.use_graph = START_IDS[start], post_sweep, use_graph
    o.mixed_levels = mixed_levels
    return o


class Ensemble:
    """Owns one ensemble handle built from instance dicts (nel, P, nu, adv, dt)."""

    def __init__(self, instances, stream=0, **kw):
        self.instances = list(instances)
        self.ens = sisdc_ens_create([make_ens_instance(d) for d in self.instances], make_ens_opts(**kw), stream)
        self.offsets, self.total = sisdc_ens_layout(self.ens, len(self.instances))

    def size(self, k):
        d = self.instances[k]
        return d["nel"][0] * d["nel"][1] * (d["P"] + 1) ** 2

    def close(self):
        if self.ens:
            sisdc_ens_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- construction from a workload description (marshalling) -------------------
PDE_IDS = {"convdiff": SISDC_PDE_CONVDIFF, "burgers": SISDC_PDE_BURGERS, "euler": SISDC_PDE_EULER,
           "ns": SISDC_PDE_NS}
NODE_IDS = {"radau_right": SISDC_RADAU_RIGHT, "lobatto": SISDC_LOBATTO}
START_IDS = {"spread": SISDC_START_SPREAD, "predictor": SISDC_START_PREDICTOR,
             "cascade": SISDC_START_CASCADE, "fmg1": SISDC_START_FMG1}


def make_problem(w, precision=SISDC_FP64, si_stages=2, cg_rtol=1e-12, cg_maxit=1000, Nc=2,
                 use_graph=0, projection="interp", fmg_cycles=1, form="incremental",
                 mixed_levels=0, nu_tilde=0.0):
    p = sisdc_problem()
    p.pde = PDE_IDS[w["pde"]]
    p.ncomp = w["ncomp"]
    p.nu = w.get("nu", 0.0)
    p.gamma = w.get("gamma", 1.4)
    adv = w.get("adv", (0.0, 0.0))
    p.adv[0], p.adv[1] = adv[0], adv[1]
    p.precision = precision
    p.si_stages = si_stages
    p.cg_rtol = cg_rtol
    p.cg_maxit = cg_maxit
    p.Nc = Nc
    p.use_graph = use_graph
    p.projection = {"interp": 0, "l2": 1}[projection]
    p.fmg_cycles = fmg_cycles
    p.form = {"incremental": 0, "zero_to_node": 1}[form]
    p.mixed_levels = mixed_levels
    p.nu_tilde = nu_tilde
    if w["pde"] == "ns":
        p.mu = 1.0 / w["Re"]
        p.Pr = w["Pr"]
        p.rho_ref = w.get("rho_ref", 1.0)
    return p


def make_level_desc(w, lvl):
    d = sisdc_level_desc()
    d.dim = w["dim"]
    d.nel[0] = lvl["nel"][0]
    d.nel[1] = lvl["nel"][1] if w["dim"] == 2 else 1
    d.P = lvl["P"]
    d.M = lvl["M"]
    d.nodes = NODE_IDS[w["nodes"]]
    d.lo[0], d.lo[1] = w["lo"][0], w["lo"][1]
    d.hi[0], d.hi[1] = w["hi"][0], w["hi"][1]
    return d


class Context:
    """Owns one sisdc context and its levels (coarse to fine)."""

    def __init__(self, w, stream=0, allocator=None, **kw):
        self.w = w
        self.ctx = sisdc_create(make_problem(w, **kw), stream)
        self.allocator = allocator           # kept alive with the context
        if allocator is not None:
            sisdc_set_allocator(self.ctx, allocator)
        if w.get("av"):                      # artificial viscosity of the workload
            av = w["av"]
            sisdc_set_av(self.ctx, av["kappa"], av["cs"], av.get("comp", 0))
        self.levels = [sisdc_create_level(self.ctx, make_level_desc(w, lv)) for lv in w["levels"]]

    def info(self, l=-1):
        return sisdc_level_info(self.levels[l])

    def close(self):
        if self.ctx:
            sisdc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
