"""ctypes binding of libhelm.so (include/helm.h).  Argument marshalling only: every step of the solver
runs in the library's CUDA kernels.  Torch supplies device memory and the current stream.

The module-level functions carry the C names (helm_setup, helm_apply_A, ...); `Solver` wraps a context.
If the library has not been built, every entry point raises instead of falling back to anything else.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "libhelm.so")

HELM_PRECOND_NONE, HELM_PRECOND_EIGT, HELM_PRECOND_PFFT, HELM_PRECOND_FFT2 = 0, 1, 2, 3
HELM_CLOSURE_THREE_POINT, HELM_CLOSURE_HIGH_ORDER = 0, 1
HELM_PREC_FP32, HELM_PREC_TF32, HELM_PREC_TF32X3, HELM_PREC_BF16, HELM_PREC_FP16 = 0, 1, 2, 3, 4
HELM_C64, HELM_C128 = 0, 1

STATUS = {0: "HELM_OK", 1: "HELM_ERR_ARG", 2: "HELM_ERR_CUDA", 3: "HELM_ERR_NOMEM", 4: "HELM_ERR_EIG",
          5: "HELM_ERR_PIVOT", 6: "HELM_ERR_NAN", 7: "HELM_ERR_BREAKDOWN", 8: "HELM_ERR_NOT_CONVERGED",
          9: "HELM_ERR_ITER_LIMIT", 10: "HELM_ERR_UNSUPPORTED"}


class HelmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "%s failed: %s (%d)" % (where, STATUS.get(code, "?"), code)
        if code in (2, 3) and _lib is not None:
            msg += ": " + _lib.helm_last_error().decode(errors="replace")
        super().__init__(msg)


class helm_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("lz", C.c_double), ("staggered", C.c_int)]


class helm_options(C.Structure):
    _fields_ = [("order", C.c_int), ("precond", C.c_int), ("precision", C.c_int), ("restart", C.c_int),
                ("max_iter", C.c_int), ("rtol", C.c_double), ("flexible", C.c_int), ("reorth", C.c_int)]


class helm_solve_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("restarts", C.c_int), ("reserved", C.c_int),
                ("relres_true", C.c_double), ("relres_est", C.c_double), ("beta0", C.c_double),
                ("seconds", C.c_double), ("cycle_its", C.c_int * 16)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("reserved", "cycle_its")}
        d["cycle_its"] = [c for c in self.cycle_its if c]
        return d


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "helm_setup": (C.c_int, [C.POINTER(helm_grid), C.c_void_p, C.c_double, C.c_void_p, C.POINTER(helm_options),
                             C.c_void_p, C.POINTER(C.c_void_p)]),
    "helm_build_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_apply_A": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "helm_set_closure": (C.c_int, [C.c_void_p, C.c_int]),
    "helm_build_rhs_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_closure_face_count": (C.c_longlong, [C.c_void_p]),
    "helm_closure_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_apply_precond": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_precond_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_get_eig": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_gmres_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(helm_solve_info), C.c_void_p]),
    "helm_gmres_solve_batched": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                           C.c_void_p, C.c_void_p]),
    "helm_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "helm_batch_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_batch_destroy": (None, [C.c_void_p]),
    "helm_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.c_void_p]),
    "helm_residual_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.c_void_p]),
    "helm_set_wait_limit": (C.c_int, [C.c_void_p, C.c_longlong]),
    "helm_set_matvec_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "helm_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "helm_profile_classes": (C.c_int, [C.c_void_p, C.c_uint]),
    "helm_profile_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "helm_destroy": (None, [C.c_void_p]),
    "helm_net_create": (C.c_int, [C.c_int, C.c_ulonglong, C.POINTER(C.c_void_p)]),
    "helm_net_destroy": (None, [C.c_void_p]),
    "helm_net_num_params": (C.c_size_t, [C.c_void_p]),
    "helm_net_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "helm_net_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "helm_net_get_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "helm_net_zero_grad": (C.c_int, [C.c_void_p, C.c_void_p]),
    "helm_net_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_void_p]),
    "helm_net_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_net_adam": (C.c_int, [C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, C.c_void_p]),
    "helm_net_mse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "helm_net_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "helm_net_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "helm_net_target": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "helm_attach_net": (C.c_int, [C.c_void_p, C.c_void_p]),
    "helm_status_str": (C.c_char_p, [C.c_int]),
    "helm_version": (C.c_char_p, []),
    "helm_last_error": (C.c_char_p, []),
}


def lib():
    """Load libhelm.so (raises if it was not built: there is no other implementation)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError("libhelm.so not found at %s; build it with __graft_entry__.build()" % library_path)
        L = C.CDLL(library_path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code, where):
    if code != 0:
        raise HelmError(code, where)


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    """Data pointer of a torch tensor (contiguous) or a numpy array (host memory)."""
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return C.c_void_p(t.ctypes.data)
    assert t.is_contiguous()
    return C.c_void_p(t.data_ptr())


def helm_setup(grid, k2, k0, k0z2, options, stream=None):
    ctx = C.c_void_p()
    z = None
    if k0z2 is not None:
        z = np.ascontiguousarray(k0z2, dtype=np.float64)
    code = lib().helm_setup(C.byref(grid), _ptr(k2), float(k0), C.c_void_p(z.ctypes.data) if z is not None else None,
                            C.byref(options), _stream(stream), C.byref(ctx))
    _check(code, "helm_setup")
    return ctx


def helm_build_rhs(ctx, f, F, stream=None):
    _check(lib().helm_build_rhs(ctx, _ptr(f), _ptr(F), _stream(stream)), "helm_build_rhs")


def helm_apply_A(ctx, x, y, dtype, stream=None):
    _check(lib().helm_apply_A(ctx, _ptr(x), _ptr(y), int(dtype), _stream(stream)), "helm_apply_A")


def helm_set_closure(ctx, closure):
    _check(lib().helm_set_closure(ctx, int(closure)), "helm_set_closure")


def helm_build_rhs_fields(ctx, fields, F, stream=None):
    _check(lib().helm_build_rhs_fields(ctx, _ptr(fields), _ptr(F), _stream(stream)), "helm_build_rhs_fields")


def helm_closure_face_count(ctx):
    return int(lib().helm_closure_face_count(ctx))


def helm_closure_rhs(ctx, faces, F_in, F_out, stream=None):
    _check(lib().helm_closure_rhs(ctx, _ptr(faces), _ptr(F_in), _ptr(F_out), _stream(stream)), "helm_closure_rhs")


def helm_apply_precond(ctx, r, z, stream=None):
    _check(lib().helm_apply_precond(ctx, _ptr(r), _ptr(z), _stream(stream)), "helm_apply_precond")


def helm_precond_step(ctx, step, x, y, stream=None):
    _check(lib().helm_precond_step(ctx, int(step), _ptr(x), _ptr(y), _stream(stream)), "helm_precond_step")


def helm_get_eig(ctx, axis, n):
    D = np.zeros(n, np.complex128)
    V = np.zeros((n, n), np.complex128)
    Vi = np.zeros((n, n), np.complex128)
    _check(lib().helm_get_eig(ctx, int(axis), _ptr(D), _ptr(V), _ptr(Vi)), "helm_get_eig")
    return D, V, Vi


def helm_gmres_solve(ctx, b, x, stream=None):
    info = helm_solve_info()
    code = lib().helm_gmres_solve(ctx, _ptr(b), _ptr(x), C.byref(info), _stream(stream))
    return code, info


def helm_gmres_solve_batched(ctxs, bs, xs, nrhs, stream=None):
    """Batched solve (include/helm.h): bs[p], xs[p] complex128 device tensors [nrhs][nz][ny][nx].
    Returns (status, [helm_solve_info per (problem, rhs), problem-major])."""
    n = len(ctxs)
    carr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    barr = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xarr = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    infos = (helm_solve_info * (n * nrhs))()
    code = lib().helm_gmres_solve_batched(carr, n, barr, xarr, int(nrhs), infos, _stream(stream))
    return code, list(infos)


class Batch:
    """A batch plan (helm_batch_*): solvers[p] with right-hand sides bs[p] and iterates xs[p]
    (complex128 device tensors [nrhs][nz][ny][nx] whose addresses stay fixed)."""

    def __init__(self, solvers, bs, xs, stream=None):
        self.solvers, self.bs, self.xs = list(solvers), list(bs), list(xs)
        self.nrhs = int(bs[0].shape[0])
        n = len(self.solvers)
        carr = (C.c_void_p * n)(*[S.ctx.value for S in self.solvers])
        barr = (C.c_void_p * n)(*[b.data_ptr() for b in self.bs])
        xarr = (C.c_void_p * n)(*[x.data_ptr() for x in self.xs])
        h = C.c_void_p()
        _check(lib().helm_batch_create(carr, n, barr, xarr, self.nrhs, _stream(stream), C.byref(h)),
               "helm_batch_create")
        self.h = h

    def run(self, stream=None):
        """Returns (status, infos[p][r])."""
        n = len(self.solvers)
        infos = (helm_solve_info * (n * self.nrhs))()
        code = lib().helm_batch_run(self.h, infos, _stream(stream))
        if code not in (0, 8):
            raise HelmError(code, "helm_batch_run")
        flat = list(infos)
        return code, [flat[p * self.nrhs:(p + 1) * self.nrhs] for p in range(n)]

    def close(self):
        if getattr(self, "h", None):
            lib().helm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def helm_autotune(ctx, stream=None):
    """(CTA count of the Arnoldi update, matvec variant, inner-product variant) chosen for the context."""
    nb = C.c_int()
    var = C.c_int()
    dv = C.c_int()
    _check(lib().helm_autotune(ctx, C.byref(nb), C.byref(var), C.byref(dv), _stream(stream)), "helm_autotune")
    return nb.value, var.value, dv.value


def helm_residual(ctx, b, x, r=None, stream=None):
    n2 = C.c_double()
    ni = C.c_double()
    _check(lib().helm_residual(ctx, _ptr(b), _ptr(x), _ptr(r) if r is not None else None, C.byref(n2), C.byref(ni),
                               _stream(stream)), "helm_residual")
    return n2.value, ni.value


def helm_residual_noalloc(ctx, b, x, r, stream=None):
    """Allocation-free residual (see include/helm.h); returns (status, ||r||_2, ||r||_inf)."""
    n2 = C.c_double()
    ni = C.c_double()
    code = lib().helm_residual_noalloc(ctx, _ptr(b), _ptr(x), _ptr(r), C.byref(n2), C.byref(ni), _stream(stream))
    return code, n2.value, ni.value


def helm_set_wait_limit(ctx, polls):
    _check(lib().helm_set_wait_limit(ctx, int(polls)), "helm_set_wait_limit")


def helm_set_matvec_variant(ctx, variant):
    _check(lib().helm_set_matvec_variant(ctx, int(variant)), "helm_set_matvec_variant")


def helm_destroy(ctx):
    if ctx:
        lib().helm_destroy(ctx)


class Net:
    """The learned-correction network (include/helm.h, helm_net_*); parameters live on the device."""

    # per layer (name, Cout, Cin) for width c, in the library's parameter order
    @staticmethod
    def layers(width):
        c = width
        return [("c1", c, 5), ("c2", c, c), ("c3", 2 * c, c), ("c4", 2 * c, 2 * c), ("c5", c, 3 * c), ("c6", 2, c)]

    def __init__(self, width=8, seed=0):
        self.width = width
        h = C.c_void_p()
        _check(lib().helm_net_create(int(width), C.c_ulonglong(seed), C.byref(h)), "helm_net_create")
        self.h = h
        self.nparam = lib().helm_net_num_params(h)
        self.step = 0

    def close(self):
        if self.h:
            lib().helm_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        a = np.zeros(self.nparam, np.float32)
        _check(lib().helm_net_get_params(self.h, _ptr(a), a.size), "helm_net_get_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        _check(lib().helm_net_set_params(self.h, _ptr(a), a.size), "helm_net_set_params")

    def get_grads(self):
        a = np.zeros(self.nparam, np.float32)
        _check(lib().helm_net_get_grads(self.h, _ptr(a), a.size), "helm_net_get_grads")
        return a

    def unflatten(self, a):
        """{name.w: [Cout][Cin][3][3][3], name.b: [Cout]} views of a flat parameter array."""
        out, off = {}, 0
        for name, co, ci in self.layers(self.width):
            nw = co * ci * 27
            out[name + ".w"] = a[off:off + nw].reshape(co, ci, 3, 3, 3)
            off += nw
            out[name + ".b"] = a[off:off + co]
            off += co
        return out

    def flatten(self, d):
        parts = []
        for name, co, ci in self.layers(self.width):
            parts += [np.asarray(d[name + ".w"], np.float32).ravel(), np.asarray(d[name + ".b"], np.float32).ravel()]
        return np.concatenate(parts)

    def zero_grad(self, stream=None):
        _check(lib().helm_net_zero_grad(self.h, _stream(stream)), "helm_net_zero_grad")

    def forward(self, x, stream=None):
        """x: bfloat16 device tensor [B][5][Z][Y][X] -> float32 [B][2][Z][Y][X]."""
        import torch
        B, _, Z, Y, X = x.shape
        y = torch.empty((B, 2, Z, Y, X), dtype=torch.float32, device=x.device)
        _check(lib().helm_net_forward(self.h, _ptr(x), _ptr(y), B, Z, Y, X, _stream(stream)), "helm_net_forward")
        return y

    def backward(self, gy, stream=None):
        _check(lib().helm_net_backward(self.h, _ptr(gy), _stream(stream)), "helm_net_backward")

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.step += 1
        _check(lib().helm_net_adam(self.h, lr, beta1, beta2, eps, self.step, _stream(stream)), "helm_net_adam")

    def stats(self):
        """[sum|v|^2, sum|M^-1 v|^2, |alpha|, dropped, applied, sum of residual-reduction ratios]."""
        a = np.zeros(6, np.float64)
        _check(lib().helm_net_stats(self.h, _ptr(a)), "helm_net_stats")
        return a


def helm_net_mse(y, t, gy, loss, stream=None):
    """loss (device float64, 1 entry) += 0.5 mean((y-t)^2); gy = (y-t)/count."""
    _check(lib().helm_net_mse(_ptr(y), _ptr(t), _ptr(gy), y.numel(), _ptr(loss), _stream(stream)), "helm_net_mse")


def solve_batched(solvers, bs, x0s=None, stream=None):
    """Solve every solver's right-hand sides bs[p] (complex128 device [nrhs][nz][ny][nx], same nrhs for all)
    in one batched call; returns (xs, infos) with infos[p][r]."""
    import torch
    nrhs = bs[0].shape[0]
    xs = [torch.zeros_like(b) if x0s is None else x0s[p] for p, b in enumerate(bs)]
    code, infos = helm_gmres_solve_batched([S.ctx for S in solvers], bs, xs, nrhs, stream)
    if code not in (0, 8):
        raise HelmError(code, "helm_gmres_solve_batched")
    return xs, [infos[p * nrhs:(p + 1) * nrhs] for p in range(len(solvers))]


class Solver:
    """One problem: grid, k^2 samples (complex128, host numpy or torch tensor), background k0, options.
    staggered=False selects the collocated grid with the three-point ABC closure (EigT only)."""

    def __init__(self, n, k2, k0, order=4, L=(1.0, 1.0, 1.0), precond=HELM_PRECOND_EIGT, precision=HELM_PREC_FP32,
                 restart=30, max_iter=300, rtol=1e-6, flexible=False, reorth=False, k0z2=None, stream=None,
                 staggered=True):
        nx, ny, nz = n
        self.shape = (nz, ny, nx)
        self.n = (nx, ny, nz)
        self.grid = helm_grid(nx, ny, nz, L[0], L[1], L[2], int(bool(staggered)))
        self.options = helm_options(order, precond, precision, restart, max_iter, rtol, int(flexible), int(reorth))
        if isinstance(k2, np.ndarray):
            k2 = np.ascontiguousarray(k2, dtype=np.complex128)
        self.ctx = helm_setup(self.grid, k2, k0, k0z2, self.options, stream)

    def close(self):
        if self.ctx:
            helm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # torch conveniences
    def _empty(self, dtype):
        import torch
        return torch.empty(self.shape, dtype=dtype, device="cuda")

    def build_rhs(self, f, stream=None):
        import torch
        F = self._empty(torch.complex128)
        helm_build_rhs(self.ctx, f, F, stream)
        return F

    def set_closure(self, closure):
        """Collocated grids: HELM_CLOSURE_THREE_POINT (default) or HELM_CLOSURE_HIGH_ORDER for the operator."""
        helm_set_closure(self.ctx, closure)

    def build_rhs_fields(self, fields, stream=None):
        """F of the scheme from caller-known fields (complex128 device tensor; layout in helm.h)."""
        import torch
        F = self._empty(torch.complex128)
        helm_build_rhs_fields(self.ctx, fields, F, stream)
        return F

    def closure_face_count(self):
        return helm_closure_face_count(self.ctx)

    def closure_rhs(self, faces, F, stream=None):
        """F - A(G_f): the f part of the high-order closure moved to the right-hand side."""
        import torch
        out = self._empty(torch.complex128)
        helm_closure_rhs(self.ctx, faces, F, out, stream)
        return out

    def apply_A(self, x, stream=None):
        import torch
        y = self._empty(x.dtype)
        helm_apply_A(self.ctx, x, y, HELM_C64 if x.dtype == torch.complex64 else HELM_C128, stream)
        return y

    def apply_precond(self, r, stream=None):
        import torch
        z = self._empty(torch.complex64)
        helm_apply_precond(self.ctx, r, z, stream)
        return z

    def precond_step(self, step, x, stream=None):
        import torch
        y = self._empty(torch.complex64)
        helm_precond_step(self.ctx, step, x, y, stream)
        return y

    def autotune(self, stream=None):
        """Pick the Arnoldi kernels' CTA count and the matvec and inner-product variants for this grid by
        timing (cached per grid size and order); returns (CTA count, matvec variant, inner-product variant)."""
        return helm_autotune(self.ctx, stream)

    def features(self, net, v, mv, stream=None):
        """The net's 5 input channels (bfloat16 [5][nz][ny][nx]) for complex64 v and mv = M^-1 v."""
        import torch
        x = torch.empty((5,) + self.shape, dtype=torch.bfloat16, device=v.device)
        _check(lib().helm_net_features(self.ctx, net.h, _ptr(v), _ptr(mv), _ptr(x), _stream(stream)),
               "helm_net_features")
        return x

    def target(self, net, xs, xk, mv, stream=None):
        """Training target (float32 [2][nz][ny][nx]) for v = b - A xk with A^-1 v = xs - xk, mv = M^-1 v."""
        import torch
        t = torch.empty((2,) + self.shape, dtype=torch.float32, device=mv.device)
        _check(lib().helm_net_target(self.ctx, net.h, _ptr(xs), _ptr(xk), _ptr(mv), _ptr(t), _stream(stream)),
               "helm_net_target")
        return t

    def attach(self, net):
        """Apply `net` after M^-1 (flexible contexts); None detaches.  The caller keeps `net` alive."""
        _check(lib().helm_attach_net(self.ctx, net.h if net is not None else None), "helm_attach_net")
        self.net = net

    def residual(self, b, x, stream=None):
        """(||b - A x||_2, ||b - A x||_inf) with complex128 device b, x."""
        return helm_residual(self.ctx, b, x, None, stream)

    def get_eig(self, axis):
        return helm_get_eig(self.ctx, axis, self.n[axis])

    def set_wait_limit(self, polls):
        """Bound of the context's mbarrier waits in polls (0 = default); a diagnosis and test hook."""
        helm_set_wait_limit(self.ctx, polls)

    def set_matvec_variant(self, variant):
        """Pin the complex64 matvec kernel (0-4, include/helm.h); helm_autotune would pick the fastest."""
        helm_set_matvec_variant(self.ctx, variant)

    def solve(self, b, x0=None, stream=None, check=True):
        """x such that A x = b (b complex128 on the device or in host memory)."""
        import torch
        if x0 is None:
            if isinstance(b, np.ndarray):
                x = np.zeros(self.shape, np.complex128)
            else:
                x = torch.zeros(self.shape, dtype=torch.complex128, device=b.device)
        else:
            x = x0
        code, info = helm_gmres_solve(self.ctx, b, x, stream)
        if check and code not in (0,):
            raise HelmError(code, "helm_gmres_solve")
        return x, info
