"""Thin ctypes binding of libclaire.so (include/claire.h).

Argument marshalling only: every field operation runs in the library's CUDA
kernels.  Arrays are torch CUDA tensors (float32, contiguous); scalar fields
have shape (n1, n2, n3) and vector fields (3, n1, n2, n3).  There is no CPU
fallback: if the library or a CUDA device is missing the calls raise.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libclaire.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ENOTCONV, ENEGCURV, ELINESEARCH, ETIMEOUT, EORDER = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENONFINITE", "ENOTCONV", "ENEGCURV",
                "ELINESEARCH", "ETIMEOUT", "EORDER"]
OP_L, OP_REG_INV, OP_LERAY_PAR, OP_NEAR_INC, OP_REG_INV_SQRT = 0, 1, 2, 3, 4

EXPORTED = [
    "claire_default_options", "claire_create", "claire_set_options", "claire_get_options",
    "claire_set_beta", "claire_workspace_bytes", "claire_set_images", "claire_transport",
    "claire_objective_gradient", "claire_hessian_matvec", "claire_solve",
    "claire_solve_continuation", "claire_solve_host", "claire_destroy", "claire_last_error",
    "claire_trace", "claire_interp", "claire_grad8", "claire_div8", "claire_spectral",
    "claire_det_deformation_gradient", "claire_profile_reset", "claire_profile_read",
    "claire_transport_noalloc", "claire_autotune", "claire_solve_batch",
    "claire_solve_batch_grouped",
    "claire_conv3d_forward", "claire_conv3d_flip_weights", "claire_conv3d_wgrad",
    "claire_unet_op", "claire_unet_bias_grad", "claire_unet_pack", "claire_unet_mse",
    "claire_unet_adam", "claire_resample", "claire_precondition", "claire_beta_search",
    "claire_wait_status", "claire_wait_selftest", "claire_far_nodes", "claire_set_tuning",
    "claire_get_tuning",
]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("hessian", ctypes.c_int),
                ("beta_w", ctypes.c_double), ("eps_opt", ctypes.c_double),
                ("max_newton", ctypes.c_int), ("max_pcg", ctypes.c_int),
                ("fixed_iters", ctypes.c_int), ("forcing", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("verbose", ctypes.c_int),
                ("gnorm0", ctypes.c_double), ("autotune", ctypes.c_int),
                ("graphs", ctypes.c_int), ("precond", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("distance", ctypes.c_int), ("warm_check", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("pcg_iters", ctypes.c_int),
                ("matvecs", ctypes.c_int), ("pde_solves", ctypes.c_int),
                ("linesearch_halvings", ctypes.c_int),
                ("J0", ctypes.c_double), ("J", ctypes.c_double),
                ("mismatch_rel", ctypes.c_double), ("grad_rel", ctypes.c_double),
                ("gnorm0", ctypes.c_double),
                ("detF_min", ctypes.c_double), ("detF_max", ctypes.c_double),
                ("detF_mean", ctypes.c_double), ("seconds", ctypes.c_double),
                ("status", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("warm_fallback", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong),
                ("timed", ctypes.c_longlong), ("bytes", ctypes.c_double),
                ("ms", ctypes.c_double), ("timed_bytes", ctypes.c_double)]


class ClaireError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 10 else status}: {msg}")


_lib = None


def load_library(path=LIB_PATH):
    """Load libclaire.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libclaire.so not built at {path}; run python -m "
                          "paper_2401_17493_b300.build")
    L = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "claire_default_options": ([ctypes.POINTER(Options)], I),
        "claire_create": ([I, I, I, I, D, D, ctypes.POINTER(P)], I),
        "claire_set_options": ([P, ctypes.POINTER(Options)], I),
        "claire_get_options": ([P, ctypes.POINTER(Options)], I),
        "claire_set_beta": ([P, D], I),
        "claire_workspace_bytes": ([P], S),
        "claire_set_images": ([P, P, P], I),
        "claire_transport": ([P, P, P], I),
        "claire_objective_gradient": ([P, P, ctypes.POINTER(D), P], I),
        "claire_hessian_matvec": ([P, P, P], I),
        "claire_precondition": ([P, P, P, ctypes.POINTER(I)], I),
        "claire_beta_search": ([P, D, D, D, D, I, P, ctypes.POINTER(D), P, P, P, I,
                                ctypes.POINTER(I), ctypes.POINTER(Stats)], I),
        "claire_solve": ([P, P, ctypes.POINTER(Stats)], I),
        "claire_solve_continuation": ([P, ctypes.POINTER(D), I, P, ctypes.POINTER(Stats)], I),
        "claire_solve_host": ([P, P, P, ctypes.POINTER(D), I, P, ctypes.POINTER(Stats)], I),
        "claire_destroy": ([P], I),
        "claire_last_error": ([P], ctypes.c_char_p),
        "claire_trace": ([P, P, P, P], I),
        "claire_interp": ([P, P, P, P], I),
        "claire_grad8": ([P, P, P], I),
        "claire_div8": ([P, P, P], I),
        "claire_spectral": ([P, I, P, P], I),
        "claire_det_deformation_gradient": ([P, P, ctypes.POINTER(D), P], I),
        "claire_profile_reset": ([P, I], I),
        "claire_profile_read": ([P, ctypes.POINTER(KernelStat), I], I),
        "claire_transport_noalloc": ([I, I, I, I, P, P, P, P, ctypes.c_char_p, S], I),
        "claire_autotune": ([P, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "claire_set_tuning": ([P, I, I, I], I),
        "claire_get_tuning": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "claire_solve_batch": ([ctypes.POINTER(P), I, ctypes.POINTER(D), I,
                                ctypes.POINTER(P), ctypes.POINTER(Stats), I], I),
        "claire_solve_batch_grouped": ([ctypes.POINTER(P), I, ctypes.POINTER(D), I,
                                        ctypes.POINTER(P), ctypes.POINTER(Stats), I,
                                        ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_longlong)], I),
        "claire_conv3d_forward": ([P, I, I, I, I, I, P, P, I, I, P, P, P], I),
        "claire_conv3d_flip_weights": ([P, I, I, P, P], I),
        "claire_conv3d_wgrad": ([P, I, I, I, I, I, P, I, P, I, P, P], I),
        "claire_unet_op": ([I, P, P, ctypes.c_longlong, I, I, I, I, I, I, I, P], I),
        "claire_unet_bias_grad": ([P, ctypes.c_longlong, I, P, P, I, P], I),
        "claire_unet_pack": ([ctypes.c_longlong, I, P, ctypes.c_float, I, P, P], I),
        "claire_unet_mse": ([ctypes.c_longlong, I, P, P, ctypes.c_float, P, P, P, I, P, P], I),
        "claire_unet_adam": ([ctypes.c_longlong, P, P, P, P, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, I, P, P], I),
        "claire_resample": ([I, I, I, P, I, I, I, P, I, P], I),
        "claire_wait_status": ([ctypes.POINTER(I)], I),
        "claire_wait_selftest": ([I, I, P], I),
        "claire_far_nodes": ([P, ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_longlong)], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(t, shape=None, what="array"):
    """Device pointer of a contiguous float32 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA torch tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{what} must be contiguous float32")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def solve_batch(contexts, vs=None, betas=None, max_threads=0, grouped=False, wait_us=-1):
    """Solve independent pairs concurrently (claire_solve_batch, or with
    grouped=True claire_solve_batch_grouped: SL / trace / FD8 march launches of
    several pairs combined into one, the first post of a round waiting up to
    wait_us microseconds, < 0: for every unfinished pair).

    contexts: list of Context (images set); vs: list of CUDA (3, n1, n2, n3)
    initial guesses (None: zeros); betas: continuation levels or None.
    Returns (vs, [Stats]) (grouped: (vs, [Stats], (grouped launches, per-pair
    launches they replaced))) and raises on an error status other than
    ENOTCONV / ELINESEARCH."""
    import torch
    L = load_library()
    n = len(contexts)
    if vs is None:
        vs = [torch.zeros(c.vshape, device="cuda") for c in contexts]
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in contexts])
    ps = (ctypes.c_void_p * n)(*[_ptr(v, c.vshape, "v").value for v, c in zip(vs, contexts)])
    stats = (Stats * n)()
    arr = None if betas is None else (ctypes.c_double * len(betas))(*map(float, betas))
    nlev = 0 if betas is None else len(betas)
    launches, ops = ctypes.c_longlong(0), ctypes.c_longlong(0)
    if grouped:
        st = L.claire_solve_batch_grouped(hs, n, arr, nlev, ps, stats, int(wait_us),
                                          ctypes.byref(launches), ctypes.byref(ops))
    else:
        st = L.claire_solve_batch(hs, n, arr, nlev, ps, stats, int(max_threads))
    if st not in (OK, ENOTCONV, ELINESEARCH):
        raise ClaireError(st, "claire_solve_batch failed: " + "; ".join(
            c.lib.claire_last_error(c.h).decode() for c in contexts))
    if grouped:
        return vs, list(stats), (launches.value, ops.value)
    return vs, list(stats)


NOALLOC_MAX_VOXELS = 1 << 20


def transport_noalloc(v, m0, out, nt=4, stream=None):
    """m(1) through claire_transport_noalloc (no device allocation in the library).

    For callers that cannot allocate device memory: the library keeps its
    scratch in a static device array for up to NOALLOC_MAX_VOXELS voxels, shared
    by all calls (serialise overlapping calls).  v (3, n1, n2, n3), m0 and out
    (n1, n2, n3) are caller-owned CUDA float32 tensors."""
    import torch
    L = load_library()
    shape = tuple(m0.shape)
    for t, name in ((v, "v"), (m0, "m0"), (out, "out")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == m0.device):
            raise ValueError(f"{name} must be a CUDA tensor on the device of m0")
    with torch.cuda.device(m0.device):
        if stream is None:
            stream = torch.cuda.current_stream()
        buf = ctypes.create_string_buffer(512)
        st = L.claire_transport_noalloc(*shape, int(nt), _ptr(v, (3,) + shape, "v"),
                                        _ptr(m0, shape, "m0"), _ptr(out, shape, "out"),
                                        ctypes.c_void_p(stream.cuda_stream), buf, 512)
    if st != OK:
        raise ClaireError(st, buf.value.decode())
    return out


class Context:
    """One registration context (grid, nt, beta_v, gamma) owning its workspace."""

    def __init__(self, shape, nt=4, beta_v=1e-2, gamma=1.0, stream=None, **options):
        import torch
        self.lib = load_library()
        self.shape = tuple(int(n) for n in shape)
        self.vshape = (3,) + self.shape
        self.nt = nt
        h = ctypes.c_void_p()
        st = self.lib.claire_create(*self.shape, int(nt), float(beta_v), float(gamma),
                                    ctypes.byref(h))
        if st != OK:
            raise ClaireError(st, "claire_create failed")
        self.h = h
        self.opts = Options()
        self.lib.claire_default_options(ctypes.byref(self.opts))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.opts.stream = ctypes.c_void_p(stream.cuda_stream)
        self.set_options(**options)

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            self.lib.claire_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st != OK:
            raise ClaireError(st, self.lib.claire_last_error(self.h).decode())
        return st

    # -- configuration
    def set_options(self, **kw):
        new = Options()
        ctypes.pointer(new)[0] = self.opts
        for k, v in kw.items():
            if not hasattr(new, k) or k.startswith("_"):
                raise KeyError(k)
            setattr(new, k, v)
        self._check(self.lib.claire_set_options(self.h, ctypes.byref(new)))
        self.opts = new

    def set_beta(self, beta_v):
        self._check(self.lib.claire_set_beta(self.h, float(beta_v)))

    @property
    def workspace_bytes(self):
        return int(self.lib.claire_workspace_bytes(self.h))

    def set_images(self, m0, m1):
        self._check(self.lib.claire_set_images(self.h, _ptr(m0, self.shape, "m0"),
                                               _ptr(m1, self.shape, "m1")))

    # -- operators
    def _new(self, shape):
        import torch
        return torch.empty(shape, device="cuda", dtype=torch.float32)

    def transport(self, v, out=None):
        out = self._new(self.shape) if out is None else out
        self._check(self.lib.claire_transport(self.h, _ptr(v, self.vshape, "v"),
                                              _ptr(out, self.shape, "out")))
        return out

    def objective_gradient(self, v, g=None, want_gradient=True):
        if want_gradient and g is None:
            g = self._new(self.vshape)
        J = ctypes.c_double()
        self._check(self.lib.claire_objective_gradient(
            self.h, _ptr(v, self.vshape, "v"), ctypes.byref(J),
            _ptr(g, self.vshape, "g") if g is not None else None))
        return J.value, g

    def hessian_matvec(self, vt, out=None):
        out = self._new(self.vshape) if out is None else out
        self._check(self.lib.claire_hessian_matvec(self.h, _ptr(vt, self.vshape, "vt"),
                                                   _ptr(out, self.vshape, "Hvt")))
        return out

    def precondition(self, r, out=None):
        """z = M^-1 r with options.precond at the last evaluation; returns (z, inner iterations)."""
        out = self._new(self.vshape) if out is None else out
        its = ctypes.c_int(0)
        self._check(self.lib.claire_precondition(self.h, _ptr(r, self.vshape, "r"),
                                                 _ptr(out, self.vshape, "z"), ctypes.byref(its)))
        return out, its.value

    def beta_search(self, v=None, eps_d=0.1, beta0=1.0, beta_min=1e-8, rtol=0.1, max_bisect=10,
                    max_trials=64):
        """Regularisation-parameter search with det F bounds (Sec. 2.6).

        Returns (beta*, v, trials, stats); trials is a list of (beta, min det F1,
        max det F1); beta* is 0.0 when beta0 already violates the bound."""
        import torch
        v = torch.zeros(self.vshape, device="cuda") if v is None else v
        tb = (ctypes.c_double * max_trials)()
        tmn = (ctypes.c_double * max_trials)()
        tmx = (ctypes.c_double * max_trials)()
        nt = ctypes.c_int(0)
        beta = ctypes.c_double(0.0)
        st = Stats()
        r = self.lib.claire_beta_search(self.h, float(eps_d), float(beta0), float(beta_min),
                                        float(rtol), int(max_bisect), _ptr(v, self.vshape, "v"),
                                        ctypes.byref(beta), tb, tmn, tmx, int(max_trials),
                                        ctypes.byref(nt), ctypes.byref(st))
        self._solve_status(r)
        trials = [(tb[i], tmn[i], tmx[i]) for i in range(min(nt.value, max_trials))]
        return beta.value, v, trials, st

    def _solve_status(self, st):
        if st not in (OK, ENOTCONV, ELINESEARCH):
            self._check(st)
        return st

    def solve(self, v=None):
        import torch
        if v is None:
            v = torch.zeros(self.vshape, device="cuda", dtype=torch.float32)
        stats = Stats()
        st = self.lib.claire_solve(self.h, _ptr(v, self.vshape, "v"), ctypes.byref(stats))
        self._solve_status(st)
        return v, stats

    def solve_continuation(self, betas, v=None):
        import torch
        if v is None:
            v = torch.zeros(self.vshape, device="cuda", dtype=torch.float32)
        arr = (ctypes.c_double * len(betas))(*[float(b) for b in betas])
        stats = Stats()
        st = self.lib.claire_solve_continuation(self.h, arr, len(betas),
                                                _ptr(v, self.vshape, "v"), ctypes.byref(stats))
        self._solve_status(st)
        return v, stats

    def solve_host(self, m0, m1, v, betas=None):
        """m0, m1, v: host torch tensors (float32, contiguous; pinned is fastest).

        betas=None solves at the context's beta_v; a list runs the continuation."""
        for t, nm in ((m0, "m0"), (m1, "m1"), (v, "v")):
            if t.is_cuda or not t.is_contiguous():
                raise TypeError(f"{nm} must be a contiguous host tensor")
        arr = None if betas is None else (ctypes.c_double * len(betas))(*map(float, betas))
        stats = Stats()
        st = self.lib.claire_solve_host(self.h, ctypes.c_void_p(m0.data_ptr()),
                                        ctypes.c_void_p(m1.data_ptr()), arr,
                                        0 if betas is None else len(betas),
                                        ctypes.c_void_p(v.data_ptr()), ctypes.byref(stats))
        self._solve_status(st)
        return v, stats

    # -- single steps
    def trace(self, v):
        df, db = self._new(self.vshape), self._new(self.vshape)
        self._check(self.lib.claire_trace(self.h, _ptr(v, self.vshape, "v"), _ptr(df), _ptr(db)))
        return df, db

    def interp(self, u, d, out=None):
        out = self._new(self.shape) if out is None else out
        self._check(self.lib.claire_interp(self.h, _ptr(u, self.shape, "u"),
                                           _ptr(d, self.vshape, "d"), _ptr(out, self.shape)))
        return out

    def grad8(self, u):
        out = self._new(self.vshape)
        self._check(self.lib.claire_grad8(self.h, _ptr(u, self.shape, "u"), _ptr(out)))
        return out

    def div8(self, w):
        out = self._new(self.shape)
        self._check(self.lib.claire_div8(self.h, _ptr(w, self.vshape, "w"), _ptr(out)))
        return out

    def spectral(self, op, x):
        out = self._new(self.vshape)
        self._check(self.lib.claire_spectral(self.h, int(op), _ptr(x, self.vshape, "x"),
                                             _ptr(out)))
        return out

    def det_deformation_gradient(self, v, want_field=False):
        mmm = (ctypes.c_double * 3)()
        det = self._new(self.shape) if want_field else None
        self._check(self.lib.claire_det_deformation_gradient(
            self.h, _ptr(v, self.vshape, "v"), mmm, _ptr(det) if det is not None else None))
        return (mmm[0], mmm[1], mmm[2]), det

    def autotune(self):
        """Pick the fastest tile shapes for this grid; returns (sl_t1, march_t1)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.claire_autotune(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    # SL gather variants of claire_set_tuning
    GATHER_TMA, GATHER_WINDOW, GATHER_CPASYNC = 0, 1, 2

    def set_tuning(self, sl_gather=0, sl_t1=8, march_t1=32):
        """Fix the tile shapes by hand (the SL gather variant, its x1 depth, the FD8
        march depth)."""
        self._check(self.lib.claire_set_tuning(self.h, sl_gather, sl_t1, march_t1))

    def tuning(self):
        """(sl_gather, sl_t1, march_t1) currently in use."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.claire_get_tuning(self.h, ctypes.byref(a), ctypes.byref(b),
                                               ctypes.byref(c)))
        return a.value, b.value, c.value

    # -- launch accounting
    def far_nodes(self):
        """(forward, backward): nodes whose departure points of the last evaluation
        leave the staged SL brick (interpolated by the global-memory gather)."""
        f, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
        self._check(self.lib.claire_far_nodes(self.h, ctypes.byref(f), ctypes.byref(b)))
        return f.value, b.value

    def profile_reset(self, timing=False):
        self._check(self.lib.claire_profile_reset(self.h, 1 if timing else 0))

    def profile_read(self):
        """{kernel class: dict(launches, timed, bytes, ms, timed_bytes)} since the last reset
        (launches inside captured graphs are counted in launches and bytes, not timed)."""
        n = self.lib.claire_profile_read(self.h, None, 0)
        arr = (KernelStat * n)()
        got = self.lib.claire_profile_read(self.h, arr, n)
        if got < 0:
            raise ClaireError(ECUDA, "claire_profile_read failed")
        return {arr[i].name.decode(): {"launches": arr[i].launches, "timed": arr[i].timed,
                                        "bytes": arr[i].bytes, "ms": arr[i].ms,
                                        "timed_bytes": arr[i].timed_bytes}
                for i in range(got)}


def wait_status():
    """Threads whose bounded tensor-core wait ran out since the last call (their
    outputs are NaN); reads and resets the device counter (synchronises)."""
    L = load_library()
    n = ctypes.c_int(0)
    st = L.claire_wait_status(ctypes.byref(n))
    if st not in (OK, ETIMEOUT):
        raise ClaireError(st, "claire_wait_status failed")
    return n.value


def wait_selftest(max_polls=1000, arrive=False, stream=None):
    """Runs the failure path of the bounded waits on purpose (an mbarrier that
    nothing arrives at unless arrive); returns OK or ETIMEOUT."""
    L = load_library()
    st = L.claire_wait_selftest(int(max_polls), 1 if arrive else 0,
                                ctypes.c_void_p(stream) if stream else None)
    if st not in (OK, ETIMEOUT):
        raise ClaireError(st, "claire_wait_selftest failed")
    return st
