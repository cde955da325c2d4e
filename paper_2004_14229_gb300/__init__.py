"""GB300 fast directional matrix-vector product (Of & Watschinger, Alg. 4).

Thin Python binding of the C ABI in include/dfdm.h: argument marshalling only.
Every step of the product runs in libdfdm.so's CUDA kernels; there is no CPU
fallback, and using a plan without the built library raises.  PyTorch is used
for device memory and streams when the caller passes CUDA tensors.
"""
import ctypes
import os

import numpy as np

__all__ = ["DFDMError", "Plan", "Batch", "Selector", "Problem", "Params", "load_library", "LIB_PATH", "EXPORTED_SYMBOLS",
           "FP64", "TC_FP16X3"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdfdm.so")

FP64 = 0
TC_FP16X3 = 1

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "NUMERIC",
          6: "UNSUPPORTED"}

EXPORTED_SYMBOLS = [
    "dfdm_params_default", "dfdm_plan_create", "dfdm_apply", "dfdm_apply_host",
    "dfdm_plan_check", "dfdm_plan_stats", "dfdm_plan_export_tree",
    "dfdm_plan_export_offsets", "dfdm_plan_destroy", "dfdm_last_error", "dfdm_version",
    "dfdm_plan_set_timing", "dfdm_plan_timing", "dfdm_plan_autotune", "dfdm_direct_rows", "dfdm_direct_rows_noalloc",
    "dfdm_batch_create", "dfdm_batch_apply", "dfdm_batch_check", "dfdm_batch_plan",
    "dfdm_batch_info", "dfdm_batch_destroy",
    "dfdm_selector_param_count", "dfdm_selector_features", "dfdm_selector_forward",
    "dfdm_selector_grad", "dfdm_selector_train", "dfdm_select_params", "dfdm_aca", "dfdm_uniform_counts",
    "dfdm_uniform_offsets",
]


class DFDMError(RuntimeError):
    """A dfdm_* call returned a status other than DFDM_OK."""

    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("max_depth", ctypes.c_int), ("n_max", ctypes.c_int),
                ("eta2", ctypes.c_double), ("l_hf", ctypes.c_int), ("root_mode", ctypes.c_int),
                ("root_lo", ctypes.c_double * 3), ("root_side", ctypes.c_double),
                ("precision", ctypes.c_int), ("nrhs_max", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_targets", ctypes.c_int64), ("n_sources", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("l_hf", ctypes.c_int32),
                ("n_coupling", ctypes.c_int64), ("n_stored_coupling", ctypes.c_int64),
                ("n_near_blocks", ctypes.c_int64), ("nf_entries", ctypes.c_int64),
                ("n_leaves_t", ctypes.c_int64), ("n_leaves_s", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("level_dirs", ctypes.c_int32 * 16),
                ("level_coupling", ctypes.c_int64 * 16), ("level_offsets", ctypes.c_int32 * 16)]


class Problem(ctypes.Structure):
    _fields_ = [("targets", ctypes.c_void_p), ("n_t", ctypes.c_int64), ("sources", ctypes.c_void_p),
                ("n_s", ctypes.c_int64), ("kappa", ctypes.c_double), ("max_depth", ctypes.c_int)]


class Timing(ctypes.Structure):
    _fields_ = [("s2m_ms", ctypes.c_double), ("m2m_ms", ctypes.c_double), ("split_ms", ctypes.c_double),
                ("l2l_ms", ctypes.c_double), ("l2t_ms", ctypes.c_double), ("near_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("m2l_ms", ctypes.c_double * 16), ("launches", ctypes.c_int64),
                ("applies", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("m2l_nsplit", ctypes.c_int * 16), ("p2p_threads", ctypes.c_int), ("p2p_chunks", ctypes.c_int),
                ("rule_ms", ctypes.c_double), ("tuned_ms", ctypes.c_double), ("products", ctypes.c_int),
                ("from_cache", ctypes.c_int)]


_lib = None


def load_library():
    """Load libdfdm.so (built by __graft_entry__.build()); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdfdm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "dfdm_params_default": [ctypes.POINTER(Params)],
        "dfdm_plan_create": [vp, i64, vp, i64, dbl, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)],
        "dfdm_apply": [vp, vp, vp, i32, vp],
        "dfdm_apply_host": [vp, vp, vp, i32, vp],
        "dfdm_plan_check": [vp, vp],
        "dfdm_plan_stats": [vp, ctypes.POINTER(Stats)],
        "dfdm_plan_export_tree": [vp, i32, i32, ctypes.POINTER(i64), vp, vp, vp, vp],
        "dfdm_plan_export_offsets": [vp, i32, i32, ctypes.POINTER(ctypes.c_int32), vp, vp],
        "dfdm_plan_destroy": [vp],
        "dfdm_plan_set_timing": [vp, i32],
        "dfdm_direct_rows": [vp, i64, vp, i64, dbl, vp, vp, i64, vp, vp],
        "dfdm_direct_rows_noalloc": [vp, i64, vp, i64, dbl, vp, vp, i64, vp, vp],
        "dfdm_plan_timing": [vp, ctypes.POINTER(Timing)],
        "dfdm_plan_autotune": [vp, vp, ctypes.c_char_p, vp, ctypes.POINTER(Tuning)],
        "dfdm_batch_create": [i32, ctypes.POINTER(Problem), ctypes.POINTER(Params), i32, vp,
                              ctypes.POINTER(vp)],
        "dfdm_batch_apply": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32, vp],
        "dfdm_batch_check": [vp, vp],
        "dfdm_batch_plan": [vp, i32, ctypes.POINTER(vp)],
        "dfdm_batch_info": [vp, ctypes.POINTER(i32), vp, ctypes.POINTER(i64)],
        "dfdm_batch_destroy": [vp],
        "dfdm_selector_param_count": [],
        "dfdm_selector_features": [dbl, dbl, i32, i64, dbl, vp],
        "dfdm_selector_forward": [vp, vp, i64, vp, vp],
        "dfdm_selector_grad": [vp, vp, vp, i64, vp, vp, vp],
        "dfdm_selector_train": [vp, vp, vp, i64, i32, ctypes.c_float, vp, vp, vp],
        "dfdm_select_params": [vp, dbl, dbl, i64, ctypes.POINTER(Params), vp],
        "dfdm_aca": [vp, i32, i32, dbl, i32, vp, vp, ctypes.POINTER(i32)],
        "dfdm_uniform_counts": [dbl, dbl, dbl, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                ctypes.POINTER(i64)],
        "dfdm_uniform_offsets": [dbl, dbl, dbl, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_int32), vp, vp],
        "dfdm_last_error": [],
        "dfdm_version": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name in ("dfdm_last_error", "dfdm_version") else ctypes.c_int
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise DFDMError(status, load_library().dfdm_last_error().decode())


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def aca(a, tol, max_rank=None):
    """Partially pivoted ACA a ~ U @ V.conj().T of a complex matrix (host
    only, dfdm_aca; Sect. 2.7).  Returns (U (m x k), V (n x k))."""
    lib = load_library()
    a = np.ascontiguousarray(a, dtype=np.complex128)
    m, n = a.shape
    kmax = min(m, n) if max_rank is None else int(max_rank)
    u = np.zeros((m, max(kmax, 1)), dtype=np.complex128)
    v = np.zeros((n, max(kmax, 1)), dtype=np.complex128)
    k = ctypes.c_int(0)
    _check(lib.dfdm_aca(a.ctypes.data, m, n, float(tol), kmax, u.ctypes.data, v.ctypes.data, ctypes.byref(k)))
    return u[:, :k.value].copy(), v[:, :k.value].copy()


def uniform_counts(kappa, depth, eta2=5.0, root_side=1.0, l_hf=None):
    """(N_C, N_SC, nearfield leaf pairs) of Alg. 2 for a uniform tree whose
    every box is occupied (dfdm_uniform_counts; host only, no GPU)."""
    lib = load_library()
    nc, ns, npr = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.dfdm_uniform_counts(float(kappa), float(eta2), float(root_side), int(depth),
                                   -2 if l_hf is None else int(l_hf), ctypes.byref(nc), ctypes.byref(ns),
                                   ctypes.byref(npr)))
    return nc.value, ns.value, npr.value


def uniform_offsets(kappa, depth, level, alpha, eta2=5.0, root_side=1.0, l_hf=None):
    """(offsets (k, 3) int32, direction indices (k,)) of Alg. 2's admissible
    leaves on `level` for targets of parity alpha, for a fully occupied uniform
    tree (dfdm_uniform_offsets; host only)."""
    lib = load_library()
    lh = -2 if l_hf is None else int(l_hf)
    cnt = ctypes.c_int32(0)
    _check(lib.dfdm_uniform_offsets(float(kappa), float(eta2), float(root_side), int(depth), lh, int(level),
                                    int(alpha), ctypes.byref(cnt), None, None))
    off = np.empty((cnt.value, 3), dtype=np.int32)
    dirs = np.empty(cnt.value, dtype=np.int32)
    _check(lib.dfdm_uniform_offsets(float(kappa), float(eta2), float(root_side), int(depth), lh, int(level),
                                    int(alpha), ctypes.byref(cnt), off.ctypes.data, dirs.ctypes.data))
    return off, dirs


def direct_rows(targets, sources, kappa, x, rows, stream=None, y=None, noalloc=False):
    """Rows of the exact product of Eq. (1), FP64 on the GPU (no plan).

    targets, sources: CUDA float64 tensors (N, 3); x: CUDA complex128 (n_s,);
    rows: CUDA int64 (nrows,).  Returns a CUDA complex128 tensor (nrows,)
    (`y` if given).  noalloc=True calls dfdm_direct_rows_noalloc, which uses
    the library's fixed device scratch instead of allocating (nrows <= 2^18).
    """
    import torch
    t = targets.contiguous()
    s = sources.contiguous()
    xx = x.contiguous()
    r = rows.contiguous()
    for name, v, dt in (("targets", t, torch.float64), ("sources", s, torch.float64),
                        ("x", xx, torch.complex128), ("rows", r, torch.int64)):
        if not (v.is_cuda and v.dtype == dt):
            raise TypeError("%s must be a CUDA tensor of dtype %s" % (name, dt))
    if y is None:
        y = torch.empty(r.shape[0], dtype=torch.complex128, device=xx.device)
    lib = load_library()
    fn = lib.dfdm_direct_rows_noalloc if noalloc else lib.dfdm_direct_rows
    _check(fn(ctypes.c_void_p(t.data_ptr()), t.shape[0], ctypes.c_void_p(s.data_ptr()),
              s.shape[0], float(kappa), ctypes.c_void_p(xx.data_ptr()),
              ctypes.c_void_p(r.data_ptr()), r.shape[0], ctypes.c_void_p(y.data_ptr()),
              _stream_handle(stream)))
    return y


def _params(lib, order, max_depth, n_max, eta2, l_hf, root, precision, nrhs_max):
    p = Params()
    _check(lib.dfdm_params_default(ctypes.byref(p)))
    p.order, p.max_depth, p.n_max, p.eta2 = int(order), int(max_depth), int(n_max), float(eta2)
    p.l_hf = -2 if l_hf is None else int(l_hf)
    if isinstance(root, str) and root == "bounding":
        p.root_mode = 1
    else:
        lo, side = root
        p.root_mode = 0
        for i in range(3):
            p.root_lo[i] = float(lo[i])
        p.root_side = float(side)
    p.precision = int(precision)
    p.nrhs_max = int(nrhs_max)
    return p


class Plan:
    """A plan of the fast directional product for fixed P_T, P_S and kappa.

    targets, sources: (N, 3) float64 arrays (host).  order: Chebyshev nodes per
    axis (m + 1).  max_depth / n_max: Alg. 1's refinement (n_max = 0 refines
    every non-empty box to max_depth).  root: (lo[3], side) for an explicit root
    cube, or "bounding" for the smallest dyadic power-of-two cube.  l_hf: None
    for the default rule.  precision: FP64 or TC_FP16X3.
    """

    def __init__(self, targets, sources, kappa, order=5, max_depth=6, n_max=0, eta2=5.0,
                 l_hf=None, root=((0.0, 0.0, 0.0), 1.0), precision=FP64, nrhs_max=1,
                 stream=None):
        lib = load_library()
        self._lib = lib
        self._h = ctypes.c_void_p(0)
        self._owned = True
        t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
        s = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, 3)
        p = _params(lib, order, max_depth, n_max, eta2, l_hf, root, precision, nrhs_max)
        self.precision = int(precision)
        self.n_targets, self.n_sources = t.shape[0], s.shape[0]
        self.nrhs_max = int(nrhs_max)
        _check(lib.dfdm_plan_create(t.ctypes.data, t.shape[0], s.ctypes.data, s.shape[0],
                                    float(kappa), ctypes.byref(p), _stream_handle(stream),
                                    ctypes.byref(self._h)))

    @classmethod
    def _borrowed(cls, lib, handle, n_targets, n_sources, precision, nrhs_max):
        self = cls.__new__(cls)
        self._lib, self._h, self._owned = lib, handle, False
        self.precision, self.n_targets, self.n_sources = precision, n_targets, n_sources
        self.nrhs_max = nrhs_max
        return self

    # -------------------------------------------------------------- apply
    @property
    def complex_dtype(self):
        return np.complex128 if self.precision == FP64 else np.complex64

    def apply(self, x, y=None, stream=None):
        """y = A x for CUDA tensors (torch): x of shape (n_s,) or (nrhs, n_s)."""
        import torch
        tdt = torch.complex128 if self.precision == FP64 else torch.complex64
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == tdt):
            raise TypeError("x must be a CUDA tensor of dtype %s" % tdt)
        x = x.contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        if x.shape[-1] != self.n_sources:
            raise ValueError("x has %d entries per vector, expected %d" % (x.shape[-1], self.n_sources))
        shape = (self.n_targets,) if x.dim() == 1 else (nrhs, self.n_targets)
        if y is None:
            y = torch.empty(shape, dtype=tdt, device=x.device)
        _check(self._lib.dfdm_apply(self._h, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), int(nrhs),
                                    _stream_handle(stream)))
        return y

    def apply_host(self, x, y=None, stream=None):
        """y = A x for host numpy arrays; copies in and out inside the call."""
        x = np.ascontiguousarray(x, dtype=self.complex_dtype)
        nrhs = 1 if x.ndim == 1 else x.shape[0]
        shape = (self.n_targets,) if x.ndim == 1 else (nrhs, self.n_targets)
        if y is None:
            y = np.empty(shape, dtype=self.complex_dtype)
        _check(self._lib.dfdm_apply_host(self._h, x.ctypes.data, y.ctypes.data, int(nrhs),
                                         _stream_handle(stream)))
        return y

    def set_timing(self, enable=True):
        """Record CUDA events around every phase of later applies (no host
        synchronisation; they accumulate until timing() reads them)."""
        _check(self._lib.dfdm_plan_set_timing(self._h, 1 if enable else 0))

    def timing(self):
        """Per-phase device milliseconds summed over the applies since timing
        was turned on or last read (dict; 'applies' counts them)."""
        t = Timing()
        _check(self._lib.dfdm_plan_timing(self._h, ctypes.byref(t)))
        out = {name: (list(getattr(t, name)) if name == "m2l_ms" else getattr(t, name))
               for name, _ in Timing._fields_}
        out["launches"] = int(out["launches"])
        out["applies"] = int(out["applies"])
        return out

    def check(self, stream=None):
        _check(self._lib.dfdm_plan_check(self._h, _stream_handle(stream)))

    def autotune(self, x, cache=None, stream=None):
        """Time candidate launch shapes (M2L chunks per level, nearfield
        blocks) on products of x (one CUDA complex64 right-hand side) and
        keep the fastest (dfdm_plan_autotune); cache: JSON-lines file path or
        None.  Returns the choice as a dict."""
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.complex64):
            raise TypeError("x must be a CUDA complex64 tensor")
        x = x.contiguous()
        if x.dim() != 1 or x.shape[0] != self.n_sources:
            raise ValueError("x must hold one right-hand side of %d entries" % self.n_sources)
        t = Tuning()
        _check(self._lib.dfdm_plan_autotune(self._h, ctypes.c_void_p(x.data_ptr()),
                                            None if cache is None else os.fsencode(cache),
                                            _stream_handle(stream), ctypes.byref(t)))
        return {"m2l_nsplit": list(t.m2l_nsplit), "p2p_threads": t.p2p_threads, "p2p_chunks": t.p2p_chunks,
                "rule_ms": t.rule_ms, "tuned_ms": t.tuned_ms, "products": t.products,
                "from_cache": bool(t.from_cache)}

    # ------------------------------------------------------------ queries
    def stats(self):
        st = Stats()
        _check(self._lib.dfdm_plan_stats(self._h, ctypes.byref(st)))
        out = {}
        for name, _ in Stats._fields_:
            v = getattr(st, name)
            out[name] = list(v) if hasattr(v, "__len__") else int(v)
        return out

    def export_tree(self, which, level, with_perm=False):
        """(keys, begin, end[, perm]) of level `level` of the target (0) or source (1) tree."""
        nb = ctypes.c_int64(0)
        _check(self._lib.dfdm_plan_export_tree(self._h, int(which), int(level), ctypes.byref(nb),
                                               None, None, None, None))
        keys = np.empty(nb.value, dtype=np.int64)
        begin = np.empty(nb.value, dtype=np.int64)
        end = np.empty(nb.value, dtype=np.int64)
        n = self.n_targets if which == 0 else self.n_sources
        perm = np.empty(n, dtype=np.int64) if with_perm else None
        _check(self._lib.dfdm_plan_export_tree(
            self._h, int(which), int(level), ctypes.byref(nb), keys.ctypes.data, begin.ctypes.data,
            end.ctypes.data, perm.ctypes.data if with_perm else None))
        return (keys, begin, end, perm) if with_perm else (keys, begin, end)

    def export_offsets(self, level, alpha):
        """(offsets (k, 3) int32, direction indices (k,)) of Alg. 2's admissible
        leaves on `level` for targets of parity alpha = ax + 2 ay + 4 az."""
        cnt = ctypes.c_int32(0)
        _check(self._lib.dfdm_plan_export_offsets(self._h, int(level), int(alpha),
                                                  ctypes.byref(cnt), None, None))
        off = np.empty((cnt.value, 3), dtype=np.int32)
        dirs = np.empty(cnt.value, dtype=np.int32)
        _check(self._lib.dfdm_plan_export_offsets(self._h, int(level), int(alpha), ctypes.byref(cnt),
                                                  off.ctypes.data, dirs.ctypes.data))
        return off, dirs

    def close(self):
        if self._h and self._owned:
            self._lib.dfdm_plan_destroy(self._h)
        self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Independent problems applied together (dfdm_batch_*): one plan each,
    launches spread over worker streams and replayed from one CUDA graph.

    problems: sequence of dicts with "targets", "sources" ((N, 3) float64
    host arrays), "kappa" and optionally "max_depth".  The other arguments are
    shared by all problems, as in Plan (n_max must be 0).
    """

    def __init__(self, problems, order=5, max_depth=6, eta2=5.0, l_hf=None,
                 root="bounding", precision=TC_FP16X3, nrhs_max=1, nstreams=0, stream=None):
        lib = load_library()
        self._lib = lib
        self._h = ctypes.c_void_p(0)
        self._keep = []
        arr = (Problem * len(problems))()
        for i, pr in enumerate(problems):
            t = np.ascontiguousarray(pr["targets"], dtype=np.float64).reshape(-1, 3)
            s = np.ascontiguousarray(pr["sources"], dtype=np.float64).reshape(-1, 3)
            self._keep += [t, s]
            arr[i].targets, arr[i].n_t = t.ctypes.data, t.shape[0]
            arr[i].sources, arr[i].n_s = s.ctypes.data, s.shape[0]
            arr[i].kappa = float(pr["kappa"])
            arr[i].max_depth = int(pr.get("max_depth", -1))
        p = _params(lib, order, max_depth, 0, eta2, l_hf, root, precision, nrhs_max)
        _check(lib.dfdm_batch_create(len(problems), arr, ctypes.byref(p), int(nstreams),
                                     _stream_handle(stream), ctypes.byref(self._h)))
        self._keep = []
        self.precision, self.nrhs_max = int(precision), int(nrhs_max)
        self.plans = []
        for i, pr in enumerate(problems):
            h = ctypes.c_void_p(0)
            _check(lib.dfdm_batch_plan(self._h, i, ctypes.byref(h)))
            self.plans.append(Plan._borrowed(lib, h, arr[i].n_t, arr[i].n_s, self.precision,
                                             self.nrhs_max))

    def apply(self, xs, ys, stream=None):
        """ys[i] = A_i xs[i] for CUDA tensors (torch) of shape (nrhs, n_s_i) /
        (nrhs, n_t_i), all problems with the same nrhs; ys are overwritten."""
        import torch
        tdt = torch.complex128 if self.precision == FP64 else torch.complex64
        n = len(self.plans)
        if len(xs) != n or len(ys) != n:
            raise ValueError("need one x and one y per problem")
        nrhs = None
        for i, (x, y, pl) in enumerate(zip(xs, ys, self.plans)):
            for name, v, m in (("x", x, pl.n_sources), ("y", y, pl.n_targets)):
                if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == tdt and v.is_contiguous()):
                    raise TypeError("%s[%d] must be a contiguous CUDA tensor of dtype %s" % (name, i, tdt))
                if v.shape[-1] != m:
                    raise ValueError("%s[%d] has %d entries per vector, expected %d" % (name, i, v.shape[-1], m))
            r = 1 if x.dim() == 1 else x.shape[0]
            if nrhs is None:
                nrhs = r
            if r != nrhs or (1 if y.dim() == 1 else y.shape[0]) != nrhs:
                raise ValueError("every problem must have the same nrhs")
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        _check(self._lib.dfdm_batch_apply(self._h, xp, yp, int(nrhs), _stream_handle(stream)))
        return ys

    def check(self, stream=None):
        _check(self._lib.dfdm_batch_check(self._h, _stream_handle(stream)))

    def info(self):
        """(worker streams, stream of each problem, launches in the graph)."""
        ns = ctypes.c_int(0)
        so = np.zeros(len(self.plans), dtype=np.int32)
        nl = ctypes.c_int64(0)
        _check(self._lib.dfdm_batch_info(self._h, ctypes.byref(ns), so.ctypes.data, ctypes.byref(nl)))
        return ns.value, so, nl.value

    def close(self):
        if self._h:
            for pl in self.plans:
                pl.close()
            self._lib.dfdm_batch_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Selector:
    """Learned parameter selector (dfdm_selector_*): a 4 -> 64 -> 64 -> 64 -> 2
    perceptron with FP16 weights, trained and evaluated by the library's GPU
    kernels.  theta: the 8770 parameters (float32)."""

    N_PARAMS = 8770

    def __init__(self, theta):
        self._lib = load_library()
        self.theta = np.ascontiguousarray(theta, dtype=np.float32).reshape(-1)
        if self.theta.size != self._lib.dfdm_selector_param_count():
            raise ValueError("theta must hold %d parameters" % self._lib.dfdm_selector_param_count())

    @staticmethod
    def features(kappa, root_side, level, n_points, tol):
        out = np.empty(4, dtype=np.float32)
        _check(load_library().dfdm_selector_features(float(kappa), float(root_side), int(level),
                                                     int(n_points), float(tol), out.ctypes.data))
        return out

    def forward(self, x, stream=None):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        y = np.empty((x.shape[0], 2), dtype=np.float32)
        _check(self._lib.dfdm_selector_forward(self.theta.ctypes.data, x.ctypes.data, x.shape[0],
                                               y.ctypes.data, _stream_handle(stream)))
        return y

    def grad(self, x, t, stream=None):
        """(loss, gradient) of the mean squared error 1/2 |y - t|^2."""
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        t = np.ascontiguousarray(t, dtype=np.float32).reshape(-1, 2)
        g = np.empty(self.theta.size, dtype=np.float32)
        loss = np.empty(1, dtype=np.float32)
        _check(self._lib.dfdm_selector_grad(self.theta.ctypes.data, x.ctypes.data, t.ctypes.data, x.shape[0],
                                            g.ctypes.data, loss.ctypes.data, _stream_handle(stream)))
        return float(loss[0]), g

    @classmethod
    def train(cls, theta0, x, t, epochs, lr=1e-3, stream=None):
        """Full-batch Adam on the GPU; returns (Selector, losses before each step)."""
        lib = load_library()
        th0 = np.ascontiguousarray(theta0, dtype=np.float32).reshape(-1)
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 4)
        t = np.ascontiguousarray(t, dtype=np.float32).reshape(-1, 2)
        out = np.empty_like(th0)
        losses = np.empty(max(int(epochs), 1), dtype=np.float32)
        _check(lib.dfdm_selector_train(th0.ctypes.data, x.ctypes.data, t.ctypes.data, x.shape[0], int(epochs),
                                       ctypes.c_float(lr), out.ctypes.data, losses.ctypes.data,
                                       _stream_handle(stream)))
        return cls(out), losses[:int(epochs)]

    def select(self, kappa, tol, n_points, max_depth, root_side=1.0, stream=None):
        """(order, l_hf) the network picks for this product (dfdm_select_params)."""
        p = _params(self._lib, 5, max_depth, 0, 5.0, None, ((0.0, 0.0, 0.0), root_side), FP64, 1)
        _check(self._lib.dfdm_select_params(self.theta.ctypes.data, float(kappa), float(tol), int(n_points),
                                            ctypes.byref(p), _stream_handle(stream)))
        return int(p.order), int(p.l_hf)
