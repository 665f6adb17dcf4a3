"""Python binding of libgp (the C ABI in include/gp.h).

Argument marshalling only: tensors are checked (device, dtype, layout) and
their data pointers handed to the C entry points of the same names; every
step of the computation runs in the library's CUDA kernels.  PyTorch provides
the device memory and the stream.

The library must have been built (``paper_1203_1269_gb300.build.build()``);
if it is missing, importing functions from here raises -- there is no CPU or
PyTorch fallback.
"""
import ctypes
import os
import sys

import torch

from . import build as _build

GP_FP64, GP_MIXED, GP_FP32, GP_AUTO = 0, 1, 2, 3
PRECISIONS = {"fp64": GP_FP64, "mixed": GP_MIXED, "fp32": GP_FP32, "auto": GP_AUTO}
PRECISION_NAMES = {v: k for k, v in PRECISIONS.items()}
# gp_correlation: eq. (2)'s power-exponential family and the Matern family
CORRELATIONS = {"powexp": 0, "matern12": 1, "matern32": 2, "matern52": 3}
# gp_call: the calls whose device memory gp_call_bytes reports
CALLS = {"nll_batch": 0, "nll_grad": 1, "fit": 2, "predict": 3}
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ENOTPD", -4: "ECUDA", -5: "ETIMEOUT",
          -6: "EDEGENERATE", -7: "ENOTSUP"}
GP_OK, GP_EINVAL, GP_ENOMEM, GP_ENOTPD, GP_ECUDA, GP_ETIMEOUT, GP_EDEGENERATE, GP_ENOTSUP = \
    0, -1, -2, -3, -4, -5, -6, -7

_c_int, _c_double, _c_size, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p


class GPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("slices", _c_int), ("panel_slices", _c_int), ("refine_iters", _c_int),
                ("nugget_in_var", _c_int), ("max_batch", _c_int), ("update_groups", _c_int),
                ("inject_timeout", _c_int), ("fuse_panels", _c_int), ("auto_tol", _c_double),
                ("update_tile", _c_int), ("assemble_cols", _c_int), ("correlation", _c_int),
                ("predict_tc", _c_int)]


class TuneTrial(ctypes.Structure):
    _fields_ = [("update_tile", _c_int), ("fuse_panels", _c_int), ("assemble_cols", _c_int),
                ("ms", _c_double)]


_lib = None


def library_path():
    return _build.LIB


def load(path=None):
    """Load libgp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libgp.so not found at {path}: build it with "
                           "paper_1203_1269_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(path)
    P = _vp
    lib.gp_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.gp_create.argtypes = [ctypes.POINTER(P), _c_int, _c_size, P]
    lib.gp_destroy.argtypes = [P]
    lib.gp_destroy.restype = None
    lib.gp_last_error.argtypes = [P]
    lib.gp_last_error.restype = ctypes.c_char_p
    lib.gp_set_stream.argtypes = [P, P]
    lib.gp_set_options.argtypes = [P, ctypes.POINTER(Options)]
    lib.gp_get_options.argtypes = [P, ctypes.POINTER(Options)]
    lib.gp_workspace_bytes.argtypes = [P]
    lib.gp_workspace_bytes.restype = _c_size
    lib.gp_set_timing.argtypes = [P, _c_int]
    lib.gp_phase_times.argtypes = [P, ctypes.POINTER(_c_double), ctypes.POINTER(ctypes.c_longlong),
                                   _c_int]
    lib.gp_launch_count.argtypes = [P]
    lib.gp_launch_count.restype = ctypes.c_longlong
    lib.gp_corr_assemble.argtypes = [P, _c_int, _c_int, P, P, _c_double, _c_double, P, _c_int]
    lib.gp_cholesky.argtypes = [P, _c_int, _c_int, P, P, _c_double, _c_double, _c_int, P,
                                ctypes.POINTER(_c_int)]
    lib.gp_nll_batch.argtypes = [P, _c_int, _c_int, P, P, _c_int, P, _c_double, _c_double, _c_int,
                                 P, P, P, P, P]
    lib.gp_nll_batch_ex.argtypes = lib.gp_nll_batch.argtypes + [P, P]
    lib.gp_nll_grad_batch.argtypes = [P, _c_int, _c_int, P, P, _c_int, P, _c_double, _c_double, P, P, P]
    lib.gp_nll_batch_host.argtypes = lib.gp_nll_batch.argtypes
    lib.gp_plan_nll_batch.argtypes = lib.gp_nll_batch.argtypes + [P, ctypes.POINTER(P)]
    lib.gp_autotune.argtypes = [P, _c_int, _c_int, P, P, _c_int, P, _c_double, _c_double, _c_int, _c_int,
                                ctypes.POINTER(TuneTrial), _c_int, ctypes.POINTER(_c_int)]
    lib.gp_plan_launch.argtypes = [P]
    lib.gp_plan_kernels.argtypes = [P]
    lib.gp_plan_kernels.restype = ctypes.c_longlong
    lib.gp_plan_bytes.argtypes = [P]
    lib.gp_plan_bytes.restype = _c_size
    lib.gp_plan_destroy.argtypes = [P]
    lib.gp_plan_destroy.restype = None
    lib.gp_nll_batch_noalloc.argtypes = [P, _c_int, _c_int, P, P, _c_int, P, _c_double, _c_double,
                                         P, P, P, P, P]
    lib.gp_fit.argtypes = [P, _c_int, _c_int, P, P, P, _c_double, _c_double, _c_int,
                           ctypes.POINTER(P)]
    lib.gp_fit_batch.argtypes = [P, _c_int, _c_int, P, P, _c_int, P, _c_double, _c_double, _c_int,
                                 P, P, P, P, P, ctypes.POINTER(_c_int), ctypes.POINTER(P)]
    lib.gp_model_scalars.argtypes = [P, ctypes.POINTER(_c_double)]
    lib.gp_predict.argtypes = [P, P, _c_int, P, P, P]
    lib.gp_model_free.argtypes = [P]
    lib.gp_model_free.restype = None
    lib.gp_model_bytes.argtypes = [P]
    lib.gp_model_bytes.restype = _c_size
    lib.gp_call_bytes.argtypes = [P, _c_int, _c_int, _c_int, _c_int, _c_int, ctypes.POINTER(_c_size)]
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def call_bytes(call, n, d, count=1, prec="mixed", ctx=None):
    """Device bytes a call would allocate (gp_call_bytes): the workspace of
    "nll_batch" (count = T, at precision prec), "nll_grad" (count = T) or
    "predict" (count = N, with variances; n, d of the model), or the model of
    "fit".  Host arithmetic only, so it needs no GPU; ctx=None sizes with the
    default options and no budget limit."""
    lib = ctx._lib if ctx is not None else load()
    h = ctx._h if ctx is not None else None
    out = _c_size()
    rc = lib.gp_call_bytes(h, CALLS[call], int(n), int(d), int(count), _prec(prec), ctypes.byref(out))
    if rc != 0:
        msg = lib.gp_last_error(h).decode() if h is not None else "gp_call_bytes"
        raise GPError(rc, msg)
    return int(out.value)


def _dev_f64(t, name, shape=None, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the context uses {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _out_tensor(t, name, shape, dtype, device):
    """A caller-supplied output: the library writes prod(shape) elements of
    `dtype` through its pointer, so everything about it is checked first.
    device=None means a host (CPU) tensor."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"out[{name!r}] must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"out[{name!r}] must be {dtype}, got {t.dtype}")
    if device is None:
        if t.is_cuda:
            raise ValueError(f"out[{name!r}] must be a CPU tensor")
    elif t.device != device:
        raise ValueError(f"out[{name!r}] is on {t.device}, the context uses {device}")
    if not t.is_contiguous():
        raise ValueError(f"out[{name!r}] must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"out[{name!r}] has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


_INT_OUTPUTS = ("status", "prec_used")


def _check_outs(out, required, optional, T, device, shapes=None):
    """Validate a caller's `out` dict: the `required` keys must be there, the
    `optional` ones may be; each is (T,) (or shapes[key]) of int32 for the
    status-like keys and float64 otherwise."""
    if not isinstance(out, dict):
        raise TypeError("out must be a dict of tensors")
    for k in required:
        if out.get(k) is None:
            raise ValueError(f"out lacks {k!r}")
    for k in tuple(required) + tuple(optional):
        if out.get(k) is not None:
            dtype = torch.int32 if k in _INT_OUTPUTS else torch.float64
            _out_tensor(out[k], k, (shapes or {}).get(k, (T,)), dtype, device)
    return out


def _host_batch_args(x, y, thetas):
    """(n, d, T) of a host-buffer batch after checking x (n x d), y (n) and
    thetas (T x d): the library copies exactly those bytes from them."""
    def host(t, name):
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU torch.float64 tensor")
        return t
    host(x, "x"); host(y, "y"); host(thetas, "thetas")
    if x.dim() != 2:
        raise ValueError("x must be n x d")
    n, d = x.shape
    if tuple(y.shape) != (n,):
        raise ValueError(f"y has shape {tuple(y.shape)}, expected {(n,)}")
    if thetas.dim() != 2 or thetas.shape[1] != d:
        raise ValueError("thetas must be T x d")
    return n, d, thetas.shape[0]


def _prec(prec):
    if isinstance(prec, str):
        return PRECISIONS[prec]
    return int(prec)


def packed_elems(n, nb=128):
    """Doubles in the tile storage of an n x n R (lower tiles, 128 x 128)."""
    nt = (n + nb - 1) // nb
    return nt * (nt + 1) // 2 * nb * nb


class Model:
    """A resident fit (device factor and weights) owned by libgp."""

    def __init__(self, ctx, handle, n, d):
        self._ctx = ctx
        self._h = handle
        self.n, self.d = n, d
        out = (_c_double * 6)()
        ctx._lib.gp_model_scalars(handle, out)
        self.nll, self.mu, self.sigma2, self.logdet, self.Q, self.aa = list(out)
        self.bytes = int(ctx._lib.gp_model_bytes(handle))

    def free(self):
        if self._h:
            self._ctx._lib.gp_model_free(self._h)
            self._h = None

    def __del__(self):
        # at interpreter shutdown the CUDA runtime may already be gone
        if sys.is_finalizing():
            return
        try:
            self.free()
        except Exception:
            pass


class Plan:
    """A gp_nll_batch call recorded as one CUDA graph (gp_plan_nll_batch).
    launch() replays it: it re-reads the bound x, y and thetas tensors and
    overwrites `out`.  Keep those tensors alive while the plan lives."""

    def __init__(self, ctx, handle, inputs, out):
        self._ctx = ctx
        self._h = handle
        self._keep = inputs           # the bound tensors stay referenced
        self.out = out
        self.kernels = int(ctx._lib.gp_plan_kernels(handle))
        self.bytes = int(ctx._lib.gp_plan_bytes(handle))

    def launch(self):
        self._ctx._check(self._ctx._lib.gp_plan_launch(self._h))
        return self.out

    def free(self):
        if self._h:
            self._ctx._lib.gp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A libgp context on one CUDA device, enqueuing on a torch stream."""

    def __init__(self, device=0, hbm_budget_bytes=0, stream=None, **options):
        self._lib = load()
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = _vp()
        rc = self._lib.gp_create(ctypes.byref(h), device, int(hbm_budget_bytes),
                                 _vp(stream.cuda_stream))
        if rc != 0:
            raise GPError(rc, "gp_create failed")
        self._h = h
        opt = Options()
        self._lib.gp_default_options(ctypes.byref(opt))
        self._opt = opt
        if options:
            self.set_options(**options)

    # -- plumbing ----------------------------------------------------------
    def _check(self, rc):
        if rc not in (0,):
            raise GPError(rc, self._lib.gp_last_error(self._h).decode())
        return rc

    def options(self):
        return {f: getattr(self._opt, f) for f, _ in Options._fields_}

    def set_options(self, **kw):
        if isinstance(kw.get("correlation"), str):
            kw["correlation"] = CORRELATIONS[kw["correlation"]]
        opt = Options(**{**self.options(), **kw})
        self._check(self._lib.gp_set_options(self._h, ctypes.byref(opt)))
        self._opt = opt

    def set_stream(self, stream):
        self.stream = stream
        self._check(self._lib.gp_set_stream(self._h, _vp(stream.cuda_stream)))

    PHASES = ("assemble", "potrf", "trsm", "update", "solve", "split", "predict", "spare")

    def set_timing(self, on=True):
        self._check(self._lib.gp_set_timing(self._h, int(bool(on))))

    def phase_times(self):
        """{phase: (milliseconds, kernel launches)} since the previous call (synchronises)."""
        ms = (_c_double * 8)()
        ln = (ctypes.c_longlong * 8)()
        self._check(self._lib.gp_phase_times(self._h, ms, ln, 8))
        return {name: (ms[i], ln[i]) for i, name in enumerate(self.PHASES)}

    def launch_count(self):
        return int(self._lib.gp_launch_count(self._h))

    def workspace_bytes(self):
        return int(self._lib.gp_workspace_bytes(self._h))

    def call_bytes(self, call, n, d, count=1, prec="mixed"):
        """gp_call_bytes with this context's options and budget."""
        return call_bytes(call, n, d, count, prec, ctx=self)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gp_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    # -- gp_corr_assemble --------------------------------------------------
    def corr_assemble(self, x, theta, p, delta, layout="dense", out=None):
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        theta = _dev_f64(theta, "theta", (d,), self.device)
        lay = {"dense": 0, "tiles": 1, "tiles_df": 2}[layout]
        size = (n, n) if lay == 0 else (packed_elems(n),)
        if out is None:
            out = torch.empty(size, dtype=torch.float64, device=self.device)
        _dev_f64(out, "out", size, self.device)
        self._check(self._lib.gp_corr_assemble(self._h, n, d, _ptr(x), _ptr(theta), float(p),
                                               float(delta), _ptr(out), lay))
        return out

    # -- gp_cholesky -------------------------------------------------------
    def cholesky(self, x, theta, p, delta, prec="fp64", out=None):
        """Factor of R(theta) + delta I in the tile layout; returns (L, status)."""
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        theta = _dev_f64(theta, "theta", (d,), self.device)
        size = (packed_elems(n),)
        if out is None:
            out = torch.zeros(size, dtype=torch.float64, device=self.device)
        _dev_f64(out, "out", size, self.device)
        st = _c_int(0)
        self._check(self._lib.gp_cholesky(self._h, n, d, _ptr(x), _ptr(theta), float(p), float(delta),
                                          _prec(prec), _ptr(out), ctypes.byref(st)))
        return out, st.value

    # -- gp_nll_batch ------------------------------------------------------
    def nll_batch(self, x, y, thetas, p, delta, prec="fp64", out=None, cond=False):
        """-2logL, mu_hat, sigma2_hat, log|R| and status at each row of thetas.
        cond=True adds out["cond"], the 1-norm condition estimate of each R
        (split precisions only); prec="auto" adds out["prec_used"] (the
        arithmetic each candidate's values come from, a GP_* code)."""
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        y = _dev_f64(y, "y", (n,), self.device)
        thetas = _dev_f64(thetas, "thetas", device=self.device)
        if thetas.dim() != 2 or thetas.shape[1] != d:
            raise ValueError("thetas must be T x d")
        T = thetas.shape[0]
        if out is None:
            kw = dict(dtype=torch.float64, device=self.device)
            out = dict(nll=torch.empty(T, **kw), mu=torch.empty(T, **kw),
                       sigma2=torch.empty(T, **kw), logdet=torch.empty(T, **kw),
                       status=torch.empty(T, dtype=torch.int32, device=self.device))
        else:
            _check_outs(out, ("nll", "mu", "sigma2", "status"), ("logdet", "cond", "prec_used"), T,
                        self.device)
        pc = _prec(prec)
        if cond and "cond" not in out:
            out["cond"] = torch.empty(T, dtype=torch.float64, device=self.device)
        if pc == GP_AUTO and "prec_used" not in out:
            out["prec_used"] = torch.empty(T, dtype=torch.int32, device=self.device)
        self._check(self._lib.gp_nll_batch_ex(
            self._h, n, d, _ptr(x), _ptr(y), T, _ptr(thetas), float(p), float(delta), pc,
            _ptr(out["nll"]), _ptr(out["mu"]), _ptr(out["sigma2"]), _ptr(out.get("logdet")),
            _ptr(out["status"]), _ptr(out.get("cond") if cond else None), _ptr(out.get("prec_used"))))
        return out

    def autotune(self, x, y, thetas, p, delta, prec="mixed", reps=2):
        """gp_autotune: time every launch-shape combination on this batch and
        keep the fastest as the context's options.  Returns the trials (list
        of dicts, in the order timed) and the chosen options."""
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        y = _dev_f64(y, "y", (n,), self.device)
        thetas = _dev_f64(thetas, "thetas", device=self.device)
        if thetas.dim() != 2 or thetas.shape[1] != d:
            raise ValueError("thetas must be T x d")
        T = thetas.shape[0]
        buf = (TuneTrial * 16)()
        cnt = _c_int(0)
        self._check(self._lib.gp_autotune(self._h, n, d, _ptr(x), _ptr(y), T, _ptr(thetas), float(p),
                                          float(delta), _prec(prec), int(reps), buf, 16, ctypes.byref(cnt)))
        trials = [{f: getattr(buf[i], f) for f, _ in TuneTrial._fields_} for i in range(cnt.value)]
        # the library changed the context's options: read them back
        opt = Options()
        self._check(self._lib.gp_get_options(self._h, ctypes.byref(opt)))
        self._opt = opt
        return trials, self.options()

    def nll_grad_batch(self, x, y, thetas, p, delta, out=None):
        """gp_nll_grad_batch: -2logL and its gradient with respect to theta
        (T x d) at each row of thetas, in double precision."""
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        y = _dev_f64(y, "y", (n,), self.device)
        thetas = _dev_f64(thetas, "thetas", device=self.device)
        if thetas.dim() != 2 or thetas.shape[1] != d:
            raise ValueError("thetas must be T x d")
        T = thetas.shape[0]
        if out is None:
            kw = dict(dtype=torch.float64, device=self.device)
            out = dict(nll=torch.empty(T, **kw), grad=torch.empty((T, d), **kw),
                       status=torch.empty(T, dtype=torch.int32, device=self.device))
        else:
            _check_outs(out, ("nll", "grad", "status"), (), T, self.device, shapes={"grad": (T, d)})
        self._check(self._lib.gp_nll_grad_batch(
            self._h, n, d, _ptr(x), _ptr(y), T, _ptr(thetas), float(p), float(delta),
            _ptr(out["nll"]), _ptr(out["grad"]), _ptr(out["status"])))
        return out

    def plan_nll_batch(self, x, y, thetas, p, delta, prec="mixed", cond=False):
        """Record nll_batch(x, y, thetas, ...) as a CUDA graph; returns a Plan
        whose launch() replays it into plan.out (also valid on return)."""
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        y = _dev_f64(y, "y", (n,), self.device)
        thetas = _dev_f64(thetas, "thetas", device=self.device)
        if thetas.dim() != 2 or thetas.shape[1] != d:
            raise ValueError("thetas must be T x d")
        T = thetas.shape[0]
        kw = dict(dtype=torch.float64, device=self.device)
        out = dict(nll=torch.empty(T, **kw), mu=torch.empty(T, **kw), sigma2=torch.empty(T, **kw),
                   logdet=torch.empty(T, **kw), status=torch.empty(T, dtype=torch.int32, device=self.device))
        if cond:
            out["cond"] = torch.empty(T, **kw)
        h = _vp()
        self._check(self._lib.gp_plan_nll_batch(
            self._h, n, d, _ptr(x), _ptr(y), T, _ptr(thetas), float(p), float(delta), _prec(prec),
            _ptr(out["nll"]), _ptr(out["mu"]), _ptr(out["sigma2"]), _ptr(out["logdet"]), _ptr(out["status"]),
            _ptr(out.get("cond")), ctypes.byref(h)))
        return Plan(self, h, (x, y, thetas), out)

    def nll_batch_noalloc(self, x, y, thetas, p, delta, out=None):
        """gp_nll_batch_noalloc: the double-precision batch with the library's
        fixed scratch array (no device allocation by the library).  Pass
        preallocated `out` tensors to keep the call itself allocation-free."""
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        y = _dev_f64(y, "y", (n,), self.device)
        thetas = _dev_f64(thetas, "thetas", device=self.device)
        if thetas.dim() != 2 or thetas.shape[1] != d:
            raise ValueError("thetas must be T x d")
        T = thetas.shape[0]
        if out is None:
            kw = dict(dtype=torch.float64, device=self.device)
            out = dict(nll=torch.empty(T, **kw), mu=torch.empty(T, **kw),
                       sigma2=torch.empty(T, **kw), logdet=torch.empty(T, **kw),
                       status=torch.empty(T, dtype=torch.int32, device=self.device))
        else:
            _check_outs(out, ("nll", "mu", "sigma2", "status"), ("logdet",), T, self.device)
        self._check(self._lib.gp_nll_batch_noalloc(
            self._h, n, d, _ptr(x), _ptr(y), T, _ptr(thetas), float(p), float(delta),
            _ptr(out["nll"]), _ptr(out["mu"]), _ptr(out["sigma2"]), _ptr(out.get("logdet")),
            _ptr(out["status"])))
        return out

    def nll_batch_host(self, x, y, thetas, p, delta, prec="fp64", out=None):
        """gp_nll_batch_host: host (CPU, optionally pinned) tensors in and out."""
        n, d, T = _host_batch_args(x, y, thetas)
        if out is None:
            out = dict(nll=torch.empty(T, dtype=torch.float64), mu=torch.empty(T, dtype=torch.float64),
                       sigma2=torch.empty(T, dtype=torch.float64),
                       logdet=torch.empty(T, dtype=torch.float64),
                       status=torch.empty(T, dtype=torch.int32))
        else:
            _check_outs(out, ("nll", "mu", "sigma2", "status"), ("logdet",), T, None)
        self._check(self._lib.gp_nll_batch_host(
            self._h, n, d, _ptr(x), _ptr(y), T, _ptr(thetas), float(p), float(delta), _prec(prec),
            _ptr(out["nll"]), _ptr(out["mu"]), _ptr(out["sigma2"]), _ptr(out.get("logdet")),
            _ptr(out["status"])))
        return out

    # -- gp_fit / gp_predict -----------------------------------------------
    def fit(self, x, y, theta, p, delta, prec="fp64"):
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        y = _dev_f64(y, "y", (n,), self.device)
        theta = _dev_f64(theta, "theta", (d,), self.device)
        h = _vp()
        rc = self._lib.gp_fit(self._h, n, d, _ptr(x), _ptr(y), _ptr(theta), float(p), float(delta),
                              _prec(prec), ctypes.byref(h))
        if rc not in (GP_OK, GP_EDEGENERATE):
            self._check(rc)
        return Model(self, h, n, d)

    def fit_batch(self, x, y, thetas, p, delta, prec="fp64", out=None):
        """gp_fit_batch: -2logL at every row of thetas (T x d), then a fit at
        the best candidate built from its own factor.  Returns (out, best,
        model); model is None when no candidate gave a likelihood."""
        x = _dev_f64(x, "x", device=self.device)
        n, d = x.shape
        y = _dev_f64(y, "y", (n,), self.device)
        thetas = _dev_f64(thetas, "thetas", device=self.device)
        if thetas.dim() != 2 or thetas.shape[1] != d:
            raise ValueError("thetas must be T x d")
        T = thetas.shape[0]
        if out is None:
            f = lambda: torch.empty(T, dtype=torch.float64, device=self.device)
            out = dict(nll=f(), mu=f(), sigma2=f(), logdet=f(),
                       status=torch.empty(T, dtype=torch.int32, device=self.device))
        else:
            _check_outs(out, ("nll", "mu", "sigma2", "status"), ("logdet",), T, self.device)
        best = _c_int(-1)
        h = _vp()
        rc = self._lib.gp_fit_batch(self._h, n, d, _ptr(x), _ptr(y), T, _ptr(thetas), float(p), float(delta),
                                    _prec(prec), _ptr(out["nll"]), _ptr(out["mu"]), _ptr(out["sigma2"]),
                                    _ptr(out.get("logdet")), _ptr(out["status"]), ctypes.byref(best),
                                    ctypes.byref(h))
        if rc == GP_ENOTPD and best.value < 0:
            return out, -1, None
        if rc not in (GP_OK, GP_EDEGENERATE):
            self._check(rc)
        return out, best.value, Model(self, h, n, d)

    def predict(self, model, xs, want_var=True, yhat=None, s2=None):
        xs = _dev_f64(xs, "xs", device=self.device)
        N = xs.shape[0]
        if xs.dim() != 2 or xs.shape[1] != model.d:
            raise ValueError("xs must be N x d")
        if yhat is None:
            yhat = torch.empty(N, dtype=torch.float64, device=self.device)
        else:
            _out_tensor(yhat, "yhat", (N,), torch.float64, self.device)
        if want_var and s2 is None:
            s2 = torch.empty(N, dtype=torch.float64, device=self.device)
        elif want_var:
            _out_tensor(s2, "s2", (N,), torch.float64, self.device)
        self._check(self._lib.gp_predict(self._h, model._h, N, _ptr(xs), _ptr(yhat),
                                         _ptr(s2) if want_var else None))
        return yhat, (s2 if want_var else None)
