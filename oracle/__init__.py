"""CPU FP64 oracle for the Gaussian-process likelihood / kriging path.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct reference that
the CUDA library is checked against.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
It shares no code with the CUDA path (``paper_1203_1269_gb300``) and neither
imports the other.

Every function follows Section 2 of Franey, Ranjan & Chipman:
  eq. (2)  power-exponential correlation R_ij = prod_k exp(-theta_k |x_ik-x_jk|^p)
  eq. (3)  mu_hat = (1'R^-1 1)^-1 1'R^-1 Y,  sigma2_hat = Q / n
  eq. (4)  -2 log L = log|R| + n log Q,  Q = (Y-1mu)'R^-1(Y-1mu)
with the Cholesky factorisation and back-solves of Section 3.  The computation
is in ``gp_oracle.c`` (plain C, double precision, unblocked loops); this
module only marshals numpy arrays through ctypes.

Parity status: every function here is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (closed forms, hand derivations, eigenvalue and
library-solve checks, invariants, the printed Table 2 row).
"""
import ctypes
import numpy as np

from .build import build_oracle

STATUS_OK = 0
STATUS_NOTPD = -3
STATUS_DEGENERATE = -6

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
NLL_FIELDS = ("nll", "mu", "sigma2", "logdet", "Q", "nll_full", "cond1")
# correlation families of gp_oracle.c (eq. 2's power-exponential, and the
# Matern family Section 2 names as an alternative, product form)
CORR = {"powexp": 0, "matern12": 1, "matern32": 2, "matern52": 3}


def _fam(corr):
    return CORR[corr] if isinstance(corr, str) else int(corr)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_dp)


class Oracle:
    """ctypes view of one build of gp_oracle.c (the default build, or a copy
    that a test compiled itself)."""

    def __init__(self, libpath):
        lib = ctypes.CDLL(libpath)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        lib.gpo_corr_matrix.argtypes = [c_int, c_int, _dp, _dp, c_double, c_int, c_double, _dp]
        lib.gpo_cross_corr.argtypes = [c_int, c_int, _dp, _dp, _dp, c_double, c_int, _dp]
        lib.gpo_cholesky.argtypes = [c_int, _dp, _dp]
        lib.gpo_cholesky.restype = c_int
        lib.gpo_forward.argtypes = [c_int, _dp, _dp, _dp]
        lib.gpo_backward.argtypes = [c_int, _dp, _dp, _dp]
        lib.gpo_cond1_est.argtypes = [c_int, _dp, _dp]
        lib.gpo_cond1_est.restype = c_double
        lib.gpo_nll.argtypes = [c_int, c_int, _dp, _dp, _dp, c_double, c_int, c_double, c_int, _dp]
        lib.gpo_nll.restype = c_int
        lib.gpo_nll_batch.argtypes = [c_int, c_int, _dp, _dp, c_int, _dp, c_double, c_int, c_double,
                                      c_int, _dp, _ip]
        lib.gpo_predict.argtypes = [c_int, c_int, _dp, _dp, _dp, c_double, c_int, c_double, c_int,
                                    _dp, c_int, _dp, _dp]
        lib.gpo_predict.restype = c_int
        lib.gpo_fit_parts.argtypes = [c_int, c_int, _dp, _dp, _dp, c_double, c_int, c_double,
                                      _dp, _dp, _dp, _dp, _dp]
        lib.gpo_fit_parts.restype = c_int
        lib.gpo_nll_grad.argtypes = [c_int, c_int, _dp, _dp, _dp, c_double, c_int, c_double, _dp, _dp]
        lib.gpo_nll_grad.restype = c_int
        lib.gpo_num_threads.restype = c_int
        self.lib = lib

    def num_threads(self) -> int:
        """Host threads the batched oracle uses (OpenMP)."""
        return int(self.lib.gpo_num_threads())

    def corr_matrix(self, x, theta, p, delta=0.0, corr="powexp"):
        """Full n x n R(theta) + delta I (eq. 2 for the power-exponential family)."""
        x = _f64(x)
        n, d = x.shape
        th = _f64(theta).reshape(d)
        R = np.empty((n, n))
        self.lib.gpo_corr_matrix(n, d, _p(x), _p(th), float(p), _fam(corr), float(delta), _p(R))
        return R

    def cross_corr(self, x, xs, theta, p, corr="powexp"):
        """r(x*) for one point xs (length d): r_i = corr(z(x*), z(x_i)), no nugget."""
        x = _f64(x)
        n, d = x.shape
        xs = _f64(xs).reshape(d)
        th = _f64(theta).reshape(d)
        r = np.empty(n)
        self.lib.gpo_cross_corr(n, d, _p(x), _p(xs), _p(th), float(p), _fam(corr), _p(r))
        return r

    def cholesky(self, R):
        """Lower Cholesky factor; returns (L, info), info = 0 or failing column + 1."""
        R = _f64(R)
        n = R.shape[0]
        L = np.empty((n, n))
        info = self.lib.gpo_cholesky(n, _p(R), _p(L))
        return L, int(info)

    def forward(self, L, b):
        L = _f64(L)
        b = _f64(b)
        z = np.empty_like(b)
        self.lib.gpo_forward(L.shape[0], _p(L), _p(b), _p(z))
        return z

    def backward(self, L, e):
        L = _f64(L)
        e = _f64(e)
        w = np.empty_like(e)
        self.lib.gpo_backward(L.shape[0], _p(L), _p(e), _p(w))
        return w

    def cond1_est(self, R, L):
        R = _f64(R)
        L = _f64(L)
        return float(self.lib.gpo_cond1_est(R.shape[0], _p(R), _p(L)))

    def nll(self, x, y, theta, p, delta=0.0, want_cond=False, corr="powexp"):
        """Profile -2 log L at one theta.  Returns (dict of NLL_FIELDS, status)."""
        x = _f64(x)
        n, d = x.shape
        y = _f64(y).reshape(n)
        th = _f64(theta).reshape(d)
        out = np.empty(7)
        st = self.lib.gpo_nll(n, d, _p(x), _p(y), _p(th), float(p), _fam(corr), float(delta),
                              int(bool(want_cond)), _p(out))
        return dict(zip(NLL_FIELDS, out.tolist())), int(st)

    def nll_batch(self, x, y, thetas, p, delta=0.0, want_cond=False, corr="powexp"):
        """-2 log L at T candidates (thetas T x d), spread over host threads.
        Returns (out T x 7 in NLL_FIELDS order, status T)."""
        x = _f64(x)
        n, d = x.shape
        y = _f64(y).reshape(n)
        th = _f64(thetas).reshape(-1, d)
        T = th.shape[0]
        out = np.empty((T, 7))
        st = np.empty(T, dtype=np.int32)
        self.lib.gpo_nll_batch(n, d, _p(x), _p(y), T, _p(th), float(p), _fam(corr), float(delta),
                               int(bool(want_cond)), _p(out), st.ctypes.data_as(_ip))
        return out, st

    def nll_grad(self, x, y, theta, p, delta=0.0, corr="powexp"):
        """d(-2logL)/dtheta at one theta.  Returns (grad (d,), dict of NLL_FIELDS, status)."""
        x = _f64(x)
        n, d = x.shape
        y = _f64(y).reshape(n)
        th = _f64(theta).reshape(d)
        g = np.empty(d)
        out = np.empty(7)
        st = self.lib.gpo_nll_grad(n, d, _p(x), _p(y), _p(th), float(p), _fam(corr), float(delta),
                                   _p(g), _p(out))
        return g, dict(zip(NLL_FIELDS, out.tolist())), int(st)

    def predict(self, x, y, theta, p, delta, xs, nugget_in_var=True, want_var=True, corr="powexp"):
        """Kriging mean and variance at the rows of xs.  Returns (yhat, s2|None, status)."""
        x = _f64(x)
        n, d = x.shape
        y = _f64(y).reshape(n)
        th = _f64(theta).reshape(d)
        xs = _f64(xs).reshape(-1, d)
        N = xs.shape[0]
        yhat = np.empty(N)
        s2 = np.empty(N) if want_var else None
        st = self.lib.gpo_predict(n, d, _p(x), _p(y), _p(th), float(p), _fam(corr), float(delta), N,
                                  _p(xs), int(bool(nugget_in_var)), _p(yhat),
                                  _p(s2) if want_var else None)
        return yhat, s2, int(st)

    def fit_parts(self, x, y, theta, p, delta=0.0, corr="powexp"):
        """R, L, a = L^-1 1, b = L^-1 Y, w = R^-1 (Y - 1 mu_hat), status."""
        x = _f64(x)
        n, d = x.shape
        y = _f64(y).reshape(n)
        th = _f64(theta).reshape(d)
        R = np.empty((n, n)); L = np.empty((n, n))
        a = np.empty(n); b = np.empty(n); w = np.empty(n)
        st = self.lib.gpo_fit_parts(n, d, _p(x), _p(y), _p(th), float(p), _fam(corr), float(delta),
                                    _p(R), _p(L), _p(a), _p(b), _p(w))
        return R, L, a, b, w, int(st)


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build_oracle())
    return _default


def num_threads():
    return default().num_threads()


def corr_matrix(*a, **k):
    return default().corr_matrix(*a, **k)


def cross_corr(*a, **k):
    return default().cross_corr(*a, **k)


def cholesky(*a, **k):
    return default().cholesky(*a, **k)


def forward(*a, **k):
    return default().forward(*a, **k)


def backward(*a, **k):
    return default().backward(*a, **k)


def cond1_est(*a, **k):
    return default().cond1_est(*a, **k)


def nll(*a, **k):
    return default().nll(*a, **k)


def nll_batch(*a, **k):
    return default().nll_batch(*a, **k)


def predict(*a, **k):
    return default().predict(*a, **k)


def fit_parts(*a, **k):
    return default().fit_parts(*a, **k)


def nll_grad(*a, **k):
    return default().nll_grad(*a, **k)
