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
module only marshals numpy arrays through ctypes.  ``extended()`` is the same
source built in long double, used only to bound the double build's own
rounding error on small cases.

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

_ip = ctypes.POINTER(ctypes.c_int)
NLL_FIELDS = ("nll", "mu", "sigma2", "logdet", "Q", "nll_full", "cond1")
# correlation families of gp_oracle.c (eq. 2's power-exponential, and the
# Matern family Section 2 names as an alternative, product form)
CORR = {"powexp": 0, "matern12": 1, "matern32": 2, "matern52": 3}


def _fam(corr):
    return CORR[corr] if isinstance(corr, str) else int(corr)


def _p(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Oracle:
    """ctypes view of one build of gp_oracle.c (the default build, or a copy
    that a test compiled itself).  extended=True marks the long-double build,
    whose arrays and scalars are numpy.longdouble: it is there to bound the
    double build's own rounding error on small cases."""

    def __init__(self, libpath, extended=False):
        lib = ctypes.CDLL(libpath)
        self.real = np.longdouble if extended else np.float64
        self._ct = ctypes.c_longdouble if extended else ctypes.c_double
        c_int, c_real = ctypes.c_int, self._ct
        _rp = ctypes.POINTER(c_real)
        lib.gpo_corr_matrix.argtypes = [c_int, c_int, _rp, _rp, c_real, c_int, c_real, _rp]
        lib.gpo_cross_corr.argtypes = [c_int, c_int, _rp, _rp, _rp, c_real, c_int, _rp]
        lib.gpo_cholesky.argtypes = [c_int, _rp, _rp]
        lib.gpo_cholesky.restype = c_int
        lib.gpo_forward.argtypes = [c_int, _rp, _rp, _rp]
        lib.gpo_backward.argtypes = [c_int, _rp, _rp, _rp]
        lib.gpo_cond1_est.argtypes = [c_int, _rp, _rp]
        lib.gpo_cond1_est.restype = c_real
        lib.gpo_nll.argtypes = [c_int, c_int, _rp, _rp, _rp, c_real, c_int, c_real, c_int, _rp]
        lib.gpo_nll.restype = c_int
        lib.gpo_nll_batch.argtypes = [c_int, c_int, _rp, _rp, c_int, _rp, c_real, c_int, c_real,
                                      c_int, _rp, _ip]
        lib.gpo_predict.argtypes = [c_int, c_int, _rp, _rp, _rp, c_real, c_int, c_real, c_int,
                                    _rp, c_int, _rp, _rp]
        lib.gpo_predict.restype = c_int
        lib.gpo_fit_parts.argtypes = [c_int, c_int, _rp, _rp, _rp, c_real, c_int, c_real,
                                      _rp, _rp, _rp, _rp, _rp]
        lib.gpo_fit_parts.restype = c_int
        lib.gpo_nll_grad.argtypes = [c_int, c_int, _rp, _rp, _rp, c_real, c_int, c_real, _rp, _rp]
        lib.gpo_nll_grad.restype = c_int
        lib.gpo_num_threads.restype = c_int
        self.lib = lib

    # marshalling in the build's arithmetic type
    def _a(self, a):
        return np.ascontiguousarray(a, dtype=self.real)

    def _e(self, shape):
        return np.empty(shape, dtype=self.real)

    def _p(self, a):
        return None if a is None else _p(a, self._ct)

    def _fields(self, out):
        # the double build hands back Python floats; the extended one keeps
        # its numpy.longdouble values
        return dict(zip(NLL_FIELDS, out.tolist() if self.real is np.float64 else list(out)))

    def num_threads(self) -> int:
        """Host threads the batched oracle uses (OpenMP)."""
        return int(self.lib.gpo_num_threads())

    def corr_matrix(self, x, theta, p, delta=0.0, corr="powexp"):
        """Full n x n R(theta) + delta I (eq. 2 for the power-exponential family)."""
        x = self._a(x)
        n, d = x.shape
        th = self._a(theta).reshape(d)
        R = self._e((n, n))
        self.lib.gpo_corr_matrix(n, d, self._p(x), self._p(th), float(p), _fam(corr), float(delta), self._p(R))
        return R

    def cross_corr(self, x, xs, theta, p, corr="powexp"):
        """r(x*) for one point xs (length d): r_i = corr(z(x*), z(x_i)), no nugget."""
        x = self._a(x)
        n, d = x.shape
        xs = self._a(xs).reshape(d)
        th = self._a(theta).reshape(d)
        r = self._e(n)
        self.lib.gpo_cross_corr(n, d, self._p(x), self._p(xs), self._p(th), float(p), _fam(corr), self._p(r))
        return r

    def cholesky(self, R):
        """Lower Cholesky factor; returns (L, info), info = 0 or failing column + 1."""
        R = self._a(R)
        n = R.shape[0]
        L = self._e((n, n))
        info = self.lib.gpo_cholesky(n, self._p(R), self._p(L))
        return L, int(info)

    def forward(self, L, b):
        L = self._a(L)
        b = self._a(b)
        z = np.empty_like(b)
        self.lib.gpo_forward(L.shape[0], self._p(L), self._p(b), self._p(z))
        return z

    def backward(self, L, e):
        L = self._a(L)
        e = self._a(e)
        w = np.empty_like(e)
        self.lib.gpo_backward(L.shape[0], self._p(L), self._p(e), self._p(w))
        return w

    def cond1_est(self, R, L):
        R = self._a(R)
        L = self._a(L)
        return float(self.lib.gpo_cond1_est(R.shape[0], self._p(R), self._p(L)))

    def nll(self, x, y, theta, p, delta=0.0, want_cond=False, corr="powexp"):
        """Profile -2 log L at one theta.  Returns (dict of NLL_FIELDS, status)."""
        x = self._a(x)
        n, d = x.shape
        y = self._a(y).reshape(n)
        th = self._a(theta).reshape(d)
        out = self._e(7)
        st = self.lib.gpo_nll(n, d, self._p(x), self._p(y), self._p(th), float(p), _fam(corr), float(delta),
                              int(bool(want_cond)), self._p(out))
        return self._fields(out), int(st)

    def nll_batch(self, x, y, thetas, p, delta=0.0, want_cond=False, corr="powexp"):
        """-2 log L at T candidates (thetas T x d), spread over host threads.
        Returns (out T x 7 in NLL_FIELDS order, status T)."""
        x = self._a(x)
        n, d = x.shape
        y = self._a(y).reshape(n)
        th = self._a(thetas).reshape(-1, d)
        T = th.shape[0]
        out = self._e((T, 7))
        st = np.empty(T, dtype=np.int32)
        self.lib.gpo_nll_batch(n, d, self._p(x), self._p(y), T, self._p(th), float(p), _fam(corr), float(delta),
                               int(bool(want_cond)), self._p(out), st.ctypes.data_as(_ip))
        return out, st

    def nll_grad(self, x, y, theta, p, delta=0.0, corr="powexp"):
        """d(-2logL)/dtheta at one theta.  Returns (grad (d,), dict of NLL_FIELDS, status)."""
        x = self._a(x)
        n, d = x.shape
        y = self._a(y).reshape(n)
        th = self._a(theta).reshape(d)
        g = self._e(d)
        out = self._e(7)
        st = self.lib.gpo_nll_grad(n, d, self._p(x), self._p(y), self._p(th), float(p), _fam(corr), float(delta),
                                   self._p(g), self._p(out))
        return g, self._fields(out), int(st)

    def predict(self, x, y, theta, p, delta, xs, nugget_in_var=True, want_var=True, corr="powexp"):
        """Kriging mean and variance at the rows of xs.  Returns (yhat, s2|None, status)."""
        x = self._a(x)
        n, d = x.shape
        y = self._a(y).reshape(n)
        th = self._a(theta).reshape(d)
        xs = self._a(xs).reshape(-1, d)
        N = xs.shape[0]
        yhat = self._e(N)
        s2 = self._e(N) if want_var else None
        st = self.lib.gpo_predict(n, d, self._p(x), self._p(y), self._p(th), float(p), _fam(corr), float(delta), N,
                                  self._p(xs), int(bool(nugget_in_var)), self._p(yhat), self._p(s2))
        return yhat, s2, int(st)

    def fit_parts(self, x, y, theta, p, delta=0.0, corr="powexp"):
        """R, L, a = L^-1 1, b = L^-1 Y, w = R^-1 (Y - 1 mu_hat), status."""
        x = self._a(x)
        n, d = x.shape
        y = self._a(y).reshape(n)
        th = self._a(theta).reshape(d)
        R = self._e((n, n)); L = self._e((n, n))
        a = self._e(n); b = self._e(n); w = self._e(n)
        st = self.lib.gpo_fit_parts(n, d, self._p(x), self._p(y), self._p(th), float(p), _fam(corr), float(delta),
                                    self._p(R), self._p(L), self._p(a), self._p(b), self._p(w))
        return R, L, a, b, w, int(st)


_default = None
_extended = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build_oracle())
    return _default


def extended() -> Oracle:
    """The long-double build of the same definitions (numpy.longdouble in and
    out), for bounding the double oracle's own rounding error."""
    global _extended
    if _extended is None:
        _extended = Oracle(build_oracle(extended=True), extended=True)
    return _extended


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
