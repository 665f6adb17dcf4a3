"""Checks that pin the CPU oracle to facts other than itself.

Each check takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees with the fact.  The facts come from the mathematics of
Section 2 (eqs. 2-4) and from the paper's printed Table 2 row, never from the
oracle's own code:

  * Kac-Murdock-Szego closed form (d = 1, equispaced x, p = 1, delta = 0):
    R_ij = rho^|i-j|, det R = (1 - rho^2)^(n-1), the Cholesky factor in closed
    form and a tridiagonal inverse, so mu_hat, Q and -2logL follow in O(n).
  * hand derivations for n = 1, 2 (with a nugget) and n = 3 (adjugate).
  * log|R| against the eigenvalues from LAPACK's symmetric eigensolver.
  * mu_hat, sigma2_hat, Q and kriging against LAPACK's general solver, and
    for n <= 16 against long-double Gauss-Jordan elimination.
  * invariants: row permutation, scaling and shifting of y, Hadamard's
    inequality, symmetry and unit diagonal.
  * the form of eq. (4) against the printed rows of Tables 1-2.

The same checks run against planted-mistake copies of the oracle in
``test_oracle_mutants.py`` to show that each plausible mistake is caught.
"""
import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# ---------------------------------------------------------------- assembly --

def check_corr_hand_values(orc):
    """Eq. (2) at points where the value is known by hand."""
    x = np.array([[0.0, 0.0], [0.5, 0.25], [1.0, 0.0]])
    # p = 2: R_01 = exp(-2*0.25) * exp(-4*0.0625) = exp(-0.75)
    R = orc.corr_matrix(x, [2.0, 4.0], 2.0, 0.0)
    assert _rel(R[0, 1], math.exp(-0.75)) < 1e-15
    # R_02: dims differ only in x1 by 1.0 -> exp(-2)
    assert _rel(R[0, 2], math.exp(-2.0)) < 1e-15
    # p = 1: R_01 = exp(-2*0.5 - 4*0.25) = exp(-2)
    R1 = orc.corr_matrix(x, [2.0, 4.0], 1.0, 0.0)
    assert _rel(R1[0, 1], math.exp(-2.0)) < 1e-15
    # p = 1.5 at distance 0.25 in dim 2 only (points 0 and a shifted copy)
    x2 = np.array([[0.0, 0.0], [0.0, 0.25]])
    R2 = orc.corr_matrix(x2, [3.0, 5.0], 1.5, 0.0)
    assert _rel(R2[0, 1], math.exp(-5.0 * 0.125)) < 1e-15   # 0.25^1.5 = 0.125
    # nugget on the diagonal only
    Rd = orc.corr_matrix(x, [2.0, 4.0], 2.0, 1e-3)
    assert np.all(np.diag(Rd) == 1.0 + 1e-3)
    assert Rd[0, 1] == R[0, 1]


def check_corr_invariants(orc, seed=3):
    g = np.random.default_rng(seed)
    for (n, d, p) in [(17, 3, 1.95), (9, 5, 1.0), (12, 2, 2.0), (7, 4, 0.5)]:
        x = g.random((n, d))
        th = 10 ** g.uniform(-2, 1, d)
        R = orc.corr_matrix(x, th, p, 0.0)
        assert np.array_equal(R, R.T)
        assert np.all(np.diag(R) == 1.0)
        assert np.all(R > 0) and np.all(R <= 1.0)
        # larger theta never raises a correlation
        R2 = orc.corr_matrix(x, th * 2, p, 0.0)
        assert np.all(R2 <= R)
        # cross-correlation to a design point reproduces that row (no nugget)
        r = orc.cross_corr(x, x[3], th, p)
        assert np.array_equal(r, R[3])


# ------------------------------------------------------------ KMS pins ------

def kms_case(n, rho_target=0.8):
    """d = 1, x_i = i h with h a power of two (exact), p = 1, delta = 0."""
    h = 1.0 / 1024.0
    x = (np.arange(n, dtype=np.float64) * h).reshape(n, 1)
    theta = -math.log(rho_target) / h
    rho = math.exp(-theta * h)
    return x, theta, rho


def kms_quadratic_forms(rho, u, v):
    """u' R^-1 v for the KMS matrix R_ij = rho^|i-j| via its tridiagonal
    inverse (1/(1-rho^2)) * [diag 1, 1+rho^2, ..., 1+rho^2, 1; off -rho]."""
    n = len(u)
    c = 1.0 / (1.0 - rho * rho)
    diag = np.full(n, 1.0 + rho * rho)
    diag[0] = diag[-1] = 1.0
    s = np.dot(u * diag, v) - rho * (np.dot(u[1:], v[:-1]) + np.dot(u[:-1], v[1:]))
    return c * s


def check_kms(orc, n=60, rho_target=0.8, seed=5):
    x, theta, rho = kms_case(n, rho_target)
    R = orc.corr_matrix(x, [theta], 1.0, 0.0)
    i = np.arange(n)
    Rk = rho ** np.abs(i[:, None] - i[None, :])
    assert np.max(np.abs(R - Rk)) < 1e-13
    L, info = orc.cholesky(R)
    assert info == 0
    s = math.sqrt(1.0 - rho * rho)
    Lk = np.zeros((n, n))
    for a in range(n):
        Lk[a, 0] = rho ** a
        for b in range(1, a + 1):
            Lk[a, b] = rho ** (a - b) * s
    assert np.max(np.abs(L - Lk)) < 1e-12
    g = np.random.default_rng(seed)
    y = g.standard_normal(n)
    one = np.ones(n)
    A = kms_quadratic_forms(rho, one, one)
    assert _rel(A, ((n - 2) * (1 - rho) + 2) / (1 + rho)) < 1e-13
    B = kms_quadratic_forms(rho, one, y)
    C = kms_quadratic_forms(rho, y, y)
    mu = B / A
    Q = C - B * B / A
    logdet = (n - 1) * math.log(1.0 - rho * rho)
    out, st = orc.nll(x, y, [theta], 1.0, 0.0)
    assert st == 0
    assert _rel(out["logdet"], logdet) < 1e-11
    assert _rel(out["mu"], mu) < 1e-10
    assert _rel(out["Q"], Q) < 1e-10
    assert _rel(out["sigma2"], Q / n) < 1e-10
    assert _rel(out["nll"], logdet + n * math.log(Q)) < 1e-11


# ---------------------------------------------------- hand derivations ------

def check_n1(orc):
    """n = 1: R = [1 + delta], mu_hat = y_1, Q = 0 -> -2logL = -inf."""
    out, st = orc.nll(np.array([[0.3, 0.7]]), np.array([2.5]), [1.0, 2.0], 1.9, 1e-3)
    assert st == -6
    assert out["nll"] == -math.inf
    assert _rel(out["mu"], 2.5) < 1e-15
    assert out["Q"] < 1e-28
    # log near 1 turns the ulp of sqrt(1.001) into ~1e-13 relative
    assert _rel(out["logdet"], math.log(1.001)) < 1e-12


def check_n2(orc):
    """n = 2 with correlation rho and nugget delta:
    mu_hat = (y1+y2)/2, Q = (y1-y2)^2 / (2 (1 + delta - rho)),
    log|R| = log((1+delta)^2 - rho^2), -2logL = log|R| + 2 log Q."""
    for delta in (0.0, 1e-2):
        x = np.array([[0.1, 0.2], [0.4, 0.6]])
        th = np.array([1.5, 0.7])
        p = 1.95
        rho = math.exp(-1.5 * 0.3 ** p) * math.exp(-0.7 * 0.4 ** p)
        y = np.array([1.25, -0.5])
        out, st = orc.nll(x, y, th, p, delta)
        assert st == 0
        Q = (y[0] - y[1]) ** 2 / (2.0 * (1.0 + delta - rho))
        logdet = math.log((1.0 + delta) ** 2 - rho * rho)
        assert _rel(out["mu"], 0.375) < 1e-14
        assert _rel(out["Q"], Q) < 1e-12
        assert _rel(out["sigma2"], Q / 2) < 1e-12
        assert _rel(out["logdet"], logdet) < 1e-12
        assert _rel(out["nll"], logdet + 2 * math.log(Q)) < 1e-12


def _inv3_adjugate(M):
    (a, b, c), (d, e, f), (g, h, i) = M
    det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g)
    adj = [[e * i - f * h, c * h - b * i, b * f - c * e],
           [f * g - d * i, a * i - c * g, c * d - a * f],
           [d * h - e * g, b * g - a * h, a * e - b * d]]
    return det, [[adj[r][s] / det for s in range(3)] for r in range(3)]


def check_n3(orc):
    """n = 3 through the 3 x 3 adjugate inverse and the determinant by cofactors."""
    x = np.array([[0.0, 0.1], [0.3, 0.5], [0.9, 0.2]])
    th = [2.0, 1.0]
    p = 2.0
    delta = 1e-4
    M = [[0.0] * 3 for _ in range(3)]
    for r in range(3):
        for s in range(3):
            q = sum(th[k] * (x[r, k] - x[s, k]) ** 2 for k in range(2))
            M[r][s] = math.exp(-q) + (delta if r == s else 0.0)
    det, Minv = _inv3_adjugate(M)
    y = [0.3, -1.2, 2.0]
    A = sum(Minv[r][s] for r in range(3) for s in range(3))
    B = sum(Minv[r][s] * y[s] for r in range(3) for s in range(3))
    mu = B / A
    e = [y[r] - mu for r in range(3)]
    Q = sum(e[r] * Minv[r][s] * e[s] for r in range(3) for s in range(3))
    out, st = orc.nll(x, np.array(y), th, p, delta)
    assert st == 0
    assert _rel(out["mu"], mu) < 1e-11
    assert _rel(out["Q"], Q) < 1e-11
    assert _rel(out["logdet"], math.log(det)) < 1e-11
    assert _rel(out["nll"], math.log(det) + 3 * math.log(Q)) < 1e-11


# ------------------------------------------------ library cross-checks ------

def check_eig_logdet(orc, seed=11):
    g = np.random.default_rng(seed)
    for (n, d, p, delta) in [(8, 2, 2.0, 1e-6), (33, 3, 1.95, 1e-8), (64, 4, 1.5, 0.0)]:
        x = g.random((n, d))
        th = 10 ** g.uniform(-0.5, 1, d)
        y = g.standard_normal(n)
        R = orc.corr_matrix(x, th, p, delta)
        lam = np.linalg.eigvalsh(R)
        out, st = orc.nll(x, y, th, p, delta)
        assert st == 0
        assert abs(out["logdet"] - np.sum(np.log(lam))) < 1e-9 * max(1.0, abs(out["logdet"]))


def check_solve_estimates(orc, seed=13):
    """mu_hat, Q, sigma2 and -2logL against LAPACK's general solver on R."""
    g = np.random.default_rng(seed)
    for (n, d, p, delta) in [(5, 2, 2.0, 1e-4), (16, 3, 1.95, 1e-6), (40, 6, 1.95, 1e-7)]:
        x = g.random((n, d))
        th = 10 ** g.uniform(0, 1, d)
        y = np.sin(3 * x).sum(axis=1) + 0.1 * g.standard_normal(n)
        R = orc.corr_matrix(x, th, p, delta)
        one = np.ones(n)
        Ri1 = np.linalg.solve(R, one)
        Riy = np.linalg.solve(R, y)
        mu = one @ Riy / (one @ Ri1)
        res = y - mu
        Q = res @ np.linalg.solve(R, res)
        sign, ld = np.linalg.slogdet(R)
        out, st = orc.nll(x, y, th, p, delta)
        assert st == 0 and sign > 0
        assert _rel(out["mu"], mu) < 1e-9
        assert _rel(out["Q"], Q) < 1e-9
        assert _rel(out["sigma2"], Q / n) < 1e-9
        assert _rel(out["nll"], ld + n * math.log(Q)) < 1e-9
        assert _rel(out["nll_full"], ld + n * math.log(Q / n) + n * (1 + math.log(2 * math.pi))) < 1e-9


def _gauss_jordan_ld(A):
    """R^-1 and log|det R| by Gauss-Jordan elimination with partial pivoting
    in numpy.longdouble, plain loops: an elimination unrelated to the
    oracle's Cholesky route, in wider arithmetic."""
    n = A.shape[0]
    M = np.hstack([np.asarray(A, dtype=np.longdouble), np.eye(n, dtype=np.longdouble)])
    logdet = np.longdouble(0)
    for c in range(n):
        piv = c + int(np.argmax(np.abs(M[c:, c])))
        if piv != c:
            M[[c, piv]] = M[[piv, c]]
        pv = M[c, c]
        logdet += np.log(np.abs(pv))
        M[c] = M[c] / pv
        for r in range(n):
            if r != c:
                M[r] = M[r] - M[r, c] * M[c]
    return M[:, n:], logdet


def check_gauss_jordan_estimates(orc, seed=53):
    """n <= 16: mu_hat, Q, sigma2_hat, log|R| and -2logL against R^-1 and
    |det R| by long-double Gauss-Jordan elimination on the oracle's own R,
    within 8 n cond(R) u of them."""
    g = np.random.default_rng(seed)
    u = 2.0 ** -53
    for (n, d, p, delta) in [(2, 1, 2.0, 0.0), (3, 2, 1.5, 1e-6), (7, 2, 1.95, 1e-8), (16, 3, 1.95, 1e-6)]:
        x = g.random((n, d))
        th = 10 ** g.uniform(-0.5, 1, d)
        y = np.cos(4 * x).sum(axis=1) + 0.1 * g.standard_normal(n)
        R = orc.corr_matrix(x, th, p, delta)
        Ri, logdet = _gauss_jordan_ld(R)
        one = np.ones(n, dtype=np.longdouble)
        yl = y.astype(np.longdouble)
        A, B, C = one @ Ri @ one, one @ Ri @ yl, yl @ Ri @ yl
        mu = B / A
        Q = C - B * B / A
        with np.errstate(invalid="ignore", divide="ignore"):   # a broken R gives Q <= 0
            nll = logdet + n * np.log(Q)
        want = {"mu": mu, "Q": Q, "sigma2": Q / n, "logdet": logdet, "nll": nll}
        out, st = orc.nll(x, y, th, p, delta)
        assert st == 0
        tol = 8 * n * np.linalg.cond(R) * u
        for k, v in want.items():
            v = float(v)
            assert abs(out[k] - v) <= tol * max(abs(v), 1.0), (n, k, out[k], v)


def check_cholesky_reconstructs(orc, seed=17):
    g = np.random.default_rng(seed)
    x = g.random((30, 3))
    R = orc.corr_matrix(x, [3.0, 5.0, 7.0], 1.95, 1e-6)
    L, info = orc.cholesky(R)
    assert info == 0
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.all(np.diag(L) > 0)
    assert np.max(np.abs(L @ L.T - R)) < 1e-14
    # forward and backward solves against LAPACK
    b = g.standard_normal(30)
    z = orc.forward(L, b)
    assert np.max(np.abs(L @ z - b)) < 1e-10
    w = orc.backward(L, b)
    assert np.max(np.abs(L.T @ w - b)) < 1e-10


def check_notpd(orc):
    """Two equal design points with delta = 0: R is singular; the first pivot
    after the duplicate is exactly zero -> NOTPD, -2logL = +inf."""
    x = np.array([[0.2, 0.3], [0.2, 0.3], [0.7, 0.1], [0.5, 0.9]])
    out, st = orc.nll(x, np.array([1.0, 2.0, 0.5, -1.0]), [1.0, 1.0], 2.0, 0.0)
    assert st == -3
    assert out["nll"] == math.inf
    # the same design with a nugget is fine
    out, st = orc.nll(x, np.array([1.0, 2.0, 0.5, -1.0]), [1.0, 1.0], 2.0, 1e-6)
    assert st == 0 and math.isfinite(out["nll"])


def check_cond_estimate(orc, seed=19):
    """Hager's estimate is a lower bound within a small factor of the exact
    cond_1 (numpy); the last case is R = I to rounding (cond_1 = 1), where
    the iteration stops after its first round, so it also fixes the scale of
    the starting vector."""
    g = np.random.default_rng(seed)
    for (n, th) in [(20, 5.0), (50, 1.0), (40, 20.0), (30, 1e4)]:
        x = g.random((n, 2))
        R = orc.corr_matrix(x, [th, th], 1.95, 1e-8)
        L, info = orc.cholesky(R)
        assert info == 0
        est = orc.cond1_est(R, L)
        true = np.linalg.cond(R, 1)
        assert est <= true * (1 + 1e-6)
        assert est >= true / 3.0


# --------------------------------------------------------- invariants -------

def check_invariants(orc, seed=23):
    g = np.random.default_rng(seed)
    n, d = 25, 3
    x = g.random((n, d))
    y = np.cos(4 * x).sum(axis=1)
    th = [2.0, 0.5, 7.0]
    p, delta = 1.95, 1e-6
    base, st = orc.nll(x, y, th, p, delta)
    assert st == 0
    perm = g.permutation(n)
    o, _ = orc.nll(x[perm], y[perm], th, p, delta)
    for k in ("nll", "mu", "sigma2", "logdet"):
        assert _rel(o[k], base[k]) < 1e-10
    c = -3.5
    o, _ = orc.nll(x, c * y, th, p, delta)
    assert _rel(o["mu"], c * base["mu"]) < 1e-10
    assert _rel(o["sigma2"], c * c * base["sigma2"]) < 1e-10
    assert abs(o["nll"] - (base["nll"] + 2 * n * math.log(abs(c)))) < 1e-9 * abs(base["nll"]) + 1e-9
    o, _ = orc.nll(x, y + 10.0, th, p, delta)
    assert _rel(o["mu"], base["mu"] + 10.0) < 1e-10
    assert _rel(o["sigma2"], base["sigma2"]) < 1e-8
    # Hadamard: unit-diagonal SPD matrix has log|R| <= 0
    o, _ = orc.nll(x, y, th, p, 0.0)
    assert o["logdet"] <= 0.0


def check_table_form(orc):
    """Eq. (4) read literally: -2logL = log|R| + n log Q with Q = n sigma2.
    (a) the oracle's outputs have exactly that structure;
    (b) on the paper's printed rows, that reading implies log|R| <= 0, which
        Hadamard's inequality requires of a unit-diagonal correlation matrix,
        while the other readings (n log sigma2, or the full Gaussian form)
        would imply log|R| > 0 on the n = 4064 single-replication row."""
    g = np.random.default_rng(29)
    x = g.random((12, 2))
    y = g.standard_normal(12)
    o, st = orc.nll(x, y, [3.0, 4.0], 2.0, 1e-8)
    assert st == 0
    assert abs((o["nll"] - o["logdet"]) - 12 * math.log(12 * o["sigma2"])) < 1e-10
    with open(os.path.join(GOLDEN, "paper_table_rows.json")) as f:
        rows = json.load(f)["rows"]
    for row in rows:
        n, nll, s2 = row["n"], row["nll"], row["sigma2"]
        assert nll - n * math.log(n * s2) < 0.0, row["cite"]
    big = rows[0]
    n, nll, s2 = big["n"], big["nll"], big["sigma2"]
    assert nll - n * math.log(s2) > 0.0
    assert nll - n * math.log(s2) - n * (1 + math.log(2 * math.pi)) > 0.0


# --------------------------------------------------------- prediction -------

def check_predict(orc, seed=31):
    g = np.random.default_rng(seed)
    n, d = 30, 2
    x = g.random((n, d))
    y = np.sin(5 * x[:, 0]) + x[:, 1] ** 2
    th = [4.0, 2.0]
    p = 1.95
    # delta = 0: interpolation at the design points, zero variance
    yh, s2, st = orc.predict(x, y, th, p, 0.0, x[:7])
    assert st == 0
    assert np.max(np.abs(yh - y[:7])) < 1e-8
    assert np.max(np.abs(s2)) < 1e-8
    # a point far from every design point: r = 0 -> mu_hat, sigma2 (1 + delta + 1/1'R^-1 1)
    delta = 1e-6
    o, _ = orc.nll(x, y, th, p, delta)
    far = np.array([[40.0, 40.0]])
    R = orc.corr_matrix(x, th, p, delta)
    A = np.ones(n) @ np.linalg.solve(R, np.ones(n))
    yh, s2, st = orc.predict(x, y, th, p, delta, far)
    assert _rel(yh[0], o["mu"]) < 1e-12
    assert _rel(s2[0], o["sigma2"] * (1 + delta + 1.0 / A)) < 1e-9
    yh, s2n, _ = orc.predict(x, y, th, p, delta, far, nugget_in_var=False)
    assert _rel(s2n[0], o["sigma2"] * (1 + 1.0 / A)) < 1e-9
    # general points against LAPACK solves
    xs = g.random((9, d))
    yh, s2, _ = orc.predict(x, y, th, p, delta, xs)
    one = np.ones(n)
    Ri1 = np.linalg.solve(R, one)
    w = np.linalg.solve(R, y - o["mu"])
    for m in range(9):
        r = np.array([math.exp(-sum(th[k] * abs(xs[m, k] - x[i, k]) ** p for k in range(d)))
                      for i in range(n)])
        Rir = np.linalg.solve(R, r)
        ref_y = o["mu"] + r @ w
        ref_s = o["sigma2"] * (1 + delta - r @ Rir + (1 - one @ Rir) ** 2 / (one @ Ri1))
        assert abs(yh[m] - ref_y) < 1e-9 * max(1, abs(ref_y))
        assert abs(s2[m] - ref_s) < 1e-9 * o["sigma2"]
    # the variance is never negative beyond rounding
    assert np.all(s2 > -1e-12)


def check_fit_parts(orc, seed=37):
    """The intermediate vectors of one fit against LAPACK: L L' = R,
    a = L^-1 1, b = L^-1 Y, w = R^-1 (Y - 1 mu_hat)."""
    g = np.random.default_rng(seed)
    n = 20
    x = g.random((n, 3))
    y = g.standard_normal(n)
    th = [2.0, 3.0, 1.5]
    R, L, a, b, w, st = orc.fit_parts(x, y, th, 1.95, 1e-6)
    assert st == 0
    assert np.max(np.abs(L @ L.T - R)) < 1e-13
    assert np.max(np.abs(L @ a - 1.0)) < 1e-10
    assert np.max(np.abs(L @ b - y)) < 1e-10
    one = np.ones(n)
    mu = (one @ np.linalg.solve(R, y)) / (one @ np.linalg.solve(R, one))
    assert np.max(np.abs(w - np.linalg.solve(R, y - mu))) < 1e-8 * max(1.0, np.max(np.abs(w)))


# ----------------------------------------------------------------- Matern --
# The Matern family (Section 2 names it as an alternative, without a formula)
# in product form over dimensions with h = theta_k |dx_k|.  The pins below do
# not retype the closed forms: nu = 1/2 must equal eq. (2) with p = 1, and
# nu = 3/2, 5/2 must equal the general Matern correlation
#   rho(h) = 2^(1-nu) / Gamma(nu) (sqrt(2 nu) h)^nu K_nu(sqrt(2 nu) h),
# evaluated with SciPy's modified Bessel function K_nu.

def _matern_bessel(nu, h):
    from scipy.special import gamma, kv
    h = np.asarray(h, dtype=np.float64)
    z = np.sqrt(2.0 * nu) * h
    out = np.ones_like(z)
    nz = z > 0
    out[nz] = 2.0 ** (1.0 - nu) / gamma(nu) * z[nz] ** nu * kv(nu, z[nz])
    return out


def check_matern_half_is_exponential(orc, seed=41):
    """nu = 1/2 is the exponential correlation: eq. (2) with p = 1."""
    g = np.random.default_rng(seed)
    x = g.random((25, 3))
    th = 10 ** g.uniform(-1, 1, 3)
    Rm = orc.corr_matrix(x, th, 1.7, 1e-3, corr="matern12")
    Rp = orc.corr_matrix(x, th, 1.0, 1e-3, corr="powexp")
    assert np.max(np.abs(Rm - Rp)) <= 1e-15
    y = g.standard_normal(25)
    om, sm = orc.nll(x, y, th, 1.7, 1e-3, corr="matern12")
    op, sp = orc.nll(x, y, th, 1.0, 1e-3, corr="powexp")
    assert sm == sp == 0 and _rel(om["nll"], op["nll"]) < 1e-13


def check_matern_bessel(orc):
    """nu = 3/2 and 5/2 against the Bessel-function definition, in one and
    two dimensions (product form), p ignored."""
    for fam, nu in (("matern32", 1.5), ("matern52", 2.5)):
        for a in (1e-3, 0.05, 0.3, 0.9):
            for th in (0.2, 1.0, 6.0):
                x = np.array([[0.0], [a]])
                R = orc.corr_matrix(x, [th], 0.5, 0.0, corr=fam)
                ref = float(_matern_bessel(nu, th * a))
                assert abs(R[0, 1] - ref) <= 1e-12 * max(ref, 1e-300) + 1e-300, (fam, a, th, R[0, 1], ref)
                assert R[0, 0] == 1.0 and R[1, 0] == R[0, 1]
        x = np.array([[0.1, 0.7], [0.45, 0.2]])
        th = np.array([2.0, 0.8])
        R = orc.corr_matrix(x, th, 2.0, 0.0, corr=fam)
        ref = float(_matern_bessel(nu, 2.0 * 0.35) * _matern_bessel(nu, 0.8 * 0.5))
        assert _rel(R[0, 1], ref) < 1e-12


def check_matern_n2(orc):
    """The n = 2 hand derivation of -2logL with a Matern correlation (rho from
    the Bessel form): mu_hat, Q, log|R| and eq. (4)."""
    x = np.array([[0.2, 0.3], [0.5, 0.1]])
    th = np.array([1.2, 3.0])
    y = np.array([0.3, 1.9])
    for fam, nu in (("matern32", 1.5), ("matern52", 2.5)):
        rho = float(_matern_bessel(nu, 1.2 * 0.3) * _matern_bessel(nu, 3.0 * 0.2))
        out, st = orc.nll(x, y, th, 2.0, 0.0, corr=fam)
        assert st == 0
        Q = (y[0] - y[1]) ** 2 / (2.0 * (1.0 - rho))
        logdet = math.log(1.0 - rho * rho)
        assert _rel(out["mu"], 1.1) < 1e-14
        assert _rel(out["Q"], Q) < 1e-11
        assert _rel(out["nll"], logdet + 2 * math.log(Q)) < 1e-11


def check_matern_predict(orc, seed=43):
    """Kriging with a Matern correlation against LAPACK solves of the
    oracle's own R (the family only enters through R and r)."""
    g = np.random.default_rng(seed)
    n, d = 30, 2
    x = g.random((n, d))
    y = np.sin(4 * x[:, 0]) + x[:, 1]
    th = np.array([3.0, 1.5])
    xs = g.random((5, d))
    R = orc.corr_matrix(x, th, 2.0, 1e-6, corr="matern52")
    one = np.ones(n)
    a = np.linalg.solve(R, one)
    mu = one @ np.linalg.solve(R, y) / (one @ a)
    w = np.linalg.solve(R, y - mu)
    yhat, s2, st = orc.predict(x, y, th, 2.0, 1e-6, xs, corr="matern52")
    assert st == 0
    for m in range(len(xs)):
        r = orc.cross_corr(x, xs[m], th, 2.0, corr="matern52")
        assert _rel(yhat[m], mu + r @ w) < 1e-9
        # r from the Bessel form, dimension by dimension
        rb = np.prod([_matern_bessel(2.5, th[k] * np.abs(x[:, k] - xs[m, k])) for k in range(d)], axis=0)
        assert np.max(np.abs(r - rb)) < 1e-12


# --------------------------------------------------------------- gradient --

def check_grad_finite_differences(orc, seed=47):
    """d(-2logL)/dtheta against central differences of the oracle's own
    -2logL (which the other pins fix), for eq. (2) and the Matern forms."""
    g = np.random.default_rng(seed)
    n, d = 25, 3
    x = g.random((n, d))
    y = np.sin(3 * x[:, 0]) + x[:, 1] * x[:, 2]
    th = np.array([2.0, 0.7, 4.0])
    for corr, p in (("powexp", 1.95), ("powexp", 1.0), ("matern12", 2.0), ("matern32", 2.0), ("matern52", 2.0)):
        grad, out, st = orc.nll_grad(x, y, th, p, 1e-3, corr=corr)
        assert st == 0
        _, st2 = orc.nll(x, y, th, p, 1e-3, corr=corr)
        for k in range(d):
            h = 1e-5 * th[k]
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fp = orc.nll(x, y, tp, p, 1e-3, corr=corr)[0]["nll"]
            fm = orc.nll(x, y, tm, p, 1e-3, corr=corr)[0]["nll"]
            fd = (fp - fm) / (2 * h)
            assert abs(grad[k] - fd) <= 1e-6 * max(abs(fd), 1.0), (corr, k, grad[k], fd)


def check_grad_n2(orc):
    """n = 2: -2logL = log((1+delta)^2 - rho^2) + 2 log Q with
    Q = (y1-y2)^2 / (2 (1 + delta - rho)), so with drho = rho dlog rho,
    d(-2logL) = drho [-2 rho / ((1+delta)^2 - rho^2) + 2 / (1 + delta - rho)]."""
    x = np.array([[0.1, 0.2], [0.4, 0.6]])
    th = np.array([1.5, 0.7])
    y = np.array([1.25, -0.5])
    p, delta = 1.95, 1e-2
    rho = math.exp(-1.5 * 0.3 ** p) * math.exp(-0.7 * 0.4 ** p)
    grad, out, st = orc.nll_grad(x, y, th, p, delta)
    assert st == 0
    common = -2 * rho / ((1 + delta) ** 2 - rho ** 2) + 2 / (1 + delta - rho)
    for k, dx in enumerate((0.3, 0.4)):
        drho = rho * -(dx ** p)
        assert _rel(grad[k], drho * common) < 1e-12


ALL_CHECKS = [
    check_corr_hand_values, check_corr_invariants, check_kms, check_n1, check_n2,
    check_n3, check_eig_logdet, check_solve_estimates, check_cholesky_reconstructs,
    check_notpd, check_cond_estimate, check_invariants, check_table_form, check_predict,
    check_fit_parts, check_matern_half_is_exponential, check_matern_bessel, check_matern_n2,
    check_matern_predict, check_grad_finite_differences, check_grad_n2, check_gauss_jordan_estimates,
]


# ----------------------------------------- the oracle's own rounding error --
#
# The long-double build of the oracle (oracle.extended()) runs the same
# definitions with a 64-bit significand.  It is pinned to the exact KMS closed
# form at 50 digits, and then bounds the double oracle's own rounding error on
# cases without a closed form.  These checks take both builds, so they stay out
# of ALL_CHECKS (a planted mistake in the double build alone would disagree
# with the intact extended build and tell nothing about the pins).

def _ld_to_mpf(v, mpmath):
    """Exact value of a numpy.longdouble as an mpmath number (a sum of three
    doubles covers the 64- and the 113-bit significand)."""
    v = np.longdouble(v)
    total = mpmath.mpf(0)
    for _ in range(3):
        h = float(v)
        total += mpmath.mpf(h)
        v = v - np.longdouble(h)
    return total


def _kms_exact(n, theta, h, y, mpmath):
    """-2logL, sigma2, log|R| of the KMS case in 50-digit arithmetic, for the
    rho the double inputs define: rho = exp(-theta h) with theta and h exact."""
    mpmath.mp.dps = 50
    rho = mpmath.exp(-mpmath.mpf(theta) * mpmath.mpf(h))
    c = 1 / (1 - rho * rho)
    ys = [mpmath.mpf(float(v)) for v in y]
    one = [mpmath.mpf(1)] * n

    def qf(u, v):
        s = mpmath.mpf(0)
        for i in range(n):
            s += u[i] * (1 if i in (0, n - 1) else 1 + rho * rho) * v[i]
        for i in range(1, n):
            s -= rho * (u[i] * v[i - 1] + u[i - 1] * v[i])
        return c * s
    A, B, C = qf(one, one), qf(one, ys), qf(ys, ys)
    Q = C - B * B / A
    logdet = (n - 1) * mpmath.log(1 - rho * rho)
    return {"nll": logdet + n * mpmath.log(Q), "mu": B / A, "sigma2": Q / n, "logdet": logdet}


def check_extended_kms_exact(ext, mpmath, seed=61):
    """The extended build within n cond(R) 2^-64 of the exact KMS values,
    relative to max(|value|, 1), for n = 2 to 120 and rho = 0.5 to 0.99, with
    cond(R) <= ((1 + rho) / (1 - rho))^2 (the KMS eigenvalue bounds).  That is
    2^11 below the double arithmetic's n cond u, whose evaluation is off by
    1e-17 to 2e-13 on these cases: the extended arithmetic is at work."""
    g = np.random.default_rng(seed)
    h = 1.0 / 1024.0
    for n in (2, 5, 33, 120):
        for rho in (0.5, 0.9, 0.99):
            theta = -math.log(rho) / h
            x = (np.arange(n, dtype=np.float64) * h).reshape(n, 1)
            y = g.standard_normal(n)
            exact = _kms_exact(n, theta, h, y, mpmath)
            out, st = ext.nll(x, y, [theta], 1.0, 0.0)
            assert st == 0
            bound = n * ((1 + rho) / (1 - rho)) ** 2 * 2.0 ** -64
            for k in ("nll", "mu", "sigma2", "logdet"):
                err = abs((_ld_to_mpf(out[k], mpmath) - exact[k]) / max(abs(exact[k]), 1))
                assert err <= bound, (n, rho, k, float(err), bound)


def check_double_within_rounding_bound(orc, ext, seed=7):
    """The double oracle's own error, measured against the extended build:
    -2logL, mu_hat, sigma2_hat, log|R|, kriging and the gradient within
    8 n cond_1(R) u (u = 2^-53) of the extended values, relative to
    max(|value|, 1) (sigma2_hat for the variance), for every family.  The
    largest ratio seen is about one."""
    from paper_1203_1269_gb300 import inputs
    u = 2.0 ** -53
    g = np.random.default_rng(seed)
    ratios = []
    for corr in ("powexp", "matern12", "matern32", "matern52"):
        for n, d in ((3, 1), (10, 2), (40, 3), (100, 4)):
            x = inputs.random_lhd(g, n, d)
            y = inputs.y_sinsum(x)
            for th in inputs.log_uniform_thetas(g, 4, d, lo=-1.0, hi=1.0):
                od, sd = orc.nll(x, y, th, 1.95, 1e-8, want_cond=True, corr=corr)
                oe, se = ext.nll(x, y, th, 1.95, 1e-8, corr=corr)
                assert sd == se
                if sd != 0:
                    continue
                bound = n * od["cond1"] * u
                for k in ("nll", "mu", "sigma2", "logdet"):
                    e = float(oe[k])
                    ratios.append(abs(od[k] - e) / max(abs(e), 1.0) / bound)
                xs = g.random((5, d))
                yd, vd, _ = orc.predict(x, y, th, 1.95, 1e-8, xs, corr=corr)
                ye, ve, _ = ext.predict(x, y, th, 1.95, 1e-8, xs, corr=corr)
                ye, ve = ye.astype(np.float64), ve.astype(np.float64)
                ratios.append(np.max(np.abs(yd - ye)) / max(1.0, np.max(np.abs(ye))) / bound)
                ratios.append(np.max(np.abs(vd - ve)) / float(oe["sigma2"]) / bound)
                if n > 1:
                    gd, _, _ = orc.nll_grad(x, y, th, 1.95, 1e-8, corr=corr)
                    ge, _, _ = ext.nll_grad(x, y, th, 1.95, 1e-8, corr=corr)
                    ge = ge.astype(np.float64)
                    ratios.append(np.max(np.abs(gd - ge)) / max(1.0, np.max(np.abs(ge))) / bound)
    assert max(ratios) <= 8.0, max(ratios)
    return max(ratios)
