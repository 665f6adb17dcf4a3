"""CPU tests: the oracle against the pins in oracle_pins.py (no GPU)."""
import numpy as np
import pytest

import oracle
import oracle_pins as pins


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(orc, check):
    check(orc)


@pytest.mark.parametrize("n,rho", [(2, 0.5), (3, 0.9), (200, 0.8), (257, 0.3)])
def test_kms_sizes(orc, n, rho):
    pins.check_kms(orc, n=n, rho_target=rho)


def test_batch_matches_single(orc):
    from paper_1203_1269_gb300 import inputs
    w = inputs.small_grid_fit(n=40, N=0)
    out, st = orc.nll_batch(w.x, w.y, w.thetas[:9], w.p, w.delta, want_cond=True)
    for t in range(9):
        o, s = orc.nll(w.x, w.y, w.thetas[t], w.p, w.delta, want_cond=True)
        assert s == st[t]
        assert np.array_equal(np.array([o[k] for k in oracle.NLL_FIELDS]), out[t])


def test_extended_build_matches_exact_kms():
    """The long-double build of the oracle against the KMS closed form in
    50-digit arithmetic."""
    mpmath = pytest.importorskip("mpmath")
    pins.check_extended_kms_exact(oracle.extended(), mpmath)


def test_double_oracle_error_within_rounding_bound(orc):
    """The double oracle's own rounding error, bounded through the extended
    build: within 8 n cond_1(R) u everywhere it is compared."""
    worst = pins.check_double_within_rounding_bound(orc, oracle.extended())
    print(f"\nworst |double - extended| / (n cond u): {worst:.2f}")
