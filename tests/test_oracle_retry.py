"""Pins of the oracle's limiter retry (Section 3.3 (1) of arXiv 2012.11130).

The paper redoes the reconstruction of a patch whose update is unphysical
with the minmod coefficient reduced by a factor 0.75, again and again, until
Eq. (Unphysical result) passes or the coefficient vanishes. The schedule is
fixed by that passage and one reading (a coefficient below 1e-2 of the
initial one is replaced by zero, piecewise-constant reconstruction), so the
coefficient of attempt k has the closed form

    theta_k = theta_0 * 0.75**k   if theta_0 * 0.75**k >= 1e-2 * theta_0,
              0                   otherwise,

and the last attempt is the first k whose closed form is 0.

These tests check the retry loop against that closed form without using
the loop's own bookkeeping: a patch that reports k retries must give,
bitwise, the output of a single attempt at theta_k (no retry), and a single
attempt at theta_{k-1} must fail (the loop took no passing coefficient
early). A wrongly compounded factor, a floor applied to the absolute instead
of the relative coefficient, or a skipped attempt changes theta_k and fails
these comparisons. CPU only."""
import numpy as np
import pytest

from paper_2012_11130_gb300 import workloads

THETA0, FACTOR, FLOOR = 1.5, 0.75, 1e-2


def theta_of_attempt(k, theta0=THETA0, factor=FACTOR, floor=FLOOR):
    """Closed form of the coefficient of attempt k (attempt 0 = no retry)."""
    t = theta0 * factor ** k
    return 0.0 if t < floor * theta0 else t


def last_attempt(theta0=THETA0, factor=FACTOR, floor=FLOOR):
    """First k whose coefficient is 0: the attempt after which a patch that
    is still unphysical is flagged."""
    k = 0
    while theta_of_attempt(k, theta0, factor, floor) > 0.0:
        k += 1
    return k


def _rough_patches(oracle, npatch, seed, spread, lg_gamma_max):
    Wp = workloads.rough_patch_prims(npatch, seed=seed, spread=spread,
                                     lg_gamma_max=lg_gamma_max)
    C, st = oracle.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1))
    assert np.all(st == 0)
    C = C.reshape(5, npatch, 12, 12, 12).transpose(1, 0, 2, 3, 4).copy()
    dh = 1.0 / 64
    dt = np.array([oracle.cfl_dt(C[q].reshape(5, -1), dh) for q in range(npatch)])
    return C, dt, dh


def _check_schedule(oracle, C, dt, dh, floor=FLOOR):
    """Every patch against single attempts at the closed-form coefficients;
    returns the retry counts."""
    K = last_attempt(floor=floor)
    ks = []
    for q in range(C.shape[0]):
        r = oracle.advance_block(C[q], (8, 8, 8), (1, 1, 1), dt[q], dh, theta_floor=floor)
        k = r["retries"]
        ks.append(k)
        assert 0 <= k <= K
        if r["status"] == oracle.BLK_UNPHYSICAL:
            # every attempt failed, the last one at theta = 0
            assert k == K
            one = oracle.advance_block(C[q], (8, 8, 8), (1, 1, 1), dt[q], dh, theta=0.0,
                                       theta_floor=floor)
            assert one["status"] == oracle.BLK_UNPHYSICAL and one["retries"] == 0
            continue
        assert r["status"] == oracle.BLK_OK
        # a single attempt at theta_k passes and gives the same bits
        one = oracle.advance_block(C[q], (8, 8, 8), (1, 1, 1), dt[q], dh,
                                   theta=theta_of_attempt(k, floor=floor), theta_floor=floor)
        assert one["retries"] == 0 and one["status"] == oracle.BLK_OK, (q, k)
        assert np.array_equal(one["out"], r["out"]), (q, k)
        if k > 0:
            # the attempt before it fails, and the next one passes: a run
            # started at theta_{k-1} (its floor rescaled so that the
            # threshold stays floor * theta_0) retries exactly once
            tp = theta_of_attempt(k - 1, floor=floor)
            prev = oracle.advance_block(C[q], (8, 8, 8), (1, 1, 1), dt[q], dh, theta=tp,
                                        theta_floor=floor * THETA0 / tp)
            assert prev["retries"] == 1, (q, k, prev["retries"])
            assert np.array_equal(prev["out"], r["out"]), (q, k)
    return np.array(ks)


def test_closed_form_schedule_of_the_defaults():
    # 1.5 * 0.75**16 = 0.01503 >= 0.015 > 1.5 * 0.75**17: attempts 0..16 use
    # a positive coefficient, attempt 17 the piecewise-constant one.
    assert theta_of_attempt(16) == pytest.approx(1.5 * 0.75 ** 16)
    assert theta_of_attempt(16) > 0.015 > 1.5 * 0.75 ** 17
    assert last_attempt() == 17
    assert theta_of_attempt(17) == 0.0


def test_retry_count_matches_single_attempt_at_theta_k(oracle):
    # Rough patches (uncorrelated cells, rho and T over +-1 decade, Lorentz
    # factors up to 10^1.5): every patch retries, most of them ten or more
    # times, so the compounding of the factor is exercised.
    C, dt, dh = _rough_patches(oracle, 12, seed=5, spread=1.0, lg_gamma_max=1.5)
    ks = _check_schedule(oracle, C, dt, dh)
    assert ks.min() >= 2 and len(set(ks.tolist())) >= 2


def test_floor_gives_piecewise_constant_attempt(oracle):
    # Rougher patches (+-2 decades, Lorentz factors up to 100): most need the
    # piecewise-constant attempt 17, and one stays unphysical even then.
    C, dt, dh = _rough_patches(oracle, 8, seed=10, spread=2.0, lg_gamma_max=2.0)
    ks = _check_schedule(oracle, C, dt, dh)
    assert np.sum(ks == last_attempt()) >= 4
    st = [oracle.advance_block(C[q], (8, 8, 8), (1, 1, 1), dt[q], dh)["status"] for q in (6, 7)]
    assert st == [oracle.BLK_OK, oracle.BLK_UNPHYSICAL]


def test_relative_floor(oracle):
    # A floor of 0.7 theta_0 leaves the attempts 1.5, 1.125 and then 0
    # (0.84375 < 1.05): the floor is relative to the initial coefficient.
    assert [theta_of_attempt(k, floor=0.7) for k in range(3)] == [1.5, 1.125, 0.0]
    C, dt, dh = _rough_patches(oracle, 4, seed=5, spread=1.0, lg_gamma_max=1.5)
    ks = _check_schedule(oracle, C, dt, dh, floor=0.7)
    assert np.all(ks == 2)
