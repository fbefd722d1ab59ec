"""Pins for the oracle's physicality-enforcing operator (Sec. 2.5)."""
import numpy as np
import pytest

import oracle
import workloads as wl

SPEC = dict(dim=2, degree=2, n_elem=[20, 15], eos="ideal", gamma_ad=5.0 / 3.0)


def node_weights(N, dim):
    w = np.polynomial.legendre.leggauss(N)[1]
    out = w
    for _ in range(dim - 1):
        out = np.multiply.outer(w, out).ravel()
    return out


def q_stable(U):
    S2 = U[1] ** 2 + U[2] ** 2 + U[3] ** 2
    return U[4] - S2 / (U[0] + np.sqrt(U[0] ** 2 + S2))


def admissible(U):
    return (U[0] > 0) & (q_stable(U) > 0)


@pytest.fixture(scope="module")
def cells():
    U = wl.random_conserved_cells(300, 9, seed=31)
    w = node_weights(3, 2)
    mean = (U * w).sum(-1) / w.sum()
    flagged = ~admissible(U).all(-1)
    good_mean = admissible(mean)
    return U, w, mean, flagged, good_mean


def test_fixture_exercises_every_branch(cells):
    U, w, mean, flagged, good_mean = cells
    assert (~flagged).sum() > 30 and (flagged & good_mean).sum() > 30 and (flagged & ~good_mean).sum() > 5


def test_identity_on_admissible_cells(cells):
    U, w, mean, flagged, good_mean = cells
    Un, s, st = oracle.enforce(SPEC, U)
    assert np.array_equal(Un[:, ~flagged], U[:, ~flagged])
    assert np.all(s[~flagged] == 1.0)


def test_output_admissible_and_mean_preserved(cells):
    U, w, mean, flagged, good_mean = cells
    Un, s, st = oracle.enforce(SPEC, U)
    fix = flagged & good_mean
    assert admissible(Un[:, fix]).all()
    new_mean = (Un * w).sum(-1) / w.sum()
    assert np.allclose(new_mean[:, fix], mean[:, fix], rtol=0, atol=1e-14 * np.abs(U).max())
    assert np.all((s[fix] > 0) & (s[fix] < 1))
    assert st["enforced_cells"] == fix.sum()
    assert st["mean_inadmissible_cells"] == (flagged & ~good_mean).sum()


def test_inadmissible_mean_left_unchanged(cells):
    U, w, mean, flagged, good_mean = cells
    Un, s, _ = oracle.enforce(SPEC, U)
    bad = flagged & ~good_mean
    assert np.array_equal(Un[:, bad], U[:, bad])
    assert np.all(s[bad] == 1.0)


def test_factor_is_largest_admissible_by_bisection(cells):
    """s equals (1 - 1e-12) times the largest s in [0, 1] for which every smoothed node
    s U_i + (1 - s) Ubar is admissible, found by 200 bisection steps per cell."""
    U, w, mean, flagged, good_mean = cells
    _, s, _ = oracle.enforce(SPEC, U)
    fix = np.where(flagged & good_mean)[0]
    lo = np.zeros(len(fix))
    hi = np.ones(len(fix))
    Uc = U[:, fix]
    Mc = mean[:, fix][:, :, None]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        ok = admissible(mid[None, :, None] * Uc + (1 - mid[None, :, None]) * Mc).all(-1)
        lo = np.where(ok, mid, lo)
        hi = np.where(ok, hi, mid)
    assert np.allclose(s[fix] / (1 - 1e-12), lo, rtol=1e-12, atol=1e-14)
