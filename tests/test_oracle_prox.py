"""Pins of the oracle's per-cell proximal map of J (section 3, step 2): the
optimality equations, the roots of the cubic from numpy.roots (companion
matrix eigenvalues, independent of Newton's method), Cardano's formula written
from the mathematics, brute-force minimisation, and the zero case."""
import numpy as np
import pytest

import oracle as o


def objective(u, v, am, af, sigma):
    J = o.J_energy([np.asarray(x, float) for x in u], np.asarray(v, float))
    pen = sum((np.asarray(u[k]) - am[k]) ** 2 for k in range(len(am)))
    return J + 0.5 * sigma * pen + 0.5 * sigma * (v - af) ** 2


def cardano_root(am2, af, sigma):
    """Largest real root of 2 (1 + s v)^2 (v - af) - s am2 = 0 by Cardano's formula.

    Expanded: 2 s^2 v^3 + (4 s - 2 s^2 af) v^2 + (2 - 4 s af) v - (2 af + s am2) = 0.
    """
    a = 2 * sigma ** 2
    b = 4 * sigma - 2 * sigma ** 2 * af
    c = 2 - 4 * sigma * af
    d = -(2 * af + sigma * am2)
    # depressed cubic t^3 + p t + q with v = t - b/(3a)
    p = (3 * a * c - b * b) / (3 * a * a)
    q = (2 * b ** 3 - 9 * a * b * c + 27 * a * a * d) / (27 * a ** 3)
    disc = (q / 2) ** 2 + (p / 3) ** 3
    if disc >= 0:
        sq = np.sqrt(disc)
        t = np.cbrt(-q / 2 + sq) + np.cbrt(-q / 2 - sq)
    else:   # three real roots: trigonometric form, take the largest
        r = np.sqrt(-p / 3)
        phi = np.arccos(np.clip(-q / (2 * r ** 3), -1, 1))
        t = 2 * r * np.cos(phi / 3)
    return t - b / (3 * a)


CASES = [
    # (a_m vector, a_f, sigma)
    ([0.3, -0.2, 0.1], 1.0, 0.3),
    ([2.0, 1.0, 0.0], 0.5, 1.0),
    ([0.01, 0.0, 0.0], 1e-3, 0.3),
    ([5.0, -3.0, 1.0], -2.0, 0.5),
    ([0.5], -0.05, 3.0),
    ([40.0, 0.0, 0.0], -100.0, 0.3),
    ([1e-4, 2e-4, 0.0], 3.0, 0.1),
]


@pytest.mark.parametrize("am,af,sigma", CASES)
def test_prox_optimality_and_cubic(am, af, sigma):
    am_a = [np.array([x]) for x in am]
    u, v = o.prox_J(am_a, np.array([af]), sigma)
    u = [x[0] for x in u]
    v = v[0]
    am2 = sum(x * x for x in am)
    assert v > 0
    # gradient of the objective vanishes (section 3, step 2)
    for k in range(len(am)):
        assert abs(u[k] / v + sigma * (u[k] - am[k])) <= 1e-12 * (1 + abs(am[k]) * sigma)
    uu = sum(x * x for x in u)
    assert abs(-0.5 * uu / v ** 2 + sigma * (v - af)) <= 1e-11 * (1 + sigma * abs(af) + sigma * v)
    # v is the largest real root of the cubic: numpy.roots and Cardano
    coeffs = [2 * sigma ** 2, 4 * sigma - 2 * sigma ** 2 * af, 2 - 4 * sigma * af, -(2 * af + sigma * am2)]
    roots = np.roots(coeffs)
    real = roots[np.abs(roots.imag) < 1e-9 * (1 + np.abs(roots.real))].real
    assert abs(v - real.max()) <= 1e-8 * (1 + v)
    assert abs(v - cardano_root(am2, af, sigma)) <= 1e-8 * (1 + v)


@pytest.mark.parametrize("am,af,sigma", CASES[:5])
def test_prox_brute_force(am, af, sigma):
    """Grid search in (v, scale of u along a_m) around the Newton answer."""
    am_a = [np.array([x]) for x in am]
    u, v = o.prox_J(am_a, np.array([af]), sigma)
    best = objective([x for x in u], v, [np.array([x]) for x in am], af, sigma)[0]
    vs = v[0] * np.linspace(0.5, 1.5, 401)
    rng = np.random.default_rng(0)
    for _ in range(20):
        pert = [x[0] * (1 + 0.2 * rng.standard_normal()) + 0.01 * rng.standard_normal() for x in u]
        for vv in vs:
            val = objective([np.array([p]) for p in pert], np.array([vv]), [np.array([x]) for x in am], af, sigma)[0]
            assert val >= best - 1e-12 * (1 + abs(best))


def test_prox_zero_case():
    """a_f + sigma |a_m|^2 / 2 <= 0 gives (0, 0), and (0, 0) beats nearby points."""
    sigma = 0.7
    am = [np.array([0.5]), np.array([-0.4])]
    af = np.array([-0.2])   # -0.2 + 0.35 * 0.41 < 0
    u, v = o.prox_J(am, af, sigma)
    assert v[0] == 0 and all(x[0] == 0 for x in u)
    f00 = objective([np.zeros(1), np.zeros(1)], np.zeros(1), am, af[0], sigma)[0]
    rng = np.random.default_rng(1)
    for _ in range(2000):
        vv = abs(rng.standard_normal()) * 0.5 + 1e-9
        uu = [rng.standard_normal(1) * 0.5 for _ in range(2)]
        assert objective(uu, np.array([vv]), am, af[0], sigma)[0] >= f00


def test_prox_vectorised_matches_scalar():
    rng = np.random.default_rng(4)
    n = 500
    am = [rng.standard_normal(n) * 2 for _ in range(3)]
    af = rng.standard_normal(n)
    u, v = o.prox_J(am, af, 0.3)
    for i in range(0, n, 37):
        us, vs = o.prox_J([np.array([a[i]]) for a in am], np.array([af[i]]), 0.3)
        assert vs[0] == pytest.approx(v[i], rel=1e-14, abs=0)
        for k in range(3):
            assert us[k][0] == pytest.approx(u[k][i], rel=1e-14, abs=1e-300)
