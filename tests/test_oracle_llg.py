"""Pins of the oracle's precessional dynamics (Eq. 9 in reduced units), CPU.

For a lone spin under uniaxial anisotropy h = 2 K s_z z, Eq. 9 with a = 1/(1 + alpha^2) and
b = alpha/(1 + alpha^2) separates in polar angles:
    d theta/d tau = -b K sin(2 theta)      -> tan(theta) = tan(theta0) exp(-2 K b tau)
    d phi/d tau   =  a 2 K cos(theta)      -> phi - phi0 = (1/alpha) [asinh(exp(2 K b tau)/tan(theta0))
                                                                    - asinh(1/tan(theta0))]  (alpha > 0)
                                           -> phi - phi0 = 2 K cos(theta0) tau                 (alpha = 0)
A dropped or mis-signed precession or damping term fails these.  Without damping the energy is
conserved on a lattice with every interaction; with damping it decreases.  The Euler variant converges
to the closed form at first order.
"""
import math

import numpy as np
import pytest

import oracle


def _spin(theta, phi):
    return np.array([[[math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)]]])


def _angles(s):
    x, y, z = s[0, 0]
    return math.atan2(math.hypot(x, y), z), math.atan2(y, x)


def _closed(theta0, K, alpha, tau):
    a, b = 1.0 / (1.0 + alpha ** 2), alpha / (1.0 + alpha ** 2)
    th = math.atan(math.tan(theta0) * math.exp(-2 * K * b * tau))
    if alpha == 0.0:
        ph = 2 * K * math.cos(theta0) * tau
    else:
        t0 = math.tan(theta0)
        ph = (math.asinh(math.exp(2 * K * b * tau) / t0) - math.asinh(1.0 / t0)) / alpha
    return th, ph


@pytest.mark.parametrize("alpha", [0.0, 0.1, 0.5, 2.0])
def test_lone_spin_precession_and_damping_closed_form(alpha):
    K, theta0, T, n = 0.8, 1.1, 0.5, 6
    m = oracle.model(1, 1, 1, 0.0, 0.0, K, 0.0)
    phi, _, _, (acc, rej) = oracle.llg_run_rk(m, _spin(theta0, 0.0), n, T, alpha, rtol=1e-11, atol=1e-13)
    th, ph = _angles(phi)
    th_want, ph_want = _closed(theta0, K, alpha, n * T)
    assert abs(th - th_want) < 1e-8
    assert abs(math.remainder(ph - ph_want, 2 * math.pi)) < 1e-8
    assert acc >= n


def test_energy_conserved_without_damping_and_decreasing_with_it():
    m = oracle.model(4, 4, 2, 1.0, 0.3, 0.1, 0.05)
    rng = np.random.default_rng(4)
    s0 = rng.standard_normal((1, 32, 3))
    s0 /= np.linalg.norm(s0, axis=-1, keepdims=True)
    e0 = oracle.energies(m, s0)[0]
    _, e, _, _ = oracle.llg_run_rk(m, s0, 4, 0.5, 0.0, rtol=1e-10, atol=1e-12)
    assert abs(e[0] - e0) < 1e-7 * abs(e0)
    prev = e0
    s = s0
    for _ in range(5):
        s, e = oracle.llg_run(m, s, 10, 0.02, 0.3)
        assert e[0] < prev
        prev = e[0]


def test_euler_converges_at_first_order():
    K, theta0, alpha, tau = 0.8, 1.1, 0.3, 1.0
    m = oracle.model(1, 1, 1, 0.0, 0.0, K, 0.0)
    th_want, ph_want = _closed(theta0, K, alpha, tau)
    errs = []
    for n in (100, 200, 400):
        phi, _ = oracle.llg_run(m, _spin(theta0, 0.0), n, tau / n, alpha)
        th, ph = _angles(phi)
        errs.append(math.hypot(th - th_want, math.remainder(ph - ph_want, 2 * math.pi)))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_images_evolve_independently():
    # no reparametrisation and no coupling: a batch equals its images run one by one
    m = oracle.model(4, 4, 1, 1.0, 0.3, 0.05, 0.02)
    rng = np.random.default_rng(6)
    s = rng.standard_normal((3, 16, 3))
    s /= np.linalg.norm(s, axis=-1, keepdims=True)
    both, _ = oracle.llg_run(m, s, 7, 0.05, 0.2)
    for k in range(3):
        one, _ = oracle.llg_run(m, s[k:k + 1], 7, 0.05, 0.2)
        np.testing.assert_allclose(both[k], one[0], atol=1e-15)
