"""Pins of the oracle's adaptive Runge-Kutta string evolution (Sec. III, Dormand-Prince 5(4)), CPU.

* the tableau satisfies the order conditions of a 5th-order method (b) with an embedded 4th-order one
  (bhat), and its rows sum to the nodes c = (0, 1/5, 3/10, 4/5, 8/9, 1, 1): a wrong coefficient fails;
* a lone spin under uniaxial anisotropy relaxes as dtheta/dtau = -K sin(2 theta) (Eq. 13 with
  h = 2K s_z z), i.e. tan(theta) = tan(theta0) exp(-2 K tau), and the integrator follows it within its
  tolerance, more closely as the tolerance tightens;
* a state where F = 0 is a fixed point (no rejected steps, no motion).
"""
import math

import numpy as np
import pytest

import oracle

C = np.array([0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1, 1])


def test_dormand_prince_order_conditions():
    a, b, bh = oracle.dp_tableau()
    A = np.zeros((7, 7))
    A[:, :6] = a
    np.testing.assert_allclose(A.sum(1), C, atol=1e-15)
    for w, order in ((b, 5), (bh, 4)):
        assert abs(w.sum() - 1) < 1e-15
        for p in range(1, order):  # quadrature conditions sum w c^p = 1/(p+1)
            assert abs(w @ C ** p - 1 / (p + 1)) < 1e-14, (order, p)
        assert abs(w @ (A @ C) - 1 / 6) < 1e-14
        assert abs(w @ (A @ C ** 2) - 1 / 12) < 1e-14
        assert abs(w @ (C * (A @ C)) - 1 / 8) < 1e-14
        assert abs(w @ (A @ (A @ C)) - 1 / 24) < 1e-14
    # fifth-order conditions hold for b only (bhat is the embedded fourth-order solution)
    assert abs(b @ (C ** 2 * (A @ C)) - 1 / 10) < 1e-14
    assert abs(b @ (A @ C ** 3) - 1 / 20) < 1e-14
    assert abs(b @ (A @ (A @ (A @ C))) - 1 / 120) < 1e-14
    assert abs(bh @ (A @ (A @ (A @ C))) - 1 / 120) > 1e-6


def _lone_spins(thetas):
    return np.array([[[math.sin(t), 0.0, math.cos(t)]] for t in thetas])


@pytest.mark.parametrize("rtol", [1e-6, 1e-9])
def test_lone_spin_anisotropy_relaxation_closed_form(rtol):
    K, T, n = 0.7, 0.5, 6
    m = oracle.model(1, 1, 1, 0.0, 0.0, K, 0.0)
    th0 = [1.0, 2.0]  # two single-spin images; a two-image string keeps both ends under reparametrisation
    phi, _, _, (acc, rej) = oracle.string_run_rk(m, _lone_spins(th0), n, T, rtol=rtol, atol=rtol * 1e-2)
    for k, t0 in enumerate(th0):
        want = math.atan2(math.tan(t0) * math.exp(-2 * K * n * T), 1.0)
        want = want + math.pi if t0 > math.pi / 2 else want
        got = math.atan2(phi[k, 0, 0], phi[k, 0, 2])
        assert abs(got - want) < 50 * rtol, (rtol, got - want)
    assert acc >= n


def test_tighter_tolerance_is_closer():
    K, T, n = 0.7, 0.5, 4
    m = oracle.model(1, 1, 1, 0.0, 0.0, K, 0.0)
    errs = []
    for rtol in (1e-4, 1e-8):
        phi, _, _, _ = oracle.string_run_rk(m, _lone_spins([1.0, 2.0]), n, T, rtol=rtol, atol=rtol * 1e-2)
        want = math.atan(math.tan(1.0) * math.exp(-2 * K * n * T))
        errs.append(abs(math.atan2(phi[0, 0, 0], phi[0, 0, 2]) - want))
    assert errs[1] < errs[0] / 100


def test_fixed_point_is_kept():
    # uniform +z on a 4x4x2 lattice with exchange and K > 0 only (DMI and the dipole field both tilt
    # the edge spins of an open sample): h is parallel to s everywhere, F = 0
    m = oracle.model(4, 4, 2, 1.0, 0.0, 0.1, 0.0)
    path = np.zeros((3, 32, 3))
    path[..., 2] = 1.0
    phi, _, _, (acc, rej) = oracle.string_run_rk(m, path, 3, 0.2)
    np.testing.assert_allclose(phi, path, atol=1e-14)
    assert rej == 0 and acc == 3


def test_per_image_systems_are_independent_single_image_runs():
    # A two-image string keeps both ends under reparametrisation, so with per-image step control each
    # image evolves as on its own.  A string of two identical copies has the same RMS error norm as one
    # copy, so the whole-string integrator run on [a, a] follows a alone: per_image([a, b]) must equal
    # (whole([a, a])[0], whole([b, b])[0]), attempt counts included, up to the summation order of the
    # norm (the error estimate is a difference of nearly equal sums, so its rounding reaches the carried
    # step at about 1e-11).
    m = oracle.model(4, 4, 1, 1.0, 0.3, 0.05, 0.02)
    rng = np.random.default_rng(3)
    a, b = (v / np.linalg.norm(v, axis=-1, keepdims=True) for v in rng.standard_normal((2, 16, 3)))
    T, n = 0.6, 3
    phi, _, steps, counts = oracle.string_run_rk(m, np.stack([a, b]), n, T, per_image=True)
    for k, v in enumerate((a, b)):
        ref, _, step, cnt = oracle.string_run_rk(m, np.stack([v, v]), n, T)
        np.testing.assert_allclose(phi[k], ref[0], rtol=0, atol=1e-14)
        assert abs(steps[k] - step) <= 1e-9 * step and tuple(counts[k]) == cnt
    assert tuple(counts[0]) != tuple(counts[1]) or steps[0] != steps[1]


def test_per_image_equals_whole_string_when_images_agree():
    # identical images: every image's norm equals the string's, so both controls take the same steps
    m = oracle.model(4, 4, 1, 1.0, 0.3, 0.05, 0.02)
    v = np.random.default_rng(5).standard_normal((16, 3))
    path = np.stack([v, v, v]) / np.linalg.norm(v, axis=-1, keepdims=True)
    p1, e1, s1, c1 = oracle.string_run_rk(m, path, 2, 0.6, per_image=True)
    p0, e0, s0, c0 = oracle.string_run_rk(m, path, 2, 0.6)
    np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-14)
    assert all(abs(s - s0) <= 1e-9 * s0 for s in s1) and all(tuple(c) == c0 for c in c1)


def test_overflowing_attempt_is_rejected_and_recovers():
    # Off the unit sphere F = h - (s.h) s grows like |s|^3, so a first attempt of length 1000 on a lone
    # spin overflows within the seven stages (a non-finite error norm); it must count as a rejection
    # with the smallest factor, and the run must still reach the closed-form relaxation.
    K, T = 0.7, 1000.0
    m = oracle.model(1, 1, 1, 0.0, 0.0, K, 0.0)
    with np.errstate(all="ignore"):
        phi, _, step, (acc, rej) = oracle.string_run_rk(m, _lone_spins([1.0, 2.0]), 1, T)
    assert rej >= 1 and step > 0
    assert abs(math.atan2(phi[0, 0, 0], phi[0, 0, 2])) < 1e-6
    assert abs(abs(math.atan2(phi[1, 0, 0], phi[1, 0, 2])) - math.pi) < 1e-6


C6 = np.array([0, 1 / 4, 3 / 8, 12 / 13, 1, 1 / 2])


def test_fehlberg_order_conditions():
    a, b4, b5 = oracle.rkf_tableau()
    A = np.zeros((6, 6))
    A[:, :5] = a
    np.testing.assert_allclose(A.sum(1), C6, atol=1e-15)
    for w, order in ((b4, 4), (b5, 5)):
        assert abs(w.sum() - 1) < 1e-15
        for p in range(1, order):
            assert abs(w @ C6 ** p - 1 / (p + 1)) < 1e-14, (order, p)
        assert abs(w @ (A @ C6) - 1 / 6) < 1e-14
        assert abs(w @ (A @ C6 ** 2) - 1 / 12) < 1e-14
        assert abs(w @ (C6 * (A @ C6)) - 1 / 8) < 1e-14
        assert abs(w @ (A @ (A @ C6)) - 1 / 24) < 1e-14
    assert abs(b5 @ (A @ (A @ (A @ C6))) - 1 / 120) < 1e-14
    assert abs(b5 @ C6 ** 4 - 1 / 5) < 1e-14
    assert abs(b4 @ C6 ** 4 - 1 / 5) > 1e-5  # b4 is fourth order only


@pytest.mark.parametrize("rtol", [1e-6, 1e-9])
def test_fehlberg_lone_spin_closed_form(rtol):
    K, T, n = 0.7, 0.5, 6
    m = oracle.model(1, 1, 1, 0.0, 0.0, K, 0.0)
    th0 = [1.0, 2.0]
    phi, _, _, (acc, rej) = oracle.string_run_rk(m, _lone_spins(th0), n, T, rtol=rtol, atol=rtol * 1e-2,
                                                 method="rkf45")
    for k, t0 in enumerate(th0):
        want = math.atan2(math.tan(t0) * math.exp(-2 * K * n * T), 1.0)
        want = want + math.pi if t0 > math.pi / 2 else want
        got = math.atan2(phi[k, 0, 0], phi[k, 0, 2])
        assert abs(got - want) < 100 * rtol, (rtol, got - want)
    assert acc >= n


def test_fehlberg_and_dormand_prince_agree_within_tolerance():
    m = oracle.model(4, 4, 1, 1.0, 0.3, 0.05, 0.02)
    rng = np.random.default_rng(8)
    path = rng.standard_normal((3, 16, 3))
    path /= np.linalg.norm(path, axis=-1, keepdims=True)
    a, _, _, ca = oracle.string_run_rk(m, path, 2, 0.5, 1e-9, 1e-11)
    b, _, _, cb = oracle.string_run_rk(m, path, 2, 0.5, 1e-9, 1e-11, method="rkf45")
    assert np.abs(a - b).max() < 1e-6
    assert ca != cb  # different pairs take different step sequences
