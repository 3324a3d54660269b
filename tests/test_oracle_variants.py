"""Pins of the oracle's reparametrisation variants and climbing image (Sec. III), CPU.

* the natural cubic spline agrees with scipy's independent implementation (natural end conditions),
  and reproduces collinear knots exactly (where it must equal linear interpolation);
* with a climbing image kc the reparametrisation is the plain one applied to [0, kc] and [kc, K-1];
* the climbing image converges to the saddle: on a lone spin under anisotropy (E = -K s_z^2) the
  barrier is K exactly, and on a small ferromagnet (exchange + anisotropy, coherent rotation) it is
  N K, while the plain string with no image on the equator stays below; the force on the climbing
  image vanishes there;
* no image climbs in the first iteration, and the climbing image is the interior maximum of the
  energies the previous iteration started from.
"""
import math

import numpy as np
import pytest

import oracle


def _unit(a):
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _random_path(K, n_sites, seed, spread=0.6):
    """A smooth but unevenly spaced path: every site turns about its own random axis by an angle
    growing unevenly with k."""
    rng = np.random.default_rng(seed)
    a = _unit(rng.standard_normal((n_sites, 3)))
    ax = _unit(rng.standard_normal((n_sites, 3)))
    out = np.empty((K, n_sites, 3))
    for k in range(K):
        th = spread * 3 * (k / (K - 1)) ** 1.7
        c, s = np.cos(th), np.sin(th)
        out[k] = a * c + np.cross(ax, a) * s + ax * (ax * a).sum(-1, keepdims=True) * (1 - c)
    return out


def test_spline_matches_scipy_natural_cubic_spline():
    interp = pytest.importorskip("scipy.interpolate")
    K, n = 9, 5
    path = _random_path(K, n, seed=1)
    got, alpha = oracle.reparam_v(path, spline=True, return_alpha=True)
    d = np.sqrt(((path[1:] - path[:-1]) ** 2).sum(axis=(1, 2)))
    x = np.concatenate([[0.0], np.cumsum(d)]) / d.sum()
    np.testing.assert_allclose(alpha, x, atol=1e-15)
    cs = interp.CubicSpline(x, path.reshape(K, -1), bc_type="natural")
    want = cs(np.arange(K) / (K - 1)).reshape(K, n, 3)
    want = _unit(want)
    want[0], want[-1] = path[0], path[-1]
    np.testing.assert_allclose(got, want, atol=1e-13)
    # and it differs from the linear interpolation (the test would not see a linear fallback)
    assert np.abs(got - oracle.reparam_v(path)).max() > 1e-4


def test_spline_reproduces_collinear_knots():
    # knots on a straight line in component space at uneven positions: the spline is that line, so it
    # equals linear interpolation (a dropped or mis-signed term of the spline breaks this)
    rng = np.random.default_rng(2)
    A, B = rng.standard_normal((2, 6, 3))
    pos = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0, 1, 5)]))
    path = A + pos[:, None, None] * (B - A)
    lin = oracle.reparam_v(path)
    spl = oracle.reparam_v(path, spline=True)
    np.testing.assert_allclose(spl, lin, atol=1e-13)
    # linear interpolation onto equal spacing puts image k at A + (k / (K - 1)) (B - A), renormalised
    want = _unit(A + (np.arange(7) / 6.0)[:, None, None] * (B - A))
    np.testing.assert_allclose(lin[1:-1], want[1:-1], atol=1e-13)


@pytest.mark.parametrize("spline", [False, True])
def test_climbing_split_is_two_plain_reparametrisations(spline):
    K, n, kc = 11, 4, 4
    path = _random_path(K, n, seed=3)
    got = oracle.reparam_v(path, spline=spline, kc=kc)
    left = oracle.reparam_v(path[:kc + 1], spline=spline)
    right = oracle.reparam_v(path[kc:], spline=spline)
    np.testing.assert_allclose(got[:kc + 1], left, atol=1e-15)
    np.testing.assert_allclose(got[kc:], right, atol=1e-15)
    np.testing.assert_array_equal(got[kc], path[kc])
    # kc = 0 or K - 1 means no climbing image: the plain reparametrisation
    np.testing.assert_allclose(oracle.reparam_v(path, spline=spline, kc=0), oracle.reparam_v(path, spline=spline),
                               atol=0)


def test_linear_variant_equals_plain_reparam():
    path = _random_path(8, 6, seed=4)
    np.testing.assert_array_equal(oracle.reparam_v(path), oracle.reparam(path))


def _great_circle_path(K, n_sites):
    th = np.linspace(0.0, math.pi, K)
    one = np.stack([np.sin(th), np.zeros(K), np.cos(th)], axis=-1)
    return np.repeat(one[:, None, :], n_sites, axis=1)


@pytest.mark.parametrize("spline", [False, True])
def test_climbing_image_reaches_lone_spin_saddle(spline):
    Ka, K = 0.5, 8  # no image on the equator of an 8-image great circle
    m = oracle.model(1, 1, 1, 0.0, 0.0, Ka, 0.0)
    path = _great_circle_path(K, 1)
    _, e_plain = oracle.string_run(m, path, 300, 0.2)
    phi, e, kc = oracle.string_run_v(m, path, 300, 0.2, spline=spline, climb=True)
    assert oracle.barrier(e_plain)[0] < Ka * 0.96
    dE, k = oracle.barrier(e)
    assert abs(dE - Ka) < 1e-9 and k == kc
    assert abs(phi[kc, 0, 2]) < 1e-5  # on the equator
    h = oracle.field(m, phi[kc])
    F = h - (h * phi[kc]).sum(-1, keepdims=True) * phi[kc]
    assert np.abs(F).max() < 1e-5


def test_climbing_image_coherent_rotation_barrier():
    # 3x3 ferromagnet, exchange and anisotropy only: the uniform rotation is the minimum energy path
    # and its saddle (all spins in plane) lies N K above the uniform minimum
    J, Ka = 1.0, 0.2
    m = oracle.model(3, 3, 1, J, 0.0, Ka, 0.0)
    path = _great_circle_path(10, 9)
    phi, e, kc = oracle.string_run_v(m, path, 300, 0.1, climb=True)
    assert abs(oracle.barrier(e)[0] - 9 * Ka) < 1e-8
    _, e_plain = oracle.string_run(m, path, 300, 0.1)
    assert oracle.barrier(e_plain)[0] < 9 * Ka - 1e-3


def test_first_iteration_has_no_climbing_image():
    m = oracle.model(4, 4, 1, 1.0, 0.3, 0.05, 0.02)
    path = _random_path(6, 16, seed=5)
    p1, e1, kc = oracle.string_run_v(m, path, 1, 0.1, climb=True)
    p0, e0 = oracle.string_run(m, path, 1, 0.1)
    np.testing.assert_array_equal(p1, p0)
    # the image that climbs next: the interior maximum of the energies of the path the iteration
    # started from
    e_start = oracle.energies(m, path)
    assert kc == 1 + int(np.argmax(e_start[1:-1]))
    # without climbing, the spline variant's first iteration is the Euler step then the spline
    p2, _, kc2 = oracle.string_run_v(m, path, 1, 0.1, spline=True)
    steps = np.stack([oracle.step(s, oracle.field(m, s), 0.1) for s in _unit(path)])
    np.testing.assert_allclose(p2, oracle.reparam_v(steps, spline=True), atol=1e-14)
    assert kc2 == -1
