"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties one oracle function to something other than itself: a closed form, finite
differences of an independently coded quantity, geometry, a library FFT, or a textbook lattice sum.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1804_07135_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def n_bonds(nx, ny, nz):
    return (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)


# --- T1: uniform ferromagnet (Eq. 1) -------------------------------------------------------------

@pytest.mark.parametrize("dims", [(5, 4, 3), (16, 16, 1), (7, 1, 1)])
def test_ferromagnet_closed_form(dims):
    nx, ny, nz = dims
    J, D, K = 1.3, 0.4, 0.07
    m = oracle.model(nx, ny, nz, J, D, K, 0.0)
    for axis in range(3):
        s = np.zeros((nx * ny * nz, 3))
        s[:, axis] = 1.0
        e = oracle.energy_terms(m, s)
        assert e["exchange"] == pytest.approx(-J * n_bonds(nx, ny, nz), rel=1e-14)
        assert e["dmi"] == 0.0  # s_i x s_j = 0 for parallel spins
        assert e["anisotropy"] == pytest.approx(-K * nx * ny * nz if axis == 2 else 0.0, abs=1e-12)


def test_ferromagnet_interior_field():
    m = oracle.model(5, 5, 5, 1.0, 0.3, 0.05, 0.0)
    s = W.ferromagnet(5, 5, 5)
    h = oracle.field(m, s).reshape(5, 5, 5, 3)
    # interior site: six neighbours (Eq. 3), DMI differences vanish (Eq. 4), 2K s_z (Eq. 5)
    np.testing.assert_allclose(h[2, 2, 2], [0.0, 0.0, 6.0 + 0.1], atol=1e-14)
    # corner: three neighbours; Eq. 4 with the missing -x and -y neighbours taken as 0
    np.testing.assert_allclose(h[0, 0, 0], [-0.3, -0.3, 3.0 + 0.1], atol=1e-14)


# --- T2: two-spin dipole (last term of Eq. 1) ----------------------------------------------------

def test_two_spin_dipole():
    g = _golden("closed_forms.json")["two_spin_dipole"]
    w = 0.37
    m = oracle.model(2, 1, 1, 0.0, 0.0, 0.0, w)
    side = np.array([[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]])  # r along x, spins along y
    line = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])  # r along x, spins along x
    assert oracle.energy_terms(m, side)["dipole"] == pytest.approx(g["side_by_side_over_w"] * w, rel=1e-14)
    assert oracle.energy_terms(m, line)["dipole"] == pytest.approx(g["head_to_tail_over_w"] * w, rel=1e-14)


def test_single_dipole_field_closed_form():
    # field of spin j at site i: w (3 (s.u) u - s) / r^3, u = unit vector of r_ij
    w = 0.2
    m = oracle.model(4, 3, 2, 0.0, 0.0, 0.0, w)
    s = np.zeros((24, 3))
    src = (1 * 3 + 1) * 4 + 3  # (x=3, y=1, z=1)
    s[src] = [0.3, -0.5, 0.81]
    h = oracle.dipole_field(m, s)
    for i in range(24):
        if i == src:
            continue
        xi, yi, zi = i % 4, (i // 4) % 3, i // 12
        r = np.array([3 - xi, 1 - yi, 1 - zi], float)
        d = np.linalg.norm(r)
        u = r / d
        exp = w * (3 * np.dot(s[src], u) * u - s[src]) / d ** 3
        np.testing.assert_allclose(h[i], exp, rtol=1e-13, atol=1e-16)


# --- T3: the dipole tensor (Eq. 7) ---------------------------------------------------------------

def test_dipole_tensor_properties():
    rng = np.random.default_rng(1)
    for _ in range(50):
        r = rng.integers(-6, 7, size=3)
        if not r.any():
            continue
        d = oracle.dipole_tensor(r)
        assert d[0] + d[1] + d[2] == pytest.approx(0.0, abs=1e-15)  # traceless away from 0
        np.testing.assert_array_equal(d, oracle.dipole_tensor(-r))  # D(r) = D(-r)
    np.testing.assert_allclose(oracle.dipole_tensor((1, 0, 0)), np.array([2, -1, -1, 0, 0, 0]) / (4 * math.pi),
                               rtol=1e-15, atol=1e-18)
    d = oracle.dipole_tensor((1, 1, 0))
    r5 = 2 ** 2.5
    np.testing.assert_allclose(d, np.array([3 / r5 - 1 / 2 ** 1.5, 3 / r5 - 1 / 2 ** 1.5, -1 / 2 ** 1.5,
                                            3 / r5, 0, 0]) / (4 * math.pi), rtol=1e-14, atol=1e-18)


def test_dipole_kernel_spectrum_is_real():
    # the zero-padded, circularly ordered tensor is even (D(r) = D(-r)), so its DFT is real
    nx, ny, nz = 6, 5, 3
    P = (2 * nx, 2 * ny, 2 * nz)
    ker = np.zeros((6,) + P)
    for dz in range(-(nz - 1), nz):
        for dy in range(-(ny - 1), ny):
            for dx in range(-(nx - 1), nx):
                if dx or dy or dz:
                    ker[:, dx % P[0], dy % P[1], dz % P[2]] = oracle.dipole_tensor((dx, dy, dz))
    spec = np.fft.fftn(ker, axes=(1, 2, 3))
    assert np.abs(spec.imag).max() < 1e-13 * np.abs(spec.real).max()


# --- T4/T5: field = -dE/ds by central differences (Eq. 2), exact for a quadratic E ------------

@pytest.mark.parametrize("dims,params", [
    ((4, 3, 2), (1.0, 0.3, 0.05, 0.02)),
    ((5, 5, 1), (1.0, 0.3, 0.05, 0.01)),
    ((3, 1, 4), (0.7, -0.2, 0.1, 0.05)),
    ((4, 4, 1), (0.0, 1.0, 0.0, 0.0)),   # DMI alone: the sign of Eq. 4
    ((2, 3, 2), (0.0, 0.0, 0.0, 1.0)),   # dipole alone
])
def test_field_is_negative_energy_gradient(dims, params):
    nx, ny, nz = dims
    m = oracle.model(nx, ny, nz, *params)
    rng = np.random.default_rng(11)
    s = rng.standard_normal((nx * ny * nz, 3))  # not unit: E is a quadratic form in the components
    h = oracle.field(m, s)
    eps = 1e-3
    g = np.zeros_like(s)
    for i in range(s.shape[0]):
        for c in range(3):
            sp, sm = s.copy(), s.copy()
            sp[i, c] += eps
            sm[i, c] -= eps
            g[i, c] = -(oracle.energy_terms(m, sp)["total"] - oracle.energy_terms(m, sm)["total"]) / (2 * eps)
    np.testing.assert_allclose(h, g, rtol=0, atol=1e-9 * max(1.0, np.abs(h).max()))


# --- T6: Eq. 8 equals the term-by-term Hamiltonian -------------------------------------------------

@pytest.mark.parametrize("dims", [(6, 5, 2), (8, 8, 1)])
def test_energy_identity(dims):
    nx, ny, nz = dims
    m = oracle.model(nx, ny, nz, 1.0, 0.3, 0.05, 0.02)
    s = W.random_spins((nx * ny * nz, 3), seed=3)
    h = oracle.field(m, s)
    assert oracle.energy_from_field(s, h) == pytest.approx(oracle.energy_terms(m, s)["total"], rel=1e-13)


# --- Eq. 6 by FFT equals the direct sum (library FFT as the step) ----------------------------------

@pytest.mark.parametrize("dims", [(5, 3, 2), (4, 6, 1), (3, 3, 3)])
def test_direct_dipole_equals_fft_convolution(dims):
    nx, ny, nz = dims
    w = 0.05
    m = oracle.model(nx, ny, nz, 0.0, 0.0, 0.0, w)
    s = W.random_spins((nx * ny * nz, 3), seed=5)
    h = oracle.dipole_field(m, s).reshape(nz, ny, nx, 3)
    P = (2 * nz, 2 * ny, 2 * nx)
    T = np.zeros((3, 3) + P)
    idx = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
    for dz in range(-(nz - 1), nz):
        for dy in range(-(ny - 1), ny):
            for dx in range(-(nx - 1), nx):
                if dx or dy or dz:
                    d = oracle.dipole_tensor((dx, dy, dz))
                    for a in range(3):
                        for b in range(3):
                            T[a, b, dz % P[0], dy % P[1], dx % P[2]] = d[idx[(a, b)]]
    S = np.zeros((3,) + P)
    S[:, :nz, :ny, :nx] = s.reshape(nz, ny, nx, 3).transpose(3, 0, 1, 2)
    That = np.fft.fftn(T, axes=(2, 3, 4))
    Shat = np.fft.fftn(S, axes=(1, 2, 3))
    Hhat = np.einsum("abxyz,bxyz->axyz", That, Shat)
    Hc = np.fft.ifftn(Hhat, axes=(1, 2, 3)).real[:, :nz, :ny, :nx] * 4 * math.pi * w
    np.testing.assert_allclose(h, Hc.transpose(1, 2, 3, 0), rtol=0, atol=1e-13)


# --- Eq. 6 on a large monolayer: the square-lattice inverse-cube sum -------------------------------

def test_monolayer_dipole_lattice_sum():
    s_inf = _golden("closed_forms.json")["square_lattice_inverse_cube_sum"]["value"]
    errs = []
    for L in (21, 41):
        m = oracle.model(L, L, 1, 0.0, 0.0, 0.0, 1.0)
        h = oracle.dipole_field(m, W.ferromagnet(L, L, 1))
        c = (L // 2) * L + L // 2
        np.testing.assert_allclose(h[c, :2], 0.0, atol=1e-12)
        S_L = -h[c, 2]
        # the sum outside the square [-L/2, L/2]^2 is int dA / r^3 = 8 sqrt(2) / L to leading order
        errs.append(abs(S_L + 8 * math.sqrt(2) / L - s_inf))
    assert errs[1] < 2e-3 and errs[1] < errs[0] / 3


# --- T8: monotone descent under the projected step (Eq. 10 with Eq. 13) ---------------------------

@pytest.mark.parametrize("dims,params", [((16, 16, 1), (1.0, 0.3, 0.05, 0.01)), ((8, 8, 4), (1.0, 0.25, 0.1, 0.02))])
def test_monotone_descent(dims, params):
    nx, ny, nz = dims
    m = oracle.model(nx, ny, nz, *params)
    s = W.skyrmion(nx, ny, nz, R=nx / 4, D=params[1])
    s = 0.7 * s + 0.3 * W.random_spins(s.shape, seed=2)
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    e_prev = None
    for _ in range(40):
        h = oracle.field(m, s)
        e = oracle.energy_from_field(s, h)
        if e_prev is not None:
            assert e <= e_prev + 1e-12
        e_prev = e
        s = oracle.step(s, h, 0.1)
        np.testing.assert_allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)


def test_step_moves_along_projected_field():
    s = np.array([[0.0, 0.0, 1.0]])
    h = np.array([[1.0, 0.0, 5.0]])  # parallel part (0,0,5) must not act
    out = oracle.step(s, h, 0.1)
    np.testing.assert_allclose(out, [[0.1 / math.hypot(1, 0.1), 0.0, 1.0 / math.hypot(1, 0.1)]], rtol=1e-15)


# --- T9: reparametrisation (Eqs. 11-12) -----------------------------------------------------------

def _circle(angles):
    return np.stack([np.cos(angles), np.sin(angles), np.zeros_like(angles)], -1)[:, None, :]


def test_reparam_on_a_great_circle_matches_geometry():
    ang = np.array([0.0, 0.05, 0.3, 0.35, 0.9, 1.2, 1.25, 1.6])
    K = len(ang)
    out, alpha = oracle.reparam(_circle(ang), return_alpha=True)
    chords = 2 * np.sin(np.diff(ang) / 2)
    s = np.concatenate([[0.0], np.cumsum(chords)])
    np.testing.assert_allclose(alpha, s / s[-1], rtol=1e-14)
    for k in range(1, K - 1):
        target = k / (K - 1) * s[-1]
        j = np.searchsorted(s, target, side="right") - 1
        t = (target - s[j]) / chords[j]
        dth = ang[j + 1] - ang[j]
        # radial projection of the chord point at fraction t
        expected = ang[j] + math.atan2(t * math.sin(dth), (1 - t) + t * math.cos(dth))
        got = math.atan2(out[k, 0, 1], out[k, 0, 0])
        assert got == pytest.approx(expected, abs=1e-13)
    np.testing.assert_array_equal(out[0], _circle(ang)[0])
    np.testing.assert_array_equal(out[-1], _circle(ang)[-1])


def test_reparam_fixed_point_and_endpoints():
    K = 9
    ang = np.linspace(0.0, 2.0, K)
    path = np.concatenate([_circle(ang), _circle(ang * 0.5)], axis=1)  # two sites, both uniform
    out = oracle.reparam(path)
    np.testing.assert_allclose(out, path, atol=1e-14)
    rnd = W.random_spins((6, 10, 3), seed=4)
    out = oracle.reparam(rnd)
    np.testing.assert_array_equal(out[0], rnd[0])
    np.testing.assert_array_equal(out[-1], rnd[-1])
    np.testing.assert_allclose(np.linalg.norm(out, axis=-1), 1.0, atol=1e-14)


def test_reparam_degenerate_paths():
    same = np.repeat(W.random_spins((1, 5, 3), seed=6), 5, axis=0)
    np.testing.assert_array_equal(oracle.reparam(same), same)  # zero total length: no-op
    # a duplicated image (zero-length segment) is skipped: largest j with alpha*_j <= alpha_k
    ang = np.array([0.0, 0.4, 0.4, 0.8, 1.2])
    out = oracle.reparam(_circle(ang))
    got = np.arctan2(out[:, 0, 1], out[:, 0, 0])
    # three equal chords of angle 0.4; targets at 0.75, 1.5 and 2.25 chords.  Target 1.5 lands on
    # segment j=2 (the largest j with alpha*_j <= alpha_k), past the zero-length segment j=1.
    proj = lambda a0, t: a0 + math.atan2(t * math.sin(0.4), (1 - t) + t * math.cos(0.4))
    np.testing.assert_allclose(got, [0.0, proj(0.0, 0.75), proj(0.4, 0.5), proj(0.8, 0.25), 1.2], atol=1e-13)


# --- T10: initial-image energies against continuum closed forms -----------------------------------

def test_initial_skyrmion_continuum_energies():
    I = _golden("closed_forms.json")["linear_profile_exchange_integral"]["value_I"]
    rel = {}
    for R in (8, 32):
        L = int(2 * R + 16)
        m = oracle.model(L, L, 1, 1.0, 1.0, 1.0, 0.0)
        e_sk = oracle.energy_terms(m, W.skyrmion(L, L, 1, R, D=1.0))
        e_fm = oracle.energy_terms(m, W.ferromagnet(L, L, 1))
        d_exc = e_sk["exchange"] - e_fm["exchange"]
        d_ani = e_sk["anisotropy"] - e_fm["anisotropy"]
        rel[R] = (abs(d_exc / (math.pi * (math.pi ** 2 / 2 + I)) - 1),
                  abs(d_ani / (math.pi * R ** 2 / 2) - 1),
                  abs(e_sk["dmi"] / (-math.pi ** 2 * R) - 1))
        assert e_sk["dmi"] < 0  # psi = pi is the low-energy helicity for D > 0
    assert rel[32][0] < 0.01 and rel[32][1] < 1e-4 and rel[32][2] < 0.005
    assert rel[32][0] < rel[8][0] and rel[32][2] < rel[8][2]


# --- the assembled loop (Sec. III) ----------------------------------------------------------------

def test_string_run_composition_and_sanity():
    wl = W.tiny_bloch()
    spec = wl.strings[0]
    m = oracle.model(spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w)
    path = spec.initial_path()
    # one iteration of string_run == field -> step per image -> reparam, composed by hand
    h = oracle.field(m, path)
    star = np.stack([oracle.step(path[k], h[k], wl.dt) for k in range(path.shape[0])])
    by_hand = oracle.reparam(star)
    phi, e = oracle.string_run(m, path, 1, wl.dt)
    np.testing.assert_allclose(phi, by_hand, atol=1e-15)
    np.testing.assert_allclose(e, oracle.energies(m, by_hand), rtol=1e-14)
    phi, e = oracle.string_run(m, path, 30, wl.dt)
    dE, k = oracle.barrier(e)
    assert dE >= 0 and 0 <= k < spec.n_images
    d = np.linalg.norm((phi[1:] - phi[:-1]).reshape(spec.n_images - 1, -1), axis=1)
    assert d.std() / d.mean() < 0.05  # roughly equal spacing after the last reparam


def test_param_gradient_is_linear_coefficient():
    m = oracle.model(5, 4, 2, 1.1, 0.3, 0.07, 0.02)
    s = W.random_spins((40, 3), seed=8)
    g = oracle.energy_param_grad(m, s)
    e0 = oracle.energy_terms(m, s)["total"]
    for i, name in enumerate("JDKw"):
        p = dict(J=1.1, D=0.3, K=0.07, w=0.02)
        p[name] += 0.5
        e1 = oracle.energy_terms(oracle.model(5, 4, 2, **p), s)["total"]
        assert (e1 - e0) / 0.5 == pytest.approx(g[i], rel=1e-11, abs=1e-12)


def test_barrier_definition():
    # Sec. III: energy of the highest image relative to the first; ties go to the lowest index
    assert oracle.barrier([1.0, 3.0, 2.5, 3.0, 0.0]) == (2.0, 1)
    assert oracle.barrier([5.0, 1.0, 2.0]) == (0.0, 0)


def test_field_at_sites_equals_full_field():
    m = oracle.model(7, 5, 3, 1.0, 0.3, 0.05, 0.02)
    s = W.random_spins((105, 3), seed=12)
    sites = [0, 6, 17, 52, 104, 33]
    np.testing.assert_array_equal(oracle.field_at(m, s, sites), oracle.field(m, s)[sites])
