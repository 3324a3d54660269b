"""Parity of the reparametrisation variants (natural cubic spline, climbing image; Sec. III) with the
FP64 oracle's `string_run_v`, through the C ABI.

FP64: paths to 1e-10 and energies to 1e-9 after tens of iterations (the spline weights are built by
columns on the GPU and per component in the oracle, so they agree to rounding); the climbing image's
index must be equal.  FP32: the bounds of the Euler trajectory tests.
"""
import numpy as np
import pytest

import oracle
from paper_1804_07135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1


def _unit(a):
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _case(spec):
    return (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)


def _model(c):
    return oracle.model(*c[:7])


def _run(ss, cases, paths, n_iter, prec, spline, climb, dt=0.1):
    with ss.StringMethod(cases, dt=dt, precision=prec) as sm:
        sm.set_reparam(ss.SS_INTERP_SPLINE if spline else ss.SS_INTERP_LINEAR, climb)
        for i, p in enumerate(paths):
            sm.set_path(i, p)
        starts = [sm.get_path(i) for i in range(len(cases))]
        assert all(sm.climbing_image(i) == -1 for i in range(len(cases)))
        sm.step(n_iter)
        outs = [dict(path=sm.get_path(i), e=sm.energies(i), kc=sm.climbing_image(i)) for i in range(len(cases))]
    return starts, outs


@pytest.mark.parametrize("spline,climb", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("prec", [FP32, FP64])
def test_variants_tiny_bloch(ss, prec, spline, climb):
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    n_iter = 70  # past one 64-iteration graph, so the captured sequence is exercised
    (s0,), (g,) = _run(ss, [c], [spec.initial_path()], n_iter, prec, spline, climb)
    ref, e_ref, kc_ref = oracle.string_run_v(_model(c), _unit(s0), n_iter, 0.1, spline=spline, climb=climb)
    assert g["kc"] == kc_ref
    if prec == FP64:
        assert np.abs(g["path"] - ref).max() < 1e-10
        np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-9)
    else:
        assert np.abs(g["path"] - ref).max() < 1e-4
        np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-4)
    if climb:
        assert 0 < g["kc"] < spec.n_images - 1


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_climbing_with_length_128_transforms(ss, prec):
    # nx = 57 pads to 128: the FP32 path runs the two-pass length-128 x-inverse kernel in its climbing
    # mode
    c = (57, 20, 1, 1.0, 0.3, 0.05, 0.02, 6)
    path = W.bloch_point_path(c[0], c[1], c[2], c[7], R=6.0, D=c[4])
    n_iter = 12
    (s0,), (g,) = _run(ss, [c], [path], n_iter, prec, True, True)
    ref, e_ref, kc_ref = oracle.string_run_v(_model(c), _unit(s0), n_iter, 0.1, spline=True, climb=True)
    assert g["kc"] == kc_ref
    assert np.abs(g["path"] - ref).max() < (1e-4 if prec == FP32 else 1e-10)
    np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-4 if prec == FP32 else 1e-9)


def test_variants_batch_in_two_groups(ss):
    # strings of 5, 9 and 3 images share a lattice (each picks its own climbing image and spline
    # weights); a fourth string has a lattice of its own
    cases = [(12, 12, 1, 1.0, 0.3, 0.05, 0.01, 5), (12, 12, 1, 1.4, 0.35, 0.1, 0.02, 9),
             (12, 12, 1, 1.0, 0.2, 0.0, 0.0, 3), (10, 9, 2, 1.0, 0.25, 0.1, 0.02, 6)]
    paths = [W.bloch_point_path(c[0], c[1], c[2], c[7], R=3.0, D=c[4]) for c in cases]
    n_iter = 25
    starts, outs = _run(ss, cases, paths, n_iter, FP64, True, True)
    for c, s0, g in zip(cases, starts, outs):
        ref, e_ref, kc_ref = oracle.string_run_v(_model(c), _unit(s0), n_iter, 0.1, spline=True, climb=True)
        assert g["kc"] == kc_ref, c
        assert np.abs(g["path"] - ref).max() < 1e-10, c
        np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-9)


def _great_circle_path(K, n_sites):
    th = np.linspace(0.0, np.pi, K)
    one = np.stack([np.sin(th), np.zeros(K), np.cos(th)], axis=-1)
    return np.repeat(one[:, None, :], n_sites, axis=1)


@pytest.mark.parametrize("spline", [False, True])
def test_climbing_image_coherent_rotation_saddle(ss, spline):
    # 3x3 ferromagnet with exchange and anisotropy only: the saddle of the uniform rotation lies N K
    # above the minimum; an 8-image string has no image on the equator, so only the climbing image
    # reaches it
    J, Ka = 1.0, 0.2
    c = (3, 3, 1, J, 0.0, Ka, 0.0, 8)
    path = _great_circle_path(8, 9)
    with ss.StringMethod([c], dt=0.1, precision=FP64) as sm:
        sm.set_path(0, path)
        sm.step(300)
        plain = sm.barrier(0)[0]
        sm.set_reparam(ss.SS_INTERP_SPLINE if spline else ss.SS_INTERP_LINEAR, True)
        sm.set_path(0, path)
        sm.step(300)
        dE, k = sm.barrier(0)
        kc = sm.climbing_image(0)
    assert plain < 9 * Ka - 1e-3
    assert abs(dE - 9 * Ka) < 1e-8 and k == kc


def test_spline_zero_length_segment_falls_back_to_linear(ss):
    # two identical adjacent images: the spline cannot take that part, which is then linear
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    path = spec.initial_path()
    path[6] = path[5]
    with ss.StringMethod([c], dt=0.1, precision=FP64) as sm:
        sm.set_reparam(ss.SS_INTERP_SPLINE, False)
        sm.set_path(0, path)
        s0 = sm.get_path(0)
        sm.step(1)
        got = sm.get_path(0)
    ref, _, _ = oracle.string_run_v(_model(c), _unit(s0), 1, 0.1, spline=True)
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_spline_long_string(ss, prec):
    # 200 images (many spline columns per thread, W rows of 200 weights, a 32-site apply tile in FP64)
    c = (4, 4, 1, 1.0, 0.3, 0.05, 0.01, 200)
    rng = np.random.default_rng(9)
    a = _unit(rng.standard_normal((16, 3)))
    ax = _unit(rng.standard_normal((16, 3)))
    th = 2.0 * (np.arange(200) / 199.0) ** 1.5
    path = np.stack([a * np.cos(t) + np.cross(ax, a) * np.sin(t) + ax * (ax * a).sum(-1, keepdims=True) * (1 - np.cos(t))
                     for t in th])
    n_iter = 3
    (s0,), (g,) = _run(ss, [c], [path], n_iter, prec, True, False)
    ref, e_ref, _ = oracle.string_run_v(_model(c), _unit(s0), n_iter, 0.1, spline=True)
    assert np.abs(g["path"] - ref).max() < (2e-5 if prec == FP32 else 1e-11)


def test_variant_state_rules(ss):
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    with ss.StringMethod([c, (4, 4, 1, 1.0, 0.3, 0.05, 0.01, 300)], dt=0.1) as sm:
        with pytest.raises(ss.SsError) as ei:
            sm.set_reparam(ss.SS_INTERP_SPLINE, False)  # a 300-image string
        assert ei.value.status == ss.SS_ERR_INVALID_ARG
        with pytest.raises(ss.SsError):
            sm.set_reparam(2, False)
        assert ss._lib.ss_set_reparam(sm.ctx, ss.SS_INTERP_LINEAR, 3) == ss.SS_ERR_INVALID_ARG  # the ABI itself
        sm.set_reparam(ss.SS_INTERP_LINEAR, True)
        with pytest.raises(ss.SsError) as ei:
            sm.set_integrator(ss.SS_INT_DOPRI5, 1e-6, 1e-8)
        assert ei.value.status == ss.SS_ERR_STATE
        sm.set_reparam(ss.SS_INTERP_LINEAR, False)
        sm.set_integrator(ss.SS_INT_DOPRI5, 1e-6, 1e-8)
        with pytest.raises(ss.SsError) as ei:
            sm.set_reparam(ss.SS_INTERP_LINEAR, True)
        assert ei.value.status == ss.SS_ERR_STATE
        assert sm.climbing_image(0) == -1


def test_first_iteration_without_climbing_matches_plain(ss):
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    with ss.StringMethod([c], dt=0.1, precision=FP64) as sm:
        sm.set_path(0, spec.initial_path())
        sm.step(1)
        plain = sm.get_path(0)
        sm.set_reparam(ss.SS_INTERP_LINEAR, True)
        sm.set_path(0, spec.initial_path())
        sm.step(1)
        assert np.array_equal(sm.get_path(0), plain)
        e0 = oracle.energies(_model(c), _unit(sm.get_path(0)))
        kc = sm.climbing_image(0)
    start = oracle.energies(_model(c), _unit(spec.initial_path()))
    assert kc == 1 + int(np.argmax(start[1:-1])) or abs(start[kc] - start[1:-1].max()) < 1e-9
    assert np.isfinite(e0).all()


def test_dopri5_with_spline(ss):
    # the spline reparametrisation after a Dormand-Prince interval with per-image control (FP64).  The
    # oracle's evolution of image k alone: its whole-string run on the two-image string [k, k] (the
    # same error norm, and no reparametrisation moves a two-image string); then the oracle's spline.
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    T = 0.5
    with ss.StringMethod([c], dt=T, precision=FP64) as sm:
        sm.set_integrator(ss.SS_INT_DOPRI5_IMAGE, 1e-6, 1e-8)
        sm.set_reparam(ss.SS_INTERP_SPLINE, False)
        sm.set_path(0, spec.initial_path())
        s0 = sm.get_path(0)
        sm.step(1)
        got = sm.get_path(0)
    evolved = np.stack([oracle.string_run_rk(_model(c), np.stack([im, im]), 1, T, 1e-6, 1e-8,
                                             with_energies=False)[0][0] for im in _unit(s0)])
    ref = oracle.reparam_v(evolved, spline=True)
    assert np.abs(got - ref).max() < 1e-10


def test_kernel_timing_follows_the_mode(ss):
    spec = W.tiny_bloch().strings[0]
    with ss.StringMethod([_case(spec)], dt=0.1) as sm:
        sm.set_path(0, spec.initial_path())
        assert len(sm.time_kernels(reps=2)) == 4  # xfwd, yz, xinv, arc
        sm.set_reparam(ss.SS_INTERP_SPLINE, True)
        ms = sm.time_kernels(reps=2)  # xfwd, yz, xinv, climbing-image pair, arc, spline
        assert len(ms) == 6 and (ms > 0).all()
        sm.set_reparam(ss.SS_INTERP_LINEAR, False)
        sm.set_integrator(ss.SS_INT_DOPRI5, 1e-6, 1e-8)
        # one attempt round: the opening, 7 stages x (assemble, xfwd, yz, xinv), finish, control, commit, arc
        ms = sm.time_kernels(reps=2)
        assert len(ms) == 1 + 7 * 4 + 4 and (ms > 0).all()
        sm.set_integrator(ss.SS_INT_RKF45, 1e-6, 1e-8)
        assert len(sm.time_kernels(reps=2)) == 1 + 6 * 4 + 4
        # the timing leaves a unit-length path, and the integrator steps on from it
        p = sm.get_path(0)
        np.testing.assert_allclose(np.linalg.norm(p, axis=-1), 1.0, atol=1e-5)
        sm.step(2)
        assert np.isfinite(sm.get_path(0)).all()


@pytest.mark.parametrize("K", [2, 3])
def test_degenerate_strings_with_spline_and_climbing(ss, K):
    # K = 2: no interior image (nothing moves, nothing climbs); K = 3: the one interior image climbs
    # and both parts have no interior image
    c = (6, 5, 2, 1.0, 0.3, 0.05, 0.02, K)
    path = W.bloch_point_path(6, 5, 2, K, R=2.0, D=0.3)
    n_iter = 6
    (s0,), (g,) = _run(ss, [c], [path], n_iter, FP64, True, True)
    ref, e_ref, kc_ref = oracle.string_run_v(_model(c), _unit(s0), n_iter, 0.1, spline=True, climb=True)
    assert g["kc"] == kc_ref == (-1 if K == 2 else 1)
    assert np.abs(g["path"] - ref).max() < 1e-11
    np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-10)


def test_spline_on_a_string_of_identical_images(ss):
    # zero arc length: the reparametrisation keeps every image
    c = (8, 8, 1, 1.0, 0.3, 0.05, 0.01, 5)
    one = W.bloch_point_path(8, 8, 1, 2, R=3.0, D=0.3)[0]
    path = np.repeat(one[None], 5, axis=0)
    (s0,), (g,) = _run(ss, [c], [path], 3, FP64, True, False)
    ref, _, _ = oracle.string_run_v(_model(c), _unit(s0), 3, 0.1, spline=True)
    assert np.abs(g["path"] - ref).max() < 1e-12
    assert np.abs(g["path"] - g["path"][0]).max() < 1e-12  # the images stay identical


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_llg_and_dopri5_on_a_one_column_lattice(ss, prec):
    # nx = 1 (no x bonds, odd x length for the paired sites), two images
    c = (1, 6, 2, 1.0, 0.3, 0.05, 0.02, 2)
    path = _unit(np.random.default_rng(12).standard_normal((2, 12, 3)))
    tol = 1e-4 if prec == FP32 else 1e-11
    with ss.StringMethod([c], dt=0.05, precision=prec) as sm:
        sm.set_dynamics(ss.SS_DYN_LLG, 0.3)
        sm.set_path(0, path)
        s0 = sm.get_path(0)
        sm.step(20)
        got = sm.get_path(0)
        sm.set_dynamics(ss.SS_DYN_STRING)
        sm.set_integrator(ss.SS_INT_DOPRI5_IMAGE, 1e-6, 1e-8)
        sm.set_path(0, path)
        s1 = sm.get_path(0)
        sm.step(4)
        got_rk = sm.get_path(0)
    ref, _ = oracle.llg_run(_model(c), _unit(s0), 20, 0.05, 0.3)
    assert np.abs(got - ref).max() < tol
    ref_rk, _, _, _ = oracle.string_run_rk(_model(c), _unit(s1), 4, 0.05, 1e-6, 1e-8, per_image=True)
    assert np.abs(got_rk - ref_rk).max() < (1e-4 if prec == FP32 else 1e-10)


def test_climbing_image_gives_exact_barrier_derivative(ss):
    # The barrier's derivative by the anisotropy constant, by the envelope theorem, is dE/dK at the saddle
    # minus dE/dK at the minimum (Eq. 1 is linear in K).  For the coherent rotation of a 3x3 ferromagnet
    # the saddle is all spins in plane (dE/dK = 0) and the minimum all along z (dE/dK = -N): the
    # climbing image yields N = 9 exactly, the plain string's highest image less.
    c = (3, 3, 1, 1.0, 0.0, 0.2, 0.0, 8)
    path = _great_circle_path(8, 9)
    out = {}
    for climb in (False, True):
        with ss.StringMethod([c], dt=0.1, precision=FP64) as sm:
            sm.set_reparam(ss.SS_INTERP_LINEAR, climb)
            sm.set_path(0, path)
            sm.step(300)
            terms = sm.energy_terms(0)  # [image][dE/dJ, dE/dD, dE/dK, dE/dw]
            k = sm.barrier(0)[1]
            out[climb] = terms[k, 2] - terms[0, 2]
    assert abs(out[True] - 9.0) < 1e-6
    assert out[False] < 9.0 - 1e-2


def test_relax_until_the_barrier_settles(ss):
    # the convergence loop on the coherent-rotation saddle with the climbing image: it stops once the
    # barrier moves by less than the tolerance between checks, at N K
    c = (3, 3, 1, 1.0, 0.0, 0.2, 0.0, 8)
    with ss.StringMethod([c], dt=0.1, precision=FP64) as sm:
        sm.set_reparam(ss.SS_INTERP_LINEAR, True)
        sm.set_path(0, _great_circle_path(8, 9))
        done, ok, hist = sm.relax(tol=1e-10, check_every=50, max_iter=5000)
    assert ok and done < 5000
    assert abs(hist[0][-1] - 1.8) < 1e-8


def test_resetting_the_graphs_of_several_size_groups(ss):
    # after a step, choosing the reparametrisation or the dynamics again drops the captured graphs; with
    # two size groups (two graph branches) the next step must recapture them and carry on exactly as an
    # uninterrupted run (the oracle's 5 iterations)
    cases = [(16, 16, 1, 1.0, 0.3, 0.05, 0.01, 5), (12, 10, 2, 1.0, 0.2, 0.1, 0.02, 4)]
    paths = [W.bloch_point_path(c[0], c[1], c[2], c[7], R=3.0, D=c[4]) for c in cases]
    with ss.StringMethod(cases, precision=FP64) as sm:
        for i, p in enumerate(paths):
            sm.set_path(i, p)
        starts = [sm.get_path(i) for i in range(2)]
        sm.step(2)
        sm.set_reparam(ss.SS_INTERP_LINEAR, False)
        sm.step(2)
        sm.set_dynamics(ss.SS_DYN_STRING, 0.0)
        sm.step(1)
        got = [sm.get_path(i) for i in range(2)]
    for c, s0, g in zip(cases, starts, got):
        ref, _ = oracle.string_run(_model(c), _unit(s0), 5, 0.1)
        assert np.abs(g - ref).max() < 1e-10
