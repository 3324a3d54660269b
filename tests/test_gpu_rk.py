"""Parity of the adaptive Dormand-Prince 5(4) evolution (Sec. III) with the FP64 oracle's run.

The GPU integrates every string over opts.dt per iteration with its own step-size history; the oracle
(`oracle.string_run_rk`) does the same with the same controller.  On the FP64 path both take the same
accept/reject decisions, so the attempt counts must agree exactly and the carried step and the path to
round-off; on the FP32 path the error norm carries FP32 round-off, so the counts may differ by a few
attempts and the path by the FP32 bound of the Euler trajectory tests.
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


def _gpu_run(ss, cases, paths, T, n_iter, prec, rtol, atol, kind=None):
    with ss.StringMethod(cases, dt=T, precision=prec) as sm:
        sm.set_integrator(ss.SS_INT_DOPRI5 if kind is None else kind, rtol, atol)
        for i, p in enumerate(paths):
            sm.set_path(i, p)
        starts = [sm.get_path(i) for i in range(len(cases))]
        sm.step(n_iter)
        out = [dict(path=sm.get_path(i), state=sm.integrator_state(i), e=sm.energies(i),
                    e_step=sm.step_energies(i),
                    images=[sm.integrator_state(i, k) for k in range(cases[i][7])]) for i in range(len(cases))]
    return starts, out


@pytest.mark.parametrize("T,rtol,atol", [(0.5, 1e-6, 1e-8), (2.0, 1e-6, 1e-8), (0.5, 1e-4, 1e-6)])
def test_dopri5_tiny_bloch_fp64(ss, T, rtol, atol):
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    n_iter = 10
    (start,), (g,) = _gpu_run(ss, [c], [spec.initial_path()], T, n_iter, FP64, rtol, atol)
    ref, e_ref, step_ref, counts_ref = oracle.string_run_rk(_model(c), _unit(start), n_iter, T, rtol, atol)
    step, acc, rej = g["state"]
    assert (acc, rej) == counts_ref
    assert rej > 0  # the controller is exercised on both branches
    assert abs(step - step_ref) <= 1e-9 * step_ref
    assert np.abs(g["path"] - ref).max() < 1e-10
    np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-9)
    # energies summed during the last iteration: those of the state after n_iter - 1 iterations
    _, e_prev, _, _ = oracle.string_run_rk(_model(c), _unit(start), n_iter - 1, T, rtol, atol)
    np.testing.assert_allclose(g["e_step"], e_prev, rtol=0, atol=1e-9)


def test_dopri5_tiny_bloch_fp32(ss):
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    n_iter, T, rtol, atol = 10, 0.5, 1e-4, 1e-6
    (start,), (g,) = _gpu_run(ss, [c], [spec.initial_path()], T, n_iter, FP32, rtol, atol)
    ref, e_ref, step_ref, (acc_ref, rej_ref) = oracle.string_run_rk(_model(c), _unit(start), n_iter, T, rtol, atol)
    step, acc, rej = g["state"]
    assert abs(acc - acc_ref) <= 3 and abs(rej - rej_ref) <= 3
    assert np.abs(g["path"] - ref).max() < 1e-4
    np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-4)
    assert abs(oracle.barrier(g["e"])[0] - oracle.barrier(e_ref)[0]) < 1e-4


def test_dopri5_batch_with_independent_step_histories(ss):
    # two strings share a size group but differ in stiffness (so their step histories differ) and a
    # third lives in a group of its own that needs more rounds of attempts than the first
    cases = [(16, 16, 1, 1.0, 0.3, 0.05, 0.01, 5), (16, 16, 1, 1.6, 0.4, 0.1, 0.02, 7),
             (12, 10, 2, 1.0, 0.2, 0.1, 0.02, 4)]
    paths = [W.bloch_point_path(c[0], c[1], c[2], c[7], R=3.0, D=c[4]) for c in cases]
    T, n_iter, rtol, atol = 1.0, 4, 1e-6, 1e-8
    starts, outs = _gpu_run(ss, cases, paths, T, n_iter, FP64, rtol, atol)
    counts = []
    for c, s0, g in zip(cases, starts, outs):
        ref, e_ref, step_ref, counts_ref = oracle.string_run_rk(_model(c), _unit(s0), n_iter, T, rtol, atol)
        assert g["state"][1:] == counts_ref, c
        assert abs(g["state"][0] - step_ref) <= 1e-9 * step_ref, c
        assert np.abs(g["path"] - ref).max() < 1e-10, c
        np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-9)
        counts.append(counts_ref)
    assert counts[0] != counts[1]


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_dopri5_per_image_control(ss, prec):
    # every image its own ODE system: per-image counts and steps against the oracle's per-image run;
    # two strings in one size group and one in another
    cases = [(16, 16, 1, 1.0, 0.3, 0.05, 0.01, 6), (16, 16, 1, 1.6, 0.4, 0.1, 0.02, 3),
             (12, 10, 2, 1.0, 0.2, 0.1, 0.02, 4)]
    paths = [W.bloch_point_path(c[0], c[1], c[2], c[7], R=3.0, D=c[4]) for c in cases]
    T, n_iter = 1.0, 3
    rtol, atol = (1e-6, 1e-8) if prec == FP64 else (1e-4, 1e-6)
    starts, outs = _gpu_run(ss, cases, paths, T, n_iter, prec, rtol, atol, kind=ss.SS_INT_DOPRI5_IMAGE)
    for c, s0, g in zip(cases, starts, outs):
        ref, e_ref, steps_ref, counts_ref = oracle.string_run_rk(_model(c), _unit(s0), n_iter, T, rtol, atol,
                                                                 per_image=True)
        got_counts = np.array([st[1:] for st in g["images"]])
        got_steps = np.array([st[0] for st in g["images"]])
        if prec == FP64:
            np.testing.assert_array_equal(got_counts, counts_ref)
            np.testing.assert_allclose(got_steps, steps_ref, rtol=1e-9)
            assert np.abs(g["path"] - ref).max() < 1e-10, c
            np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-9)
        else:
            assert np.abs(got_counts - counts_ref).max() <= 3, c
            assert np.abs(g["path"] - ref).max() < 1e-4, c
            np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-4)
        assert g["state"] == (got_steps.min(), *got_counts.sum(0))
        assert len({tuple(x) for x in counts_ref}) > 1  # the images do take different step histories


def test_dopri5_state_resets_and_euler_resumes(ss):
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    T = 0.5
    with ss.StringMethod([c], dt=T, precision=FP64) as sm:
        assert sm.integrator_state(0) == (T, 0, 0)  # before the integrator is chosen
        sm.set_integrator(ss.SS_INT_DOPRI5, 1e-6, 1e-8)
        sm.set_path(0, spec.initial_path())
        sm.step(3)
        step, acc, rej = sm.integrator_state(0)
        assert acc > 0 and step != T
        sm.set_path(0, spec.initial_path())  # a new path restarts the controller at opts.dt
        assert sm.integrator_state(0) == (T, 0, 0)
        sm.step(3)
        assert sm.integrator_state(0) == (step, acc, rej)  # deterministic
        # back to the projected Euler step with dt = 0.5: one iteration against the oracle's
        sm.set_integrator(ss.SS_INT_EULER, 1e-6, 1e-8)
        s0 = sm.get_path(0)
        sm.step(1)
        got = sm.get_path(0)
    ref, _ = oracle.string_run(_model(c), _unit(s0), 1, T)
    assert np.abs(got - ref).max() < 1e-12


def test_dopri5_invalid_arguments(ss):
    spec = W.tiny_bloch().strings[0]
    with ss.StringMethod([_case(spec)], dt=0.1) as sm:
        for kind, rtol, atol in [(7, 1e-6, 1e-8), (ss.SS_INT_DOPRI5, 0.0, 1e-8), (ss.SS_INT_DOPRI5, 1e-6, -1.0),
                                 (ss.SS_INT_DOPRI5, float("nan"), 1e-8)]:
            with pytest.raises(ss.SsError) as ei:
                sm.set_integrator(kind, rtol, atol)
            assert ei.value.status == ss.SS_ERR_INVALID_ARG
        with pytest.raises(ss.SsError):
            sm.integrator_state(3)
        with pytest.raises(ss.SsError):
            sm.integrator_state(0, spec.n_images)


@pytest.mark.parametrize("per_image", [False, True])
@pytest.mark.parametrize("prec", [FP32, FP64])
def test_rkf45_against_oracle(ss, prec, per_image):
    # the Runge-Kutta-Fehlberg 4(5) pair (six stages, fourth-order solution carried)
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    n_iter, T = 6, 0.5
    rtol, atol = (1e-6, 1e-8) if prec == FP64 else (1e-4, 1e-6)
    kind = ss.SS_INT_RKF45_IMAGE if per_image else ss.SS_INT_RKF45
    (start,), (g,) = _gpu_run(ss, [c], [spec.initial_path()], T, n_iter, prec, rtol, atol, kind=kind)
    ref, e_ref, steps_ref, counts_ref = oracle.string_run_rk(_model(c), _unit(start), n_iter, T, rtol, atol,
                                                             per_image=per_image, method="rkf45")
    if per_image:
        got_counts = np.array([st[1:] for st in g["images"]])
        got_steps = np.array([st[0] for st in g["images"]])
    else:
        got_counts = np.array([g["state"][1:]])
        got_steps = np.array([g["state"][0]])
        counts_ref, steps_ref = np.array([counts_ref]), np.array([steps_ref])
    if prec == FP64:
        np.testing.assert_array_equal(got_counts, counts_ref)
        np.testing.assert_allclose(got_steps, steps_ref, rtol=1e-6)
        assert np.abs(g["path"] - ref).max() < 1e-10
        np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-9)
    else:
        assert np.abs(got_counts - counts_ref).max() <= 3
        assert np.abs(g["path"] - ref).max() < 1e-4
        np.testing.assert_allclose(g["e"], e_ref, rtol=0, atol=1e-4)
    # the pairs differ: Dormand-Prince takes another step sequence on the same problem
    _, _, _, counts_dp = oracle.string_run_rk(_model(c), _unit(start), n_iter, T, rtol, atol, per_image=per_image)
    assert not np.array_equal(np.asarray(counts_dp).reshape(-1, 2), np.asarray(counts_ref).reshape(-1, 2))


def test_dopri5_with_direct_dipole_sums(ss):
    # the attempt rounds of the graph's WHILE node with the direct O(N^2) dipole sums in place of the FFT
    # convolution (SS_DIPOLE_DIRECT): attempt counts and path as the oracle's, which sums directly too;
    # 9 iterations run the 8-iteration graph and the one-iteration graph
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    T, n_iter, rtol, atol = 0.5, 9, 1e-6, 1e-8
    with ss.StringMethod([c], dt=T, precision=FP64, dipole=ss.SS_DIPOLE_DIRECT) as sm:
        sm.set_integrator(ss.SS_INT_DOPRI5, rtol, atol)
        sm.set_path(0, spec.initial_path())
        start = sm.get_path(0)
        sm.step(n_iter)
        got, (step, acc, rej) = sm.get_path(0), sm.integrator_state(0)
        # the round's kernels one by one: the direct sums take the y/z entry's place in every stage
        assert len(sm.time_kernels(reps=1)) == 1 + 7 * 4 + 4
    ref, _, step_ref, counts_ref = oracle.string_run_rk(_model(c), _unit(start), n_iter, T, rtol, atol)
    assert (acc, rej) == counts_ref
    assert abs(step - step_ref) <= 1e-9 * step_ref
    assert np.abs(got - ref).max() < 1e-10
