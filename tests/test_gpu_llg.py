"""Parity of the precessional dynamics (Eq. 9, reduced units) with the FP64 oracle's `llg_run` and
`llg_run_rk`, through the C ABI: every image an independent system, no reparametrisation.

FP64: states to 1e-11 (Euler) and 1e-10 (Dormand-Prince, equal attempt counts; the carried steps to
1e-6 relative, since the error estimate sum (b - bhat) k is a difference of nearly equal sums whose
relative rounding is about eps |k| / |e|, here up to 1e-7); FP32: 1e-4.
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


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", [(16, 16, 1, 1.0, 0.3, 0.05, 0.01, 16),   # x kernels of length 32
                                  (57, 20, 1, 1.0, 0.3, 0.05, 0.02, 3)])   # length 128 (FP32 two-pass kernels)
def test_llg_euler(ss, prec, case):
    dt, alpha, n = 0.05, 0.2, 40
    path = W.bloch_point_path(case[0], case[1], case[2], case[7], R=4.0, D=case[4])
    with ss.StringMethod([case], dt=dt, precision=prec) as sm:
        sm.set_dynamics(ss.SS_DYN_LLG, alpha)
        sm.set_path(0, path)
        s0 = sm.get_path(0)
        sm.step(n)
        got = sm.get_path(0)
        e = sm.energies(0)
        e_step = sm.step_energies(0)
    ref, e_ref = oracle.llg_run(_model(case), _unit(s0), n, dt, alpha)
    _, e_prev = oracle.llg_run(_model(case), _unit(s0), n - 1, dt, alpha)
    tol = 1e-4 if prec == FP32 else 1e-11
    assert np.abs(got - ref).max() < tol
    np.testing.assert_allclose(e, e_ref, rtol=0, atol=100 * tol)
    np.testing.assert_allclose(e_step, e_prev, rtol=0, atol=100 * tol)


@pytest.mark.parametrize("kind", ["string", "image"])
def test_llg_dopri5_fp64(ss, kind):
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    T, alpha, n, rtol, atol = 0.5, 0.1, 6, 1e-7, 1e-9
    per_image = kind == "image"
    with ss.StringMethod([c], dt=T, precision=FP64) as sm:
        sm.set_dynamics(ss.SS_DYN_LLG, alpha)
        sm.set_integrator(ss.SS_INT_DOPRI5_IMAGE if per_image else ss.SS_INT_DOPRI5, rtol, atol)
        sm.set_path(0, spec.initial_path())
        s0 = sm.get_path(0)
        sm.step(n)
        got = sm.get_path(0)
        states = [sm.integrator_state(0, k) for k in range(spec.n_images)] if per_image else [sm.integrator_state(0)]
    ref, _, steps, counts = oracle.llg_run_rk(_model(c), _unit(s0), n, T, alpha, rtol, atol, per_image=per_image)
    assert np.abs(got - ref).max() < 1e-10
    if per_image:
        np.testing.assert_array_equal(np.array([st[1:] for st in states]), counts)
        np.testing.assert_allclose([st[0] for st in states], steps, rtol=1e-6)
    else:
        assert states[0][1:] == counts
        assert abs(states[0][0] - steps) <= 1e-6 * steps


def test_llg_without_damping_conserves_energy(ss):
    # every interaction including the FFT dipole field; pure precession keeps E (the Dormand-Prince
    # evolution at a tight tolerance, FP64)
    c = (24, 20, 3, 1.0, 0.3, 0.1, 0.05, 2)
    rng = np.random.default_rng(11)
    s = _unit(rng.standard_normal((2, 24 * 20 * 3, 3)))
    with ss.StringMethod([c], dt=0.25, precision=FP64) as sm:
        sm.set_dynamics(ss.SS_DYN_LLG, 0.0)
        sm.set_integrator(ss.SS_INT_DOPRI5, 1e-10, 1e-12)
        sm.set_path(0, s)
        e0 = sm.energies(0)
        sm.step(8)
        e1 = sm.energies(0)
        moved = np.abs(sm.get_path(0) - _unit(s)).max()
    assert moved > 0.1
    np.testing.assert_allclose(e1, e0, rtol=1e-8)


def test_llg_state_rules_and_return_to_string(ss):
    spec = W.tiny_bloch().strings[0]
    c = _case(spec)
    with ss.StringMethod([c], dt=0.1, precision=FP64) as sm:
        for alpha in (-0.1, float("nan"), float("inf")):
            with pytest.raises(ss.SsError) as ei:
                sm.set_dynamics(ss.SS_DYN_LLG, alpha)
            assert ei.value.status == ss.SS_ERR_INVALID_ARG
        with pytest.raises(ss.SsError):
            sm.set_dynamics(5, 0.1)
        sm.set_reparam(ss.SS_INTERP_LINEAR, True)
        with pytest.raises(ss.SsError) as ei:
            sm.set_dynamics(ss.SS_DYN_LLG, 0.1)
        assert ei.value.status == ss.SS_ERR_STATE
        sm.set_reparam(ss.SS_INTERP_LINEAR, False)
        sm.set_dynamics(ss.SS_DYN_LLG, 0.1)
        with pytest.raises(ss.SsError) as ei:
            sm.set_reparam(ss.SS_INTERP_LINEAR, True)
        assert ei.value.status == ss.SS_ERR_STATE
        sm.set_path(0, spec.initial_path())
        sm.step(5)
        sm.set_dynamics(ss.SS_DYN_STRING)
        s0 = sm.get_path(0)
        sm.step(3)
        got = sm.get_path(0)
    ref, _ = oracle.string_run(_model(c), _unit(s0), 3, 0.1)
    assert np.abs(got - ref).max() < 1e-12
