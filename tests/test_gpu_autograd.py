"""Differentiation through libss (torch.autograd.Function) against the FP64 oracle.

dE/ds (Eq. 2) and dE/d(J, D, K, w) (Eq. 1 is linear in each constant) are checked against central
finite differences (h = 1e-4) of the oracle's Hamiltonian on the 16x16x4 crop of the 64x64x8
workload, and at the full 64x64x8 size against the oracle's field (itself pinned to finite
differences) at sampled sites and the oracle's parameter terms at the barrier image and image 0.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_07135_gb300 import autograd as ag
from paper_1804_07135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-4


def _relaxed(ss, case, path, n_iter):
    sm = ss.StringMethod([case])
    sm.set_path(0, path)
    sm.step(n_iter)
    return sm, sm.get_path(0)


def test_autograd_against_oracle_finite_differences_on_crop(ss):
    full = W.bloch_collapse().strings[0]
    case = (16, 16, 4, full.J, full.D, full.K, full.w, full.n_images)
    sm, state = _relaxed(ss, case, W.bloch_collapse_crop_path(full.initial_path()), 100)
    try:
        state = state / np.linalg.norm(state, axis=-1, keepdims=True)
        spins = torch.tensor(state, dtype=torch.float32, device="cuda", requires_grad=True)
        params = torch.tensor([full.J, full.D, full.K, full.w], dtype=torch.float64, requires_grad=True)
        e = ag.string_energies(sm, 0, spins, params)
        k = int(torch.argmax(e).item())
        assert k != 0, "the relaxed crop string should have its maximum away from image 0"
        barrier = e[k] - e[0]
        barrier.backward()
        g_s = spins.grad.double().cpu().numpy()
        g_p = params.grad.cpu().numpy()
        stored = sm.get_path(0)  # the FP32 state the library evaluated
    finally:
        sm.close()
    m = oracle.model(16, 16, 4, full.J, full.D, full.K, full.w)
    h = 1e-4
    rng = np.random.default_rng(0)
    for img, sign in ((k, 1.0), (0, -1.0)):
        s = stored[img] / np.linalg.norm(stored[img], axis=-1, keepdims=True)
        for _ in range(64):
            i, c = int(rng.integers(0, s.shape[0])), int(rng.integers(0, 3))
            sp, sm_ = s.copy(), s.copy()
            sp[i, c] += h
            sm_[i, c] -= h
            fd = (oracle.energy_terms(m, sp)["total"] - oracle.energy_terms(m, sm_)["total"]) / (2 * h)
            scale = max(1.0, abs(fd))
            assert abs(g_s[img, i, c] - sign * fd) <= REL * scale, (img, i, c)
    # barrier = E_k - E_0 is linear in each constant at fixed spins
    sk = stored[k] / np.linalg.norm(stored[k], axis=-1, keepdims=True)
    s0 = stored[0] / np.linalg.norm(stored[0], axis=-1, keepdims=True)
    base = dict(J=full.J, D=full.D, K=full.K, w=full.w)
    for q, name in enumerate("JDKw"):
        def b(v):
            p = dict(base)
            p[name] = v
            mm = oracle.model(16, 16, 4, **p)
            return oracle.energy_terms(mm, sk)["total"] - oracle.energy_terms(mm, s0)["total"]
        fd = (b(base[name] + h) - b(base[name] - h)) / (2 * h)
        assert abs(g_p[q] - fd) <= REL * max(1.0, abs(fd)), name


def test_autograd_full_size_against_oracle_field_and_terms(ss):
    spec = W.bloch_collapse().strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    sm, state = _relaxed(ss, case, spec.initial_path(), 200)
    try:
        spins = torch.tensor(state, dtype=torch.float32, device="cuda", requires_grad=True)
        params = torch.tensor([spec.J, spec.D, spec.K, spec.w], dtype=torch.float64, requires_grad=True)
        e = ag.string_energies(sm, 0, spins, params)
        e.sum().backward()
        g_s = spins.grad.double().cpu().numpy()
        d_barrier, kb, dE = ag.barrier_param_grad(sm, 0)
        stored = sm.get_path(0)
    finally:
        sm.close()
    m = oracle.model(spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w)
    rng = np.random.default_rng(1)
    sites = rng.integers(0, spec.n_sites, size=24)
    for img in (0, kb):
        s = stored[img] / np.linalg.norm(stored[img], axis=-1, keepdims=True)
        ref = -oracle.field_at(m, s, sites)
        assert np.abs(g_s[img][sites] - ref).max() <= REL * np.abs(ref).max()
    sk = stored[kb] / np.linalg.norm(stored[kb], axis=-1, keepdims=True)
    s0 = stored[0] / np.linalg.norm(stored[0], axis=-1, keepdims=True)
    ref = oracle.energy_param_grad(m, sk) - oracle.energy_param_grad(m, s0)
    np.testing.assert_allclose(d_barrier, ref, rtol=REL, atol=REL)
    assert dE >= 0.0


def test_autograd_fp32_against_the_fp64_gpu_method(ss):
    # the same state through an FP32 context and through the plain FP64 GPU method: dE/ds (the field,
    # Eq. 2) agrees to the FP32 field tolerance; the energies and the barrier's parameter derivatives
    # d(barrier)/d(J, D, K, w), both FP64 evaluations of that state, agree to FP64 rounding.  The FP64
    # context is given the FP32 context's stored state, so both evaluate the same spins.
    spec = W.bloch_collapse().strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    sm32, state = _relaxed(ss, case, spec.initial_path(), 100)
    out = {}
    try:
        with ss.StringMethod([case], precision=ss.SS_PREC_FP64) as sm64:
            for name, sm, dt in (("fp32", sm32, torch.float32), ("fp64", sm64, torch.float64)):
                spins = torch.tensor(state, dtype=dt, device="cuda", requires_grad=True)
                params = torch.tensor([spec.J, spec.D, spec.K, spec.w], dtype=torch.float64, requires_grad=True)
                e = ag.string_energies(sm, 0, spins, params)
                k = int(torch.argmax(e).item())
                (e[k] - e[0]).backward()
                out[name] = dict(e=e.detach().cpu().numpy(), k=k, g_s=spins.grad.double().cpu().numpy(),
                                 g_p=params.grad.cpu().numpy(), bpg=ag.barrier_param_grad(sm, 0))
                if name == "fp32":
                    state = sm32.get_path(0)  # the FP32 state, handed to the FP64 context
    finally:
        sm32.close()
    a, b = out["fp32"], out["fp64"]
    assert a["k"] == b["k"] and a["bpg"][1] == b["bpg"][1]
    scale = np.abs(b["g_s"]).max()
    assert np.abs(a["g_s"] - b["g_s"]).max() <= 1e-5 * scale
    np.testing.assert_allclose(a["e"], b["e"], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(a["g_p"], b["g_p"], rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(a["bpg"][0], b["bpg"][0], rtol=1e-10, atol=1e-9)
