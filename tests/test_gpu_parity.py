"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, on seeded inputs.

Tolerances:
  * field (Eqs. 2-7): max |h_gpu - h_oracle| <= 1e-5 * max |h_oracle| on the FP32 path, 1e-12 on FP64;
  * energies (Eq. 8) evaluated on the same stored state: |dE| <= w * (the FFT round-off bound of the
    dipole term derived in test_energy_and_terms_parity) + 1e-9;
  * trajectories (Sec. III loop): final path and barrier against the oracle run from the GPU's own
    starting state, with bounds stated in each test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1804_07135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1


def _sm(ss, strings, **kw):
    return ss.StringMethod(strings, **kw)


def _unit(a):
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _model(t):
    nx, ny, nz, J, D, K, w, _ = t
    return oracle.model(nx, ny, nz, J, D, K, w)


FIELD_CASES = [
    (16, 16, 1, 1.0, 0.3, 0.05, 0.01, 3),   # odd image count: one pair has an empty partner
    (5, 3, 2, 1.0, 0.3, 0.05, 0.02, 2),     # padded lengths 9 and 6 (radix 3)
    (12, 7, 3, 0.8, -0.25, 0.1, 0.05, 4),   # negative D, ragged rows
    (1, 6, 2, 1.0, 0.3, 0.05, 0.02, 2),     # nx = 1
    (33, 10, 1, 1.0, 0.3, 0.05, 0.02, 2),   # padded length 72 = 8*9
    (20, 21, 5, 1.0, 0.25, 0.1, 0.02, 3),   # rows not a multiple of the CTA row count
    (9, 9, 4, 1.0, 0.0, 0.0, 0.5, 2),       # dipole only, strong
    # padded length 128 along x and/or y: the two-pass register transforms (FP32)
    (64, 64, 4, 1.0, 0.3, 0.05, 0.02, 2),   # x and y/z kernels, nz = 4
    (57, 61, 8, 1.0, 0.3, 0.05, 0.03, 3),   # ragged x and y, nz = 8, odd image count
    (60, 20, 3, 1.0, 0.3, 0.05, 0.02, 2),   # x kernels only (Py = 48), ragged CTA rows
    (20, 58, 4, 0.9, -0.3, 0.05, 0.04, 2),  # y/z kernel only (Px = 48)
    # two kx columns per y/z CTA (four layers, Py = 192 and 256)
    (20, 90, 4, 1.0, 0.3, 0.05, 0.03, 3),
    (22, 112, 4, 1.0, 0.25, 0.1, 0.02, 2),
]


def _padded(n):
    """The zero-padded transform length: the smallest 2^a 3^b >= 2n - 1, or the power of two >= 2n - 1
    when that is at most 1/8 longer."""
    m = 2 * n - 1
    best = None
    a = 1
    while a < 4 * m:
        b = a
        while b < 4 * m:
            if b >= m and (best is None or b < best):
                best = b
            b *= 3
        a *= 2
    p2 = 1
    while p2 < m:
        p2 *= 2
    return p2 if 8 * p2 <= 9 * best else best


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", FIELD_CASES)
def test_field_parity(ss, case, prec):
    nx, ny, nz, J, D, K, w, n = case
    path = W.random_spins((n, nx * ny * nz, 3), seed=nx * 100 + ny)
    with _sm(ss, [case], precision=prec) as sm:
        sm.set_path(0, path)
        state = sm.get_path(0)
        h = sm.field(0)
    ref = oracle.field(_model(case), _unit(state))
    tol = (1e-5 if prec == FP32 else 1e-12) * np.abs(ref).max()
    assert np.abs(h - ref).max() <= tol


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", [(12, 10, 3, 1.0, 0.3, 0.05, 0.02, 4), (60, 58, 4, 1.0, 0.3, 0.05, 0.02, 2)])
def test_energy_and_terms_parity(ss, case, prec):
    m = _model(case)
    path = W.random_spins((case[7], case[0] * case[1] * case[2], 3), seed=3)
    n_img = case[7]
    with _sm(ss, [case], precision=prec) as sm:
        sm.set_path(0, path)
        state = _unit(sm.get_path(0))
        e = sm.energies(0)
        grads = [sm.grad(0, k) for k in range(n_img)]
    e_ref = oracle.energies(m, state)
    h_ref = oracle.field(m, state)
    nx, ny, nz, w = case[0], case[1], case[2], case[6]
    # The J, D, K terms are FP64 sums over the stored spins (atol 1e-9).  The unit-w dipole term
    # t_w = -(1/2) sum_i conv_i . s_i is an FP64 sum of the convolution computed in the path's
    # precision, whose round-off is bounded by ||d conv||_2 <= eps ||conv||_2 with
    # eps = u (2 log2(Px Py) + 3 nz + 4) (forward and inverse 2-D FFTs, the z sum over 3 nz lines, the
    # pair packing); by Cauchy-Schwarz over unit spins |d t_w| <= (1/2) eps ||conv||_2 sqrt(N), and the
    # energy (Eq. 1) inherits w times that.  1e-9 covers the FP64 rounding of the sums on both sides.
    u = 2.0 ** -24 if prec == FP32 else 2.0 ** -53
    eps = u * (2 * np.log2(_padded(nx) * _padded(ny)) + 3 * nz + 4)
    for k, (ds, terms) in enumerate(grads):
        ref_terms = oracle.energy_param_grad(m, state[k])
        np.testing.assert_allclose(terms[:3], ref_terms[:3], rtol=0, atol=1e-9)
        conv = oracle.dipole_field(m, state[k]) / w
        tol_w = 0.5 * eps * np.linalg.norm(conv) * np.sqrt(state.shape[1])
        assert abs(terms[3] - ref_terms[3]) <= tol_w + 1e-9, (terms[3], ref_terms[3], tol_w)
        assert abs(e[k] - e_ref[k]) <= w * tol_w + 1e-9, (k, e[k], e_ref[k], w * tol_w)
        assert np.abs(ds + h_ref[k]).max() <= (1e-5 if prec == FP32 else 1e-12) * np.abs(h_ref[k]).max()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_single_step_without_reparam(ss, prec):
    spec = W.tiny_bloch().strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    with _sm(ss, [case], precision=prec, reparam_every=0) as sm:
        sm.set_path(0, spec.initial_path())
        start = sm.get_path(0)
        sm.step(1)
        got = sm.get_path(0)
        e_pre = sm.step_energies(0)
    m = _model(case)
    h = oracle.field(m, start)
    ref = np.stack([oracle.step(start[k], h[k], 0.1) for k in range(spec.n_images)])
    assert np.abs(got - ref).max() <= (2e-6 if prec == FP32 else 1e-13)
    e_ref = np.array([oracle.energy_from_field(start[k], h[k]) for k in range(spec.n_images)])
    np.testing.assert_allclose(e_pre, e_ref, rtol=0, atol=1e-4 if prec == FP32 else 1e-10)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_one_iteration_with_reparam(ss, prec):
    spec = W.tiny_bloch().strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    with _sm(ss, [case], precision=prec) as sm:
        sm.set_path(0, spec.initial_path())
        start = sm.get_path(0)
        sm.step(1)
        got = sm.get_path(0)
    ref, _ = oracle.string_run(_model(case), start, 1, 0.1)
    assert np.abs(got - ref).max() <= (5e-6 if prec == FP32 else 1e-12)


def _run_both(ss, case, path, n_iter, prec):
    with _sm(ss, [case], precision=prec) as sm:
        sm.set_path(0, path)
        start = sm.get_path(0)
        sm.step(n_iter)
        got = sm.get_path(0)
        e = sm.energies(0)
        b = sm.barrier(0)
    ref, e_ref = oracle.string_run(_model(case), _unit(start), n_iter, 0.1)
    return got, e, b, ref, e_ref, oracle.barrier(e_ref)


def _barrier_split(case, got, e, b, ref, e_ref, b_ref):
    """The barrier error split into the evaluation (the reported energies against the oracle's energies of
    the GPU's own final state) and the trajectory drift (the oracle's energies of the two final states),
    with the drift's first-order bound: to first order E(s + ds) - E(s) = -sum_i F_i . ds_i with
    F = h - (s.h) s (energies are taken of renormalised spins, so the normal part of ds does not count),
    hence |dE_k| <= max_i |F_k,i| sum_i |ds_k,i| + (second order, ~ |dF/ds| |ds|^2, below 1e-12 here)."""
    m = _model(case)
    state = _unit(got)
    e_own = oracle.energies(m, state)
    b_own = oracle.barrier(e_own)
    h = oracle.field(m, state)
    F = h - (h * state).sum(-1, keepdims=True) * state
    drift_bound = np.array([np.abs(F[k]).max() * np.abs(got[k] - ref[k]).sum() for k in range(len(e))])
    return dict(total=b[0] - b_ref[0], evaluation=b[0] - b_own[0], drift=b_own[0] - b_ref[0],
                e_eval=np.abs(e - e_own), e_drift=np.abs(e_own - e_ref), drift_bound=drift_bound, k_own=b_own[1])


# The barrier target: |dE| <= 1e-6 in units of J against the FP64 oracle.  The reported energies are
# evaluated in FP64 (the FP64 pipeline applied to the FP32 state), so the evaluation part is at the FP64
# rounding level (1e-9 allows for sums of 3N terms in two orders) and the rest is the drift of the FP32
# trajectory, bounded per image as in _barrier_split.
BARRIER_TOL = 1e-6


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_trajectory_tiny_bloch_200_iterations(ss, prec):
    wl = W.tiny_bloch()
    spec = wl.strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    got, e, (dE, k), ref, e_ref, (dE_ref, k_ref) = _run_both(ss, case, spec.initial_path(), wl.n_iter, prec)
    if prec == FP64:
        assert np.abs(got - ref).max() < 1e-10
        assert abs(dE - dE_ref) < 1e-10 and k == k_ref
    else:
        assert np.abs(got - ref).max() < 1e-5
        sp = _barrier_split(case, got, e, (dE, k), ref, e_ref, (dE_ref, k_ref))
        assert (sp["e_eval"] <= 1e-9).all(), sp["e_eval"].max()
        assert (sp["e_drift"] <= sp["drift_bound"] + 1e-9).all()
        assert abs(sp["evaluation"]) <= 2e-9 and sp["k_own"] == k
        assert abs(dE - dE_ref) <= BARRIER_TOL and k == k_ref, sp


@pytest.mark.parametrize("n_iter", [60, 200])
def test_trajectory_bloch_collapse_crop(ss, n_iter):
    full = W.bloch_collapse().strings[0]
    crop = W.bloch_collapse_crop_path(full.initial_path())
    case = (16, 16, 4, full.J, full.D, full.K, full.w, full.n_images)
    got, e, (dE, k), ref, e_ref, (dE_ref, k_ref) = _run_both(ss, case, crop, n_iter, FP32)
    assert np.abs(got - ref).max() < 1e-5
    sp = _barrier_split(case, got, e, (dE, k), ref, e_ref, (dE_ref, k_ref))
    assert (sp["e_eval"] <= 1e-9).all(), sp["e_eval"].max()
    assert (sp["e_drift"] <= sp["drift_bound"] + 1e-9).all()
    assert abs(sp["evaluation"]) <= 2e-9
    assert abs(dE - dE_ref) <= BARRIER_TOL and k == k_ref, sp


def test_batched_strings_of_uneven_size(ss):
    cases = [(16, 16, 1, 1.0, 0.3, 0.05, 0.01, 5), (12, 10, 2, 1.0, 0.2, 0.1, 0.02, 4),
             (16, 16, 1, 1.0, 0.35, 0.0, 0.02, 3), (7, 9, 3, 1.0, 0.25, 0.15, 0.0, 4)]
    paths = [W.bloch_point_path(c[0], c[1], c[2], c[7], R=3.0, D=c[4]) for c in cases]
    n_iter = 15
    with _sm(ss, cases) as sm:
        for i, p in enumerate(paths):
            sm.set_path(i, p)
        starts = [sm.get_path(i) for i in range(len(cases))]
        sm.step(n_iter)
        got = [sm.get_path(i) for i in range(len(cases))]
        es = [sm.energies(i) for i in range(len(cases))]
    for c, s0, g, e in zip(cases, starts, got, es):
        ref, e_ref = oracle.string_run(_model(c), _unit(s0), n_iter, 0.1)
        assert np.abs(g - ref).max() < 1e-5
        np.testing.assert_allclose(e, e_ref, rtol=0, atol=1e-5)


def _rotation_path(K, n_sites, seed):
    """Smooth, unevenly spaced path: every site turns about its own axis by 2 (k/(K-1))^1.5 rad."""
    rng = np.random.default_rng(seed)
    a = _unit(rng.standard_normal((n_sites, 3)))
    ax = _unit(rng.standard_normal((n_sites, 3)))
    out = np.empty((K, n_sites, 3))
    for k in range(K):
        th = 2.0 * (k / (K - 1)) ** 1.5
        c, s_ = np.cos(th), np.sin(th)
        out[k] = a * c + np.cross(ax, a) * s_ + ax * (ax * a).sum(-1, keepdims=True) * (1 - c)  # Rodrigues
    return out


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_long_and_short_strings_in_one_size_group(ss, prec):
    # K = 300 (several images per thread in the arc-length scan, 38 chunks of differences), K = 2 (one
    # chunk, one difference) and K = 9 (a chunk that also sums the last image's energy) share a lattice,
    # so one arc launch serves strings that use different numbers of chunks
    cases = [(4, 4, 1, 1.0, 0.3, 0.05, 0.01, 300), (4, 4, 1, 1.0, 0.2, 0.1, 0.02, 2),
             (4, 4, 1, 0.9, 0.3, 0.0, 0.03, 9)]
    paths = [_rotation_path(c[7], 16, seed=40 + i) for i, c in enumerate(cases)]
    n_iter = 5
    with _sm(ss, cases, precision=prec) as sm:
        for i, p in enumerate(paths):
            sm.set_path(i, p)
        starts = [sm.get_path(i) for i in range(len(cases))]
        sm.step(n_iter)
        got = [sm.get_path(i) for i in range(len(cases))]
        es = [sm.step_energies(i) for i in range(len(cases))]
    tol = 2e-5 if prec == FP32 else 1e-12
    for c, s0, g, e in zip(cases, starts, got, es):
        ref, e_ref = oracle.string_run(_model(c), _unit(s0), n_iter, 0.1)
        assert np.abs(g - ref).max() < tol, c
        # energies of the state before the last step (summed by the arc kernel's chunk CTAs): the
        # oracle's path after n_iter - 1 iterations
        _, e_prev = oracle.string_run(_model(c), _unit(s0), n_iter - 1, 0.1)
        np.testing.assert_allclose(e, e_prev, rtol=0, atol=tol * 10)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_paper_monolayer(ss, prec):
    # the paper's 112x112x1 monolayer (Sec. IV constants, d = 5.30 meV, padded length 256): the field at
    # sampled sites of two images, then three iterations of a six-image sub-string (images 0, 12, ..., 48
    # and the last) against the oracle
    spec = W.paper_monolayer()
    path = spec.initial_path()
    sub = np.concatenate([path[:-1:12], path[-1:]])
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, sub.shape[0])
    m = _model(case)
    sites = np.random.default_rng(5).integers(0, spec.n_sites, size=64)
    with _sm(ss, [case], precision=prec) as sm:
        sm.set_path(0, sub)
        start = sm.get_path(0)
        h = sm.field(0)
        sm.step(3)
        got = sm.get_path(0)
        e = sm.energies(0)
        dE, k = sm.barrier(0)
    for img in (1, 3):
        ref = oracle.field_at(m, _unit(start[img]), sites)
        assert np.abs(h[img][sites] - ref).max() <= (1e-5 if prec == FP32 else 1e-12) * np.abs(ref).max()
    ref, e_ref = oracle.string_run(m, _unit(start), 3, 0.1)
    dE_ref, k_ref = oracle.barrier(e_ref)
    assert np.abs(got - ref).max() < (1e-5 if prec == FP32 else 1e-12)
    # FP32: the two states differ by rounding, so to first order dE = -sum h . ds with independent
    # per-component errors of about u |s| per step: RMS u |h| sqrt(3N) ~ 6e-8 * 4 * 194 ~ 5e-5 per step,
    # 1.4e-4 after three; 1e-3 leaves a margin of seven.  FP64: energies near -2.5e4 are sums of 3N terms
    # in different orders on the two sides, so 1e-12 relative
    tol = 1e-3 if prec == FP32 else 1e-12 * np.abs(e_ref).max()
    np.testing.assert_allclose(e, e_ref, rtol=0, atol=tol)
    assert abs(dE - dE_ref) < tol and k == k_ref


@pytest.mark.parametrize("dims", [(64, 64, 8), (192, 192, 8)])
def test_full_size_field_on_sampled_sites(ss, dims):
    nx, ny, nz = dims
    case = (nx, ny, nz, 1.0, 0.25, 0.1, 0.02, 2)
    N = nx * ny * nz
    path = np.stack([W.skyrmion(nx, ny, nz, R=nx / 8, D=0.25), W.random_spins((N, 3), seed=21)])
    with _sm(ss, [case]) as sm:
        sm.set_path(0, path.astype(np.float32))
        state = sm.get_path(0)
        h = sm.field(0)
    rng = np.random.default_rng(5)
    sites = np.concatenate([[0, N - 1, nx - 1, nx * ny - 1], rng.integers(0, N, size=28)])
    m = _model(case)
    for k in range(2):
        ref = oracle.field_at(m, _unit(state[k]), sites)
        scale = np.abs(ref).max()
        assert np.abs(h[k][sites] - ref).max() <= 1e-5 * scale


def test_deterministic_and_resumable(ss):
    spec = W.tiny_bloch().strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    outs = []
    for split in (False, True):
        with _sm(ss, [case]) as sm:
            sm.set_path(0, spec.initial_path())
            if split:
                sm.step(17)
                sm.step(23)
            else:
                sm.step(40)
            outs.append((sm.get_path(0, np.float32), sm.energies(0), sm.step_energies(0)))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])


def test_device_and_host_buffers_agree(ss):
    spec = W.tiny_bloch().strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    path = spec.initial_path()
    with _sm(ss, [case]) as sm:
        sm.set_path(0, torch.from_numpy(path.astype(np.float32)).cuda())
        sm.step(5)
        dev = torch.zeros(path.shape, dtype=torch.float32, device="cuda")
        ss.ss_get_path(sm.ctx, 0, dev)
        host = sm.get_path(0, np.float32)
        np.testing.assert_array_equal(dev.cpu().numpy(), host)


def test_invalid_inputs_and_state(ss):
    case = (8, 8, 1, 1.0, 0.3, 0.05, 0.01, 3)
    with _sm(ss, [case]) as sm:
        with pytest.raises(ss.SsError) as e:
            sm.step(1)
        assert e.value.status == ss.SS_ERR_STATE
        bad = W.random_spins((3, 64, 3), seed=1)
        bad[1, 7] = 0.0
        with pytest.raises(ss.SsError) as e:
            sm.set_path(0, bad)
        assert e.value.status == ss.SS_ERR_INVALID_ARG
        bad[1, 7] = [np.nan, 0, 1]
        with pytest.raises(ss.SsError) as e:
            sm.set_path(0, bad)
        assert e.value.status == ss.SS_ERR_INVALID_ARG
        with pytest.raises(ss.SsError) as e:
            ss.ss_energies(sm.ctx, 3)
        assert e.value.status == ss.SS_ERR_INVALID_ARG
        sm.set_path(0, W.random_spins((3, 64, 3), seed=2))  # recovers
        sm.step(2)
        assert np.isfinite(sm.energies(0)).all()


def test_overflow_is_reported_as_nonfinite(ss):
    # a finite but huge exchange constant overflows the FP32 field: the energy reduction sees inf
    case = (8, 8, 1, 1e38, 0.0, 0.0, 0.0, 3)
    with _sm(ss, [case]) as sm:
        sm.set_path(0, W.random_spins((3, 64, 3), seed=4))
        sm.step(1)
        with pytest.raises(ss.SsError) as e:
            sm.step_energies(0)
        assert e.value.status == ss.SS_ERR_NONFINITE


def test_uneven_parameter_study_batch(ss):
    # the 20-string, four-size parameter study in one context (one launch per kernel and size)
    wl = W.uneven_study()
    cases = [(s.nx, s.ny, s.nz, s.J, s.D, s.K, s.w, s.n_images) for s in wl.strings]
    with _sm(ss, cases) as sm:
        for i, s in enumerate(wl.strings):
            sm.set_path(i, s.initial_path().astype(np.float32))
        sm.step(3)
        assert sm.kernels_per_iteration() == 4 * len({(c[0], c[1], c[2]) for c in cases})
        rng = np.random.default_rng(3)
        checked = set()
        for i, s in enumerate(wl.strings):
            e = sm.energies(i)
            assert np.isfinite(e).all()
            if (s.nx, s.nz) in checked:
                continue
            checked.add((s.nx, s.nz))
            state = sm.get_path(i)
            h = sm.field(i)
            m = _model(cases[i])
            sites = rng.integers(0, s.n_sites, size=12)
            for k in (0, s.n_images // 2):
                ref = oracle.field_at(m, _unit(state[k]), sites)
                assert np.abs(h[k][sites] - ref).max() <= 1e-5 * np.abs(ref).max()
    assert len(checked) == 4


def test_torch_caching_allocator(ss):
    # device memory from PyTorch's caching allocator: accounted by torch while the context lives,
    # returned by ss_destroy, and the results equal those of a cudaMalloc context
    spec = W.tiny_bloch().strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    ss.use_torch_allocator()
    try:
        with _sm(ss, [case], precision=FP64) as sm:
            assert torch.cuda.memory_allocated() > before
            sm.set_integrator(ss.SS_INT_DOPRI5, 1e-6, 1e-8)  # variant buffers come from it too
            grown = torch.cuda.memory_allocated()
            sm.set_integrator(ss.SS_INT_EULER, 1e-6, 1e-8)
            sm.set_path(0, spec.initial_path())
            sm.step(20)
            got = sm.get_path(0)
        assert grown > before
    finally:
        ss.use_cuda_malloc()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    with _sm(ss, [case], precision=FP64) as sm:
        sm.set_path(0, spec.initial_path())
        sm.step(20)
        ref = sm.get_path(0)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("case", [FIELD_CASES[0], FIELD_CASES[1], FIELD_CASES[2], FIELD_CASES[5], FIELD_CASES[6]])
def test_direct_dipole_field_parity(ss, case, prec):
    # SS_DIPOLE_DIRECT: the O(N^2) sum on the GPU against the oracle's direct sum
    nx, ny, nz, J, D, K, w, n = case
    path = W.random_spins((n, nx * ny * nz, 3), seed=nx * 100 + ny + 7)
    with _sm(ss, [case], precision=prec, dipole=ss.SS_DIPOLE_DIRECT) as sm:
        sm.set_path(0, path)
        state = sm.get_path(0)
        h = sm.field(0)
        terms = sm.energy_terms(0)
    ref = oracle.field(_model(case), _unit(state))
    tol = (1e-5 if prec == FP32 else 1e-12) * np.abs(ref).max()
    assert np.abs(h - ref).max() <= tol
    want = np.array([[t for t in oracle.energy_param_grad(_model(case), s)] for s in _unit(state)])
    np.testing.assert_allclose(terms, want, rtol=0, atol=(1e-3 if prec == FP32 else 1e-9))


def test_direct_dipole_trajectory_matches_fft_and_oracle(ss):
    wl = W.tiny_bloch()
    spec = wl.strings[0]
    case = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    out = {}
    for mode in (ss.SS_DIPOLE_DIRECT, ss.SS_DIPOLE_FFT):
        with _sm(ss, [case], precision=FP64, dipole=mode) as sm:
            sm.set_path(0, spec.initial_path())
            start = sm.get_path(0)
            sm.step(100)
            out[mode] = (sm.get_path(0), sm.barrier(0))
    ref, e_ref = oracle.string_run(_model(case), _unit(start), 100, 0.1)
    assert np.abs(out[ss.SS_DIPOLE_DIRECT][0] - ref).max() < 1e-10
    assert np.abs(out[ss.SS_DIPOLE_DIRECT][0] - out[ss.SS_DIPOLE_FFT][0]).max() < 1e-10
    assert abs(out[ss.SS_DIPOLE_DIRECT][1][0] - oracle.barrier(e_ref)[0]) < 1e-9


@pytest.mark.parametrize("n_iter", [0, 7, 40])
def test_barrier_from_selected_images_equals_full_fp64(ss, n_iter):
    # ss_barrier on an FP32 context evaluates in FP64 only the images whose FP32 energy bound can reach
    # the maximum; the result must equal the barrier over every image's FP64 energy (ss_energies) exactly
    cases = [(16, 16, 1, 1.0, 0.3, 0.05, 0.01, 16), (16, 16, 1, 1.0, 0.2, 0.1, 0.02, 9),
             (12, 10, 3, 1.0, 0.25, 0.1, 0.05, 6), (20, 21, 2, 1.0, 0.3, 0.0, 0.0, 5)]
    paths = [W.bloch_point_path(c[0], c[1], c[2], c[7], R=3.5, D=c[4]) for c in cases]
    with _sm(ss, cases) as sm:
        for i, p in enumerate(paths):
            sm.set_path(i, p)
        sm.step(n_iter)
        bars = [sm.barrier(i) for i in range(len(cases))]
        full = [sm.energies(i) for i in range(len(cases))]
    for (dE, k), e in zip(bars, full):
        kf = int(np.argmax(e))
        assert k == kf and dE == e[kf] - e[0]
