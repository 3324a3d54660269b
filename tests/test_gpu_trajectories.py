"""Trajectory parity of the CUDA path with the FP64 oracle on the kernel sets the timed workloads use.

Each test runs a few full iterations (field, step, per-image energies, equal-arc-length
reparametrisation; Sec. III) through the C ABI and compares the final path element by element with the
oracle's run from the GPU's own starting state, then the reported energies with the oracle's energies
of the GPU's final state (the evaluation, Eq. 8) and of the oracle's final state (evaluation plus the
drift of the FP32 trajectory).

Tolerances:
  * path: 1e-5 (FP32) after three iterations -- each iteration rounds every component once in the
    step and once in the gather (u = 6e-8) and the projected step amplifies a perturbation by at most
    1 + dt |dF/ds| ~ 2.3 (dt = 0.1, |dF/ds| <= 2 (6 J + |D| + 2 K + w 4 zeta(3/2) beta(3/2)) ~ 13);
    1e-12 (FP64);
  * energies of the GPU's own final state: w times the FFT round-off bound of the dipole term
    (||d conv||_2 <= eps ||conv||_2, eps = u (2 log2(Px Py) + 3 nz + 4), so
    |dE| <= w (1/2) eps ||conv||_2 sqrt(N)), with u the unit round-off of the FFT's precision (the
    reported energies come from the FP64 evaluation, so u = 2^-53 on both paths), plus 1e-9 + 1e-13 |E|
    for the FP64 sums taken in different orders;
  * energies against the oracle's trajectory: the evaluation bound plus the drift, which to first order
    is -sum F . ds over the state difference ds (F = h - (s.h) s; the normal part of ds does not count
    since energies are taken of renormalised spins): |dE| <= max|F| ||ds||_1, with ds the measured
    path difference.
"""
import numpy as np
import pytest

import oracle
from paper_1804_07135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1


def _unit(a):
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _model(c):
    nx, ny, nz, J, D, K, w, _ = c
    return oracle.model(nx, ny, nz, J, D, K, w)


def _padded(n):
    """The library's padded transform length (smallest 2^a 3^b >= 2n - 1, or the power of two >= 2n - 1
    when that is at most 1/8 longer)."""
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


def _eval_bound(c, state, prec):
    """Bound on |E_gpu - E_oracle| of each image of `state` (see the module docstring): the reported
    energies are FP64 evaluations on both paths."""
    nx, ny, nz, w = c[0], c[1], c[2], c[6]
    if w == 0.0:
        return np.full(state.shape[0], 1e-9)
    m = _model(c)
    u = 2.0 ** -53
    eps = u * (2 * np.log2(_padded(nx) * _padded(ny)) + 3 * nz + 4)
    out = []
    for s in state:
        conv = oracle.dipole_field(m, s) / w
        out.append(w * 0.5 * eps * np.linalg.norm(conv) * np.sqrt(s.shape[0]) + 1e-9)
    return np.array(out)


def _run_batch(ss, cases, paths, n_iter, prec):
    with ss.StringMethod(cases, precision=prec) as sm:
        for i, p in enumerate(paths):
            sm.set_path(i, p)
        starts = [sm.get_path(i) for i in range(len(cases))]
        cfgs = [sm.launch_config(i) for i in range(len(cases))]
        sm.step(n_iter)
        got = [sm.get_path(i) for i in range(len(cases))]
        es = [sm.energies(i) for i in range(len(cases))]
        bs = [sm.barrier(i) for i in range(len(cases))]
    return starts, cfgs, got, es, bs


def _check(c, start, got, e, b, n_iter, prec):
    m = _model(c)
    ref, e_ref = oracle.string_run(m, _unit(start), n_iter, 0.1)
    path_err = np.abs(got - ref).max()
    assert path_err < (1e-5 if prec == FP32 else 1e-12), (c, path_err)
    state = _unit(got)
    e_own = oracle.energies(m, state)
    # plus the FP64 rounding of energies of size |E| summed over 3N terms in different orders
    bound = _eval_bound(c, state, prec) + 1e-13 * np.abs(e_own)
    assert (np.abs(e - e_own) <= bound).all(), (c, np.abs(e - e_own).max(), bound.max())
    force = oracle.field(m, state)
    force -= (force * state).sum(-1, keepdims=True) * state
    drift = np.array([np.abs(force[k]).max() * np.abs(got[k] - ref[k]).sum() for k in range(len(e))])
    assert (np.abs(e - e_ref) <= bound + drift + 1e-9).all(), (c, np.abs(e - e_ref).max())
    dE_ref, k_ref = oracle.barrier(e_ref)
    dE_own, k_own = oracle.barrier(e_own)
    assert b[1] == k_own
    assert abs(b[0] - dE_own) <= 2 * bound.max()
    return path_err


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_trajectory_on_the_64x64x8_kernel_set(ss, prec):
    # Padded lengths 128 in x and y with eight layers: the bench workload's kernels -- the gather and
    # length-128 x transform, the length-128 y/z kernel with the eight-layer z-convolution, the x-inverse
    # step kernel -- over three iterations with reparametrisation (ragged x and y extents, so the last
    # CTA rows and the zero padding are both exercised), element by element against the oracle.
    c = (57, 61, 8, 1.0, 0.25, 0.1, 0.02, 4)
    path = W.bloch_point_path(c[0], c[1], c[2], c[7], R=7.0, D=c[4])
    starts, cfgs, got, es, bs = _run_batch(ss, [c], [path], 3, prec)
    assert (cfgs[0]["Px"], cfgs[0]["Py"]) == (128, 128)
    _check(c, starts[0], got[0], es[0], bs[0], 3, prec)


# one lattice per compile-time kernel family of the batch workloads: padded length 128, 192, 256 or 384
# along x (x kernels) or along y (y/z kernel) with 1, 4 or 8 layers; three images each (one image pair
# has an empty partner), all in one context as separate size groups
FAMILY_CASES = [
    (60, 60, 4, 1.0, 0.30, 0.05, 0.02, 3),    # Px = Py = 128, nz = 4 (64^2 x 4 study strings)
    (90, 10, 4, 1.0, 0.20, 0.10, 0.02, 3),    # Px = 192
    (10, 90, 4, 1.0, 0.35, 0.15, 0.02, 3),    # Py = 192, nz = 4 (96^2 x 4 study strings)
    (120, 8, 8, 1.0, 0.25, 0.05, 0.02, 3),    # Px = 256
    (8, 120, 8, 1.0, 0.25, 0.10, 0.02, 3),    # Py = 256, nz = 8 (128^2 x 8 study strings)
    (7, 118, 4, 1.0, 0.30, 0.00, 0.02, 3),    # Py = 256, nz = 4 (boundary sweep)
    (112, 112, 1, 1.0, 0.098, 0.018, 0.05, 3),  # Px = Py = 256, nz = 1 (the paper's monolayer)
    (170, 6, 8, 1.0, 0.20, 0.10, 0.02, 3),    # Px = 384
    (6, 170, 8, 1.0, 0.40, 0.20, 0.02, 3),    # Py = 384, nz = 8 (192^2 x 8 study strings)
]


def test_uneven_batch_through_every_kernel_family(ss):
    # A reduced uneven parameter study: strings whose lattices select each compile-time transform
    # length and layer count the 20-string study, the boundary sweep and the monolayer use, stepped
    # together in one context for three iterations and compared with the oracle string by string.
    paths = [(W.bloch_point_path if i % 2 == 0 else W.boundary_path)(c[0], c[1], c[2], c[7],
                                                                    R=max(2.0, min(c[0], c[1]) / 3.0), D=c[4])
             for i, c in enumerate(FAMILY_CASES)]
    starts, cfgs, got, es, bs = _run_batch(ss, FAMILY_CASES, paths, 3, FP32)
    seen = set()
    for c, cfg in zip(FAMILY_CASES, cfgs):
        assert cfg["Px"] == _padded(c[0]) and cfg["Py"] == _padded(c[1])
        seen.add(cfg["Px"])
        seen.add(cfg["Py"])
    assert {128, 192, 256, 384} <= seen
    for c, s0, g, e, b in zip(FAMILY_CASES, starts, got, es, bs):
        _check(c, s0, g, e, b, 3, FP32)


@pytest.mark.parametrize("case", [(30, 120, 1, 1.0, 0.3, 0.05, 0.05, 5),   # Py = 256, nz = 1: 8 or 4 columns
                                  (20, 90, 4, 1.0, 0.3, 0.05, 0.05, 4),    # Py = 192, nz = 4: 2 or 1 column
                                  (12, 170, 1, 1.0, 0.3, 0.05, 0.05, 3),   # Py = 384 (XOR line layout), nz = 1
                                  (12, 170, 4, 1.0, 0.3, 0.05, 0.05, 3)])  # Py = 384, nz = 4
def test_yz_columns_per_cta_do_not_change_the_field(ss, case, monkeypatch):
    # the autotuner picks the two-pass y/z kernel's kx columns per CTA; every column is transformed and
    # convolved the same way whatever the count, so both counts give bit-identical fields (and the
    # default one is pinned to the oracle by the family test)
    nz = case[2]
    counts = (8, 4) if nz == 1 else (2, 1)
    path = W.random_spins((case[7], case[0] * case[1] * case[2], 3), seed=77 + nz)
    fields = []
    for kxb in counts:
        monkeypatch.setenv("SS_X_CONFIG", f"256:4:256:4:{kxb}")
        with ss.StringMethod([case]) as sm:
            sm.set_path(0, path)
            fields.append(sm.field(0, dtype=np.float32))
    np.testing.assert_array_equal(fields[0], fields[1])
    ref = oracle.field(_model(case), _unit(path))
    assert np.abs(fields[0] - ref).max() <= 1e-5 * np.abs(ref).max()
