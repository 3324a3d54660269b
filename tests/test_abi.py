"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/ss.h declares.

No compute calls: these run without a GPU.
"""
import ctypes
import os
import re

import pytest

from paper_1804_07135_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ss.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ss_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ss_create", "ss_create_batch", "ss_set_path", "ss_get_path", "ss_step", "ss_energies",
                     "ss_barrier", "ss_field", "ss_grad", "ss_destroy", "ss_last_error"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(binding._SIGNATURES)
    binding.load()


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.SsError) as e:
        binding.ss_create(8, 8, 1, 1.0, 0.3, 0.05, 0.01, 4)
    assert e.value.status == binding.SS_ERR_CUDA


def test_argument_validation_on_host():
    with pytest.raises(binding.SsError) as e:
        binding.ss_create(0, 8, 1, 1.0, 0.3, 0.05, 0.01, 4)
    assert e.value.status == binding.SS_ERR_INVALID_ARG
    with pytest.raises(binding.SsError) as e:
        binding.ss_create(8, 8, 1, 1.0, 0.3, 0.05, 0.01, 1)
    assert e.value.status == binding.SS_ERR_INVALID_ARG
    with pytest.raises(binding.SsError) as e:
        binding.ss_create(8, 8, 1, float("nan"), 0.3, 0.05, 0.01, 4)
    assert e.value.status == binding.SS_ERR_INVALID_ARG
    with pytest.raises(binding.SsError) as e:
        binding.ss_create(8, 8, 1, 1.0, 0.3, 0.05, 0.01, 4, binding.make_opts(dt=-1.0))
    assert e.value.status == binding.SS_ERR_INVALID_ARG


def test_allocator_pair_must_be_complete():
    # one callback without the other is refused (host-side check, no GPU involved)
    binding.load()
    alloc = binding.SS_ALLOC_FN(lambda n, d, s, u: None)
    assert binding._lib.ss_set_allocator(alloc, binding.SS_FREE_FN(), None) == binding.SS_ERR_INVALID_ARG
    assert binding._lib.ss_set_allocator(binding.SS_ALLOC_FN(), binding.SS_FREE_FN(), None) == binding.SS_OK


def test_options_validation_on_host():
    # checked before any device work: an unknown dipole mode, a reparametrisation period other than
    # 0 or 1, a non-positive dt
    for kw in ({"dipole": 3}, {"reparam_every": 2}, {"dt": 0.0}, {"dt": float("nan")}):
        with pytest.raises(binding.SsError) as e:
            binding.ss_create(8, 8, 1, 1.0, 0.3, 0.05, 0.01, 4, binding.make_opts(**kw))
        assert e.value.status == binding.SS_ERR_INVALID_ARG, kw


def test_product_path_never_touches_the_oracle():
    # the package (binding, workloads, study, autograd, build) neither imports nor loads the oracle:
    # only the tests, the smoke check and the benchmark's CPU baseline may
    import ast
    pkg = os.path.join(ROOT, "paper_1804_07135_gb300")
    for name in os.listdir(pkg):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, name)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(a.name.split(".")[0] != "oracle" for a in node.names), name
            if isinstance(node, ast.ImportFrom):
                assert (node.module or "").split(".")[0] != "oracle", name
            if isinstance(node, ast.Constant) and isinstance(node.value, str):
                assert "ssm_oracle" not in node.value, name


def test_relax_loop_logic(monkeypatch):
    # the convergence loop of StringMethod.relax on a stand-in context whose barrier settles
    class Fake(binding.StringMethod):
        def __init__(self):
            self.ctx = None
            self.t = 0

        def step(self, n):
            self.t += n

        def barrier(self, string=0):
            return (1.0 - 0.5 ** (self.t / 100.0), 0)

    monkeypatch.setattr(binding, "ss_num_strings", lambda ctx: 2)
    sm = Fake()
    done, ok, hist = sm.relax(tol=1e-3, check_every=100, max_iter=10000)
    assert ok and done % 100 == 0 and abs(hist[0][-1] - hist[0][-2]) <= 1e-3 < abs(hist[0][-2] - hist[0][-3])
    sm = Fake()
    done, ok, _ = sm.relax(tol=0.0, check_every=50, max_iter=120)
    assert not ok and done == 120
    with pytest.raises(ValueError):
        sm.relax(check_every=0)
