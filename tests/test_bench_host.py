"""Host-side arithmetic of bench.py (no GPU): the zero-padded transform length, the y/z kernel's
FLOP count and the variant table."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_1804_07135_gb300 import binding, workloads  # noqa: E402


def _padded_brute(n):
    # the linear convolution of n samples needs a length >= 2n - 1; take the smallest 3-smooth length
    # (2^a 3^b), or the power of two when it is at most 1/8 longer
    m = 2 * n - 1
    smooth = min(L for L in range(m, 4 * m + 1) if L == 2 ** round(math.log2(L)) or
                 all(p in (2, 3) for p in _factors(L)))
    p2 = 1 << (m - 1).bit_length()
    return p2 if 8 * p2 <= 9 * smooth else smooth


def _factors(L):
    out, d = [], 2
    while d * d <= L:
        while L % d == 0:
            out.append(d)
            L //= d
        d += 1
    if L > 1:
        out.append(L)
    return out


def test_padded_length_rule():
    for n in range(1, 400):
        assert bench.padded(n) == _padded_brute(n), n
    assert [bench.padded(n) for n in (64, 96, 112, 192)] == [128, 192, 256, 384]


def test_yz_flop_count_of_the_bench_workload():
    spec = workloads.bloch_collapse().strings[0]
    # 16 pairs x (2 x 128 kx x 3 x 8 lines x 5 x 128 x 7 + 128 x 128 x 36 x 64)
    want = 16 * (2 * 128 * 3 * 8 * 5 * 128 * 7 + 128 * 128 * 36 * 64)
    assert bench.yz_flops(spec) == want


def test_variants_map_to_library_modes():
    assert set(bench.VARIANTS) >= {"plain", "spline", "climbing_image", "dopri5_per_string", "llg_euler"}
    for name, (interp, climb, integ, dyn) in bench.VARIANTS.items():
        assert interp in ("linear", "spline") and integ in ("euler", "dopri5", "dopri5_image")
        assert dyn in ("string", "llg") and not (climb and integ != "euler")
    assert binding.SS_INT_DOPRI5 == 1 and binding.SS_INTERP_SPLINE == 1 and binding.SS_DYN_LLG == 1


def test_group_flop_count_matches_the_string_count():
    # a single-string group gives the per-string count; pairs are formed over the group's images
    spec = workloads.bloch_collapse().strings[0]
    assert bench.yz_flops_group(spec.nx, spec.ny, spec.nz, spec.n_images) == bench.yz_flops(spec)
    assert bench.yz_flops_group(64, 64, 8, 33) == 17 * bench.yz_flops_group(64, 64, 8, 2)


def test_headline_is_the_largest_workload():
    wl = bench.headline_workload()
    assert wl.name == "uneven-study-20x32" and len(wl.strings) == 20
    assert wl.spin_updates_per_iter > workloads.boundary_sweep().spin_updates_per_iter
    keys, imgs = bench.group_keys(wl)
    assert len(keys) == 4 and sum(imgs.values()) == 640
    assert bench.oracle_sample_spec().nx == 64


def test_selected_workload_subsets():
    wl = bench.selected_workload(bench.HEADLINE, "192x192x8", 1)
    assert len(wl.strings) == 1 and (wl.strings[0].nx, wl.strings[0].nz) == (192, 8)
    assert wl.name == "uneven-study-20x32[192x192x8, 1 of 20 strings]"
    assert bench.selected_workload(bench.HEADLINE) is bench.WORKLOADS[bench.HEADLINE]
    assert len(bench.selected_workload("boundary-sweep-128x128x4-8x48", None, 3).strings) == 3
    # the CPU sample's N^2 cost stays bounded: fewer images for larger lattices
    for w in bench.WORKLOADS.values():
        spec = bench.oracle_sample_spec(w)
        assert spec.n_sites == min(s.n_sites for s in w.strings)
        assert bench.oracle_sample_images(spec) * spec.n_sites ** 2 <= 8 * 16384 ** 2 * 4
