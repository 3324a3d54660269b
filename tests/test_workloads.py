"""The synthetic workloads (CPU): the paper's monolayer constants come from the numbers the paper prints
(tests/golden/paper_constants.json, Sec. IV), converted to the library's reduced units."""
import json
import math
import os

import numpy as np

from paper_1804_07135_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_monolayer_uses_the_printed_constants():
    c = json.load(open(GOLDEN))
    assert (W.PAPER_A_NM, W.PAPER_MOMENT_MUB, W.PAPER_J_MEV) == (c["lattice_constant_nm"], c["moment_bohr_magnetons"], c["exchange_meV"])
    s = W.paper_monolayer()
    assert [s.nx, s.ny, s.nz] == c["lattice"] and s.n_images == c["images_per_string"]
    # Fig. 4's d = 5.30 meV in units of J
    assert abs(s.D - c["dmi_fig4_meV"] / c["exchange_meV"]) < 1e-15


def test_reduced_dipole_strength():
    # w = mu0 |S|^2 / (4 pi a^3) in units of J; mu0/(4 pi) = 1e-7 N/A^2 to 1e-10 relative
    c = json.load(open(GOLDEN))
    S = c["moment_bohr_magnetons"] * 9.2740100783e-24
    a = c["lattice_constant_nm"] * 1e-9
    w = 1e-7 * S * S / a ** 3 / (c["exchange_meV"] * 1.602176634e-22)
    assert abs(W.paper_w() - w) <= 1e-9 * w
    assert abs(w - 2.79e-4) < 0.005e-4  # the value quoted among the readings


def test_phase_diagram_grid_and_paths():
    wl = W.paper_phase_diagram()
    assert len(wl.strings) == 2 * len(W.PHASE_D_MEV) * len(W.PHASE_K_MEV)
    assert {s.path for s in wl.strings} == {"bloch", "boundary"}
    for s in wl.strings[:: len(W.PHASE_K_MEV)]:
        p = s.initial_path()
        assert np.allclose(np.linalg.norm(p, axis=-1), 1.0)
        assert np.allclose(p[-1], [0.0, 0.0, 1.0])  # the last image is the ferromagnet
        assert p[0][:, 2].min() < -0.9  # the first image holds a skyrmion core
