"""Phase-diagram run on the paper's monolayer (Sec. IV): annihilation barriers over a (d, k) grid for
the Bloch-point and the boundary path, through the library's public API only.

    python -m paper_1804_07135_gb300.study [--checkpoints 1000,2000,5000] [--spline] [--climb]
                                           [--integrator euler|dopri5|dopri5_image|rkf45|rkf45_image]

For every string it reports the barrier max_k E_k - E_0 (in units of J and in meV) at each checkpoint,
the index of the highest image, and the diameter of the first image's skyrmion (the distance between
the two zero crossings of s_z along y through the lattice centre, in lattice constants and nm), which
the paper relates to k (Fig. 4).  One JSON line per string, then a markdown table.
"""
import argparse
import json

import numpy as np

from . import binding, workloads


def skyrmion_diameter(image: np.ndarray, nx: int, ny: int) -> float:
    """Distance between the outermost zero crossings of s_z along y at x = nx // 2, layer 0 (lattice
    constants); 0 when s_z has no sign change there."""
    sz = image.reshape(-1, ny, nx, 3)[0, :, nx // 2, 2]
    cross = [y + sz[y] / (sz[y] - sz[y + 1]) for y in range(ny - 1) if sz[y] * sz[y + 1] < 0]
    return float(cross[-1] - cross[0]) if len(cross) >= 2 else 0.0


INTEGRATORS = {"euler": binding.SS_INT_EULER, "dopri5": binding.SS_INT_DOPRI5,
               "dopri5_image": binding.SS_INT_DOPRI5_IMAGE, "rkf45": binding.SS_INT_RKF45,
               "rkf45_image": binding.SS_INT_RKF45_IMAGE}


def run(wl, checkpoints, stream=None, spline=False, climb=False, integrator="euler", rtol=1e-6, atol=1e-8):
    descs = [(s.nx, s.ny, s.nz, s.J, s.D, s.K, s.w, s.n_images) for s in wl.strings]
    rows = [{"path": s.path, "d_meV": s.D * workloads.PAPER_J_MEV, "k_meV": s.K * workloads.PAPER_J_MEV,
             "barrier_J": {}, "barrier_meV": {}} for s in wl.strings]
    with binding.StringMethod(descs, dt=wl.dt, stream=stream) as sm:
        sm.set_reparam(binding.SS_INTERP_SPLINE if spline else binding.SS_INTERP_LINEAR, climb)
        if integrator != "euler":
            sm.set_integrator(INTEGRATORS[integrator], rtol, atol)
        for i, s in enumerate(wl.strings):
            sm.set_path(i, s.initial_path().astype(np.float32))
        done = 0
        for cp in sorted(checkpoints):
            sm.step(cp - done)
            done = cp
            for i, r in enumerate(rows):
                dE, k = sm.barrier(i)
                r["barrier_J"][cp] = dE
                r["barrier_meV"][cp] = dE * workloads.PAPER_J_MEV
                r["k_max"] = k
                if climb:
                    r["climbing_image"] = sm.climbing_image(i)
        for i, (s, r) in enumerate(zip(wl.strings, rows)):
            diam = skyrmion_diameter(sm.get_path(i)[0], s.nx, s.ny)
            r["diameter_a"] = diam
            r["diameter_nm"] = diam * workloads.PAPER_A_NM
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--checkpoints", default="1000,2000,5000")
    ap.add_argument("--spline", action="store_true", help="natural cubic spline reparametrisation")
    ap.add_argument("--climb", action="store_true", help="climbing image (Euler step only)")
    ap.add_argument("--integrator", default="euler", choices=tuple(INTEGRATORS))
    args = ap.parse_args()
    cps = [int(x) for x in args.checkpoints.split(",")]
    rows = run(workloads.paper_phase_diagram(), cps, spline=args.spline, climb=args.climb,
               integrator=args.integrator)
    for r in rows:
        print(json.dumps(r))
    print(f"\n| path | d (meV) | k (meV) | barrier (meV) at {', '.join(map(str, sorted(cps)))} | highest image | "
          f"skyrmion diameter (nm) |")
    print("|---|---|---|---|---|---|")
    for r in rows:
        b = " / ".join(f"{r['barrier_meV'][c]:.1f}" for c in sorted(cps))
        print(f"| {r['path']} | {r['d_meV']:.2f} | {r['k_meV']:.2f} | {b} | {r['k_max']} | {r['diameter_nm']:.2f} |")


if __name__ == "__main__":
    main()
