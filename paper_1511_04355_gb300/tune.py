"""Search the FP32 far-field launch shapes on this GPU and write the tuning table.

For icosphere meshes of 320, 1280, 5120 and 20480 triangles (the range of the uneven-instance
workload) the library's autotuner (bem_autotune) times one FP32 operator application with every
launch shape, for launches of 1, 2, 4, ..., 128 frequencies, and keeps the fastest shape per
launch size.  The table is written to far32_tuning.txt beside this file, one entry per line
(ne_max nfl_max ft tiles waves ms ms_fixed), which bem_load_tuning reads.

Run on the GPU the table is for: python -m paper_1511_04355_gb300.tune  (about 2.5 minutes)
"""
from __future__ import annotations

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LEVELS = (2, 3, 4, 5)
NFL = (1, 2, 4, 8, 16, 32, 64, 128)


def main(path=None):
    import workloads as W
    import paper_1511_04355_gb300 as P

    path = path or P.TUNING_TABLE
    lines = ["# FP32 far-field launch shapes chosen by bem_autotune on this GPU",
             "# icosphere cavities, mu 1e9 Pa, nu 0.25, rho 2000 kg/m^3, s_k = 250 + i k pi / 0.02",
             "# ne_max nfl_max ft tiles waves ms ms_fixed   (ms: one FP32 operator application)"]
    for level in LEVELS:
        prob = W.spherical_cavity(level=level, n_freq=max(NFL))
        c = P.Context(0)
        c.set_mesh(prob.verts, prob.tris)
        m = prob.material
        c.set_material(m.mu, m.nu, m.rho)
        c.set_bc(prob.bc_type, prob.bc_value)
        t0 = time.perf_counter()
        for e in P.bem_autotune(c.h, prob.s, list(NFL)):
            lines.append(f"{e['ne_max']} {e['nfl_max']} {e['ft']} {e['tiles']} {e['waves']} "
                         f"{e['ms']:.4f} {e['ms_fixed']:.4f}")
        print(f"{len(prob.tris)} triangles: {time.perf_counter() - t0:.1f} s", flush=True)
        c.close()
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
