"""Writes cavity5120_lu.npz: dense-LU solutions of the 5120-triangle spherical cavity.

The workload is the batched benchmark's: icosphere of radius 1 m with 5120 flat triangles
(15360 complex unknowns), mu = 1e9 Pa, nu = 0.25, rho = 2000 kg/m^3, step pressure 1e6 Pa,
frequencies s_k = 250 + i k pi / 0.02.  For k = 0, 64 and 127 this assembles the dense
collocation system A(s_k) a = b(s_k) of Sec. 2.1, Eq. (Aa_b), with the oracle and solves it by
LU, which is the exact solution of the discrete system the GPU path solves iteratively.  Only
the oracle and the input generators are used.  Stored: s (3,), x (3, 15360) complex128 and the
LU residuals ||A x - b|| / ||b||.

Run from the repository root: python tests/golden/make_cavity5120_lu.py  (about 5 minutes per
frequency and 30 GB of host memory).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import bem as OB  # noqa: E402

KS = (0, 64, 127)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity5120_lu.npz")


def main():
    prob = W.spherical_cavity(level=4, n_freq=128, T=0.02, sigma=250.0)
    g = OB.geometry(prob.verts, prob.tris)
    xs, res = [], []
    for k in KS:
        t0 = time.perf_counter()
        A, b = OB.assemble(g, prob.s[k], prob.material, prob.bc_type, prob.bc_value)
        x = np.linalg.solve(A, b)
        res.append(np.linalg.norm(A @ x - b) / np.linalg.norm(b))
        del A
        xs.append(x)
        print(f"k={k}: {time.perf_counter() - t0:.0f} s, LU residual {res[-1]:.2e}", flush=True)
    np.savez(OUT, s=prob.s[list(KS)], k=np.array(KS), x=np.array(xs), lu_residual=np.array(res))


if __name__ == "__main__":
    main()
