"""Writes the dense direct solutions of two three-level arrays for the GPU solve
parity tests.  Calls only the oracle (dense float64 assembly of Zs and b, then
numpy's LU solve of the same discrete system, Sec. 6.2's reference solution)
and the seeded input generators.

    python tests/golden/make_multilevel_golden.py

Output (tests/golden/):
  mid_8x8_nv3.npz     8 x 8 array of 3^3-voxel cubes (6,912 unknowns, quadtree
                      levels 2 and 3): normal incidence + 2 angles x 2 polarisations
  graded_8x8_nv3.npz  8 x 8 graded array (three cube sides by lens phase, seed 0),
                      3^3 voxels: normal incidence + 3 random directions (seed 0)
Each file holds khat (nrhs x 3), pol (nrhs x 3 complex) and I (n x nrhs complex).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads  # noqa: E402
from oracle import problem_from_geometry, assembly as A  # noqa: E402


def cases():
    kn, pn = workloads.normal_incidence()
    ka, pa = workloads.angle_sweep(2, 40.0)
    kr, pr = workloads.random_directions(3, 0)
    return {
        "mid_8x8_nv3": (workloads.square_array(8, 3), np.vstack([kn, ka]), np.vstack([pn, pa])),
        "graded_8x8_nv3": (workloads.graded_array(8, 3, 0), np.vstack([kn, kr]), np.vstack([pn, pr])),
    }


def main():
    for name, (g, kh, pol) in cases().items():
        t0 = time.time()
        P = problem_from_geometry(g)
        Z = A.dense_matrix(P)
        B = np.stack([A.rhs(P, kh[c], pol[c]) for c in range(len(kh))], 1)
        I = np.linalg.solve(Z, B)
        np.savez(os.path.join(HERE, name + ".npz"), khat=kh, pol=pol, I=I)
        print(f"{name}: n = {P.n}, {len(kh)} right-hand sides, {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
