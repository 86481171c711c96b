"""The stored dense solutions of the three-level arrays (written by
tests/golden/make_multilevel_golden.py from the oracle) are checked against
fresh oracle rows: for two atoms per file, the rows of Zs (the atom's self
block and its blocks with every other atom) applied to the stored current
give the right-hand side to float64 rounding, and the stored incident waves
are the generator's."""
import os
import sys

import numpy as np
import pytest

from oracle import problem_from_geometry, assembly as A

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_multilevel_golden as MG  # noqa: E402


@pytest.mark.parametrize("name", ["mid_8x8_nv3", "graded_8x8_nv3"])
def test_stored_solution_solves_the_oracle_system(name):
    g, kh, pol = MG.cases()[name]
    d = np.load(os.path.join(HERE, "golden", name + ".npz"))
    assert np.array_equal(d["khat"], kh) and np.array_equal(d["pol"], pol)
    P = problem_from_geometry(g)
    I = d["I"]
    assert I.shape == (P.n, len(kh))
    for a in (0, P.n_atoms - 19):
        rows = slice(P.offsets[a], P.offsets[a + 1])
        Zr = np.hstack([A.self_block(P, P.types[a]) if b == a else A.cross_block(P, a, b)
                        for b in range(P.n_atoms)])
        for c in range(len(kh)):
            br = A.rhs(P, kh[c], pol[c])[rows]
            assert np.linalg.norm(Zr @ I[:, c] - br) <= 1e-9 * np.linalg.norm(br)
