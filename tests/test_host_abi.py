"""CPU tests of libvie's C-ABI surface and host logic (no GPU needed): the
library loads and exports every function include/vie.h declares, and the
host-side grid hierarchy and greedy map agree with the oracle."""
import os
import re

import numpy as np
import pytest

import workloads
from oracle import tree as OT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_10586_gb300 import build, vie
    if not os.path.exists(vie.LIB_PATH):
        build.build()
    return vie.load()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(vie_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_2603_10586_gb300 import vie
    assert declared_functions() == set(vie.EXPORTS)


@pytest.mark.parametrize("layout", ["square5", "square16", "graded8", "vogel100", "vogel300"])
def test_host_far_blocks_match_oracle(lib, layout):
    from paper_2603_10586_gb300 import vie
    if layout.startswith("square"):
        g = workloads.square_array(int(layout[6:]), 1)
    elif layout.startswith("graded"):
        g = workloads.graded_array(int(layout[6:]), 1, seed=3)
    else:
        g = workloads.vogel_spiral(int(layout[5:]))
    L, mine = vie.plan_far_blocks(g.centres)
    Lo, ref = OT.build_tree(g.centres)
    assert L == Lo
    assert mine == [(l, list(t), list(s)) for l, t, s in ref]


def test_host_rejects_coincident_atoms(lib):
    from paper_2603_10586_gb300 import vie
    with pytest.raises(vie.VieError):
        vie.plan_far_blocks(np.zeros((3, 3)))


def test_host_lpt_matches_oracle(lib):
    from paper_2603_10586_gb300 import vie
    rng = np.random.default_rng(4)
    for n, p in ((1, 1), (17, 4), (500, 64), (3000, 7)):
        w = rng.integers(1, 1000, n).astype(float)
        owner, loads = vie.lpt_assign(w, p)
        o_ref, l_ref, _ = OT.lpt_assign(w, p)
        assert np.array_equal(owner, o_ref)
        assert np.allclose(loads, l_ref)


def test_footprint_model_is_monotone(lib):
    from paper_2603_10586_gb300 import vie
    a = vie.footprint_bytes(10000, 108, 1, 60, 10 ** 7)
    assert vie.footprint_bytes(20000, 108, 1, 60, 10 ** 7) > a
    assert vie.footprint_bytes(10000, 108, 4, 60, 10 ** 7) > a
    assert vie.footprint_bytes(10000, 108, 1, 60, 10 ** 8) > a
