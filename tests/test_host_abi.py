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


STRUCTS = {  # C struct of include/vie.h -> ctypes class of the binding
    "vie_ctx_opts": "CtxOpts", "vie_geometry": "GeometryC", "vie_op_info": "OpInfo",
    "vie_incident": "IncidentC", "vie_solve_opts": "SolveOpts", "vie_tune_result": "TuneResult",
    "vie_solve_stats": "SolveStats", "vie_serve_opts": "ServeOpts", "vie_request": "RequestC",
    "vie_result": "ResultC",
}


def test_struct_layouts_match_binding(tmp_path):
    # a layout drift between the header and the ctypes binding would pass wrong
    # arguments silently: compile the header with the host compiler and compare
    # every struct's size and every field's offset
    import ctypes
    import shutil
    import subprocess
    from paper_2603_10586_gb300 import vie
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vie.h"', "int main(void) {"]
    expect = []
    for cname, pyname in STRUCTS.items():
        cls = getattr(vie, pyname)
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {fname}));')
            expect.append(getattr(cls, fname).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


def test_header_constants_match_binding():
    from paper_2603_10586_gb300 import vie
    src = open(os.path.join(ROOT, "include", "vie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\b(VIE_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    consts.update({k: int(v) for k, v in re.findall(r"#define\s+(VIE_[A-Z0-9_]+)\s+(-?\d+)\b", src)})
    consts["VIE_NOALLOC_SCRATCH_ELEMS"] = 1 << 22
    assert re.search(r"#define\s+VIE_NOALLOC_SCRATCH_ELEMS\s+\(1LL << 22\)", src)
    rename = {"VIE_APPLY_FUSE_PRECOND": "FUSE_PRECOND", "VIE_APPLY_DENSE": "DENSE",
              "VIE_NOALLOC_SCRATCH_ELEMS": "NOALLOC_SCRATCH_ELEMS"}
    checked = 0
    for name, value in consts.items():
        if name in rename:
            py = rename[name]
        elif name.startswith("VIE_VAR_"):
            py = name[4:]
        elif name.startswith("VIE_ERR_") or name == "VIE_OK":
            py = name
        else:
            py = name[4:]
        if not hasattr(vie, py):
            continue
        assert getattr(vie, py) == value, (name, py)
        checked += 1
    for name in ("VIE_OK", "VIE_ERR_INVALID_ARG", "VIE_C64", "VIE_BF16X3", "VIE_VAR_SIMT_SHARED",
                 "VIE_APPLY_FUSE_PRECOND"):
        assert name in consts
    assert checked >= 20
