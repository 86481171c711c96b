"""CPU float64 oracle for the QR-compressed VIE solver. TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import, call or execute anything in this package.  The CUDA library
(``paper_2603_10586_gb300``) never imports it and shares no code with it.
"""
from .discretization import AtomMesh, Problem
from . import quadrature, assembly


def problem_from_geometry(g):
    """Oracle Problem from a ``workloads.Geometry`` (plain data)."""
    return Problem(g.centres, g.types, g.sides, g.nvs, g.eps, g.wavelength)
