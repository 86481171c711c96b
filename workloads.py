"""Seeded synthetic inputs shared by the oracle tests, the CUDA path tests and bench.py.

This module holds input generation only (array layouts, material tables,
incident-wave directions, request streams, random vectors).  It contains none
of the method's arithmetic, so the oracle and the CUDA path stay independent.

The paper's own workload (Vogel spirals of gold spheres meshed with
tetrahedra, Sec. 6.1) is not reproducible here: the meshes are not published.
These generators stand in for it with square arrays of dielectric cubes of
the same kind (sub-wavelength meta-atoms in the z = 0 plane).  Lengths are in
units of the wavelength unless stated.

Atom (ix, iy) of an ns x ns array sits at ((ix - (ns-1)/2) p, (iy - (ns-1)/2) p, 0)
and has index iy * ns + ix (row-major).
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass
class Geometry:
    """Plain description of a metasurface (what the C-ABI's vie_geometry carries)."""
    centres: np.ndarray          # (N, 3) float64
    types: np.ndarray            # (N,) int32
    sides: np.ndarray            # (T,) float64 cube side per type
    nvs: np.ndarray              # (T,) int32 voxels per edge per type
    eps: np.ndarray              # (T,) complex128 relative permittivity per type
    wavelength: float = 1.0

    @property
    def n_atoms(self):
        return len(self.types)

    def unknowns(self):
        nv = self.nvs[self.types]
        return int(np.sum(3 * (nv + 1) * nv * nv))


def square_array(ns, nv, side=0.2, pitch=0.4, eps=12.0, wavelength=1.0):
    """ns x ns array of identical cubes (one type)."""
    i = np.arange(ns)
    ix, iy = np.meshgrid(i, i, indexing="xy")
    c = np.zeros((ns * ns, 3))
    c[:, 0] = (ix.ravel() - (ns - 1) / 2.0) * pitch
    c[:, 1] = (iy.ravel() - (ns - 1) / 2.0) * pitch
    return Geometry(c, np.zeros(ns * ns, np.int32), np.array([side], float),
                    np.array([nv], np.int32), np.array([eps], complex), float(wavelength))


def graded_array(ns, nv, seed, sides=(0.15, 0.2, 0.25), pitch=0.4, eps=12.0, wavelength=1.0):
    """ns x ns array whose cube side follows a lens phase profile.

    rho = distance from the array centre, psi = k (sqrt(rho^2 + F^2) - F) with
    the focal length F ~ U[10, 40] wavelengths drawn from ``seed``; the type is
    floor(3 (psi mod 2 pi) / (2 pi)) and selects the side from ``sides``.
    """
    g = square_array(ns, nv, sides[0], pitch, eps, wavelength)
    rng = np.random.default_rng(seed)
    F = rng.uniform(10.0, 40.0) * wavelength
    k = 2 * np.pi / wavelength
    rho = np.hypot(g.centres[:, 0], g.centres[:, 1])
    psi = k * (np.sqrt(rho ** 2 + F ** 2) - F)
    t = np.floor(3.0 * np.mod(psi, 2 * np.pi) / (2 * np.pi)).astype(np.int32)
    t = np.clip(t, 0, len(sides) - 1)
    g.types = t
    g.sides = np.array(sides, float)
    g.nvs = np.full(len(sides), nv, np.int32)
    g.eps = np.full(len(sides), eps, complex)
    return g


def vogel_spiral(n_atoms, radius=0.1, nv=1, eps=12.0, wavelength=1.0):
    """Sec. 6.1 layout: centres r_i (cos(i a), sin(i a), 0), r_i = c sqrt(i),
    c = sqrt(3) R, a = 2 pi / phi^2 with phi = (1 + sqrt 5)/2 (the printed
    "(1+sqrt5/2)" is read as the golden ratio), i = 1..N.  Cubes of side R
    stand in for the spheres of radius R."""
    i = np.arange(1, n_atoms + 1, dtype=float)
    phi = (1.0 + np.sqrt(5.0)) / 2.0
    alpha = 2.0 * np.pi / phi ** 2
    r = np.sqrt(3.0) * radius * np.sqrt(i)
    c = np.stack([r * np.cos(i * alpha), r * np.sin(i * alpha), np.zeros_like(r)], 1)
    return Geometry(c, np.zeros(n_atoms, np.int32), np.array([radius], float),
                    np.array([nv], np.int32), np.array([eps], complex), float(wavelength))


# Sec. 6.1: spheres of radius 100 nm at a wavelength of 600 nm, gold with
# eps_r = -9.428 + 1.513 i at that frequency.  The paper's "+ i" belongs to the
# exp(-i w t) convention; under this code's exp(j w t) a lossy medium has
# Im eps < 0, so the same gold is -9.428 - 1.513 j.
GOLD_600NM = complex(-9.428, -1.513)


def vogel_gold(n_atoms, nv=2, wavelength=1.0):
    """The Sec. 6.1 workload on this voxel basis: n_atoms gold meta-atoms of
    radius R = wavelength / 6 on the Vogel spiral (c = sqrt(3) R), each a cube
    of the sphere's volume (side (4 pi / 3)^(1/3) R) standing in for the
    sphere."""
    R = wavelength / 6.0
    g = vogel_spiral(n_atoms, radius=R, nv=nv, eps=GOLD_600NM, wavelength=wavelength)
    return Geometry(g.centres, g.types, np.array([(4.0 * np.pi / 3.0) ** (1.0 / 3.0) * R]), g.nvs, g.eps,
                    g.wavelength)


def single_cube(side, nv, eps=12.0, wavelength=1.0):
    return Geometry(np.zeros((1, 3)), np.zeros(1, np.int32), np.array([side], float),
                    np.array([nv], np.int32), np.array([eps], complex), float(wavelength))


def two_cubes(distance, side=0.2, nv=1, eps=12.0, wavelength=1.0):
    c = np.array([[0.0, 0.0, 0.0], [distance, 0.0, 0.0]])
    return Geometry(c, np.zeros(2, np.int32), np.array([side], float),
                    np.array([nv], np.int32), np.array([eps], complex), float(wavelength))


# ----------------------------------------------------------------------------
# incident plane waves: (khat, polarisation) per right-hand side
# ----------------------------------------------------------------------------
def normal_incidence():
    """Incidence from +z (khat = -z), x-polarised."""
    return np.array([[0.0, 0.0, -1.0]]), np.array([[1.0, 0.0, 0.0]], complex)


def angle_sweep(n_angles=32, max_deg=60.0):
    """n_angles polar angles uniform in [0, max_deg] (ends included) at azimuth 0,
    each with TE (y) and TM (theta-hat) polarisation; RHS index = 2 i + pol."""
    th = np.deg2rad(max_deg) * np.arange(n_angles) / max(n_angles - 1, 1)
    khat, pol = [], []
    for t in th:
        kh = -np.array([np.sin(t), 0.0, np.cos(t)])
        te = np.array([0.0, 1.0, 0.0])
        tm = np.array([np.cos(t), 0.0, -np.sin(t)])
        khat += [kh, kh]
        pol += [te, tm]
    return np.array(khat), np.array(pol, complex)


def random_directions(n, seed, max_deg=20.0):
    """n incidence directions near normal incidence with random linear polarisation."""
    rng = np.random.default_rng(seed)
    th = np.deg2rad(max_deg) * rng.uniform(0, 1, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    kh = -np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    eth = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1)
    eph = np.stack([-np.sin(ph), np.cos(ph), np.zeros(n)], 1)
    a = rng.uniform(0, 2 * np.pi, n)
    pol = np.cos(a)[:, None] * eth + np.sin(a)[:, None] * eph
    return kh, pol.astype(complex)


def random_complex(n, seed=1234, cols=None):
    """Complex standard normal vector(s) (float64), seed 1234 by default."""
    rng = np.random.default_rng(seed)
    shape = (n,) if cols is None else (n, cols)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


# ----------------------------------------------------------------------------
# the named configurations
# ----------------------------------------------------------------------------
def config(name, seed=0):
    """(geometry, khat, pol) of a named workload."""
    if name == "tiny":        # 4x4 of 3^3-voxel cubes, 1,728 unknowns
        g = square_array(4, 3)
        kh, p = normal_incidence()
    elif name == "scale":     # 16x16 of 6^3-voxel cubes, 193,536 unknowns
        g = square_array(16, 6)
        kh, p = normal_incidence()
    elif name == "multirhs":  # 32x32 of 4^3-voxel cubes, 245,760 unknowns, 64 RHS
        g = square_array(32, 4)
        kh, p = angle_sweep(32, 60.0)
    elif name == "graded":    # 64x64 graded, 4^3 voxels, 983,040 unknowns, 16 RHS
        g = graded_array(64, 4, seed)
        kh, p = random_directions(16, seed)
    elif name == "mid":       # 8x8 of 3^3-voxel cubes, 6,912 unknowns
        g = square_array(8, 3)
        kh, p = normal_incidence()
    else:
        raise KeyError(name)
    return g, kh, p


@dataclass
class Request:
    arrival_s: float
    ns: int
    wavelength: float
    eps: float
    khat: np.ndarray
    pol: np.ndarray
    geometry: Geometry = field(default=None)


def serving_stream(n_requests, seed=0, rate_hz=20.0, ns_range=(8, 48), nv=3):
    """Poisson request stream: inter-arrival Exp(1/rate), side ns ~ U{8..48},
    lambda ~ U[0.9, 1.1], eps_r ~ U[8, 14], 1..8 RHS near normal incidence.
    Geometry is fixed in absolute units (side 0.2, pitch 0.4)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        ns = int(rng.integers(ns_range[0], ns_range[1] + 1))
        lam = float(rng.uniform(0.9, 1.1))
        eps = float(rng.uniform(8.0, 14.0))
        s = int(rng.integers(1, 9))
        kh, p = random_directions(s, seed * 100003 + i)
        r = Request(t, ns, lam, eps, kh, p)
        r.geometry = square_array(ns, nv, 0.2, 0.4, eps, lam)
        out.append(r)
    return out
