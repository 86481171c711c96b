"""Pins of the oracle's discretisation and assembly: closed-form mass matrix,
charge neutrality, reciprocity, quadrature convergence, the optical theorem
and the quasi-static dipole limit of a small cube."""
import numpy as np
import pytest

import workloads
from oracle import problem_from_geometry, assembly as A, fields as F


@pytest.fixture(scope="module")
def tiny(tiny_dense):
    P, Z, _, kh, pol = tiny_dense
    return P, Z, kh, pol


def test_unknown_counts():
    for nv, n in ((3, 108), (6, 756), (4, 240)):
        assert problem_from_geometry(workloads.square_array(1, nv)).n == n


def test_mass_matrix_closed_form_against_quadrature():
    # M_ij = int w_i . w_j by 3-point Gauss (exact for the quadratic integrand)
    from oracle.discretization import AtomMesh
    m = AtomMesh(0.3, 3)
    P, w, xi = A.voxel_points(m, np.zeros(3), 3)
    ps = A._profiles(xi)
    M = np.zeros((m.n_faces, m.n_faces))
    for i in range(m.n_faces):
        for j in range(m.n_faces):
            if m.face_dir[i] != m.face_dir[j]:
                continue
            d = m.face_dir[i]
            for va, sa in m.face_voxels(i):
                for vb, sb in m.face_voxels(j):
                    if va == vb:
                        M[i, j] += np.sum(w * ps[d, 0 if sa > 0 else 1] * ps[d, 0 if sb > 0 else 1])
    M /= m.h ** 4
    assert np.allclose(A.mass_matrix(m), M, rtol=0, atol=1e-12 / m.h)
    diag = np.diag(A.mass_matrix(m)) * m.h
    interior = (m.face_lo_vox >= 0) & (m.face_hi_vox >= 0)
    assert np.allclose(diag[interior], 2 / 3) and np.allclose(diag[~interior], 1 / 3)


def test_every_rooftop_is_charge_neutral():
    from oracle.discretization import AtomMesh
    m = AtomMesh(0.2, 4)
    for f in range(m.n_faces):
        vol, sur = m.face_charges(f)
        total = sum(c * m.h ** 3 for _, c in vol) + sum(c * m.h ** 2 for _, c in sur)
        assert abs(total) < 1e-12


def test_reciprocity(tiny):
    P, Z, _, _ = tiny
    n = P.offsets[1]
    # different atoms: the symmetric Gauss rule makes Z_IJ = Z_JI^T to rounding
    cross = Z[:n, n:]
    assert np.linalg.norm(cross - Z[n:, :n].T) <= 1e-12 * np.linalg.norm(cross)
    # touching pairs (inner analytic, outer Gauss) are not symmetrised: measured asymmetry
    asym = np.linalg.norm(Z - Z.T) / np.linalg.norm(Z)
    assert asym < 1e-4


def test_self_block_touching_rule_converges():
    # the static part of touching pairs converges as the outer rule grows;
    # the 6-point rule (the definition) is within 1e-3 of the 12-point one
    g = workloads.single_cube(0.2, 2)
    P = problem_from_geometry(g)
    old = A.Q_OUTER
    Zq = {}
    try:
        for q in (3, 4, 6, 8, 12):
            A.Q_OUTER = q
            Zq[q] = A.self_block(P, 0)
    finally:
        A.Q_OUTER = old
    err = {q: np.linalg.norm(Zq[q] - Zq[12]) / np.linalg.norm(Zq[12]) for q in (3, 4, 6, 8)}
    assert err[3] > err[4] > err[6] > err[8]
    assert err[6] < 1e-3


def test_cross_rule_accuracy():
    # 2-point rule between atoms (the definition) against 4 points: relative 1e-3
    g = workloads.square_array(2, 3)
    P = problem_from_geometry(g)
    Z2 = A.cross_block(P, 0, 1)
    old = A.Q_CROSS
    try:
        A.Q_CROSS = 4
        Z4 = A.cross_block(P, 0, 1)
    finally:
        A.Q_CROSS = old
    assert np.linalg.norm(Z2 - Z4) / np.linalg.norm(Z4) < 1e-3


def test_optical_theorem_lossless(tiny):
    P, Z, kh, pol = tiny
    v0 = A.rhs_v0(P, kh, pol)
    I = np.linalg.solve(Z, 1j * P.k * v0)
    se, ss = F.sigma_ext(I, v0), F.sigma_sca(P, I)
    assert se > 0
    assert abs(se - ss) / se < 1e-4


def test_lossy_permittivity_absorbs():
    # eps with negative imaginary part (e^{jwt}): extinction exceeds scattering
    g = workloads.square_array(2, 2, eps=12.0 - 2.0j)
    P = problem_from_geometry(g)
    Z = A.dense_matrix(P)
    v0 = A.rhs_v0(P, [0, 0, -1.0], [1, 0, 0])
    I = np.linalg.solve(Z, 1j * P.k * v0)
    se, ss = F.sigma_ext(I, v0), F.sigma_sca(P, I)
    assert se > ss * 1.01 and ss > 0


def _single_cube_alpha(a, nv, eps=12.0):
    g = workloads.single_cube(a, nv, eps)
    P = problem_from_geometry(g)
    Z = A.dense_matrix(P)
    kh, pol = np.array([0, 0, -1.0]), np.array([1, 0, 0.0])
    v0 = A.rhs_v0(P, kh, pol)
    I = np.linalg.solve(Z, 1j * P.k * v0)
    return P, I, v0, F.dipole_moment(P, I)


def test_quasi_static_dipole_limit():
    a = 0.01
    alphas = []
    for nv in (2, 3, 4):
        P, I, v0, p = _single_cube_alpha(a, nv)
        alpha = p[0]
        k = P.k
        # radiation damping of a lossless dipole: Im(1/alpha) = +k^3/(6 pi)  (e^{jwt})
        assert abs(np.imag(1 / alpha) * 6 * np.pi / k ** 3 - 1) < 1e-3
        # scattered power equals the dipole formula
        assert abs(F.sigma_sca(P, I) / (k ** 4 * abs(alpha) ** 2 / (6 * np.pi)) - 1) < 1e-3
        assert abs(p[1]) < 1e-9 * abs(alpha) and abs(p[2]) < 1e-9 * abs(alpha)
        alphas.append(alpha.real / a ** 3)
    # between the equal-volume Clausius-Mossotti sphere and eps - 1, converging upward
    assert all(3 * 11 / 14 < x < 11 for x in alphas)
    assert alphas[0] < alphas[1] < alphas[2]
    assert (alphas[2] - alphas[1]) < (alphas[1] - alphas[0])


def test_volume_charge_fraction_decreases_with_refinement():
    # App. A: the exact current is divergence-free inside; the discrete volume
    # charge must shrink relative to the surface charge as the mesh is refined
    frac = []
    for nv in (2, 3, 4):
        P, I, _, _ = _single_cube_alpha(0.05, nv)
        m = P.meshes[0]
        qv = np.zeros(m.n_vox, complex)
        qs = np.zeros(len(m.surf_face), complex)
        for f in range(m.n_faces):
            vol, sur = m.face_charges(f)
            for v, c in vol:
                qv[v] += I[f] * c * m.h ** 3
            for s, c in sur:
                qs[s] += I[f] * c * m.h ** 2
        frac.append(np.sum(np.abs(qv)) / (np.sum(np.abs(qv)) + np.sum(np.abs(qs))))
    assert frac[0] > frac[1] > frac[2]


def test_cross_rule_solution_sensitivity():
    # the 2-point rule between atoms (the definition) moves the solved current by
    # far less than the compression tolerance: against a 4-point rule on a 3x3
    # array of 2^3-voxel cubes the currents differ by < 1e-4 relative (on the
    # 4x4 array of 3^3 cubes the difference is 1.6e-5)
    g = workloads.square_array(3, 2)
    P = problem_from_geometry(g)
    kh, pol = np.array([0, 0, -1.0]), np.array([1, 0, 0.0])
    b = A.rhs(P, kh, pol)
    I2 = np.linalg.solve(A.dense_matrix(P), b)
    old = A.Q_CROSS
    try:
        A.Q_CROSS = 4
        I4 = np.linalg.solve(A.dense_matrix(P), b)
    finally:
        A.Q_CROSS = old
    assert np.linalg.norm(I2 - I4) / np.linalg.norm(I4) < 1e-4


def test_current_at_voxel_centres_uniform_field():
    # a uniform current density J0 e_d carries the flux J0 h^2 through every
    # face of direction d: the rooftop expansion reproduces J0 e_d at every
    # voxel centre (boundary faces included), and nothing in the other axes
    g = workloads.single_cube(0.3, 3)
    P = problem_from_geometry(g)
    m = P.meshes[0]
    for d, J0 in ((0, 2.0 - 1.0j), (1, 0.5j), (2, -3.0)):
        I = np.where(m.face_dir == d, J0 * m.h ** 2, 0.0).astype(complex)
        J = F.current_at_voxel_centres(P, I)
        want = np.zeros((m.n_vox, 3), complex)
        want[:, d] = J0
        assert np.allclose(J, want, rtol=0, atol=1e-12)


def test_current_at_voxel_centres_integrates_to_dipole_moment():
    # J is linear along its own axis inside a voxel, so the centre value is the
    # voxel average: sum_v J(c_v) h^3 = int J dV = j k p for any coefficients
    g = workloads.square_array(2, 3)
    P = problem_from_geometry(g)
    I = workloads.random_complex(P.n, 77)
    J = F.current_at_voxel_centres(P, I)
    vol = np.concatenate([np.full(P.mesh(a).n_vox, P.mesh(a).h ** 3) for a in range(P.n_atoms)])
    total = (J * vol[:, None]).sum(0)
    p = F.dipole_moment(P, I)
    assert np.allclose(total, 1j * P.k * p, rtol=1e-12, atol=0)


def test_near_field_tends_to_far_field(tiny):
    # far from the array the near field is F(rhat) exp(-j k r) / r up to terms
    # of relative order 1/(k r) and k D^2 / r
    P, Z, kh, pol = tiny
    I = np.linalg.solve(Z, A.rhs(P, kh, pol))
    dirs = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8], [0.0, -0.6, -0.8], [1.0, 0.0, 0.0]])
    r = 2.0e4
    E = F.near_field(P, I, r * dirs)
    ref = F.far_field(P, I, dirs) * np.exp(-1j * P.k * r) / r
    assert np.linalg.norm(E - ref) <= 1e-3 * np.linalg.norm(ref)


def test_near_field_of_small_cube_is_the_dipole_field():
    # a cube of side 0.01 lambda seen from 0.3 lambda: the field of its dipole
    # moment p, k^2 (n x p) x n / r + (3 n (n.p) - p) (1/r^3 + j k/r^2), times
    # exp(-j k r) / (4 pi), to the cube's octupole order (a/r)^2
    P, I, v0, p = _single_cube_alpha(0.01, 2)
    k = P.k
    pts = np.array([[0.3, 0.0, 0.0], [0.0, 0.3, 0.0], [0.0, 0.0, -0.3], [0.2, 0.1, 0.15]])
    E = F.near_field(P, I, pts)
    for i, x in enumerate(pts):
        rr = np.linalg.norm(x)
        n = x / rr
        Ed = (k * k * np.cross(np.cross(n, p), n) / rr + (3 * n * np.dot(n, p) - p) * (1 / rr ** 3 + 1j * k / rr ** 2))
        Ed = Ed * np.exp(-1j * k * rr) / (4 * np.pi)
        assert np.linalg.norm(E[i] - Ed) <= 5e-3 * np.linalg.norm(Ed), i
