"""Oracle assembly of the scaled VIE matrix and right-hand side (CPU, float64).
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3, eq. matrixeq: Z I = v0 with Z = R + j w mu0 L + D / (j w eps0) and
R_ij = int w_i . w_j / (j w eps0 chi)  (sigma = 0, eq. const_rel).  The oracle
solves the equivalent scaled system (units eps0 = mu0 = c = 1, so w = k)

    Zs = j k Z = M / chi - k^2 L + D,        b = j k v0,

with M_ij = int w_i . w_j, L_ij = int int w_i(r) . w_j(r') g(r - r'),
D_ij = int int q_i(r) g(r - r') q_j(r') (q = distributional divergence of w,
volume and surface parts: for div-free loop/star functions this is the
paper's D^SS), g = exp(-j k R) / (4 pi R) (Sec. 2, below eq. IntEq; the
"k ... free-space wavelength" there is the wavenumber 2 pi / lambda).

Quadrature rule (the paper is silent; this is the reading used throughout):
  * element pairs in different atoms: tensor Gauss-Legendre, Q_CROSS = 2
    points per axis on both elements;
  * element pairs in one atom that do not touch: Gauss-Legendre, Q_SELF = 3;
  * touching element pairs (closed elements intersect): g = 1/(4 pi R) + g_s.
    The static part uses the closed-form inner integral over the source
    element (uniform or linear density) and Q_OUTER = 6 Gauss points per axis
    on the test element; g_s = (exp(-j k R) - 1)/(4 pi R) (limit -jk/(4 pi))
    uses Gauss-Legendre Q_SELF on both elements.  No symmetrisation.
  * right-hand side v0_i = int w_i . E0 with Q_SELF points per axis.
"""
import numpy as np

from .quadrature import (gauss_legendre_01, box_potential, box_linear_potential,
                         rect_potential)

Q_CROSS = 2
Q_SELF = 3
Q_OUTER = 6
FOUR_PI = 4.0 * np.pi


def green(R, k):
    return np.exp(-1j * k * R) / (FOUR_PI * R)


def green_smooth(R, k):
    """(exp(-jkR) - 1) / (4 pi R), written without cancellation; -jk/(4 pi) at R = 0."""
    with np.errstate(divide="ignore", invalid="ignore"):
        val = (-2.0 * np.sin(0.5 * k * R) ** 2 - 1j * np.sin(k * R)) / (FOUR_PI * R)
    return np.where(R > 0, val, -1j * k / FOUR_PI)


# ----------------------------------------------------------------------------
# Gauss point sets of all voxels / surface elements of one atom
# ----------------------------------------------------------------------------
def voxel_points(mesh, origin, q):
    """Points (nvox, q^3, 3), weights (q^3,), local coordinates xi (q^3, 3)."""
    x, w = gauss_legendre_01(q)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    xi = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=-1)
    wt = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel() * mesh.h ** 3
    lo = origin + mesh.h * mesh.vox_idx.astype(float)
    return lo[:, None, :] + mesh.h * xi[None, :, :], wt, xi


def surface_points(mesh, origin, q):
    """Points (nsurf, q^2, 3) and weights (q^2,) of the boundary faces."""
    x, w = gauss_legendre_01(q)
    A, B = np.meshgrid(x, x, indexing="ij")
    ns = len(mesh.surf_face)
    pts = np.zeros((ns, q * q, 3))
    for s in range(ns):
        f = mesh.surf_face[s]
        d = mesh.face_dir[f]
        a, b = [e for e in range(3) if e != d]
        base = origin + mesh.h * mesh.face_idx[f].astype(float)
        pts[s, :, d] = base[d]
        pts[s, :, a] = base[a] + mesh.h * A.ravel()
        pts[s, :, b] = base[b] + mesh.h * B.ravel()
    wt = (w[:, None] * w[None, :]).ravel() * mesh.h ** 2
    return pts, wt


def _profiles(xi):
    """psi[d, s, p]: s = 0 -> xi_d, s = 1 -> 1 - xi_d at point p."""
    return np.stack([np.stack([xi[:, d], 1.0 - xi[:, d]]) for d in range(3)])


# ----------------------------------------------------------------------------
# element-pair integral tables
# ----------------------------------------------------------------------------
class PairTables:
    """Integrals between the elements of a test atom and a source atom.

    U[A, B]            = int_A int_B g                       (voxel, voxel)
    W[d, sa, sb, A, B] = int_A psi_sa int_B psi_sb g          (profiles along d)
    VS[A, t], SV[s, B], SS[s, t]: uniform voxel/surface combinations.
    """

    def __init__(self, nA, nB, nsA, nsB):
        self.U = np.zeros((nA, nB), complex)
        self.W = np.zeros((3, 2, 2, nA, nB), complex)
        self.VS = np.zeros((nA, nsB), complex)
        self.SV = np.zeros((nsA, nB), complex)
        self.SS = np.zeros((nsA, nsB), complex)


def _gauss_vv(PA, wA, xiA, PB, wB, xiB, kern, out_U, out_W, rowsA=None, colsB=None, chunk=16):
    """Gauss-Gauss voxel/voxel integrals for all pairs (rowsA x colsB) or listed pairs."""
    psA = _profiles(xiA) * wA
    psB = _profiles(xiB) * wB
    nA = PA.shape[0]
    for a0 in range(0, nA, chunk):
        a1 = min(nA, a0 + chunk)
        D = PA[a0:a1, None, :, None, :] - PB[None, :, None, :, :]
        G = kern(np.sqrt((D * D).sum(-1)))
        out_U[a0:a1] = np.einsum("p,q,abpq->ab", wA, wB, G)
        for d in range(3):
            for sa in range(2):
                for sb in range(2):
                    out_W[d, sa, sb, a0:a1] = np.einsum("p,q,abpq->ab", psA[d, sa], psB[d, sb], G)


def _gauss_generic(PA, wA, PB, wB, kern):
    D = PA[:, None, :, None, :] - PB[None, :, None, :, :]
    G = kern(np.sqrt((D * D).sum(-1)))
    return np.einsum("p,q,abpq->ab", wA, wB, G)


def cross_tables(prob, I, J):
    """Tables for two different atoms: Gauss-Legendre Q_CROSS everywhere."""
    mI, mJ = prob.mesh(I), prob.mesh(J)
    oI, oJ = prob.origin(I), prob.origin(J)
    k = prob.k
    kern = lambda R: green(R, k)
    T = PairTables(mI.n_vox, mJ.n_vox, len(mI.surf_face), len(mJ.surf_face))
    PA, wA, xiA = voxel_points(mI, oI, Q_CROSS)
    PB, wB, xiB = voxel_points(mJ, oJ, Q_CROSS)
    SA, swA = surface_points(mI, oI, Q_CROSS)
    SB, swB = surface_points(mJ, oJ, Q_CROSS)
    _gauss_vv(PA, wA, xiA, PB, wB, xiB, kern, T.U, T.W)
    T.VS[:] = _gauss_generic(PA, wA, SB, swB, kern)
    T.SV[:] = _gauss_generic(SA, swA, PB, wB, kern)
    T.SS[:] = _gauss_generic(SA, swA, SB, swB, kern)
    return T


def _surf_extent(mesh, s):
    """Integer index extent [lo, hi] (3, 2) of a surface element."""
    f = mesh.surf_face[s]
    d = mesh.face_dir[f]
    ijk = mesh.face_idx[f]
    ext = np.stack([ijk, ijk + 1], axis=1)
    ext[d, 1] = ijk[d]
    return ext


def _vox_extent(mesh, v):
    ijk = mesh.vox_idx[v]
    return np.stack([ijk, ijk + 1], axis=1)


def _touch(e1, e2):
    return bool(np.all(np.maximum(e1[:, 0], e2[:, 0]) <= np.minimum(e1[:, 1], e2[:, 1])))


def self_tables(mesh, k):
    """Tables of one atom with itself, in local coordinates (corner at origin).

    Identical atoms therefore get bit-identical self blocks (Sec. 4: Z_11 = ... = Z_NN
    when all meta-atoms are identical)."""
    o = np.zeros(3)
    h = mesh.h
    nA, nS = mesh.n_vox, len(mesh.surf_face)
    T = PairTables(nA, nA, nS, nS)
    kern = lambda R: green(R, k)
    kern_s = lambda R: green_smooth(R, k)
    P3, w3, xi3 = voxel_points(mesh, o, Q_SELF)
    S3, sw3 = surface_points(mesh, o, Q_SELF)
    Po, wo, xio = voxel_points(mesh, o, Q_OUTER)
    So, swo = surface_points(mesh, o, Q_OUTER)

    # separated pairs (every pair first; touching pairs, where the plain rule
    # may hit R = 0, are overwritten below)
    with np.errstate(divide="ignore", invalid="ignore"):
        _gauss_vv(P3, w3, xi3, P3, w3, xi3, kern, T.U, T.W)
        T.VS[:] = _gauss_generic(P3, w3, S3, sw3, kern)
        T.SV[:] = _gauss_generic(S3, sw3, P3, w3, kern)
        T.SS[:] = _gauss_generic(S3, sw3, S3, sw3, kern)

    vext = [_vox_extent(mesh, v) for v in range(nA)]
    sext = [_surf_extent(mesh, s) for s in range(nS)]
    vlo = h * mesh.vox_idx.astype(float)
    vhi = vlo + h
    psio = _profiles(xio) * wo
    ps3 = _profiles(xi3) * w3

    def rect_of(s):
        return mesh.surf_rect(s, o)

    # --- voxel / voxel touching pairs
    for A in range(nA):
        for B in range(nA):
            if not _touch(vext[A], vext[B]):
                continue
            pts = Po[A]
            phi = box_potential(pts, vlo[B], vhi[B]) / FOUR_PI
            T.U[A, B] = np.dot(wo, phi)
            for d in range(3):
                lin = box_linear_potential(pts, vlo[B], vhi[B], d) / FOUR_PI
                inner = (lin, phi - lin)
                for sa in range(2):
                    for sb in range(2):
                        T.W[d, sa, sb, A, B] = np.dot(psio[d, sa], inner[sb])
            D = P3[A][:, None, :] - P3[B][None, :, :]
            G = kern_s(np.sqrt((D * D).sum(-1)))
            T.U[A, B] += w3 @ G @ w3
            for d in range(3):
                for sa in range(2):
                    for sb in range(2):
                        T.W[d, sa, sb, A, B] += ps3[d, sa] @ G @ ps3[d, sb]
    # --- voxel / surface and surface / voxel touching pairs
    for A in range(nA):
        for s in range(nS):
            if not _touch(vext[A], sext[s]):
                continue
            ax, c, lo, hi = rect_of(s)
            T.VS[A, s] = np.dot(wo, rect_potential(Po[A], ax, c, lo, hi)) / FOUR_PI
            D = P3[A][:, None, :] - S3[s][None, :, :]
            T.VS[A, s] += w3 @ kern_s(np.sqrt((D * D).sum(-1))) @ sw3
            T.SV[s, A] = np.dot(swo, box_potential(So[s], vlo[A], vhi[A])) / FOUR_PI
            D = S3[s][:, None, :] - P3[A][None, :, :]
            T.SV[s, A] += sw3 @ kern_s(np.sqrt((D * D).sum(-1))) @ w3
    # --- surface / surface touching pairs
    for s in range(nS):
        for t in range(nS):
            if not _touch(sext[s], sext[t]):
                continue
            ax, c, lo, hi = rect_of(t)
            T.SS[s, t] = np.dot(swo, rect_potential(So[s], ax, c, lo, hi)) / FOUR_PI
            D = S3[s][:, None, :] - S3[t][None, :, :]
            T.SS[s, t] += sw3 @ kern_s(np.sqrt((D * D).sum(-1))) @ sw3
    return T


# ----------------------------------------------------------------------------
# from element tables to face (basis-function) entries
# ----------------------------------------------------------------------------
def incidence(mesh):
    """Profile incidence Inc[s] (nf, nvox), volume charges Cv (nf, nvox),
    sheet charges Cs (nf, nsurf) of every rooftop of the atom."""
    nf, nv, ns = mesh.n_faces, mesh.n_vox, len(mesh.surf_face)
    inc = np.zeros((2, nf, nv))
    Cv = np.zeros((nf, nv))
    Cs = np.zeros((nf, ns))
    for f in range(nf):
        for v, prof in mesh.face_voxels(f):
            inc[0 if prof > 0 else 1, f, v] = 1.0
        vol, sur = mesh.face_charges(f)
        for v, c in vol:
            Cv[f, v] = c
        for s, c in sur:
            Cs[f, s] = c
    return inc, Cv, Cs


def mass_matrix(mesh):
    """M_ij = int w_i . w_j (closed form per voxel: 1/3 for equal profiles,
    1/6 for xi against 1 - xi, times h^3 h^-4)."""
    inc, _, _ = incidence(mesh)
    same = inc[0] @ inc[0].T + inc[1] @ inc[1].T
    diff = inc[0] @ inc[1].T + inc[1] @ inc[0].T
    sd = mesh.face_dir[:, None] == mesh.face_dir[None, :]
    return np.where(sd, (same / 3.0 + diff / 6.0) / mesh.h, 0.0)


def block_from_tables(mI, mJ, T, k):
    """-k^2 L + D for the face pairs of (test atom mI, source atom mJ)."""
    incI, CvI, CsI = incidence(mI)
    incJ, CvJ, CsJ = incidence(mJ)
    L = np.zeros((mI.n_faces, mJ.n_faces), complex)
    for d in range(3):
        rows = mI.face_dir == d
        cols = mJ.face_dir == d
        acc = np.zeros((rows.sum(), cols.sum()), complex)
        for sa in range(2):
            for sb in range(2):
                acc += incI[sa][rows] @ T.W[d, sa, sb] @ incJ[sb][cols].T
        L[np.ix_(rows, cols)] = acc / (mI.h ** 2 * mJ.h ** 2)
    D = CvI @ T.U @ CvJ.T + CvI @ T.VS @ CsJ.T + CsI @ T.SV @ CvJ.T + CsI @ T.SS @ CsJ.T
    return -k * k * L + D


def self_block(prob, t):
    """Scaled self block Zs_ii of atom type t."""
    mesh = prob.meshes[t]
    T = self_tables(mesh, prob.k)
    chi = complex(prob.eps[t]) - 1.0
    return mass_matrix(mesh) / chi + block_from_tables(mesh, mesh, T, prob.k)


def cross_block(prob, I, J):
    """Scaled interaction block Zs_IJ between two different atoms."""
    T = cross_tables(prob, I, J)
    return block_from_tables(prob.mesh(I), prob.mesh(J), T, prob.k)


def dense_matrix(prob, self_blocks=None):
    """The full scaled matrix Zs (n x n), atom-major ordering (eq. bp)."""
    n = prob.n
    Z = np.zeros((n, n), complex)
    if self_blocks is None:
        self_blocks = {t: self_block(prob, t) for t in sorted(set(prob.types.tolist()))}
    off = prob.offsets
    for I in range(prob.n_atoms):
        for J in range(prob.n_atoms):
            blk = self_blocks[prob.types[I]] if I == J else cross_block(prob, I, J)
            Z[off[I]:off[I + 1], off[J]:off[J + 1]] = blk
    return Z


# ----------------------------------------------------------------------------
# right-hand side
# ----------------------------------------------------------------------------
def plane_wave(khat, pol, k):
    """E0(r) = pol exp(-j k khat . r)  (e^{j w t} convention)."""
    khat = np.asarray(khat, float)
    pol = np.asarray(pol, complex)
    return lambda r: pol * np.exp(-1j * k * (r @ khat))[..., None]


def rhs_v0(prob, khat, pol):
    """v0_i = int w_i . E0 (eq. matrixeq), Gauss-Legendre Q_SELF per voxel."""
    E0 = plane_wave(khat, pol, prob.k)
    v0 = np.zeros(prob.n, complex)
    for I in range(prob.n_atoms):
        mesh = prob.mesh(I)
        P, w, xi = voxel_points(mesh, prob.origin(I), Q_SELF)
        E = E0(P)                                   # (nvox, q^3, 3)
        ps = _profiles(xi) * w                      # (3, 2, q^3)
        for f in range(mesh.n_faces):
            d = mesh.face_dir[f]
            acc = 0.0
            for v, prof in mesh.face_voxels(f):
                acc += np.dot(ps[d, 0 if prof > 0 else 1], E[v, :, d])
            v0[prob.offsets[I] + f] = acc / mesh.h ** 2
    return v0


def rhs(prob, khat, pol):
    """Scaled right-hand side b = j k v0."""
    return 1j * prob.k * rhs_v0(prob, khat, pol)
