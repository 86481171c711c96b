"""Oracle outputs: current density, far field, cross sections, dipole moment.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Units eps0 = mu0 = c = 1 (so omega = k and the wave impedance is 1), e^{j w t}.
  J(r)      = sum_f I_f w_f(r)                                  (Sec. 3, eq. eqn04)
  N(rhat)   = int J(r') exp(+j k rhat . r') dV'
  F(rhat)   = -j k / (4 pi) (N - rhat (rhat . N))   so that E_sca ~ F exp(-j k r) / r
  sigma_sca = closed-surface integral of |F|^2 over the unit sphere
  sigma_ext = Re(I^H v0) / |E0|^2     (power taken from the incident wave)
  p         = int J dV / (j w)                                  (dipole moment)
  E_sca(r)  = -j k int J g dV' + (1 / (j k)) grad int q g dV'    (scattered near field,
              r outside the atoms; q = div J with the boundary sheets: Sec. 2, eq. IntEq)
The far and near fields use Gauss-Legendre with Q_SELF points per voxel axis
(per face axis for the charge sheets).
"""
import numpy as np

from .assembly import voxel_points, surface_points, _profiles, Q_SELF, FOUR_PI


def _voxel_moments(prob, I, rhat, q=Q_SELF):
    """int_A psi_s(xi_d) exp(j k rhat . r) dV for every voxel A, profile s, axis d.

    Returns (ndir, nvox, 3, 2) complex."""
    mesh = prob.mesh(I)
    P, w, xi = voxel_points(mesh, prob.origin(I), q)
    ph = np.exp(1j * prob.k * np.einsum("vpc,tc->tvp", P, rhat))      # (ndir, nvox, q^3)
    ps = _profiles(xi) * w                                            # (3, 2, q^3)
    return np.einsum("tvp,dsp->tvds", ph, ps)


def radiation_vector(prob, I_sol, rhat):
    """N(rhat) for unit directions rhat (ndir, 3)."""
    rhat = np.atleast_2d(rhat)
    N = np.zeros((len(rhat), 3), complex)
    for a in range(prob.n_atoms):
        mesh = prob.mesh(a)
        mom = _voxel_moments(prob, a, rhat)
        coeff = I_sol[prob.offsets[a]:prob.offsets[a + 1]] / mesh.h ** 2
        for f in range(mesh.n_faces):
            d = mesh.face_dir[f]
            for v, prof in mesh.face_voxels(f):
                N[:, d] += coeff[f] * mom[:, v, d, 0 if prof > 0 else 1]
    return N


def far_field(prob, I_sol, rhat):
    rhat = np.atleast_2d(np.asarray(rhat, float))
    N = radiation_vector(prob, I_sol, rhat)
    Nt = N - rhat * np.sum(rhat * N, axis=1, keepdims=True)
    return -1j * prob.k / (4.0 * np.pi) * Nt


def sphere_rule(n_theta=24, n_phi=48):
    """Gauss-Legendre in cos(theta) times trapezoid in phi: directions and weights."""
    x, w = np.polynomial.legendre.leggauss(n_theta)
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    st = np.sqrt(1 - x * x)
    dirs = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)),
                     np.outer(x, np.ones(n_phi))], -1).reshape(-1, 3)
    wts = np.outer(w, np.full(n_phi, 2 * np.pi / n_phi)).ravel()
    return dirs, wts


def sigma_sca(prob, I_sol, n_theta=24, n_phi=48):
    dirs, wts = sphere_rule(n_theta, n_phi)
    F = far_field(prob, I_sol, dirs)
    return float(np.sum(wts * np.sum(np.abs(F) ** 2, axis=1)))


def sigma_ext(I_sol, v0, e0_norm=1.0):
    return float(np.real(np.vdot(I_sol, v0))) / e0_norm ** 2


def dipole_moment(prob, I_sol):
    """p = int J dV / (j k); int w_f dV = (h / 2) (number of voxels beside f) e_d."""
    p = np.zeros(3, complex)
    for a in range(prob.n_atoms):
        mesh = prob.mesh(a)
        Ia = I_sol[prob.offsets[a]:prob.offsets[a + 1]]
        nvox = (mesh.face_lo_vox >= 0).astype(float) + (mesh.face_hi_vox >= 0)
        for d in range(3):
            sel = mesh.face_dir == d
            p[d] += np.sum(Ia[sel] * nvox[sel]) * mesh.h / 2.0
    return p / (1j * prob.k)


def current_at_voxel_centres(prob, I_sol):
    """J at every voxel centre (atom-major, voxel order of the mesh): (nvox_total, 3)."""
    out = []
    for a in range(prob.n_atoms):
        mesh = prob.mesh(a)
        Ia = I_sol[prob.offsets[a]:prob.offsets[a + 1]]
        J = np.zeros((mesh.n_vox, 3), complex)
        for f in range(mesh.n_faces):
            for v, prof in mesh.face_voxels(f):
                J[v, mesh.face_dir[f]] += Ia[f] * 0.5 / mesh.h ** 2
        out.append(J)
    return np.concatenate(out)


def near_field(prob, I_sol, points, q=Q_SELF):
    """Scattered field E_sca at points outside the atoms (npts, 3) -> (npts, 3).

    From the potentials of the current and its charge (units eps0 = mu0 = 1,
    w = k): E = -j k A + (1 / (j k)) grad Phi, A = int J g, Phi = int q g, with
    q the distributional divergence of J (volume density per voxel plus the
    boundary sheets), so that -E_sca tested with w_i gives the (j k L + D /
    (j k)) rows of the Galerkin system (Sec. 3).  grad_r g(r - r') =
    -(1 + j k R) exp(-j k R) / (4 pi R^2) Rhat."""
    pts = np.atleast_2d(np.asarray(points, float))
    k = prob.k
    E = np.zeros((len(pts), 3), complex)
    for a in range(prob.n_atoms):
        mesh = prob.mesh(a)
        org = prob.origin(a)
        Ia = I_sol[prob.offsets[a]:prob.offsets[a + 1]]
        P, w, xi = voxel_points(mesh, org, q)                      # (nvox, q^3, 3)
        ps = _profiles(xi)                                         # (3, 2, q^3)
        J = np.zeros((mesh.n_vox, len(w), 3), complex)
        qv = np.zeros(mesh.n_vox, complex)
        qs = np.zeros(len(mesh.surf_face), complex)
        for f in range(mesh.n_faces):
            d = mesh.face_dir[f]
            for v, prof in mesh.face_voxels(f):
                J[v, :, d] += Ia[f] * ps[d, 0 if prof > 0 else 1] / mesh.h ** 2
            vol, sur = mesh.face_charges(f)
            for v, c in vol:
                qv[v] += Ia[f] * c
            for s_, c in sur:
                qs[s_] += Ia[f] * c
        S, sw = surface_points(mesh, org, q)                       # (nsurf, q^2, 3)
        src_v = P.reshape(-1, 3)
        for i, r in enumerate(pts):
            D = r[None, :] - src_v
            R = np.sqrt((D * D).sum(1))
            g = np.exp(-1j * k * R) / (FOUR_PI * R)
            dg = (-(1 + 1j * k * R) * g / R ** 2)[:, None] * D     # grad_r g
            wv = np.tile(w, mesh.n_vox)
            E[i] += -1j * k * (wv[:, None] * g[:, None] * J.reshape(-1, 3)).sum(0)
            E[i] += (1.0 / (1j * k)) * ((wv * np.repeat(qv, len(w)))[:, None] * dg).sum(0)
            if len(qs):
                Ds = r[None, :] - S.reshape(-1, 3)
                Rs = np.sqrt((Ds * Ds).sum(1))
                gs = np.exp(-1j * k * Rs) / (FOUR_PI * Rs)
                dgs = (-(1 + 1j * k * Rs) * gs / Rs ** 2)[:, None] * Ds
                ws = np.tile(sw, len(qs)) * np.repeat(qs, len(sw))
                E[i] += (1.0 / (1j * k)) * (ws[:, None] * dgs).sum(0)
    return E
