"""Oracle preconditioner and GMRES (float64 complex).
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 4, eq. diagprecond: left preconditioner P = Z_D = diag(Z_11, ..., Z_NN),
factored once per distinct atom type (O(N_p^3)) and applied per atom (O(N_p^2)).
Sec. 6: GMRES (Saad-Schultz) with the Arnoldi process.  Readings: x0 = 0;
modified Gram-Schmidt; Givens rotations; restart length m (None = no
restart); stop when the preconditioned relative residual
||P^-1 (b - Z x)|| / ||P^-1 b|| <= tol.
"""
import numpy as np

from .direct import lu_factor, lu_solve


class BlockJacobi:
    def __init__(self, prob, self_blocks):
        self.prob = prob
        self.fact = {t: lu_factor(B) for t, B in self_blocks.items()}

    def apply(self, y):
        p = self.prob
        z = np.zeros_like(np.asarray(y, complex))
        for a in range(p.n_atoms):
            s = slice(p.offsets[a], p.offsets[a + 1])
            LU, piv = self.fact[p.types[a]]
            z[s] = lu_solve(LU, piv, y[s])
        return z


def gmres(apply_A, b, precond=None, tol=1e-6, restart=None, maxiter=5000):
    """Left-preconditioned GMRES(m).  Returns (x, info) with info = dict(iterations,
    history (preconditioned relative residual after each iteration), converged)."""
    M = precond if precond is not None else (lambda v: v)
    b = np.asarray(b, complex)
    n = b.shape[0]
    x = np.zeros(n, complex)
    r = M(b)
    beta0 = np.linalg.norm(r)
    hist = []
    it = 0
    if beta0 == 0:
        return x, dict(iterations=0, history=hist, converged=True)
    m = restart if restart is not None else maxiter
    while True:
        beta = np.linalg.norm(r)
        V = np.zeros((n, m + 1), complex)
        H = np.zeros((m + 1, m), complex)
        cs = np.zeros(m, complex)
        sn = np.zeros(m, complex)
        g = np.zeros(m + 1, complex)
        g[0] = beta
        V[:, 0] = r / beta
        j_done = 0
        conv = False
        for j in range(m):
            w = M(apply_A(V[:, j]))
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[:, j + 1] = w / H[j + 1, j]
            # Givens rotation G = [[conj(c), conj(s)], [-s, c]], c = a/rho, s = b/rho,
            # maps [a; b] to [rho; 0]; apply the previous ones, then the new one
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = a / den if den != 0 else 1.0
            sn[j] = c / den if den != 0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_done = j + 1
            res = abs(g[j + 1]) / beta0
            hist.append(res)
            if res <= tol or it >= maxiter:
                conv = res <= tol
                break
        y = np.zeros(j_done, complex)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + V[:, :j_done] @ y
        if conv or it >= maxiter:
            return x, dict(iterations=it, history=hist, converged=conv)
        r = M(b - apply_A(x))
        if np.linalg.norm(r) / beta0 <= tol:
            return x, dict(iterations=it, history=hist, converged=True)


def bicgstab(apply_A, b, precond=None, tol=1e-6, maxiter=5000):
    """Left-preconditioned BiCGStab (van der Vorst, 1992), the Krylov method the
    paper weighs against GMRES in Sec. 6, on M^-1 A x = M^-1 b with x0 = 0.
    Complex inner products <u, v> = sum conj(u) v; the shadow residual is the
    initial residual.  Stops when the (recursively updated) preconditioned
    residual satisfies ||r|| / ||M^-1 b|| <= tol.  Returns (x, info) with info =
    dict(iterations, history, converged)."""
    M = precond if precond is not None else (lambda v: v)
    op = lambda v: M(apply_A(v))  # noqa: E731
    b = np.asarray(b, complex)
    x = np.zeros_like(b)
    r = M(b)
    beta0 = np.linalg.norm(r)
    hist = []
    if beta0 == 0:
        return x, dict(iterations=0, history=hist, converged=True)
    rhat = r.copy()
    rho = alpha = omega = 1.0 + 0.0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxiter + 1):
        rho_new = np.vdot(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = op(p)
        alpha = rho_new / np.vdot(rhat, v)
        s = r - alpha * v
        t = op(s)
        tt = np.vdot(t, t)
        omega = np.vdot(t, s) / tt if tt != 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        res = np.linalg.norm(r) / beta0
        hist.append(res)
        if res <= tol:
            return x, dict(iterations=it, history=hist, converged=True)
        if omega == 0:
            break
    return x, dict(iterations=len(hist), history=hist, converged=False)
