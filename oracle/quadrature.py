"""Oracle quadrature primitives (CPU, float64). TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package; the product path never does.

The paper assembles the Galerkin entries of Sec. 3 (R, L, D and v0 below
eq. matrixeq) but does not say how the singular integrals are evaluated (it
defers to its references).  The rule used here is the reading stated in the
package header (``oracle/__init__.py``): tensor Gauss-Legendre for separated
element pairs, and for touching pairs a split of the Green's function into
its static part 1/(4 pi R), integrated with an analytic inner integral, plus a
smooth remainder integrated with Gauss-Legendre.

Closed forms used for the analytic inner integrals (u, v, w are source minus
field coordinates, R = sqrt(u^2+v^2+w^2)):

  box    : d^3 F / du dv dw = 1/R,
           F = vw ln(u+R) + uw ln(v+R) + uv ln(w+R)
               - u^2/2 atan(vw/(uR)) - v^2/2 atan(uw/(vR)) - w^2/2 atan(uv/(wR))
  rect   : d^2 G / du dv = 1/R,   G = u ln(v+R) + v ln(u+R) - w atan(uv/(wR))
  rect R : d^2 H / du dv = R,
           H = uvR/3 + (u^3+3uw^2)/6 ln(v+R) + (v^3+3vw^2)/6 ln(u+R)
               - w^3/3 atan(uv/(wR))

(each verified by differentiation; the tests pin them against brute force and
against textbook values).
"""
import numpy as np


def gauss_legendre_01(q):
    """Gauss-Legendre nodes and weights on [0, 1] (q points)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def _log_a_plus_R(a, R, rest2):
    """ln(a + R) with R = sqrt(a^2 + rest2); stable for a < 0.

    For a < 0, a + R = rest2 / (R - a).  Where rest2 == 0 and a < 0 the value
    is -inf (likewise at R == 0); every caller multiplies it by a coefficient
    that vanishes there, so 0 is returned in those cases.
    """
    with np.errstate(divide="ignore", invalid="ignore"):
        pos = np.log(np.where((a >= 0) & (R > 0), a + R, 1.0))
        neg = np.log(np.where(rest2 > 0, rest2, 1.0)) - np.log(np.where(a < 0, R - a, 1.0))
    out = np.where(a >= 0, pos, neg)
    return np.where(((a < 0) & (rest2 <= 0)) | (R == 0), 0.0, out)


def _atan_term(num, den):
    """atan(num/den), returning 0 where den == 0 (its coefficient vanishes there)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(den != 0, np.arctan(num / np.where(den != 0, den, 1.0)), 0.0)


def _F_box(u, v, w):
    R = np.sqrt(u * u + v * v + w * w)
    t = (v * w * _log_a_plus_R(u, R, v * v + w * w)
         + u * w * _log_a_plus_R(v, R, u * u + w * w)
         + u * v * _log_a_plus_R(w, R, u * u + v * v))
    t -= 0.5 * u * u * _atan_term(v * w, u * R)
    t -= 0.5 * v * v * _atan_term(u * w, v * R)
    t -= 0.5 * w * w * _atan_term(u * v, w * R)
    return t


def _G_rect(u, v, w):
    R = np.sqrt(u * u + v * v + w * w)
    return (u * _log_a_plus_R(v, R, u * u + w * w)
            + v * _log_a_plus_R(u, R, v * v + w * w)
            - w * _atan_term(u * v, w * R))


def _H_rectR(u, v, w):
    R = np.sqrt(u * u + v * v + w * w)
    return (u * v * R / 3.0
            + (u ** 3 + 3.0 * u * w * w) / 6.0 * _log_a_plus_R(v, R, u * u + w * w)
            + (v ** 3 + 3.0 * v * w * w) / 6.0 * _log_a_plus_R(u, R, v * v + w * w)
            - w ** 3 / 3.0 * _atan_term(u * v, w * R))


def box_potential(pts, lo, hi):
    """int_box dV' / |r - r'| at points ``pts`` (..., 3); box = [lo, hi].

    lo/hi are (..., 3) arrays broadcasting against ``pts[..., 0]``."""
    pts = np.asarray(pts, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    out = 0.0
    for sx, ex in ((-1.0, lo[..., 0]), (1.0, hi[..., 0])):
        u = ex - pts[..., 0]
        for sy, ey in ((-1.0, lo[..., 1]), (1.0, hi[..., 1])):
            v = ey - pts[..., 1]
            for sz, ez in ((-1.0, lo[..., 2]), (1.0, hi[..., 2])):
                w = ez - pts[..., 2]
                out += sx * sy * sz * _F_box(u, v, w)
    return out


def _rect_generic(kernel, pts, axis, coord, lo, hi):
    pts = np.asarray(pts, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    a, b = [d for d in range(3) if d != axis]
    w = coord - pts[..., axis]
    out = 0.0
    for su, eu in ((-1.0, lo[..., a]), (1.0, hi[..., a])):
        u = eu - pts[..., a]
        for sv, ev in ((-1.0, lo[..., b]), (1.0, hi[..., b])):
            v = ev - pts[..., b]
            out += su * sv * kernel(u, v, w)
    return out


def rect_potential(pts, axis, coord, lo, hi):
    """int_rect dA' / |r - r'| for the axis-aligned rectangle {r'_axis = coord,
    lo <= r'_other <= hi}; lo/hi are (..., 3) arrays whose ``axis`` entry is
    ignored, ``coord`` broadcasts like ``pts[..., 0]``."""
    return _rect_generic(_G_rect, pts, axis, coord, lo, hi)


def rect_R_integral(pts, axis, coord, lo, hi):
    """int_rect |r - r'| dA' over the same rectangle as :func:`rect_potential`."""
    return _rect_generic(_H_rectR, pts, axis, coord, lo, hi)


def box_linear_potential(pts, lo, hi, d):
    """int_box xi_d(r') / |r - r'| dV' with xi_d = (r'_d - lo_d)/(hi_d - lo_d).

    Uses (r'_d - lo_d) = (r'_d - r_d) + (r_d - lo_d) and
    (r'_d - r_d)/R = dR/dr'_d, so the first part is a difference of two
    rectangle integrals of R over the faces r'_d = hi_d and r'_d = lo_d.
    """
    pts = np.asarray(pts, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    hd = hi[..., d] - lo[..., d]
    top = rect_R_integral(pts, d, hi[..., d], lo, hi)
    bot = rect_R_integral(pts, d, lo[..., d], lo, hi)
    return (top - bot + (pts[..., d] - lo[..., d]) * box_potential(pts, lo, hi)) / hd


def box_gauss_points(lo, hi, q):
    """Tensor Gauss-Legendre points (q^3, 3) and weights (q^3,) on a box."""
    x, w = gauss_legendre_01(q)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ext = hi - lo
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    pts = lo + np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=-1) * ext
    return pts, W * np.prod(ext)


def rect_gauss_points(axis, coord, lo, hi, q):
    """Tensor Gauss-Legendre points (q^2, 3) and weights on an axis-aligned rectangle."""
    x, w = gauss_legendre_01(q)
    a, b = [d for d in range(3) if d != axis]
    A, B = np.meshgrid(x, x, indexing="ij")
    pts = np.zeros((q * q, 3))
    pts[:, axis] = coord
    pts[:, a] = lo[a] + A.ravel() * (hi[a] - lo[a])
    pts[:, b] = lo[b] + B.ravel() * (hi[b] - lo[b])
    W = (w[:, None] * w[None, :]).ravel() * (hi[a] - lo[a]) * (hi[b] - lo[b])
    return pts, W
