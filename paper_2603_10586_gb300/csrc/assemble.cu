// Galerkin entries of the scaled VIE matrix (paper Sec. 3, eq. matrixeq):
//   Zs = M / chi - k^2 L + D,
// M_ij = int w_i.w_j, L_ij = int int w_i g w_j, D_ij = int int q_i g q_j with
// q = div w (volume charge on the voxels beside a face plus a sheet on a
// boundary face), g = exp(-j k R) / (4 pi R).
//
// Quadrature rule (the paper leaves it to its references; this is the
// library's definition):
//   * elements in different atoms: Gauss-Legendre, 2 points per axis on both;
//   * separated elements of one atom: Gauss-Legendre, 3 points per axis;
//   * touching elements of one atom: g = 1/(4 pi R) + g_s; the static part
//     integrates the source element in closed form (uniform box, linear box,
//     uniform rectangle) and the test element with 6 Gauss points per axis;
//     g_s = (exp(-j k R) - 1)/(4 pi R) (limit -j k/(4 pi)) uses 3 points.
//
// Work is organised in two kernels per atom pair: element-pair tables
// (U = int int g over voxel pairs, W[d][sa][sb] with the rooftop profiles
// xi / 1 - xi along d, and the uniform voxel/sheet combinations VS, SV, SS),
// then one thread per matrix entry gathers its (at most 2 x 2) element pairs.
#include <cmath>

#include "common.h"
#include "cplx.cuh"

namespace vie {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv4Pi = 1.0 / (4.0 * kPi);

// Gauss-Legendre on [0, 1]
__constant__ double c_gl3_x[3] = {0.11270166537925831148, 0.5, 0.88729833462074168852};
__constant__ double c_gl3_w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
__constant__ double c_gl6_x[6] = {0.03376524289842398609, 0.16939530676686774317, 0.38069040695840154568,
                                  0.61930959304159845432, 0.83060469323313225683, 0.96623475710157601391};
__constant__ double c_gl6_w[6] = {0.08566224618958517252, 0.18038078652406930378, 0.23395696728634552369,
                                  0.23395696728634552369, 0.18038078652406930378, 0.08566224618958517252};
// 2-point nodes xi = 1/2 -+ 1/(2 sqrt 3); weights 1/2
constexpr double kGl2Off = 0.28867513459481288225;  // 1/(2 sqrt 3)

// --------------------------------------------------------------------------
// closed-form inner integrals (source minus field coordinates u, v, w)
// --------------------------------------------------------------------------
__device__ double log_a_plus_R(double a, double R, double rest2) {
    if (R == 0.0) return 0.0;
    if (a >= 0.0) return log(a + R);
    if (rest2 <= 0.0) return 0.0;
    return log(rest2) - log(R - a);   // a + R = rest2 / (R - a) for a < 0
}
__device__ double atan_ratio(double num, double den) { return den != 0.0 ? atan(num / den) : 0.0; }

// d^3 F / du dv dw = 1/R
__device__ double F_box(double u, double v, double w) {
    double u2 = u * u, v2 = v * v, w2 = w * w;
    double R = sqrt(u2 + v2 + w2);
    double t = v * w * log_a_plus_R(u, R, v2 + w2) + u * w * log_a_plus_R(v, R, u2 + w2) +
               u * v * log_a_plus_R(w, R, u2 + v2);
    t -= 0.5 * u2 * atan_ratio(v * w, u * R);
    t -= 0.5 * v2 * atan_ratio(u * w, v * R);
    t -= 0.5 * w2 * atan_ratio(u * v, w * R);
    return t;
}
// d^2 G / du dv = 1/R
__device__ double G_rect(double u, double v, double w) {
    double R = sqrt(u * u + v * v + w * w);
    return u * log_a_plus_R(v, R, u * u + w * w) + v * log_a_plus_R(u, R, v * v + w * w) -
           w * atan_ratio(u * v, w * R);
}
// d^2 H / du dv = R
__device__ double H_rectR(double u, double v, double w) {
    double R = sqrt(u * u + v * v + w * w);
    return u * v * R / 3.0 + (u * u * u + 3.0 * u * w * w) / 6.0 * log_a_plus_R(v, R, u * u + w * w) +
           (v * v * v + 3.0 * v * w * w) / 6.0 * log_a_plus_R(u, R, v * v + w * w) -
           w * w * w / 3.0 * atan_ratio(u * v, w * R);
}

// int_box dV'/|r - r'|
__device__ double box_pot(const double r[3], const double lo[3], const double hi[3]) {
    double acc = 0.0;
    for (int ix = 0; ix < 2; ++ix)
        for (int iy = 0; iy < 2; ++iy)
            for (int iz = 0; iz < 2; ++iz) {
                double u = (ix ? hi[0] : lo[0]) - r[0];
                double v = (iy ? hi[1] : lo[1]) - r[1];
                double w = (iz ? hi[2] : lo[2]) - r[2];
                // sign = product over axes of (+1 for hi, -1 for lo)
                double s = (ix ? 1.0 : -1.0) * (iy ? 1.0 : -1.0) * (iz ? 1.0 : -1.0);
                acc += s * F_box(u, v, w);
            }
    return acc;
}

// rectangle {r'_axis = c, lo <= r'_other <= hi}: kernel K(u, v, w) summed over corners
template <int KIND>  // 0: 1/R, 1: R
__device__ double rect_int(const double r[3], int axis, double c, const double lo[3], const double hi[3]) {
    int a = axis == 0 ? 1 : 0;
    int b = axis == 2 ? 1 : 2;
    double w = c - r[axis];
    double acc = 0.0;
    for (int iu = 0; iu < 2; ++iu)
        for (int iv = 0; iv < 2; ++iv) {
            double u = (iu ? hi[a] : lo[a]) - r[a];
            double v = (iv ? hi[b] : lo[b]) - r[b];
            double s = (iu ? 1.0 : -1.0) * (iv ? 1.0 : -1.0);
            acc += s * (KIND == 0 ? G_rect(u, v, w) : H_rectR(u, v, w));
        }
    return acc;
}

// int_box xi_d(r') / |r - r'| dV',  xi_d = (r'_d - lo_d) / (hi_d - lo_d)
__device__ double box_lin_pot(const double r[3], const double lo[3], const double hi[3], int d, double phi) {
    double top = rect_int<1>(r, d, hi[d], lo, hi);
    double bot = rect_int<1>(r, d, lo[d], lo, hi);
    return (top - bot + (r[d] - lo[d]) * phi) / (hi[d] - lo[d]);
}

// full and smooth Green's functions (times 4 pi)
template <class T>
__device__ __forceinline__ typename C2<T>::t green4pi(T R, T two_over_lambda) {
    T s, c;
    sincospi_t(R * two_over_lambda, &s, &c);
    T inv = T(1) / R;
    return mk(c * inv, -s * inv);
}
__device__ __forceinline__ double2 green4pi_smooth(double R, double k) {
    if (R == 0.0) return make_double2(0.0, -k);
    double s = sin(0.5 * k * R);
    return make_double2(-2.0 * s * s / R, -sin(k * R) / R);
}

// --------------------------------------------------------------------------
// self tables (one atom type, float64, local coordinates)
// tables layout (test element index fastest, so that the entry kernel's
// neighbouring threads, which differ in the test face, read neighbouring
// words): plane 0 = U, planes 1 + 4 d + 2 sa + sb = W[d][sa][sb], each
// nvox x nvox at B * nvox + A; then VS at t * nvox + A, SV at B * nsurf + s,
// SS at t * nsurf + s (A, s: test voxel / sheet; B, t: source voxel / sheet).
// --------------------------------------------------------------------------
__device__ void vox_box(const DevMesh& m, int A, double h, double lo[3], double hi[3]) {
    for (int d = 0; d < 3; ++d) {
        lo[d] = h * m.vox_ijk[3 * A + d];
        hi[d] = lo[d] + h;
    }
}
// surface element: axis, plane coordinate, lo/hi (hi[axis] = lo[axis])
__device__ int surf_rect(const DevMesh& m, int s, double h, double lo[3], double hi[3], int ext[6]) {
    int f = m.surf_face[s];
    int4 fi = m.face[f];
    int d = fi.x;
    // recover (i, j, k) of face f from its position in the direction-major numbering
    int nv = m.nv;
    int per_dir = (nv + 1) * nv * nv;
    int g = f - d * per_dir;
    int ijk[3];
    if (d == 0) { ijk[0] = g / (nv * nv); ijk[1] = (g / nv) % nv; ijk[2] = g % nv; }
    else if (d == 1) { ijk[0] = g / (nv * (nv + 1)); ijk[1] = (g / nv) % (nv + 1); ijk[2] = g % nv; }
    else { ijk[0] = g / (nv * (nv + 1)); ijk[1] = (g / (nv + 1)) % nv; ijk[2] = g % (nv + 1); }
    for (int e = 0; e < 3; ++e) {
        lo[e] = h * ijk[e];
        hi[e] = (e == d) ? lo[e] : lo[e] + h;
        ext[2 * e] = ijk[e];
        ext[2 * e + 1] = (e == d) ? ijk[e] : ijk[e] + 1;
    }
    return d;
}

// The voxel/voxel integrals of one atom depend only on the relative offset of
// the two voxels (uniform voxels, local coordinates), so they are computed
// once per offset o = ijk_B - ijk_A in [-(nv-1), nv-1]^3, one warp each: the
// lanes split the outer points of both rules and all-reduce the sums; a
// second kernel copies them to every voxel pair.  Rules: 3-point Gauss per
// axis on both voxels (full g apart, smooth remainder when touching); for
// touching voxels the static part with a 6-point outer rule and the closed-form
// box potentials inside.
__device__ __forceinline__ double warp_allsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(128) self_vv_offset_kernel(int nv, double h, double k, double2* otab) {
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int w1 = 2 * nv - 1, noff = w1 * w1 * w1;
    if (warp >= noff) return;  // whole warps
    const int o[3] = {warp / (w1 * w1) - (nv - 1), (warp / w1) % w1 - (nv - 1), warp % w1 - (nv - 1)};
    double loA[3], loB[3], hiB[3];
    bool touch = true;
    for (int d = 0; d < 3; ++d) {
        const int ia = o[d] < 0 ? -o[d] : 0;
        loA[d] = h * ia;
        loB[d] = h * (ia + o[d]);
        hiB[d] = loB[d] + h;
        touch &= abs(o[d]) <= 1;
    }
    const double two_over_lambda = k / kPi;
    double2 G[3][3][3];
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[d][a][b] = make_double2(0, 0);
    if (lane < 27) {
        const int pa = lane;
        const int ax = pa / 9, ay = (pa / 3) % 3, az = pa % 3;
        const double ra[3] = {loA[0] + h * c_gl3_x[ax], loA[1] + h * c_gl3_x[ay], loA[2] + h * c_gl3_x[az]};
        const double wa = c_gl3_w[ax] * c_gl3_w[ay] * c_gl3_w[az];
        for (int pb = 0; pb < 27; ++pb) {
            const int bx = pb / 9, by = (pb / 3) % 3, bz = pb % 3;
            const double dx = ra[0] - (loB[0] + h * c_gl3_x[bx]);
            const double dy = ra[1] - (loB[1] + h * c_gl3_x[by]);
            const double dz = ra[2] - (loB[2] + h * c_gl3_x[bz]);
            const double R = sqrt(dx * dx + dy * dy + dz * dz);
            double2 g = touch ? green4pi_smooth(R, k) : green4pi<double>(R, two_over_lambda);
            g = (wa * c_gl3_w[bx] * c_gl3_w[by] * c_gl3_w[bz]) * g;
            G[0][ax][bx] += g;
            G[1][ay][by] += g;
            G[2][az][bz] += g;
        }
    }
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                G[d][a][b].x = warp_allsum(G[d][a][b].x);
                G[d][a][b].y = warp_allsum(G[d][a][b].y);
            }
    const double scale = h * h * h * h * h * h * kInv4Pi;
    double2 U = make_double2(0, 0);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) U += G[0][a][b];
    U = scale * U;
    double2 W[3][2][2];
    for (int d = 0; d < 3; ++d)
        for (int sa = 0; sa < 2; ++sa)
            for (int sb = 0; sb < 2; ++sb) {
                double2 acc = make_double2(0, 0);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        const double pa = sa ? 1.0 - c_gl3_x[a] : c_gl3_x[a];
                        const double pb = sb ? 1.0 - c_gl3_x[b] : c_gl3_x[b];
                        acc += (pa * pb) * G[d][a][b];
                    }
                W[d][sa][sb] = scale * acc;
            }
    if (touch) {
        // static part: outer 6-point rule on A split over the lanes, closed-form inner over B
        const double h3 = h * h * h;
        double us = 0.0, ws[3][2][2];
        for (int d = 0; d < 3; ++d)
            for (int sa = 0; sa < 2; ++sa)
                for (int sb = 0; sb < 2; ++sb) ws[d][sa][sb] = 0.0;
        for (int p = lane; p < 216; p += 32) {
            const int ix = p / 36, iy = (p / 6) % 6, iz = p % 6;
            const double xi[3] = {c_gl6_x[ix], c_gl6_x[iy], c_gl6_x[iz]};
            const double r[3] = {loA[0] + h * xi[0], loA[1] + h * xi[1], loA[2] + h * xi[2]};
            const double wp = h3 * c_gl6_w[ix] * c_gl6_w[iy] * c_gl6_w[iz] * kInv4Pi;
            const double phi = box_pot(r, loB, hiB);
            us += wp * phi;
            for (int d = 0; d < 3; ++d) {
                const double lin = box_lin_pot(r, loB, hiB, d, phi);
                const double inner[2] = {lin, phi - lin};
                const double prof[2] = {xi[d], 1.0 - xi[d]};
                for (int sa = 0; sa < 2; ++sa)
                    for (int sb = 0; sb < 2; ++sb) ws[d][sa][sb] += wp * prof[sa] * inner[sb];
            }
        }
        U.x += warp_allsum(us);
        for (int d = 0; d < 3; ++d)
            for (int sa = 0; sa < 2; ++sa)
                for (int sb = 0; sb < 2; ++sb) W[d][sa][sb].x += warp_allsum(ws[d][sa][sb]);
    }
    if (lane == 0) {
        otab[warp] = U;
        for (int d = 0; d < 3; ++d)
            for (int sa = 0; sa < 2; ++sa)
                for (int sb = 0; sb < 2; ++sb) otab[(size_t)(1 + 4 * d + 2 * sa + sb) * noff + warp] = W[d][sa][sb];
    }
}

__global__ void self_vv_expand_kernel(DevMesh m, const double2* __restrict__ otab, double2* __restrict__ tab) {
    const int nv2 = m.nvox * m.nvox;
    const int tt = blockIdx.x * blockDim.x + threadIdx.x;
    if (tt >= nv2) return;
    const int B = tt / m.nvox, A = tt % m.nvox;
    const int w1 = 2 * m.nv - 1, noff = w1 * w1 * w1;
    int idx = 0;
    for (int d = 0; d < 3; ++d) idx = idx * w1 + (m.vox_ijk[3 * B + d] - m.vox_ijk[3 * A + d] + m.nv - 1);
    for (int q = 0; q < 13; ++q) tab[(size_t)q * nv2 + tt] = otab[(size_t)q * noff + idx];
}

// uniform voxel/sheet combinations of one atom with itself
// mode 0: VS (voxel A, sheet s), 1: SV (sheet s, voxel B), 2: SS
__global__ void self_surf_kernel(DevMesh m, double h, double k, double2* tab) {
    int mode = blockIdx.y;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int nA = mode == 2 ? m.nsurf : (mode == 0 ? m.nvox : m.nsurf);
    int nB = mode == 2 ? m.nsurf : (mode == 0 ? m.nsurf : m.nvox);
    if (t >= nA * nB) return;
    int ia = t / nB, ib = t % nB;
    const double two_over_lambda = k / kPi;
    // element descriptions
    double loA[3], hiA[3], loB[3], hiB[3];
    int extA[6], extB[6];
    int axA = -1, axB = -1;
    if (mode == 0 || mode == 1) {
        int v = mode == 0 ? ia : ib;
        int s = mode == 0 ? ib : ia;
        double lo[3], hi[3], slo[3], shi[3];
        int vext[6], sext[6];
        vox_box(m, v, h, lo, hi);
        for (int e = 0; e < 3; ++e) { vext[2 * e] = m.vox_ijk[3 * v + e]; vext[2 * e + 1] = vext[2 * e] + 1; }
        int ax = surf_rect(m, s, h, slo, shi, sext);
        if (mode == 0) {
            for (int e = 0; e < 3; ++e) { loA[e] = lo[e]; hiA[e] = hi[e]; loB[e] = slo[e]; hiB[e] = shi[e]; }
            for (int e = 0; e < 6; ++e) { extA[e] = vext[e]; extB[e] = sext[e]; }
            axB = ax;
        } else {
            for (int e = 0; e < 3; ++e) { loA[e] = slo[e]; hiA[e] = shi[e]; loB[e] = lo[e]; hiB[e] = hi[e]; }
            for (int e = 0; e < 6; ++e) { extA[e] = sext[e]; extB[e] = vext[e]; }
            axA = ax;
        }
    } else {
        axA = surf_rect(m, ia, h, loA, hiA, extA);
        axB = surf_rect(m, ib, h, loB, hiB, extB);
    }
    bool touch = true;
    for (int e = 0; e < 3; ++e) touch &= max(extA[2 * e], extB[2 * e]) <= min(extA[2 * e + 1], extB[2 * e + 1]);

    // Gauss-Gauss part with 3 points per axis of each element
    auto npts = [](int ax) { return ax < 0 ? 27 : 9; };
    auto point = [&](int ax, const double lo[3], int p, double r[3], double& w) {
        if (ax < 0) {
            int i0 = p / 9, i1 = (p / 3) % 3, i2 = p % 3;
            r[0] = lo[0] + h * c_gl3_x[i0];
            r[1] = lo[1] + h * c_gl3_x[i1];
            r[2] = lo[2] + h * c_gl3_x[i2];
            w = h * h * h * c_gl3_w[i0] * c_gl3_w[i1] * c_gl3_w[i2];
        } else {
            int a = ax == 0 ? 1 : 0, b = ax == 2 ? 1 : 2;
            int i0 = p / 3, i1 = p % 3;
            r[ax] = lo[ax];
            r[a] = lo[a] + h * c_gl3_x[i0];
            r[b] = lo[b] + h * c_gl3_x[i1];
            w = h * h * c_gl3_w[i0] * c_gl3_w[i1];
        }
    };
    double2 acc = make_double2(0, 0);
    for (int p = 0; p < npts(axA); ++p) {
        double ra[3], wa;
        point(axA, loA, p, ra, wa);
        for (int q = 0; q < npts(axB); ++q) {
            double rb[3], wb;
            point(axB, loB, q, rb, wb);
            double dx = ra[0] - rb[0], dy = ra[1] - rb[1], dz = ra[2] - rb[2];
            double R = sqrt(dx * dx + dy * dy + dz * dz);
            double2 g = touch ? green4pi_smooth(R, k) : green4pi<double>(R, two_over_lambda);
            acc += (wa * wb) * g;
        }
    }
    acc = kInv4Pi * acc;
    if (touch) {
        // static part: outer 6-point rule on the test element, closed-form inner
        int nq = axA < 0 ? 216 : 36;
        for (int p = 0; p < nq; ++p) {
            double r[3], wp;
            if (axA < 0) {
                int i0 = p / 36, i1 = (p / 6) % 6, i2 = p % 6;
                r[0] = loA[0] + h * c_gl6_x[i0];
                r[1] = loA[1] + h * c_gl6_x[i1];
                r[2] = loA[2] + h * c_gl6_x[i2];
                wp = h * h * h * c_gl6_w[i0] * c_gl6_w[i1] * c_gl6_w[i2];
            } else {
                int a = axA == 0 ? 1 : 0, b = axA == 2 ? 1 : 2;
                int i0 = p / 6, i1 = p % 6;
                r[axA] = loA[axA];
                r[a] = loA[a] + h * c_gl6_x[i0];
                r[b] = loA[b] + h * c_gl6_x[i1];
                wp = h * h * c_gl6_w[i0] * c_gl6_w[i1];
            }
            double inner = axB < 0 ? box_pot(r, loB, hiB) : rect_int<0>(r, axB, loB[axB], loB, hiB);
            acc.x += wp * inner * kInv4Pi;
        }
    }
    size_t nv2 = (size_t)m.nvox * m.nvox;
    size_t base = 13 * nv2;
    if (mode == 0) tab[base + (size_t)ib * m.nvox + ia] = acc;
    else if (mode == 1) tab[base + (size_t)m.nvox * m.nsurf + (size_t)ib * m.nsurf + ia] = acc;
    else tab[base + 2 * (size_t)m.nvox * m.nsurf + (size_t)ib * m.nsurf + ia] = acc;
}

// --------------------------------------------------------------------------
// tables between two different atoms (2-point Gauss-Legendre everywhere)
// --------------------------------------------------------------------------
struct GeoPtrs {
    const double* centres;
    const int* types;
    const double* sides;
};

__device__ __forceinline__ void vox_centre(const DevMesh& m, const GeoPtrs& g, int atom, int v, double c[3],
                                           double& h) {
    const double side = g.sides[g.types[atom]];
    h = side / m.nv;
    const float4 l = m.vox_c[v];
    c[0] = g.centres[3 * atom] - 0.5 * side + h * l.x;
    c[1] = g.centres[3 * atom + 1] - 0.5 * side + h * l.y;
    c[2] = g.centres[3 * atom + 2] - 0.5 * side + h * l.z;
}

// centre of a boundary face (its plane coordinate along the normal axis)
__device__ __forceinline__ int surf_centre(const DevMesh& m, const GeoPtrs& g, int atom, int s, double c[3],
                                           double& h) {
    const double side = g.sides[g.types[atom]];
    h = side / m.nv;
    const float4 l = m.surf_c[s];
    c[0] = g.centres[3 * atom] - 0.5 * side + h * l.x;
    c[1] = g.centres[3 * atom + 1] - 0.5 * side + h * l.y;
    c[2] = g.centres[3 * atom + 2] - 0.5 * side + h * l.z;
    return (int)l.w;
}

template <class T>
__global__ void cross_vv_kernel(const PairJob* jobs, DevMesh m, GeoPtrs geo, T two_over_lambda,
                                typename C2<T>::t* tab, size_t job_stride) {
    using T2 = typename C2<T>::t;
    const int job = blockIdx.y;
    const int nv2 = m.nvox * m.nvox;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nv2) return;
    const int B = t / m.nvox, A = t % m.nvox;  // table index t = B * nvox + A
    const PairJob jb = jobs[job];
    double cA[3], cB[3], hA, hB;
    vox_centre(m, geo, jb.a, A, cA, hA);
    vox_centre(m, geo, jb.b, B, cB, hB);
    // displacement in float64, then the small node offsets in T
    T D[3] = {T(cA[0] - cB[0]), T(cA[1] - cB[1]), T(cA[2] - cB[2])};
    const T oA = T(hA * kGl2Off), oB = T(hB * kGl2Off);
    T dd[3][2][2];
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) dd[d][a][b] = D[d] + (a ? oA : -oA) - (b ? oB : -oB);
    T2 G[3][2][2];
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) G[d][a][b] = mk(T(0), T(0));
#pragma unroll
    for (int ax = 0; ax < 2; ++ax)
#pragma unroll
        for (int bx = 0; bx < 2; ++bx) {
            T x2 = dd[0][ax][bx] * dd[0][ax][bx];
#pragma unroll
            for (int ay = 0; ay < 2; ++ay)
#pragma unroll
                for (int by = 0; by < 2; ++by) {
                    T xy2 = x2 + dd[1][ay][by] * dd[1][ay][by];
#pragma unroll
                    for (int az = 0; az < 2; ++az)
#pragma unroll
                        for (int bz = 0; bz < 2; ++bz) {
                            T r2 = xy2 + dd[2][az][bz] * dd[2][az][bz];
                            T inv = rsqrt_t(r2);
                            T R = r2 * inv;
                            T s, c;
                            sincospi_t(R * two_over_lambda, &s, &c);
                            T2 g = mk(c * inv, -s * inv);
                            G[0][ax][bx] += g;
                            G[1][ay][by] += g;
                            G[2][az][bz] += g;
                        }
                }
        }
    const T scale = T(hA * hA * hA * hB * hB * hB / 64.0 * kInv4Pi);
    const T xn[2] = {T(0.5 - kGl2Off), T(0.5 + kGl2Off)};
    T2* out = tab + (size_t)job * job_stride;
    T2 U = G[0][0][0] + G[0][0][1] + G[0][1][0] + G[0][1][1];
    out[t] = scale * U;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int sa = 0; sa < 2; ++sa)
#pragma unroll
            for (int sb = 0; sb < 2; ++sb) {
                T2 acc = mk(T(0), T(0));
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        T pa = sa ? T(1) - xn[a] : xn[a];
                        T pb = sb ? T(1) - xn[b] : xn[b];
                        acc += (pa * pb) * G[d][a][b];
                    }
                out[(size_t)(1 + 4 * d + 2 * sa + sb) * nv2 + t] = scale * acc;
            }
}

// uniform voxel/sheet integrals between two atoms, 2 points per axis:
// mode 0: VS (test voxel, source sheet), 1: SV (test sheet, source voxel), 2: SS
template <class T, int NA, int NB>
__device__ __forceinline__ typename C2<T>::t surf_pair(const T D[3], const T (*pa)[3], const T (*pb)[3],
                                                       T two_over_lambda) {
    using T2 = typename C2<T>::t;
    T2 acc = mk(T(0), T(0));
#pragma unroll
    for (int p = 0; p < NA; ++p) {
        T ra[3] = {D[0] + pa[p][0], D[1] + pa[p][1], D[2] + pa[p][2]};
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            T dx = ra[0] - pb[q][0], dy = ra[1] - pb[q][1], dz = ra[2] - pb[q][2];
            T r2 = dx * dx + dy * dy + dz * dz;
            T inv = rsqrt_t(r2);
            T sn, cs;
            sincospi_t(r2 * inv * two_over_lambda, &sn, &cs);
            acc += mk(cs * inv, -sn * inv);
        }
    }
    return acc;
}

// node offsets of the 2-point rule on a voxel (8) or on a sheet normal to `ax` (4)
template <class T>
__device__ __forceinline__ void rule_points(int ax, T o, T (*pts)[3]) {
    if (ax < 0) {
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            pts[p][0] = (p & 4) ? o : -o;
            pts[p][1] = (p & 2) ? o : -o;
            pts[p][2] = (p & 1) ? o : -o;
        }
    } else {
        // the normal axis is a runtime value: select per (compile-time) component
        const int a = ax == 0 ? 1 : 0;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int d = 0; d < 3; ++d)
                pts[p][d] = d == ax ? T(0) : (d == a ? ((p & 2) ? o : -o) : ((p & 1) ? o : -o));
    }
}

template <class T>
__global__ void cross_surf_kernel(const PairJob* jobs, DevMesh m, GeoPtrs geo, T two_over_lambda,
                                  typename C2<T>::t* tab, size_t job_stride) {
    using T2 = typename C2<T>::t;
    const int job = blockIdx.z;
    const int mode = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nA = mode == 0 ? m.nvox : m.nsurf;  // test elements (fastest)
    const int nB = mode == 1 ? m.nvox : m.nsurf;  // source elements
    if (t >= nA * nB) return;
    const int ib = t / nA, ia = t % nA;
    const PairJob jb = jobs[job];
    double cA[3], cB[3], hA, hB;
    int axA = -1, axB = -1;
    if (mode == 0) vox_centre(m, geo, jb.a, ia, cA, hA);
    else axA = surf_centre(m, geo, jb.a, ia, cA, hA);
    if (mode == 1) vox_centre(m, geo, jb.b, ib, cB, hB);
    else axB = surf_centre(m, geo, jb.b, ib, cB, hB);
    const T D[3] = {T(cA[0] - cB[0]), T(cA[1] - cB[1]), T(cA[2] - cB[2])};
    T pa[8][3], pb[8][3];
    rule_points<T>(axA, T(hA * kGl2Off), pa);
    rule_points<T>(axB, T(hB * kGl2Off), pb);
    T2 acc;
    if (mode == 0) acc = surf_pair<T, 8, 4>(D, pa, pb, two_over_lambda);
    else if (mode == 1) acc = surf_pair<T, 4, 8>(D, pa, pb, two_over_lambda);
    else acc = surf_pair<T, 4, 4>(D, pa, pb, two_over_lambda);
    const double wA = axA < 0 ? hA * hA * hA / 8.0 : hA * hA / 4.0;
    const double wB = axB < 0 ? hB * hB * hB / 8.0 : hB * hB / 4.0;
    acc = T(wA * wB * kInv4Pi) * acc;
    const size_t nv2 = (size_t)m.nvox * m.nvox;
    T2* out = tab + (size_t)job * job_stride + 13 * nv2;
    if (mode == 0) out[(size_t)ib * m.nvox + ia] = acc;
    else if (mode == 1) out[(size_t)m.nvox * m.nsurf + (size_t)ib * m.nsurf + ia] = acc;
    else out[2 * (size_t)m.nvox * m.nsurf + (size_t)ib * m.nsurf + ia] = acc;
}

// --------------------------------------------------------------------------
// entries from tables: -k^2 L + D (+ M / chi for a self block)
// --------------------------------------------------------------------------
// One CTA: 128 test faces i (threads) x kEntCols source faces j (loop), so the
// source-face data are loaded once per column and the index arithmetic stays
// 32-bit.  Optionally accumulates the squared norm of the written entries per
// CTA (fixed reduction order) into norm_part.
constexpr int kEntRows = 128, kEntCols = 8;

template <class T, class TO, bool SELF>
__global__ void __launch_bounds__(kEntRows) entries_kernel(const PairJob* jobs, DevMesh m, GeoPtrs geo, double k2,
                                                           const typename C2<T>::t* __restrict__ tab,
                                                           size_t job_stride, TO* const* dst, const int64_t* ld,
                                                           const double2* inv_chi, double* norm_part) {
    using T2 = typename C2<T>::t;
    const int job = blockIdx.y;
    const int np = m.np, nvox = m.nvox, nsurf = m.nsurf;
    const int nv2 = nvox * nvox;
    const int i = blockIdx.x * kEntRows + threadIdx.x;
    const PairJob jb = jobs[job];
    const double hA = geo.sides[geo.types[jb.a]] / m.nv;
    const double hB = geo.sides[geo.types[jb.b]] / m.nv;
    const T2* __restrict__ tb = tab + (size_t)job * job_stride;
    const T2* __restrict__ VS = tb + 13 * (size_t)nv2;
    const T2* __restrict__ SV = VS + (size_t)nvox * nsurf;
    const T2* __restrict__ SS = SV + (size_t)nsurf * nvox;
    const T cvA = T(1.0 / (hA * hA * hA)), cvB = T(1.0 / (hB * hB * hB));
    const T lscale = T(1.0 / (hA * hA * hB * hB)), tk2 = T(k2);
    TO* out = dst[jb.dst];
    const int64_t ldo = ld[jb.dst];
    const bool active = i < np;
    int4 fi = make_int4(0, -1, -1, -1);
    T csA = T(0);
    if (active) {
        fi = m.face[i];
        if (fi.w >= 0) csA = T(m.sheet_sign[i] / (hA * hA));
    }
    const int vi0 = fi.y, vi1 = fi.z, si = fi.w;
    double nrm = 0.0;
    const int j0 = blockIdx.z * kEntCols;
    for (int jj = 0; jj < kEntCols; ++jj) {
        const int j = j0 + jj;
        if (j >= np || !active) continue;
        const int4 fj = m.face[j];
        const int vj0 = fj.y, vj1 = fj.z, sj = fj.w;
        const T csB = sj >= 0 ? T(m.sheet_sign[j] / (hB * hB)) : T(0);
        T2 L = mk(T(0), T(0)), D = mk(T(0), T(0));
        // volume charges (+h^-3 below the face, -h^-3 above) and profiles (xi, 1 - xi)
        if (fi.x == fj.x) {
            const T2* W = tb + (size_t)(1 + 4 * fi.x) * nv2;
            if (vi0 >= 0 && vj0 >= 0) L += W[0 * nv2 + vj0 * nvox + vi0];
            if (vi0 >= 0 && vj1 >= 0) L += W[1 * (size_t)nv2 + vj1 * nvox + vi0];
            if (vi1 >= 0 && vj0 >= 0) L += W[2 * (size_t)nv2 + vj0 * nvox + vi1];
            if (vi1 >= 0 && vj1 >= 0) L += W[3 * (size_t)nv2 + vj1 * nvox + vi1];
        }
        T2 Uc = mk(T(0), T(0));
        if (vi0 >= 0) {
            if (vj0 >= 0) Uc += tb[vj0 * nvox + vi0];
            if (vj1 >= 0) Uc -= tb[vj1 * nvox + vi0];
            if (sj >= 0) D += (cvA * csB) * VS[sj * nvox + vi0];
        }
        if (vi1 >= 0) {
            if (vj0 >= 0) Uc -= tb[vj0 * nvox + vi1];
            if (vj1 >= 0) Uc += tb[vj1 * nvox + vi1];
            if (sj >= 0) D -= (cvA * csB) * VS[sj * nvox + vi1];
        }
        D += (cvA * cvB) * Uc;
        if (si >= 0) {
            T2 Sv = mk(T(0), T(0));
            if (vj0 >= 0) Sv += SV[vj0 * nsurf + si];
            if (vj1 >= 0) Sv -= SV[vj1 * nsurf + si];
            D += (csA * cvB) * Sv;
            if (sj >= 0) D += (csA * csB) * SS[sj * nsurf + si];
        }
        T2 z = D - (tk2 * lscale) * L;
        if (SELF && fi.x == fj.x) {
            // M_ij = sum over shared voxels of (1/3 equal profiles, 1/6 opposite) / h
            double Mij = 0.0;
            if (vi0 >= 0 && vi0 == vj0) Mij += 1.0 / 3.0;
            if (vi0 >= 0 && vi0 == vj1) Mij += 1.0 / 6.0;
            if (vi1 >= 0 && vi1 == vj0) Mij += 1.0 / 6.0;
            if (vi1 >= 0 && vi1 == vj1) Mij += 1.0 / 3.0;
            if (Mij != 0.0) {
                Mij /= hA;
                double2 ic = inv_chi[geo.types[jb.a]];
                z += mk(T(Mij * ic.x), T(Mij * ic.y));
            }
        }
        const TO zo = cvt<TO>(z);
        out[(int64_t)jb.row_off + i + ((int64_t)jb.col_off + j) * ldo] = zo;
        nrm += (double)zo.x * zo.x + (double)zo.y * zo.y;
    }
    if (norm_part) {
        __shared__ double red[kEntRows];
        red[threadIdx.x] = nrm;
        __syncthreads();
        for (int st = kEntRows / 2; st > 0; st >>= 1) {
            if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            norm_part[((size_t)job * gridDim.z + blockIdx.z) * gridDim.x + blockIdx.x] = red[0];
    }
}

// --------------------------------------------------------------------------
// right-hand side b = j k v0, v0_i = int w_i . E0, 3-point Gauss per axis
// --------------------------------------------------------------------------
__global__ void rhs_kernel(DevMesh m, GeoPtrs geo, int N, double k, const double* khat, const double* pol,
                           int nrhs, double2* b, int64_t ld) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = (int64_t)N * m.np;
    if (t >= n * nrhs) return;
    int c = (int)(t / n);
    int64_t row = t % n;
    int atom = (int)(row / m.np), f = (int)(row % m.np);
    double side = geo.sides[geo.types[atom]];
    double h = side / m.nv;
    int4 fi = m.face[f];
    int d = fi.x;
    const double* kh = khat + 3 * c;
    double2 pd = make_double2(pol[6 * c + 2 * d], pol[6 * c + 2 * d + 1]);
    double2 acc = make_double2(0, 0);
    int vox[2] = {fi.y, fi.z};
    for (int s = 0; s < 2; ++s) {
        if (vox[s] < 0) continue;
        double lo[3];
        for (int e = 0; e < 3; ++e)
            lo[e] = geo.centres[3 * atom + e] - 0.5 * side + h * m.vox_ijk[3 * vox[s] + e];
        for (int p = 0; p < 27; ++p) {
            int ix[3] = {p / 9, (p / 3) % 3, p % 3};
            double r[3], w = h * h * h;
            for (int e = 0; e < 3; ++e) {
                r[e] = lo[e] + h * c_gl3_x[ix[e]];
                w *= c_gl3_w[ix[e]];
            }
            double xi = c_gl3_x[ix[d]];
            double prof = s ? 1.0 - xi : xi;
            double ph = k * (kh[0] * r[0] + kh[1] * r[1] + kh[2] * r[2]);
            double sn, cs;
            sincos(ph, &sn, &cs);
            acc += (w * prof) * make_double2(cs, -sn);
        }
    }
    double2 v0 = cmul(acc, pd);
    v0 = (1.0 / (h * h)) * v0;
    b[row + (int64_t)c * ld] = make_double2(-k * v0.y, k * v0.x);  // j k v0
}

// radiation vector N(rhat) = int J exp(j k rhat . r) dV, one block per (direction, rhs)
__global__ void radiation_kernel(DevMesh m, GeoPtrs geo, int N, double k, const double2* I, int nrhs,
                                 const double* dirs, int npts, double2* out) {
    int dir = blockIdx.x, c = blockIdx.y;
    const double* rh = dirs + 3 * dir;
    int64_t n = (int64_t)N * m.np;
    double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int64_t row = threadIdx.x; row < n; row += blockDim.x) {
        int atom = (int)(row / m.np), f = (int)(row % m.np);
        double side = geo.sides[geo.types[atom]];
        double h = side / m.nv;
        int4 fi = m.face[f];
        int d = fi.x;
        int vox[2] = {fi.y, fi.z};
        double2 sum = make_double2(0, 0);
        for (int s = 0; s < 2; ++s) {
            if (vox[s] < 0) continue;
            double lo[3];
            for (int e = 0; e < 3; ++e)
                lo[e] = geo.centres[3 * atom + e] - 0.5 * side + h * m.vox_ijk[3 * vox[s] + e];
            for (int p = 0; p < 27; ++p) {
                int ix[3] = {p / 9, (p / 3) % 3, p % 3};
                double r[3], w = h * h * h;
                for (int e = 0; e < 3; ++e) {
                    r[e] = lo[e] + h * c_gl3_x[ix[e]];
                    w *= c_gl3_w[ix[e]];
                }
                double xi = c_gl3_x[ix[d]];
                double prof = s ? 1.0 - xi : xi;
                double ph = k * (rh[0] * r[0] + rh[1] * r[1] + rh[2] * r[2]);
                double sn, cs;
                sincos(ph, &sn, &cs);
                sum += (w * prof) * make_double2(cs, sn);
            }
        }
        acc[d] += (1.0 / (h * h)) * cmul(I[row + (int64_t)c * n], sum);
    }
    __shared__ double2 red[3][256];
    for (int d = 0; d < 3; ++d) red[d][threadIdx.x] = acc[d];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int d = 0; d < 3; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) out[((size_t)c * npts + dir) * 3 + d] = red[d][0];
}

// rooftop face numbering of an atom (x-faces, then y, then z; each direction
// lexicographic in (i, j, k) with the normal index 0..nv)
__device__ __forceinline__ int face_index(int nv, int d, int i, int j, int k) {
    const int base = d * nv * nv * (nv + 1);
    if (d == 0) return base + (i * nv + j) * nv + k;
    if (d == 1) return base + (i * (nv + 1) + j) * nv + k;
    return base + (i * nv + j) * (nv + 1) + k;
}

// scattered near field E = -j k A + (1 / (j k)) grad Phi at points outside the
// atoms, A = int J g, Phi = int q g (q = div J with the boundary sheets), one
// block per (point, rhs): threads take (atom, voxel) pairs, form J at the
// voxel's 27 Gauss points and its volume charge from the six faces, then the
// boundary sheets (9 points each); grad_r g = -(1 + j k R) g / R^2 (r - r')
__global__ void near_field_kernel(DevMesh m, GeoPtrs geo, int N, double k, const double2* I, int nrhs,
                                  const double* pts, int npts, double2* out) {
    const int ip = blockIdx.x, c = blockIdx.y;
    const double px = pts[3 * ip], py = pts[3 * ip + 1], pz = pts[3 * ip + 2];
    const int64_t n = (int64_t)N * m.np;
    const double2* Ic = I + (int64_t)c * n;
    double2 A[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    double2 G[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    const int nv = m.nv;
    // one Gauss point: w (J (3 components) g, q grad g) added to A and G
    auto add = [&](double rx, double ry, double rz, double w, const double2* Jp, double2 q) {
        const double dx = px - rx, dy = py - ry, dz = pz - rz;
        const double R = sqrt(dx * dx + dy * dy + dz * dz);
        double sn, cs;
        sincos(k * R, &sn, &cs);
        const double2 g = (1.0 / (4.0 * M_PI * R)) * make_double2(cs, -sn);     // exp(-j k R) / (4 pi R)
        const double2 f = (-1.0 / (R * R)) * cmul(make_double2(1.0, k * R), g);  // grad g = f (r - r')
        if (Jp)
            for (int d = 0; d < 3; ++d) A[d] += w * cmul(Jp[d], g);
        const double2 qf = w * cmul(q, f);
        G[0] += dx * qf;
        G[1] += dy * qf;
        G[2] += dz * qf;
    };
    for (int64_t e = threadIdx.x; e < (int64_t)N * m.nvox; e += blockDim.x) {
        const int atom = (int)(e / m.nvox), v = (int)(e % m.nvox);
        const double side = geo.sides[geo.types[atom]], h = side / nv;
        const int vi = m.vox_ijk[3 * v], vj = m.vox_ijk[3 * v + 1], vk = m.vox_ijk[3 * v + 2];
        const double2* Ia = Ic + (int64_t)atom * m.np;
        double2 lo_f[3], up_f[3];
        for (int d = 0; d < 3; ++d) {
            int a0[3] = {vi, vj, vk};
            lo_f[d] = Ia[face_index(nv, d, a0[0], a0[1], a0[2])];
            a0[d] += 1;
            up_f[d] = Ia[face_index(nv, d, a0[0], a0[1], a0[2])];
        }
        const double2 q = (1.0 / (h * h * h)) * ((up_f[0] - lo_f[0]) + (up_f[1] - lo_f[1]) + (up_f[2] - lo_f[2]));
        const double ox = geo.centres[3 * atom] - 0.5 * side + h * vi;
        const double oy = geo.centres[3 * atom + 1] - 0.5 * side + h * vj;
        const double oz = geo.centres[3 * atom + 2] - 0.5 * side + h * vk;
        for (int p = 0; p < 27; ++p) {
            const int ix = p / 9, iy = (p / 3) % 3, iz = p % 3;
            const double xi[3] = {c_gl3_x[ix], c_gl3_x[iy], c_gl3_x[iz]};
            const double w = h * h * h * c_gl3_w[ix] * c_gl3_w[iy] * c_gl3_w[iz];
            double2 Jp[3];
            for (int d = 0; d < 3; ++d) Jp[d] = (1.0 / (h * h)) * ((1.0 - xi[d]) * lo_f[d] + xi[d] * up_f[d]);
            add(ox + h * xi[0], oy + h * xi[1], oz + h * xi[2], w, Jp, q);
        }
    }
    for (int64_t e = threadIdx.x; e < (int64_t)N * m.nsurf; e += blockDim.x) {
        const int atom = (int)(e / m.nsurf), sf = (int)(e % m.nsurf);
        const double side = geo.sides[geo.types[atom]], h = side / nv;
        const int f = m.surf_face[sf];
        const int4 fi = m.face[f];
        const int d = fi.x, v = fi.y >= 0 ? fi.y : fi.z;
        const double2 sig = (m.sheet_sign[f] / (h * h)) * Ic[(int64_t)atom * m.np + f];
        double o[3];
        for (int a = 0; a < 3; ++a) o[a] = geo.centres[3 * atom + a] - 0.5 * side + h * m.vox_ijk[3 * v + a];
        if (fi.y >= 0) o[d] += h;  // the face is the top of its lower voxel
        const int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
        for (int p = 0; p < 9; ++p) {
            const int i1 = p / 3, i2 = p % 3;
            double r[3] = {o[0], o[1], o[2]};
            r[a1] += h * c_gl3_x[i1];
            r[a2] += h * c_gl3_x[i2];
            add(r[0], r[1], r[2], h * h * c_gl3_w[i1] * c_gl3_w[i2], nullptr, sig);
        }
    }
    __shared__ double2 red[6][256];
    for (int d = 0; d < 3; ++d) {
        red[d][threadIdx.x] = A[d];
        red[3 + d][threadIdx.x] = G[d];
    }
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int d = 0; d < 6; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) {
            const double2 a = red[d][0], gr = red[3 + d][0];
            // -j k A + grad Phi / (j k) = (k A.y + gr.y / k, -k A.x - gr.x / k)
            out[((size_t)c * npts + ip) * 3 + d] = make_double2(k * a.y + gr.y / k, -k * a.x - gr.x / k);
        }
}

GeoPtrs geo_of(Op& op) {
    return GeoPtrs{op.d_centres.as<double>(), op.d_types.as<int>(), op.d_sides.as<double>()};
}

size_t table_stride(const DevMesh& m) {
    size_t nv2 = (size_t)m.nvox * m.nvox;
    return 13 * nv2 + 2 * (size_t)m.nvox * m.nsurf + (size_t)m.nsurf * m.nsurf;
}

}  // namespace

// ---------------------------------------------------------------------------
// self blocks Zs_ii in float64, one per type
// ---------------------------------------------------------------------------
void assemble_self_blocks(Op& op) {
    const DevMesh& m = op.dmesh;
    const int np = m.np;
    size_t stride = table_stride(m);
    DevBuf tab(stride * sizeof(double2));
    const int w1o = 2 * m.nv - 1;
    DevBuf otab((size_t)13 * w1o * w1o * w1o * sizeof(double2));  // voxel/voxel integrals per offset
    op.d_zself64.alloc((size_t)op.T * np * np * sizeof(double2));
    DevBuf jobs(sizeof(PairJob)), dst(sizeof(void*)), ldb(sizeof(int64_t));
    cudaStream_t s = op.ctx->stream;
    for (int t = 0; t < op.T; ++t) {
        double h = op.h[t];
        int nv2 = m.nvox * m.nvox;
        const int w1 = 2 * m.nv - 1, noff = w1 * w1 * w1;
        self_vv_offset_kernel<<<(noff * 32 + 127) / 128, 128, 0, s>>>(m.nv, h, op.k, otab.as<double2>());
        VIE_CHECK_LAUNCH();
        self_vv_expand_kernel<<<(nv2 + 255) / 256, 256, 0, s>>>(m, otab.as<double2>(), tab.as<double2>());
        VIE_CHECK_LAUNCH();
        int ns = std::max(m.nvox, m.nsurf) * m.nsurf;
        self_surf_kernel<<<dim3((ns + 63) / 64, 3), 64, 0, s>>>(m, h, op.k, tab.as<double2>());
        VIE_CHECK_LAUNCH();
        // an atom of this type (entries only need its type); a type without
        // atoms gets an identity block so that its inverse stays defined
        int atom = op.atoms_of_type[t].empty() ? -1 : op.atoms_of_type[t][0];
        if (atom < 0) {
            std::vector<double2> eye((size_t)np * np, make_double2(0, 0));
            for (int i = 0; i < np; ++i) eye[(size_t)i * np + i] = make_double2(1, 0);
            VIE_CUDA(cudaMemcpyAsync(op.d_zself64.as<double2>() + (size_t)t * np * np, eye.data(),
                                     eye.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
            VIE_CUDA(cudaStreamSynchronize(s));
            continue;
        }
        PairJob jb{atom, atom, 0, 0, 0};
        void* dptr = op.d_zself64.as<double2>() + (size_t)t * np * np;
        int64_t ldv = np;
        VIE_CUDA(cudaMemcpyAsync(jobs.p, &jb, sizeof(jb), cudaMemcpyHostToDevice, s));
        VIE_CUDA(cudaMemcpyAsync(dst.p, &dptr, sizeof(dptr), cudaMemcpyHostToDevice, s));
        VIE_CUDA(cudaMemcpyAsync(ldb.p, &ldv, sizeof(ldv), cudaMemcpyHostToDevice, s));
        entries_kernel<double, double2, true>
            <<<dim3((np + kEntRows - 1) / kEntRows, 1, (np + kEntCols - 1) / kEntCols), kEntRows, 0, s>>>(
                jobs.as<PairJob>(), m, geo_of(op), op.k * op.k, tab.as<double2>(), stride,
                dst.as<double2* const>(), ldb.as<int64_t>(), op.d_inv_chi.as<double2>(), nullptr);
        VIE_CHECK_LAUNCH();
        VIE_CUDA(cudaStreamSynchronize(s));
    }
}

// ---------------------------------------------------------------------------
// interaction blocks of atom pairs (a != b), written into destination matrices
// ---------------------------------------------------------------------------
__global__ void k_sum_rows(const double* part, int per, int nrows, double* out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    double acc = 0.0;
    for (int c = 0; c < per; ++c) acc += part[(size_t)r * per + c];
    out[r] = acc;
}

namespace {
// tables and entry sums in T, entries written as TO
template <class T, class TO>
void assemble_pairs_as(Op& op, const PairJob* d_jobs, int n_jobs, void* const* d_dst, const int64_t* d_ld,
                       cudaStream_t s, double* norm_out) {
    using T2 = typename C2<T>::t;
    const DevMesh& m = op.dmesh;
    size_t stride = table_stride(m);
    // scratch for a chunk of jobs (<= 2 GiB)
    size_t per_job = stride * sizeof(T2);
    int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_jobs, ((size_t)2 << 30) / per_job));
    chunk = std::min(chunk, 65535);  // jobs run along grid y / z
    DevBuf tab((size_t)chunk * per_job);
    const T tol = T(2.0 / op.wavelength);
    const int nv2 = m.nvox * m.nvox;
    const int ns = std::max(m.nvox, m.nsurf) * m.nsurf;
    DevBuf npart;
    if (norm_out)
        npart.alloc((size_t)chunk * ((m.np + kEntRows - 1) / kEntRows) * ((m.np + kEntCols - 1) / kEntCols) *
                    sizeof(double));
    for (int j0 = 0; j0 < n_jobs; j0 += chunk) {
        int nj = std::min(chunk, n_jobs - j0);
        cross_vv_kernel<T><<<dim3((nv2 + 127) / 128, nj), 128, 0, s>>>(d_jobs + j0, m, geo_of(op), tol,
                                                                        tab.as<T2>(), stride);
        VIE_CHECK_LAUNCH();
        cross_surf_kernel<T><<<dim3((ns + 127) / 128, 3, nj), 128, 0, s>>>(d_jobs + j0, m, geo_of(op), tol,
                                                                           tab.as<T2>(), stride);
        VIE_CHECK_LAUNCH();
        const dim3 eg((m.np + kEntRows - 1) / kEntRows, nj, (m.np + kEntCols - 1) / kEntCols);
        entries_kernel<T, TO, false><<<eg, kEntRows, 0, s>>>(
            d_jobs + j0, m, geo_of(op), op.k * op.k, tab.as<T2>(), stride, (TO* const*)d_dst, d_ld,
            op.d_inv_chi.as<double2>(), norm_out ? npart.as<double>() : nullptr);
        VIE_CHECK_LAUNCH();
        if (norm_out) {
            k_sum_rows<<<(nj + 127) / 128, 128, 0, s>>>(npart.as<double>(), (int)(eg.x * eg.z), nj, norm_out + j0);
            VIE_CHECK_LAUNCH();
        }
    }
    // keep the scratch alive until the work is done
    VIE_CUDA(cudaStreamSynchronize(s));
}
}  // namespace

template <class T>
void assemble_pairs(Op& op, const PairJob* d_jobs, int n_jobs, void* const* d_dst, const int64_t* d_ld,
                    cudaStream_t s, double* norm_out) {
    assemble_pairs_as<T, typename C2<T>::t>(op, d_jobs, n_jobs, d_dst, d_ld, s, norm_out);
}

void assemble_pairs_f32_from_f64(Op& op, const PairJob* d_jobs, int n_jobs, void* const* d_dst, const int64_t* d_ld,
                                 cudaStream_t s, double* norm_out) {
    assemble_pairs_as<double, float2>(op, d_jobs, n_jobs, d_dst, d_ld, s, norm_out);
}

template void assemble_pairs<float>(Op&, const PairJob*, int, void* const*, const int64_t*, cudaStream_t, double*);

namespace {
// y[a] = sum_b Z_ab x_b for the atoms of a chunk; blocks of atom a_local are
// stored at blk + (a_local * N + b) * np^2 (self block pointer for b == a)
template <class T2>
__global__ void dense_rows_kernel(const T2* blk, const T2* zself, const int* types, int N, int np, int a0,
                                  const T2* x, T2* y) {
    const int al = blockIdx.y;
    const int a = a0 + al;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    using R = decltype(x[0].x);
    T2 acc = mk(R(0), R(0));
    const size_t np2 = (size_t)np * np;
    for (int b = 0; b < N; ++b) {
        const T2* Zb = b == a ? zself + (size_t)types[a] * np2 : blk + ((size_t)al * N + b) * np2;
        const T2* xb = x + (size_t)b * np;
        for (int j = 0; j < np; ++j) cfma(acc, Zb[i + (size_t)j * np], xb[j]);
    }
    y[(size_t)a * np + i] = acc;
}
}  // namespace

// y = Zs x with every interaction block regenerated on the fly (never stored):
// the uncompressed operator, for accuracy checks of the compressed one and as
// the plain dense product it replaces.
template <class T>
void dense_apply(Op& op, const typename C2<T>::t* x, typename C2<T>::t* y, cudaStream_t s) {
    using T2 = typename C2<T>::t;
    const int N = op.N, np = op.np;
    const size_t np2 = (size_t)np * np;
    const T2* zself;
    DevBuf z32;
    if (sizeof(T) == 8) zself = (const T2*)op.d_zself64.p;
    else zself = (const T2*)op.d_zself32.p;
    int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)N, ((size_t)4 << 30) / (N * np2 * sizeof(T2))));
    DevBuf blk((size_t)chunk * N * np2 * sizeof(T2));
    std::vector<void*> dst{blk.p};
    std::vector<int64_t> ld{np};
    DevBuf dd, dl;
    upload(dd, dst);
    upload(dl, ld);
    for (int a0 = 0; a0 < N; a0 += chunk) {
        int na = std::min(chunk, N - a0);
        std::vector<PairJob> jobs;
        for (int al = 0; al < na; ++al)
            for (int b = 0; b < N; ++b)
                if (b != a0 + al) {
                    // block (al, b) at column offset (al * N + b) * np of an np-row matrix
                    jobs.push_back(PairJob{a0 + al, b, 0, 0, (al * N + b) * np});
                }
        DevBuf dj;
        upload(dj, jobs);
        // the blocks the compression forms (complex float32 entries from float64 tables)
        if (!jobs.empty() && sizeof(T) == 4)
            assemble_pairs_f32_from_f64(op, dj.as<PairJob>(), (int)jobs.size(), dd.as<void* const>(),
                                        dl.as<int64_t>(), s);
        else if (!jobs.empty())
            assemble_pairs<T>(op, dj.as<PairJob>(), (int)jobs.size(), dd.as<void* const>(), dl.as<int64_t>(), s);
        dense_rows_kernel<T2><<<dim3((np + 127) / 128, na), 128, 0, s>>>(blk.as<T2>(), zself, op.d_types.as<int>(),
                                                                         N, np, a0, x, y);
        VIE_CHECK_LAUNCH();
        VIE_CUDA(cudaStreamSynchronize(s));
    }
}
void dense_apply_c64(Op& op, const float2* x, float2* y, cudaStream_t s) { dense_apply<float>(op, x, y, s); }
void dense_apply_c128(Op& op, const double2* x, double2* y, cudaStream_t s) { dense_apply<double>(op, x, y, s); }
template void assemble_pairs<double>(Op&, const PairJob*, int, void* const*, const int64_t*, cudaStream_t, double*);

void rhs_kernel_launch(Op& op, const double* d_khat, const double* d_pol, int nrhs, void* b, int64_t ld,
                       cudaStream_t s) {
    int64_t total = op.n() * nrhs;
    rhs_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(op.dmesh, geo_of(op), op.N, op.k, d_khat, d_pol,
                                                                nrhs, (double2*)b, ld);
    VIE_CHECK_LAUNCH();
}

void near_field_launch(Op& op, const void* d_I, int nrhs, const double* d_pts, int npts, void* d_out, cudaStream_t s) {
    near_field_kernel<<<dim3(npts, nrhs), 256, 0, s>>>(op.dmesh, geo_of(op), op.N, op.k, (const double2*)d_I, nrhs,
                                                       d_pts, npts, (double2*)d_out);
    VIE_CHECK_LAUNCH();
}

void far_field_launch(Op& op, const void* d_I, int nrhs, const double* d_dirs, int npts, void* d_out,
                      cudaStream_t s) {
    radiation_kernel<<<dim3(npts, nrhs), 256, 0, s>>>(op.dmesh, geo_of(op), op.N, op.k, (const double2*)d_I,
                                                       nrhs, d_dirs, npts, (double2*)d_out);
    VIE_CHECK_LAUNCH();
}

}  // namespace vie
