// Host-side tables: Legendre polynomials, reduced associated Legendre kernels,
// harmonic-projection quadratures, and the E/B recombination of native moments.
#include <math.h>

#include "lpp_internal.h"

namespace lpp {

static const double kPi = 3.14159265358979323846;

// Power-series coefficients of the Legendre polynomial L_l from the three-term
// recurrence (k+1) L_{k+1} = (2k+1) mu L_k - k L_{k-1}.
void legendre_poly(int l, double* c) {
    double p0[16] = {0}, p1[16] = {0}, p2[16] = {0};
    p0[0] = 1.0;
    if (l == 0) { for (int i = 0; i <= l; ++i) c[i] = p0[i]; return; }
    p1[1] = 1.0;
    for (int k = 1; k < l; ++k) {
        for (int i = 0; i <= k + 1; ++i) {
            const double shifted = i > 0 ? p1[i - 1] : 0.0;
            p2[i] = ((2.0 * k + 1.0) * shifted - k * p0[i]) / (k + 1.0);
        }
        for (int i = 0; i < 16; ++i) { p0[i] = p1[i]; p1[i] = p2[i]; }
    }
    for (int i = 0; i <= l; ++i) c[i] = p1[i];
}

// m-th derivative of a power series of degree deg (in place), returning the new degree.
static int derive(double* c, int deg, int m) {
    for (int t = 0; t < m; ++t) {
        for (int i = 0; i < deg; ++i) c[i] = (i + 1) * c[i + 1];
        c[deg] = 0.0;
        --deg;
    }
    return deg;
}

void build_kernel_polys(KernelPolys& kp) {
    for (int i = 0; i < 4; ++i) for (int j = 0; j < 8; ++j) kp.cross[i][j] = 0.0;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 8; ++j) kp.plus[i][j] = 0.0;
    for (int i = 0; i < 5; ++i) for (int j = 0; j < 9; ++j) kp.minus[i][j] = 0.0;
    double c[16];
    // Lm_L(mu)/(1-mu^2)^(m/2) = (-1)^m d^m L_L / dmu^m (m even: sign +1)
    for (int L = 2; L <= 6; L += 2) {
        for (int i = 0; i < 16; ++i) c[i] = 0.0;
        legendre_poly(L, c);
        const int d = derive(c, L, 2);
        for (int i = 0; i <= d; ++i) kp.cross[L / 2 - 1][i] = c[i];
    }
    for (int l = 0; l <= 4; l += 2) {
        for (int i = 0; i < 16; ++i) c[i] = 0.0;
        legendre_poly(l, c);
        for (int i = 0; i <= l; ++i) kp.plus[l / 2][i] = c[i];
    }
    for (int L = 4; L <= 12; L += 2) {
        for (int i = 0; i < 16; ++i) c[i] = 0.0;
        legendre_poly(L, c);
        const int d = derive(c, L, 4);
        for (int i = 0; i <= d; ++i) kp.minus[L / 2 - 2][i] = c[i];
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on L_n.
void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = n == 1 ? z : p1;
            const double pm = n == 1 ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Exact projection onto the 2L+1 real harmonics of degree L: integrands of degree
// 2L are integrated exactly by L+1 Gauss-Legendre nodes in cos(theta) times 2L+1
// equally spaced azimuths.
void build_quadrature(int L, Quadrature& q) {
    q.L = L;
    const int nmu = L + 1, nphi = 2 * L + 1;
    q.S = nmu * nphi;
    q.dirs.assign(3 * q.S, 0.0);
    q.table.assign((size_t)(2 * L + 1) * q.S, 0.0);
    double x[16], w[16];
    gauss_legendre(nmu, x, w);
    int s = 0;
    for (int i = 0; i < nmu; ++i) {
        const double st = sqrt(1.0 - x[i] * x[i]);
        for (int j = 0; j < nphi; ++j, ++s) {
            const double ph = 2.0 * kPi * j / nphi;
            const double kx = st * cos(ph), ky = st * sin(ph), kz = x[i];
            q.dirs[3 * s] = kx;
            q.dirs[3 * s + 1] = ky;
            q.dirs[3 * s + 2] = kz;
            const double wt = w[i] * 2.0 * kPi / nphi;
            for (int n = -L; n <= L; ++n)
                q.table[(size_t)(n + L) * q.S + s] = wt * ylm_norm(L, n) * ylm_poly<double>(L, n, kx, ky, kz);
        }
    }
}

}  // namespace lpp

// (2l+1)/2 int_{-1}^{1} Lm_L(mu) L_l(mu) dmu by 24-node Gauss-Legendre (exact to rounding:
// the integrands are polynomials of degree <= 12).
static double legendre_overlap(int m, int L, int l) {
    double x[24], w[24];
    lpp::gauss_legendre(24, x, w);
    double cl[16] = {0}, cL[16] = {0};
    lpp::legendre_poly(l, cl);
    lpp::legendre_poly(L, cL);
    // m-th derivative of L_L times (1 - mu^2)^(m/2)
    int deg = L;
    for (int t = 0; t < m; ++t) {
        for (int i = 0; i < deg; ++i) cL[i] = (i + 1) * cL[i + 1];
        cL[deg] = 0.0;
        --deg;
    }
    double s = 0.0;
    for (int i = 0; i < 24; ++i) {
        double a = 0.0, b = 0.0;
        for (int k = deg; k >= 0; --k) a = a * x[i] + cL[k];
        for (int k = l; k >= 0; --k) b = b * x[i] + cl[k];
        double f = 1.0;
        for (int t = 0; t < m / 2; ++t) f *= (1.0 - x[i] * x[i]);
        s += w[i] * a * f * b;
    }
    return 0.5 * (2 * l + 1) * s;
}

namespace lpp {
// N[l][L] = (2l+1)/2 int Lm2_L L_l (l = 0, 2; L = 2, 4, 6), M[l][L] = (2l+1)/2 int Lm4_L L_l
// (l = 0, 2, 4; L = 4, 6, 8): native associated-Legendre moments -> Legendre multipoles.
void eb_matrices(double N[2][3], double M[3][3]) {
    for (int li = 0; li < 2; ++li)
        for (int j = 0; j < 3; ++j) N[li][j] = legendre_overlap(2, 2 + 2 * j, 2 * li);
    for (int li = 0; li < 3; ++li)
        for (int j = 0; j < 3; ++j) M[li][j] = legendre_overlap(4, 4 + 2 * j, 2 * li);
}
}  // namespace lpp

extern "C" lpp_status lpp_derive_eb(const double* p, int n_bins, double* ge, double* ee, double* bb) {
    if (!p || n_bins <= 0 || !ge || !ee || !bb) return LPP_ERR_INVALID_ARG;
    const int crossL[3] = {2, 4, 6}, minusL[3] = {4, 6, 8};
    const int crossSlot[3] = {LPP_MOM_CROSS2, LPP_MOM_CROSS4, LPP_MOM_CROSS6};
    const int minusSlot[3] = {LPP_MOM_MINUS4, LPP_MOM_MINUS6, LPP_MOM_MINUS8};
    const int plusSlot[3] = {LPP_MOM_PLUS0, LPP_MOM_PLUS2, LPP_MOM_PLUS4};
    for (int b = 0; b < n_bins; ++b) {
        for (int li = 0; li < 2; ++li) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += legendre_overlap(2, crossL[j], 2 * li) * p[(crossSlot[j] * n_bins + b) * 2];
            ge[li * n_bins + b] = s;
        }
        for (int li = 0; li < 3; ++li) {
            double mm = 0.0;
            for (int j = 0; j < 3; ++j) mm += legendre_overlap(4, minusL[j], 2 * li) * p[(minusSlot[j] * n_bins + b) * 2];
            const double pl = p[(plusSlot[li] * n_bins + b) * 2];
            ee[li * n_bins + b] = 0.5 * (pl + mm);
            bb[li * n_bins + b] = 0.5 * (pl - mm);
        }
    }
    return LPP_OK;
}

extern "C" lpp_status lpp_gaussian_sigma(const double* p0, const double* k_edges, int n_bins, double volume,
                                         double noise_g, double noise_e, double* sigma) {
    if (!p0 || !k_edges || !sigma || n_bins < 1 || !(volume > 0.0) || noise_g < 0.0 || noise_e < 0.0)
        return LPP_ERR_INVALID_ARG;
    const double pi = 3.14159265358979323846;
    const int ell[8] = {0, 2, 0, 2, 4, 0, 2, 4};
    for (int b = 0; b < n_bins; ++b) {
        const double k0 = k_edges[b], k1 = k_edges[b + 1];
        if (!(k1 > k0) || k0 < 0.0) return LPP_ERR_INVALID_ARG;
        const double nk = volume * (k1 * k1 * k1 - k0 * k0 * k0) / (6.0 * pi * pi);
        const double gg = p0[b] + noise_g, ge = p0[n_bins + b];
        const double ee = p0[2 * n_bins + b] + noise_e, bb = p0[3 * n_bins + b] + noise_e;
        for (int c = 0; c < 8; ++c) {
            const double f = 2 * ell[c] + 1;
            double v;
            if (c < 2) v = f * (gg * ee + ge * ge) / nk;
            else if (c < 5) v = 2.0 * f * ee * ee / nk;
            else v = 2.0 * f * bb * bb / nk;
            sigma[c * n_bins + b] = sqrt(v);
        }
    }
    return LPP_OK;
}
