// Internal declarations shared by the liblpp translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lpp.h"

namespace lpp {

// ------------------------------------------------------------------ complex helpers
template <typename T> struct cplx;
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<double> { using t = double2; };
template <typename T> using c2 = typename cplx<T>::t;

template <typename T> __host__ __device__ __forceinline__ c2<T> mk(T re, T im) { c2<T> r; r.x = re; r.y = im; return r; }
template <typename T> __host__ __device__ __forceinline__ c2<T> cadd(c2<T> a, c2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ c2<T> csub(c2<T> a, c2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ c2<T> cmul(c2<T> a, c2<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ c2<T> cconj(c2<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __host__ __device__ __forceinline__ c2<T> cscale(c2<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by -i
template <typename T> __host__ __device__ __forceinline__ c2<T> cmul_mi(c2<T> a) { return mk<T>(a.y, -a.x); }

// ------------------------------------------------ real spherical harmonics, degree <= 12
// Real orthonormal harmonics on the unit sphere:
//   Y_{L,0}  = N_L0 Q_L^0(z)
//   Y_{L,+m} = sqrt(2) N_Lm Q_L^m(z) Re[(x + i y)^m]
//   Y_{L,-m} = sqrt(2) N_Lm Q_L^m(z) Im[(x + i y)^m]
// with P_L^m(z) = (1 - z^2)^{m/2} Q_L^m(z) (no Condon-Shortley sign), Q_m^m = (2m-1)!!,
// Q_{m+1}^m = (2m+1) z Q_m^m and (L-m) Q_L^m = (2L-1) z Q_{L-1}^m - (L+m-1) Q_{L-2}^m,
// N_Lm = sqrt((2L+1)/(4 pi) (L-m)!/(L+m)!).  (x + i y)^m carries the sin^m(theta) factor,
// so every Y is a polynomial in the components of the unit vector.
__host__ __device__ inline double ylm_norm(int L, int n) {
    int m = n < 0 ? -n : n;
    double r = 1.0;
    for (int j = L - m + 1; j <= L + m; ++j) r *= (double)j;
    double v = sqrt((2.0 * L + 1.0) / (4.0 * 3.14159265358979323846) / r);
    return m == 0 ? v : v * 1.41421356237309504880;
}

// Q_L^m(z) * {1, Re, Im}[(x+iy)^m]: the harmonic without its normalisation constant.
template <typename T>
__host__ __device__ __forceinline__ T ylm_poly(int L, int n, T x, T y, T z) {
    int m = n < 0 ? -n : n;
    T qmm = (T)1;
    for (int i = 1; i <= m; ++i) qmm *= (T)(2 * i - 1);
    T q = qmm;
    if (L > m) {
        T q0 = qmm, q1 = (T)(2 * m + 1) * z * qmm;
        for (int l = m + 2; l <= L; ++l) {
            T q2 = ((T)(2 * l - 1) * z * q1 - (T)(l + m - 1) * q0) / (T)(l - m);
            q0 = q1;
            q1 = q2;
        }
        q = q1;
    }
    if (m == 0) return q;
    T re = (T)1, im = (T)0;
    for (int i = 0; i < m; ++i) {
        T t = re * x - im * y;
        im = re * y + im * x;
        re = t;
    }
    return q * (n > 0 ? re : im);
}

// (L - |n|)! * ylm_poly(L, n, x, y, z) without divisions: with q~_l = (l - m)! Q_l^m the
// recurrence (l - m) Q_l = (2l - 1) z Q_{l-1} - (l + m - 1) Q_{l-2} becomes
// q~_l = (2l - 1) z q~_{l-1} - (l + m - 1)(l - m - 1) q~_{l-2}, integer coefficients only.
template <typename T>
__host__ __device__ __forceinline__ T ylm_poly_scaled(int L, int n, T x, T y, T z) {
    int m = n < 0 ? -n : n;
    T qmm = (T)1;
    for (int i = 1; i <= m; ++i) qmm *= (T)(2 * i - 1);
    T q = qmm;
    if (L > m) {
        T q0 = qmm, q1 = (T)(2 * m + 1) * z * qmm;
        for (int l = m + 2; l <= L; ++l) {
            T q2 = (T)(2 * l - 1) * z * q1 - (T)((l + m - 1) * (l - m - 1)) * q0;
            q0 = q1;
            q1 = q2;
        }
        q = q1;
    }
    if (m == 0) return q;
    T re = (T)1, im = (T)0;
    for (int i = 0; i < m; ++i) {
        T t = re * x - im * y;
        im = re * y + im * x;
        re = t;
    }
    return q * (n > 0 ? re : im);
}

// ylm_norm(L, n) / (L - |n|)!: the constant that goes with ylm_poly_scaled.
__host__ __device__ inline double ylm_norm_scaled(int L, int n) {
    int m = n < 0 ? -n : n;
    double f = 1.0;
    for (int j = 2; j <= L - m; ++j) f *= (double)j;
    return ylm_norm(L, n) / f;
}

// ------------------------------------------------------------------ channel tables
enum Kind { KIND_CROSS = 0, KIND_PLUS = 1, KIND_MINUS = 2, KIND_DENS = 3 };
enum Part { PART_RE = 0, PART_IM = 1 };

// One real k-space field of the estimate: the projection of the real or imaginary
// part of a moment kernel onto the real harmonic Y_{L,n}.
struct Channel {
    int kind;     // Kind
    int L;        // degree
    int n;        // harmonic index -L..L
    int part;     // Part
    int moment;   // output slot LPP_MOM_*
    int coeff;    // row of the per-particle coefficient array
};

// Per-degree quadrature: samples khat_s (x,y,z) and table[n + L][s] = w_s Y_{L,n}(khat_s).
struct Quadrature {
    int L;
    int S;
    std::vector<double> dirs;   // [S][3]
    std::vector<double> table;  // [2L+1][S]
};

// Polynomial coefficients (power series in mu) of the reduced kernels.
struct KernelPolys {
    // cross: Lm2_L / (1 - mu^2);  minus: Lm4_L / (1 - mu^2)^2;  plus: L_l
    double cross[4][8];   // L = 2,4,6 (index L/2 - 1); up to mu^6
    double plus[3][8];    // l = 0,2,4 (index l/2)
    double minus[5][9];   // L = 4,6,8,10,12 (index L/2 - 2); up to mu^8
};

void build_quadrature(int L, Quadrature& q);
void build_kernel_polys(KernelPolys& kp);
void legendre_poly(int l, double* c);  // power-series coefficients, c[0..l]
void gauss_legendre(int n, double* x, double* w);
void eb_matrices(double N[2][3], double M[3][3]);

// --------------------------------------------------------------------- device params
struct DevTables;  // opaque pointer bundle filled by the C API

// Per-kernel timing bookkeeping (kernel kinds as in lpp_plan_kernel_stats).
enum KernelKind { KK_ASSIGN = 0, KK_FFT = 1, KK_COMBINE = 2, KK_COEFF = 3, KK_PARTNER = 4, KK_OTHER = 5, KK_COUNT = 6 };

}  // namespace lpp
