// Window-convolved theory templates by FFTLog (Sec. 3.2, Eqs. window_convolution_X_hankel,
// def_of_Q_llp; Appendix D).
//
//   Pt^(L)_X(k) = H_L[ sum_L' Q^X_LL'(r) xi^(L')_X(r) ](k),   xi^(L')_X = H^-1_L'[P^(L')_X]
//
// Both Hankel transforms use the log-Fourier method of Hamilton (2000): A(x) x^-q is
// expanded in a discrete Fourier series in ln x and each term is transformed with the Mellin
// transform of j_l,  int_0^inf x^(s-1) j_l(x) dx = 2^(s-2) sqrt(pi) G((l+s)/2) / G((3+l-s)/2).
// One CTA evaluates one parameter set: the BBKS model and its sigma_8 normalisation, three
// inverse transforms (L' = 0, 2, 4), then for each of the fourteen output slots (the
// estimator's order: the density quadrupole and hexadecapole, whose templates are the
// leakage of the monopole through Q_2 and Q_4, Sec. 4.3, then the minus moments L = 10, 12,
// which the model leaves zero and only the window fills) the mixture with the window
// multipoles, one forward transform and the shell averages.  Everything is FP64.
//
// Grid (shared with the tests): 2048 log-spaced k in [1e-4, 10], zero padding to 4096,
// k_0 r_0 = exp(-(N-1) Delta), biases 1.5 (inverse) and 0.5 (forward), the input tapered by
// t - sin(2 pi t)/(2 pi) over the outer 10% of the log-k range at both ends.
#include <math.h>
#include <string.h>

#include <complex>
#include <vector>

#include "lpp_internal.h"
#include "lpp_kernels.h"
#include "lpp_fft_dev.cuh"

namespace {

constexpr int kNin = 2048;
constexpr int kNfft = 4096;
constexpr int kLogN = 12;
constexpr double kKmin = 1e-4, kKmax = 10.0, kQinv = 1.5, kQfwd = 0.5, kTaper = 0.1;
constexpr double kPi = 3.14159265358979323846;
constexpr int kSlots = LPP_N_MOMENTS;
// the slots the derived curves read: cross L = 2, 4, 6, plus l = 0, 2, 4, minus L = 4, 6, 8
constexpr unsigned kEbSlots = 0x3FEu;
constexpr int kNfwd = 7;      // forward transforms of order l = 0, 2, ..., 12 (the output slots' L)
constexpr int kMaxTerms = 3;   // model multipoles L' feeding one output slot

struct SlotDesc {
    int kind;      // 0 dd, 1 cross, 2 plus, 3 minus
    int L;
    int n_terms;
    int lp[kMaxTerms];      // L' of each term (0, 2, 4)
    int coef[kMaxTerms];    // model coefficient id (see model_coef)
    int qx[kMaxTerms];      // row of the mixed window table Q^X_LL'(r_m)
};

struct TemplateArgs {
    const double* params;   // [n][6]: A, b_g, sigma8, tilt, Gamma, shot-noise scale
    int n_templates;
    double* out;            // [n][LPP_N_MOMENTS][nb]
    const double* kin;      // [2048] k_n
    const double* s8w;      // [2048] sigma_8 quadrature weight w_n k^3 W^2(8k) / (2 pi^2)
    const double* ain;      // [2048] k^3 taper k^-q_inv
    const double2* uinv;    // [3][4096] inverse kernels (1/N folded in)
    const double* rinv;     // [4096] r^-q_inv / (2 pi^2)
    const double2* ufwd;    // [7][4096] forward kernels of l = 0, 2, ..., 12 (1/N folded in)
    const double* rfwd;     // [4096] r^(3 - q_fwd)
    const double* kfwd;     // [2048] 4 pi k^-q_fwd
    const double* qx;       // [rows][4096] mixed window Q^X_LL'(r_m)
    const double2* tw;      // [4096] e^{-2 pi i j / N}
    const int* bin_lo;      // [nb] first k_n of each shell
    const int* bin_hi;      // [nb] one past the last
    const double* bin_w;    // [2048] k_n^3
    int nb;
    double shot_plus;
    SlotDesc slots[kSlots];
    // optional derived curves gE_0,2, EE_0,2,4, BB_0,2,4 per shell, standardised as
    // (value - ref) / sigma and stored FP32 [n][8][nb]
    float* eb;
    const double* eb_ref;
    const double* eb_sigma;
    double N[2][3], M[3][3];
    // spin-2 primordial non-Gaussianity (Sec. 5): 12 f_NL^(s=2) delta b_IA and (c / H0)^2 / Omega_m;
    // png_amp = 0: Gaussian initial conditions
    double png_amp, png_len2;
    unsigned slot_mask;     // output slots to compute; the others are written as zeros
};

// BBKS transfer function T(q), q = k / Gamma (Bardeen, Bond, Kaiser & Szalay 1986)
__device__ __forceinline__ double bbks_transfer(double k, double gam) {
    const double q = k / gam;
    return log(1.0 + 2.34 * q) / (2.34 * q) *
           pow(1.0 + 3.89 * q + (16.1 * q) * (16.1 * q) + (5.46 * q) * (5.46 * q) * (5.46 * q) +
                   (6.71 * q) * (6.71 * q) * (6.71 * q) * (6.71 * q),
               -0.25);
}

// The shape response to spin-2 PNG: P -> [1 + 12 f_NL delta b_IA / M(k)] P for each shape field
// (Sec. 5), M(k) = (2/3) k^2 T(k) D (c/H0)^2 / Omega_m with D = 1 (z = 0).
__device__ __forceinline__ double png_factor(double k, double gam, double amp, double len2) {
    return 1.0 + amp / ((2.0 / 3.0) * k * k * bbks_transfer(k, gam) * len2);
}

__device__ __forceinline__ double bbks_shape(double k, double gam, double tilt) {
    const double q = k / gam;
    const double t = log(1.0 + 2.34 * q) / (2.34 * q) *
                     pow(1.0 + 3.89 * q + (16.1 * q) * (16.1 * q) + (5.46 * q) * (5.46 * q) * (5.46 * q) +
                             (6.71 * q) * (6.71 * q) * (6.71 * q) * (6.71 * q),
                         -0.25);
    return pow(k, 1.0 + tilt) * t * t;
}

__device__ __forceinline__ double model_coef(int id, double A, double b) {
    switch (id) {
        case 0: return b * b;                  // dd, L' = 0
        case 1: return -A * b / 6.0;           // cross, L' = 2
        case 2: return 2.0 * A * A / 15.0;     // plus, L' = 0
        case 3: return -4.0 * A * A / 21.0;    // plus, L' = 2
        case 4: return 2.0 * A * A / 35.0;     // plus, L' = 4
        default: return A * A / 420.0;         // minus, L' = 4
    }
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    __syncthreads();
    return s;
}

// wk <- FFT(wk) * u ; FFT again (the log-Fourier transform between the two grids)
__device__ void log_fourier(double2* wk, const double2* __restrict__ u, const double2* __restrict__ tw) {
    const int tid = threadIdx.x;
    lpp::fft_columns<double, kLogN, false, 1, 1>(wk, 0, tid, tw);
    for (int i = tid; i < kNfft; i += blockDim.x) wk[i] = lpp::cmul<double>(wk[i], u[i]);
    __syncthreads();
    lpp::fft_columns<double, kLogN, false, 1, 1>(wk, 0, tid, tw);
}

__global__ void __launch_bounds__(512, 1) k_template(TemplateArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* wk = reinterpret_cast<double2*>(smem_raw);        // [4096]
    double* xi = reinterpret_cast<double*>(wk + kNfft);        // [3][4096]
    double* av = xi + 3 * kNfft;                               // [2048]
    __shared__ double red[32];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int t = blockIdx.x;
    if (t >= a.n_templates) return;
    const double* p = a.params + 6 * (size_t)t;
    const double A = p[0], b = p[1], s8 = p[2], tilt = p[3], gam = p[4], shot = p[5];

    // model spectrum and its sigma_8 normalisation
    double loc = 0.0;
    for (int n = tid; n < kNin; n += nthr) {
        const double sh = bbks_shape(a.kin[n], gam, tilt);
        av[n] = sh;
        loc += a.s8w[n] * sh;
    }
    const double s2 = block_sum(loc, red);
    const double norm = s8 * s8 / s2;
    for (int n = tid; n < kNin; n += nthr) av[n] *= norm * a.ain[n];
    __syncthreads();

    // xi^(L') = H^-1_L'[P_X], one phase of at most three transforms: Gaussian: P at L' = 0, 2, 4
    // for every slot; with PNG the shape spectra carry the response factor once (cross, phase 0
    // with the density's P) or twice (plus and minus, phase 1)
    const bool png = a.png_amp != 0.0;
    for (int phase = 0; phase < (png ? 2 : 1); ++phase) {
    int nrow = 3, rowL[3] = {0, 2, 4}, rowP[3] = {0, 0, 0};
    if (png && phase == 0) { nrow = 2; rowL[1] = 2; rowP[1] = 1; }
    if (png && phase == 1) { rowP[0] = rowP[1] = rowP[2] = 2; }
    for (int r = 0; r < nrow; ++r) {
        for (int m = tid; m < kNfft; m += nthr) {
            double v = 0.0;
            if (m < kNin) {
                v = av[m];
                if (rowP[r] > 0) {
                    const double f = png_factor(a.kin[m], gam, a.png_amp, a.png_len2);
                    v *= rowP[r] == 1 ? f : f * f;
                }
            }
            wk[m] = make_double2(v, 0.0);
        }
        __syncthreads();
        log_fourier(wk, a.uinv + (size_t)(rowL[r] / 2) * kNfft, a.tw);
        const double sgn = (rowL[r] == 2) ? -1.0 : 1.0;   // i^L'
        for (int m = tid; m < kNfft; m += nthr) xi[r * kNfft + m] = sgn * wk[m].x * a.rinv[m];
        __syncthreads();
    }

    // each output slot of this phase: mixture with the window, forward transform, shell averages
    for (int s = 0; s < kSlots; ++s) {
        const SlotDesc& sd = a.slots[s];
        if (png && (sd.kind >= 2 ? 1 : 0) != phase) continue;
        if (!((a.slot_mask >> s) & 1u)) {
            for (int bb = tid; bb < a.nb; bb += nthr) a.out[((size_t)t * kSlots + s) * a.nb + bb] = 0.0;
            continue;
        }
        double cf[kMaxTerms];
        int row[kMaxTerms];
        for (int j = 0; j < sd.n_terms; ++j) {
            cf[j] = model_coef(sd.coef[j], A, b);
            row[j] = 0;
            for (int r = 0; r < nrow; ++r)
                if (rowL[r] == sd.lp[j]) row[j] = r;
        }
        for (int m = tid; m < kNfft; m += nthr) {
            double g = 0.0;
            for (int j = 0; j < sd.n_terms; ++j)
                g += cf[j] * a.qx[(size_t)sd.qx[j] * kNfft + m] * xi[row[j] * kNfft + m];
            wk[m] = make_double2(g * a.rfwd[m], 0.0);
        }
        __syncthreads();
        log_fourier(wk, a.ufwd + (size_t)(sd.L / 2) * kNfft, a.tw);
        const double sgn = ((sd.L / 2) & 1) ? -1.0 : 1.0;   // (-i)^L
        const double add = (sd.kind == 2 && sd.L == 0) ? shot * a.shot_plus : 0.0;
        // one warp per shell
        const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
        for (int bb = wid; bb < a.nb; bb += nw) {
            double num = 0.0, den = 0.0;
            for (int n = a.bin_lo[bb] + lane; n < a.bin_hi[bb]; n += 32) {
                const double w = a.bin_w[n];
                num += w * sgn * wk[n].x * a.kfwd[n];
                den += w;
            }
            for (int o = 16; o > 0; o >>= 1) {
                num += __shfl_down_sync(0xffffffffu, num, o);
                den += __shfl_down_sync(0xffffffffu, den, o);
            }
            if (lane == 0) a.out[((size_t)t * kSlots + s) * a.nb + bb] = den > 0.0 ? num / den + add : 0.0;
        }
        __syncthreads();
    }
    }
    if (a.eb) {
        // Legendre multipoles of P_gE = Re P_gd and P_EE/BB = (P_+ +- P_-)/2 (Sec. 2.4, Eq. relation_pm_EB)
        const double* o = a.out + (size_t)t * kSlots * a.nb;
        for (int bb = tid; bb < a.nb; bb += nthr) {
            double v[8];
            for (int li = 0; li < 2; ++li)
                v[li] = a.N[li][0] * o[1 * a.nb + bb] + a.N[li][1] * o[2 * a.nb + bb] + a.N[li][2] * o[3 * a.nb + bb];
            for (int li = 0; li < 3; ++li) {
                const double mm = a.M[li][0] * o[7 * a.nb + bb] + a.M[li][1] * o[8 * a.nb + bb] +
                                  a.M[li][2] * o[9 * a.nb + bb];
                const double pl = o[(4 + li) * a.nb + bb];
                v[2 + li] = 0.5 * (pl + mm);
                v[5 + li] = 0.5 * (pl - mm);
            }
            for (int c = 0; c < 8; ++c) {
                const int i = c * a.nb + bb;
                const double ref = a.eb_ref ? a.eb_ref[i] : 0.0;
                const double sg = a.eb_sigma ? a.eb_sigma[i] : 1.0;
                a.eb[(size_t)t * 8 * a.nb + i] = (float)((v[c] - ref) / sg);
            }
        }
    }
}

// ------------------------------------------------------------------ host tables
double lfact(int n) { return lgamma((double)n + 1.0); }

// Wigner 3j symbol by the Racah formula.
double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
    const double ldelta = lfact(j1 + j2 - j3) + lfact(j1 - j2 + j3) + lfact(-j1 + j2 + j3) - lfact(j1 + j2 + j3 + 1);
    const double lpre = 0.5 * (ldelta + lfact(j1 + m1) + lfact(j1 - m1) + lfact(j2 + m2) + lfact(j2 - m2) +
                               lfact(j3 + m3) + lfact(j3 - m3));
    double sum = 0.0;
    for (int k = 0; k <= j1 + j2 + j3; ++k) {
        const int a1 = j3 - j2 + k + m1, a2 = j3 - j1 + k - m2, a3 = j1 + j2 - j3 - k, a4 = j1 - k - m1,
                  a5 = j2 - k + m2;
        if (a1 < 0 || a2 < 0 || a3 < 0 || a4 < 0 || a5 < 0) continue;
        const double term = exp(lpre - lfact(k) - lfact(a1) - lfact(a2) - lfact(a3) - lfact(a4) - lfact(a5));
        sum += (k & 1) ? -term : term;
    }
    const int ph = j1 - j2 - m3;
    return ((ph % 2) != 0 ? -1.0 : 1.0) * sum;
}

// Coefficient of Q_l'' in Q^X_LL' (Eq. def_of_Q_llp).
double mixing(int m, int L, int Lp, int lpp) {
    const double pref = (2.0 * L + 1.0) * exp(0.5 * (lfact(L - m) - lfact(L + m) + lfact(Lp + m) - lfact(Lp - m)));
    return pref * wigner3j(lpp, L, Lp, 0, 0, 0) * wigner3j(lpp, L, Lp, 0, m, -m);
}

// ln Gamma(z) for Re z > 0: upward recurrence to Re z >= 12, then the Stirling series with
// Bernoulli numbers B_2 .. B_14.
std::complex<double> lgamma_c(std::complex<double> z) {
    std::complex<double> shift = 0.0;
    while (z.real() < 12.0) {
        shift -= std::log(z);
        z += 1.0;
    }
    const double B[7] = {1.0 / 6, -1.0 / 30, 1.0 / 42, -1.0 / 30, 5.0 / 66, -691.0 / 2730, 7.0 / 6};
    const std::complex<double> iz = 1.0 / z, iz2 = iz * iz;
    std::complex<double> series = 0.0, pw = iz;
    for (int k = 1; k <= 7; ++k) {
        series += B[k - 1] / (2.0 * k * (2.0 * k - 1.0)) * pw;
        pw *= iz2;
    }
    return shift + (z - 0.5) * std::log(z) - z + 0.5 * log(2.0 * kPi) + series;
}

// u_alpha = (k_0 r_0)^{-i eta} M_l(q + i eta) / N, eta = 2 pi alpha / (N Delta), alpha in DFT order;
// the Nyquist coefficient is kept real.
void fftlog_kernel(int ell, double q, double delta, double kr0, double2* u) {
    for (int i = 0; i < kNfft; ++i) {
        const int alpha = i < kNfft / 2 ? i : i - kNfft;
        const double eta = 2.0 * kPi * alpha / (kNfft * delta);
        const std::complex<double> s(q, eta);
        const std::complex<double> lm = (s - 2.0) * log(2.0) + 0.5 * log(kPi) + lgamma_c(0.5 * (double(ell) + s)) -
                                        lgamma_c(0.5 * (3.0 + double(ell) - s));
        std::complex<double> v = std::exp(lm - std::complex<double>(0.0, eta * log(kr0))) / double(kNfft);
        if (i == kNfft / 2) v = std::complex<double>(v.real(), 0.0);
        u[i] = make_double2(v.real(), v.imag());
    }
}

double top_hat(double x) {
    if (x < 1e-2) return 1.0 - x * x / 10.0 + x * x * x * x / 280.0;
    return 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
}

double taper_at(int n) {
    const double x = double(n) / (kNin - 1);
    double out = 1.0;
    for (double t : {x / kTaper, (1.0 - x) / kTaper}) {
        if (t >= 1.0) continue;
        const double tt = t < 0.0 ? 0.0 : t;
        out *= tt - sin(2.0 * kPi * tt) / (2.0 * kPi);
    }
    return out;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct lpp_template_s {
    int nb = 0;
    double shot_plus = 0.0;
    double png_amp = 0.0, png_len2 = 0.0;   // 12 f_NL delta b_IA and (c/H0)^2 / Omega_m
    unsigned slot_mask = (1u << kSlots) - 1u;
    int qx_rows = 0;
    std::vector<double> kin, s8w, ain, rinv, rfwd, kfwd, qx, bin_w;
    std::vector<double2> uinv, ufwd, tw;
    std::vector<int> bin_lo, bin_hi;
    SlotDesc slots[kSlots];
    // device
    char* ws = nullptr;
    size_t ws_need = 0, o_kin, o_s8w, o_ain, o_uinv, o_rinv, o_ufwd, o_rfwd, o_kfwd, o_qx, o_tw, o_lo, o_hi, o_bw;
    bool ready = false;
};

extern "C" lpp_status lpp_template_create(const double* q, const double* s, int n_s, const double* k_edges,
                                          int n_bins, double shot_plus, lpp_template_t* out) {
    if (!q || !s || !k_edges || !out || n_s < 1 || n_bins < 1 || n_bins > 256) return LPP_ERR_INVALID_ARG;
    for (int i = 0; i + 1 < n_s; ++i)
        if (!(s[i] < s[i + 1])) return LPP_ERR_INVALID_ARG;
    for (int i = 0; i < n_bins; ++i)
        if (!(k_edges[i] < k_edges[i + 1])) return LPP_ERR_INVALID_ARG;
    lpp_template_t t = new lpp_template_s();
    t->nb = n_bins;
    t->shot_plus = shot_plus;
    const double delta = log(kKmax / kKmin) / (kNin - 1);
    const double r0 = exp(-(kNfft - 1) * delta) / kKmin;
    const double kr0 = kKmin * r0;
    t->kin.resize(kNin);
    t->s8w.resize(kNin);
    t->ain.resize(kNin);
    t->kfwd.resize(kNin);
    t->bin_w.resize(kNin);
    for (int n = 0; n < kNin; ++n) {
        const double k = kKmin * exp(n * delta);
        const double wtr = (n == 0 || n == kNin - 1) ? 0.5 * delta : delta;
        const double th = top_hat(8.0 * k);
        t->kin[n] = k;
        t->s8w[n] = wtr * k * k * k / (2.0 * kPi * kPi) * th * th;
        t->ain[n] = k * k * k * taper_at(n) * pow(k, -kQinv);
        t->kfwd[n] = 4.0 * kPi * pow(k, -kQfwd);
        t->bin_w[n] = k * k * k;
    }
    t->rinv.resize(kNfft);
    t->rfwd.resize(kNfft);
    std::vector<double> r(kNfft);
    for (int m = 0; m < kNfft; ++m) {
        r[m] = r0 * exp(m * delta);
        t->rinv[m] = pow(r[m], -kQinv) / (2.0 * kPi * kPi);
        t->rfwd[m] = pow(r[m], 3.0 - kQfwd);
    }
    t->uinv.resize(3 * kNfft);
    for (int li = 0; li < 3; ++li) fftlog_kernel(2 * li, kQinv, delta, kr0, &t->uinv[li * kNfft]);
    t->ufwd.resize(kNfwd * kNfft);
    for (int li = 0; li < kNfwd; ++li) fftlog_kernel(2 * li, kQfwd, delta, kr0, &t->ufwd[li * kNfft]);
    t->tw.resize(kNfft);
    for (int j = 0; j < kNfft; ++j) t->tw[j] = make_double2(cos(2.0 * kPi * j / kNfft), -sin(2.0 * kPi * j / kNfft));
    // window multipoles on the r grid: linear in s, held below s_0, zero beyond the last s
    std::vector<double> qr(5 * kNfft, 0.0);
    for (int li = 0; li < 5; ++li)
        for (int m = 0; m < kNfft; ++m) {
            const double x = r[m];
            double v;
            if (x <= s[0]) v = q[li * n_s];
            else if (x > s[n_s - 1]) v = 0.0;
            else {
                int j = 0;
                while (j + 1 < n_s && s[j + 1] < x) ++j;
                const double f = (x - s[j]) / (s[j + 1] - s[j]);
                v = q[li * n_s + j] + f * (q[li * n_s + j + 1] - q[li * n_s + j]);
            }
            qr[li * kNfft + m] = v;
        }
    // output slots: kind, L and the model multipoles feeding them
    const int kinds[kSlots] = {0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 0, 0, 3, 3};
    const int Ls[kSlots] = {0, 2, 4, 6, 0, 2, 4, 4, 6, 8, 2, 4, 10, 12};
    const int mX[4] = {0, 2, 0, 4};
    int rows = 0;
    for (int sl = 0; sl < kSlots; ++sl) {
        SlotDesc& sd = t->slots[sl];
        sd.kind = kinds[sl];
        sd.L = Ls[sl];
        sd.n_terms = 0;
        auto add = [&](int lp, int cid) {
            const int j = sd.n_terms++;
            sd.lp[j] = lp;
            sd.coef[j] = cid;
            sd.qx[j] = rows++;
            std::vector<double> mix(5);
            for (int lpp = 0; lpp <= 8; lpp += 2) mix[lpp / 2] = mixing(mX[sd.kind], sd.L, lp, lpp);
            for (int m = 0; m < kNfft; ++m) {
                double v = 0.0;
                for (int li = 0; li < 5; ++li) v += mix[li] * qr[li * kNfft + m];
                t->qx.push_back(v);
            }
        };
        if (sd.kind == 0) add(0, 0);
        else if (sd.kind == 1) add(2, 1);
        else if (sd.kind == 2) { add(0, 2); add(2, 3); add(4, 4); }
        else add(4, 5);
    }
    t->qx_rows = rows;
    t->bin_lo.resize(n_bins);
    t->bin_hi.resize(n_bins);
    for (int bb = 0; bb < n_bins; ++bb) {
        int lo = kNin, hi = 0;
        for (int n = 0; n < kNin; ++n)
            if (t->kin[n] >= k_edges[bb] && t->kin[n] < k_edges[bb + 1]) {
                lo = n < lo ? n : lo;
                hi = n + 1;
            }
        t->bin_lo[bb] = lo < hi ? lo : 0;
        t->bin_hi[bb] = lo < hi ? hi : 0;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    t->o_kin = take(kNin * 8);
    t->o_s8w = take(kNin * 8);
    t->o_ain = take(kNin * 8);
    t->o_uinv = take(3 * kNfft * 16);
    t->o_rinv = take(kNfft * 8);
    t->o_ufwd = take(kNfwd * kNfft * 16);
    t->o_rfwd = take(kNfft * 8);
    t->o_kfwd = take(kNin * 8);
    t->o_qx = take((size_t)rows * kNfft * 8);
    t->o_tw = take(kNfft * 16);
    t->o_lo = take(n_bins * 4);
    t->o_hi = take(n_bins * 4);
    t->o_bw = take(kNin * 8);
    t->ws_need = off;
    *out = t;
    return LPP_OK;
}

extern "C" void lpp_template_destroy(lpp_template_t t) { delete t; }

extern "C" lpp_status lpp_template_workspace_size(lpp_template_t t, size_t* bytes) {
    if (!t || !bytes) return LPP_ERR_INVALID_ARG;
    *bytes = t->ws_need;
    return LPP_OK;
}

extern "C" lpp_status lpp_template_set_workspace(lpp_template_t t, void* dev, size_t bytes, void* stream) {
    if (!t || !dev) return LPP_ERR_INVALID_ARG;
    if (((uintptr_t)dev & 255) != 0) return LPP_ERR_INVALID_ARG;
    if (bytes < t->ws_need) return LPP_ERR_WORKSPACE;
    t->ws = (char*)dev;
    cudaStream_t st = (cudaStream_t)stream;
    auto put = [&](size_t o, const void* src, size_t b) {
        return cudaMemcpyAsync(t->ws + o, src, b, cudaMemcpyHostToDevice, st);
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = put(t->o_kin, t->kin.data(), kNin * 8);
    if (e == cudaSuccess) e = put(t->o_s8w, t->s8w.data(), kNin * 8);
    if (e == cudaSuccess) e = put(t->o_ain, t->ain.data(), kNin * 8);
    if (e == cudaSuccess) e = put(t->o_uinv, t->uinv.data(), 3 * kNfft * 16);
    if (e == cudaSuccess) e = put(t->o_rinv, t->rinv.data(), kNfft * 8);
    if (e == cudaSuccess) e = put(t->o_ufwd, t->ufwd.data(), kNfwd * kNfft * 16);
    if (e == cudaSuccess) e = put(t->o_rfwd, t->rfwd.data(), kNfft * 8);
    if (e == cudaSuccess) e = put(t->o_kfwd, t->kfwd.data(), kNin * 8);
    if (e == cudaSuccess) e = put(t->o_qx, t->qx.data(), t->qx.size() * 8);
    if (e == cudaSuccess) e = put(t->o_tw, t->tw.data(), kNfft * 16);
    if (e == cudaSuccess) e = put(t->o_lo, t->bin_lo.data(), t->nb * 4);
    if (e == cudaSuccess) e = put(t->o_hi, t->bin_hi.data(), t->nb * 4);
    if (e == cudaSuccess) e = put(t->o_bw, t->bin_w.data(), kNin * 8);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LPP_ERR_CUDA;
    t->ready = true;
    return LPP_OK;
}

static lpp_status convolve(lpp_template_t t, const double* params, int n_templates, double* out, float* eb,
                           const double* eb_ref, const double* eb_sigma, void* stream);

extern "C" lpp_status lpp_template_set_png(lpp_template_t t, double f_nl, double db_ia, double omega_m) {
    if (!t || !(omega_m > 0.0) || !(db_ia == db_ia) || !(f_nl == f_nl)) return LPP_ERR_INVALID_ARG;
    const double c_over_h0 = 2997.92458;   // Mpc/h: c / (100 km/s/Mpc)
    t->png_amp = 12.0 * f_nl * db_ia;
    t->png_len2 = c_over_h0 * c_over_h0 / omega_m;
    return LPP_OK;
}

extern "C" lpp_status lpp_template_set_slots(lpp_template_t t, unsigned mask) {
    if (!t || (mask >> kSlots) != 0u) return LPP_ERR_INVALID_ARG;
    t->slot_mask = mask;
    return LPP_OK;
}

extern "C" lpp_status lpp_convolve_template(lpp_template_t t, const double* params, int n_templates, double* out,
                                            void* stream) {
    return convolve(t, params, n_templates, out, nullptr, nullptr, nullptr, stream);
}

extern "C" lpp_status lpp_convolve_template_eb(lpp_template_t t, const double* params, int n_templates, double* out,
                                               float* eb, const double* eb_ref, const double* eb_sigma, void* stream) {
    if (n_templates > 0 && !eb) return LPP_ERR_INVALID_ARG;
    if (t && (t->slot_mask & kEbSlots) != kEbSlots) return LPP_ERR_INVALID_ARG;
    return convolve(t, params, n_templates, out, eb, eb_ref, eb_sigma, stream);
}

static lpp_status convolve(lpp_template_t t, const double* params, int n_templates, double* out, float* eb,
                           const double* eb_ref, const double* eb_sigma, void* stream) {
    if (!t || (n_templates > 0 && (!params || !out)) || n_templates < 0) return LPP_ERR_INVALID_ARG;
    if (!t->ready) return LPP_ERR_NOT_READY;
    if (n_templates == 0) return LPP_OK;
    TemplateArgs a;
    memset(&a, 0, sizeof(a));
    a.params = params;
    a.n_templates = n_templates;
    a.out = out;
    a.kin = (const double*)(t->ws + t->o_kin);
    a.s8w = (const double*)(t->ws + t->o_s8w);
    a.ain = (const double*)(t->ws + t->o_ain);
    a.uinv = (const double2*)(t->ws + t->o_uinv);
    a.rinv = (const double*)(t->ws + t->o_rinv);
    a.ufwd = (const double2*)(t->ws + t->o_ufwd);
    a.rfwd = (const double*)(t->ws + t->o_rfwd);
    a.kfwd = (const double*)(t->ws + t->o_kfwd);
    a.qx = (const double*)(t->ws + t->o_qx);
    a.tw = (const double2*)(t->ws + t->o_tw);
    a.bin_lo = (const int*)(t->ws + t->o_lo);
    a.bin_hi = (const int*)(t->ws + t->o_hi);
    a.bin_w = (const double*)(t->ws + t->o_bw);
    a.nb = t->nb;
    a.shot_plus = t->shot_plus;
    a.png_amp = t->png_amp;
    a.png_len2 = t->png_len2;
    a.slot_mask = t->slot_mask;
    for (int s = 0; s < kSlots; ++s) a.slots[s] = t->slots[s];
    a.eb = eb;
    a.eb_ref = eb_ref;
    a.eb_sigma = eb_sigma;
    lpp::eb_matrices(a.N, a.M);
    const size_t smem = (size_t)kNfft * 16 + (size_t)3 * kNfft * 8 + (size_t)kNin * 8;
    cudaFuncSetAttribute(k_template, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_template<<<n_templates, 512, smem, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? LPP_OK : LPP_ERR_CUDA;
}
