/*
 * lpp.h -- C ABI of the GB300 LPP projected-tensor multipole library (liblpp.so).
 *
 * The library measures the multipoles of the power spectrum of a projected rank-2
 * tensor field (galaxy shapes) with the local-plane-parallel (LPP) FFT estimators of
 * Kurita & Takada (2022), "Analysis method for 3D power spectrum of projected tensor
 * fields with fast estimator and window convolution modelling":
 *
 *   cross  P^(L)_gd, L = 2,4,6   Sec. 3.1.2, Eqs. lpp_estimator_cross_Xiij, def_of_Xiij
 *   plus   P^(l)_+,  l = 0,2,4   Eq. lpp_estimator_auto_+ (Appendix B)
 *   minus  P^(L)_-,  L = 4..12   Eqs. lpp_estimator_auto_-, def_of_Xiijkl (Appendix B)
 *   density   P^(l)_dd, l = 0,2,4 Sec. 3.1.1, Eqs. lpp_dens_app, delta_ell
 *
 * The shear of each galaxy is gamma = e_ij(x) s_ij (Eq. gamma_def), with
 * e_ij = e+_i e+_j and e+ = (e_theta + i e_phi)/sqrt(2) (Eqs. def_of_eij_+2,
 * def_polarization_vector) in the sky frame about a plan pole p:
 * e_phi = unit(p x xhat), e_theta = e_phi x xhat (for p = z this is the frame of
 * the rotation S(d), Eq. def_standard_rotation).
 *
 * Conventions shared by every entry point:
 *  - All device work runs asynchronously on the plan's stream; lpp_multipoles
 *    synchronises that stream before it writes host outputs.
 *  - The library never allocates device memory: the caller supplies one device
 *    workspace of lpp_plan_workspace_size() bytes (e.g. a torch uint8 tensor).
 *  - Every function returns an lpp_status; none aborts or throws.  On an error the
 *    host outputs are left untouched.  After LPP_ERR_CUDA the plan must be destroyed.
 *  - Grids are cubic: n^3 nodes over a box of side `box`, n a power of two in
 *    [8, 1024].  Particles must lie in [origin, origin + box] on every axis.
 */
#ifndef LPP_H
#define LPP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LPP_OK = 0,
    LPP_ERR_INVALID_ARG = 1,  /* bad descriptor, size, pointer or flag                         */
    LPP_ERR_CUDA = 2,         /* a CUDA runtime call failed; destroy the plan                  */
    LPP_ERR_NOT_READY = 3,    /* workspace or required catalogue not supplied yet              */
    LPP_ERR_WORKSPACE = 4,    /* workspace smaller than lpp_plan_workspace_size()              */
    LPP_ERR_UNSUPPORTED = 5,  /* grid size or option combination not built                      */
    LPP_ERR_DOMAIN = 6,       /* a particle lies outside the box, on the observer or the pole  */
    LPP_ERR_BOUNDS = 7        /* checking builds (liblpp_check.so, LPP_CHECK): a device index fell
                                 outside its buffer; the access was skipped, the results are void */
} lpp_status;

/* assignment schemes: the exponent p of the window sinc^p */
enum { LPP_CIC = 2, LPP_TSC = 3 };
/* arithmetic of grids, FFTs and per-mode products (shell sums are always FP64) */
enum { LPP_FP32 = 0, LPP_FP64 = 1 };
/* line of sight used for the projection / for the estimator:
 * LOCAL = unit(x - observer) per galaxy (case (a) of Sec. 4.2),
 * GLOBAL = the plan's los_global for every galaxy (cases (b), (c)). */
enum { LPP_LOS_LOCAL = 0, LPP_LOS_GLOBAL = 1 };
/* catalogue roles for lpp_assign */
enum { LPP_SHAPES = 0, LPP_DENSITY = 1, LPP_RANDOMS = 2 };
/* shape inputs */
enum { LPP_SHAPE_NONE = 0, LPP_SHAPE_GAMMA12 = 1, LPP_SHAPE_TENSOR6 = 2 };

/* Moment slots of every output array, in this order.  Slots 10 and 11 are the density
 * quadrupole and hexadecapole P^(2,4)_dd of Eq. lpp_dens_app (Yamamoto form: each
 * catalogue's delta^(l) with its own endpoint lines of sight, Eq. delta_ell).  Slots 12 and 13
 * are the minus moments L = 10, 12. */
#define LPP_N_MOMENTS 14
enum {
    LPP_MOM_DD0 = 0,
    LPP_MOM_CROSS2 = 1, LPP_MOM_CROSS4 = 2, LPP_MOM_CROSS6 = 3,
    LPP_MOM_PLUS0 = 4, LPP_MOM_PLUS2 = 5, LPP_MOM_PLUS4 = 6,
    LPP_MOM_MINUS4 = 7, LPP_MOM_MINUS6 = 8, LPP_MOM_MINUS8 = 9,
    LPP_MOM_DD2 = 10, LPP_MOM_DD4 = 11,
    LPP_MOM_MINUS10 = 12, LPP_MOM_MINUS12 = 13
};
/* bitmask of requested moments: bit i enables slot i.  LPP_WANT_ALL is the ten slots of
 * the density monopole and the tensor estimators; LPP_WANT_DENSITY adds the density
 * quadrupole and hexadecapole (2l+1 fields each, from the density catalogue and the
 * randoms).  LPP_WANT_CROSS_B adds the B (imaginary) part of the cross moments, which
 * costs 2L+1 extra fields per L. */
#define LPP_WANT_ALL 0x3FFu
#define LPP_WANT_DD2 (1u << LPP_MOM_DD2)
#define LPP_WANT_DD4 (1u << LPP_MOM_DD4)
#define LPP_WANT_DENSITY (LPP_WANT_DD2 | LPP_WANT_DD4)
/* the minus moments beyond L = 8 (Eq. lpp_estimator_auto_- with L = 10, 12; 2 (2L+1) fields each),
 * for the completeness of the minus-spectrum expansion (Sec. 2.4) and its systematics tests */
#define LPP_WANT_MINUS_HIGH ((1u << LPP_MOM_MINUS10) | (1u << LPP_MOM_MINUS12))
#define LPP_WANT_CROSS_B (1u << 16)

typedef struct lpp_plan_s* lpp_plan_t;

typedef struct {
    int n;                   /* grid side, power of two, 8..1024                               */
    double box;              /* side of the cubic box                                          */
    double origin[3];        /* lower corner of the box                                        */
    double observer[3];      /* observer position (LOCAL line of sight)                        */
    double pole[3];          /* pole p of the sky frame; must not be parallel to any LOS       */
    int scheme;              /* LPP_CIC or LPP_TSC                                             */
    int interlace;           /* 1: average with the grid shifted by half a cell (all axes)     */
    int compensate;          /* 1: divide by the assignment window prod sinc^p                 */
    int precision;           /* LPP_FP32 or LPP_FP64                                           */
    int los_proj;            /* LPP_LOS_LOCAL / GLOBAL for gamma = e_ij(x) s_ij                 */
    int los_est;             /* LPP_LOS_LOCAL / GLOBAL inside the estimator kernels            */
    double los_global[3];    /* global line of sight (normalised by the library)               */
    unsigned moments;        /* LPP_WANT_* bitmask                                             */
    int n_bins;              /* number of |k| shells, 1..256                                   */
    const double* k_edges;   /* host, n_bins+1 increasing edges; copied at create              */
    double norm_override;    /* > 0: use this I for every moment instead of the estimate      */
    int subtract_shot;       /* 1: subtract shot noise from P_+^(0) and P_dd^(0)               */
    long long max_shapes;    /* capacity (particles) reserved in the workspace per role       */
    long long max_density;
    long long max_randoms;
    int host_inputs;         /* 1: reserve staging so lpp_assign accepts host catalogues       */
    int batch;               /* complex grids per field pass; 0 = library default             */
    int fused_slots;         /* channel fields per CTA of the fused assignment + x-FFT pass:
                                0 = library choice (two for FP32 interlaced 256^3 and 512^3 grids
                                when a batch holds an even number), 1 = always one (a tuning knob;
                                results agree within the FP32 tolerance)                          */
} lpp_plan_desc;

typedef struct {
    const void* pos;    /* [3][count] SoA x,y,z; float for LPP_FP32 plans, double for FP64   */
    const void* w;      /* [count] weights or NULL (all 1)                                   */
    const void* nbar;   /* [count] mean density (randoms, for I = alpha sum nbar w^2) or NULL */
    const void* shape;  /* TENSOR6: [6][count] (xx,yy,zz,xy,xz,yz); GAMMA12: [2][count]       */
    long long count;    /* number of particles, 0..max for the role                          */
    int shape_kind;     /* LPP_SHAPE_*; only the LPP_SHAPES role reads shapes                */
    int on_host;        /* 1: pointers are host memory (copied during lpp_assign)            */
} lpp_particles;

typedef struct {
    double* p;            /* out [LPP_N_MOMENTS][n_bins][2] normalised (re, im)               */
    double* raw;          /* out, optional: the same before normalisation and shot noise      */
    double* k_mean;       /* out, optional [n_bins]: mean |k| of the modes in each shell      */
    long long* n_modes;   /* out, optional [n_bins]: modes of the n^3 grid in each shell      */
    double norm_auto;     /* out: I for plus/minus                                            */
    double norm_cross;    /* out: I for cross                                                 */
    double norm_dd;       /* out: I for the density monopole                                  */
    double shot_plus;     /* out: sum_s w^2 |gamma|^2 / I (subtracted from P_+^(0))           */
    double shot_dd;       /* out: density shot noise (subtracted from P_dd^(0))               */
    double alpha;         /* out: sum w_density / sum w_randoms (0 without randoms)           */
} lpp_result;

/* Create a plan from a descriptor; validates sizes and flags on the host only.  The plan
 * fixes what every estimate of it computes (Sec. 3.1.2): the grid of Eq. lpp_estimator_cross_Xiij
 * (n^3 nodes over the box, CIC/TSC assignment, optional interlacing and window deconvolution),
 * the |k| shells of the multipoles (Eq. multipole_cross_def), the requested moments and, from
 * them, the real harmonic fields (2L+1 per moment order and projected part, because each
 * kernel of Eqs. def_of_Xiij, def_of_Xiijkl and lpp_estimator_auto_+ is a pure degree-L
 * spherical harmonic in khat), the sky frame of Eq. gamma_def about `pole`, and the line of
 * sight of the projection and of the estimator (cases (a)-(c) of Sec. 4.2).
 * Errors: LPP_ERR_UNSUPPORTED for a grid that is not a power of two in [8, 1024],
 * LPP_ERR_INVALID_ARG for any other bad field (shells, scheme, precision, moments, a zero
 * pole or global line of sight).  On success *plan is owned by the caller (lpp_plan_destroy). */
lpp_status lpp_plan_create(const lpp_plan_desc* desc, lpp_plan_t* plan);
void lpp_plan_destroy(lpp_plan_t plan);

/* Device bytes the caller must provide through lpp_plan_set_workspace. */
lpp_status lpp_plan_workspace_size(lpp_plan_t plan, size_t* bytes);
/* Hand the plan a device buffer of at least lpp_plan_workspace_size() bytes,
 * 256-byte aligned; the caller keeps ownership and must keep it alive. */
lpp_status lpp_plan_set_workspace(lpp_plan_t plan, void* device_ptr, size_t bytes);
/* CUDA stream (cudaStream_t) for all work of this plan; NULL = legacy default stream. */
lpp_status lpp_plan_set_stream(lpp_plan_t plan, void* stream);
/* Number of real k-space fields one estimate transforms (channels plus partners). */
lpp_status lpp_plan_field_count(lpp_plan_t plan, int* n_fields);

/* Attach a catalogue to a role: the galaxies whose shapes form gamma (Eq. gamma_def) and
 * the shear field of Eq. lpp_estimator_cross_Xiij (LPP_SHAPES), the density tracer delta
 * (LPP_DENSITY), or the randoms that describe the survey window (LPP_RANDOMS; delta = data -
 * alpha randoms, Sec. 4.3).  Device pointers are referenced (they must stay valid until
 * lpp_multipoles returns); host pointers are copied into the workspace on the plan's
 * stream.  LPP_SHAPES is required; LPP_DENSITY defaults to the shapes' positions and
 * weights; LPP_RANDOMS is optional (none = periodic box).  Errors: LPP_ERR_INVALID_ARG for a
 * count above the role's capacity, a null pointer, a bad shape kind or missing shapes that
 * the requested moments need, host memory on a plan without staging; LPP_ERR_NOT_READY for
 * host memory before the workspace is set.  Positions are checked against the box during
 * lpp_multipoles (LPP_ERR_DOMAIN). */
lpp_status lpp_assign(lpp_plan_t plan, int role, const lpp_particles* particles);
/* Forget a role's catalogue (e.g. to run a periodic estimate after a survey one). */
lpp_status lpp_clear(lpp_plan_t plan, int role);

/* Run the estimator (Secs. 3.1.1-3.1.2): sky frames and shears, harmonic weights,
 * CIC/TSC assignment with optional interlacing, 3D FFTs, k-space contraction with
 * the partner field and FP64 shell sums; then normalise and subtract shot noise.
 * Density multipoles (slots 10, 11): P^(l)_dd = (2l+1) < delta^(l)(k) delta(-k) > / I_dd
 * with delta^(l) = FT[w L_l(khat . xhat)] of the density catalogue minus alpha times that
 * of the randoms, computed through the addition theorem L_l(khat . xhat) =
 * 4 pi / (2l+1) sum_n Y_ln(khat) Y_ln(xhat) as 2l+1 real fields FT[w Y_ln(xhat)]; no shot
 * noise for l > 0 (its shell average of L_l vanishes).  With los_est = GLOBAL the plan's
 * global line of sight replaces xhat (Eq. gpp_dens).
 * Synchronises the plan's stream.  Returns LPP_ERR_DOMAIN if a particle was outside
 * the box, at the observer, or on the frame pole. */
lpp_status lpp_multipoles(lpp_plan_t plan, lpp_result* result);

/* Window multipoles Q_l(s), l = 0,2,4,6,8 (Eq. windowQ_ell, endpoint line of sight d = x):
 * Q_l(s) = (2l+1) < int_x W(x) W(x+s) L_l(s.x) >_shell / I, with W = alpha times the
 * assigned randoms (LPP_RANDOMS, required), alpha = sum w_density / sum w_randoms when a
 * density or shape catalogue is assigned (else 1), and I = alpha sum_r nbar w^2, the
 * estimator's normalisation.  Computed by FFT cross-correlations of W Y_{l,n}(x) with W on
 * the plan's grid (CIC/TSC, deconvolved when the plan compensates, never interlaced); the
 * box must exceed the survey extent plus the largest separation, or pairs wrap around.
 * Separation shells are [s_edges[b], s_edges[b+1]) over the grid separations (s = 0
 * excluded).  Outputs: q [5][n_s]; s_mean [n_s] and n_points [n_s] (optional); *norm = I
 * (optional).  Synchronises the plan's stream. */
lpp_status lpp_window_Q(lpp_plan_t plan, int n_s, const double* s_edges, double* q, double* s_mean,
                        long long* n_points, double* norm);

/* Window multipoles by pair counting, the paper's own method for Q_l (Sec. 4.3; Eq. windowQ_ell
 * with the endpoint line of sight d = xhat_r, W = alpha sum_r w_r delta_D(x - x_r)):
 *   Q_l(b) = (2l+1) alpha^2 / (I V_b) sum_{r != r', |s_rr'| in b} w_r w_r' L_l(shat_rr' . xhat_r),
 * s_rr' = x_r' - x_r (minimal image when box > 0, else none), V_b = 4 pi (e_{b+1}^3 - e_b^3) / 3,
 * I = alpha sum_r nbar_r w_r^2 (the estimator's normalisation), xhat_r = unit(x_r - observer).
 * A cross-check of lpp_window_Q (FFT correlations on a grid) for a subsample of the randoms: the
 * cost grows as n^2 (every unordered pair once, FP64).  The shell of a pair is decided in FP64
 * on e_b <= sqrt(dx^2 + dy^2 + dz^2) < e_{b+1} with correctly rounded operations.
 * pos [3][n], w [n] (NULL: 1) and nbar [n] (NULL: 1) are FP64 device arrays; observer [3] and
 * s_edges [n_s + 1] (increasing, >= 0) are host; q [5][n_s] (l = 0, 2, 4, 6, 8) is host output.
 * workspace: a 256-byte aligned device buffer of lpp_window_Q_pairs_workspace_size() bytes,
 * owned by the caller.  Runs on `stream` and synchronises it.  Errors: LPP_ERR_INVALID_ARG
 * (bad sizes, pointers, alpha <= 0, box < 0, n_s outside 1..256), LPP_ERR_WORKSPACE (buffer too
 * small), LPP_ERR_CUDA. */
lpp_status lpp_window_Q_pairs_workspace_size(int n_s, size_t* bytes);
lpp_status lpp_window_Q_pairs(const double* pos, const double* w, const double* nbar, long long n,
                              const double* observer, double box, double alpha, int n_s, const double* s_edges,
                              double* q, void* workspace, size_t bytes, void* stream);

/* ------------------------------------------------------------------ batches of catalogues
 * Many catalogues (mocks) through a set of plans in one launch: the estimator of Secs.
 * 3.1.1-3.1.2 (each mock exactly as lpp_multipoles would compute it on its plan) over many
 * realisations, as in the validation of Sec. 4 (1000 realisations of the tidal field, Sec.
 * 4.1, whose mean Secs. 4.2-4.3 compare between estimators and with the template).  plans[0..n_plans) are
 * distinct plans with their workspaces set (they may differ in grid size and bins); mock j
 * runs on plans[plan_of[j]] with the device catalogues shapes[j] (shape kind GAMMA12 or
 * TENSOR6) and randoms[j] (randoms == NULL or randoms[j].count == 0: periodic box).  Mocks
 * of one plan run in order on a stream of the batch, different plans concurrently.  With
 * use_graph != 0 the whole batch is captured once into a CUDA graph at creation and every
 * lpp_batch_launch is one graph launch; otherwise each launch enqueues the kernels anew.
 * The catalogue buffers are borrowed: they must stay valid, with the same addresses and
 * counts, for the batch's lifetime (their contents may change between launches).  Host
 * memory for the per-mock sums is pinned and owned by the batch.  While a batch is in
 * flight its plans must not be used otherwise.  Errors: LPP_ERR_INVALID_ARG (bad indices,
 * counts above a plan's capacity, host catalogues, a plan listed twice), LPP_ERR_NOT_READY
 * (a plan without workspace), LPP_ERR_CUDA (stream, event, pinned memory or capture). */
typedef struct lpp_batch_s* lpp_batch_t;

lpp_status lpp_batch_create(lpp_plan_t* plans, int n_plans, const int* plan_of, const lpp_particles* shapes,
                            const lpp_particles* randoms, int n_mocks, int use_graph, lpp_batch_t* batch);
void lpp_batch_destroy(lpp_batch_t batch);
/* Runs every mock, ordered after the work already on `stream` and before later work on it;
 * asynchronous. */
lpp_status lpp_batch_launch(lpp_batch_t batch, void* stream);
/* Waits for the last launch and fills results[n_mocks] (caller-owned arrays as for
 * lpp_multipoles); returns the first failing mock's status (e.g. LPP_ERR_DOMAIN). */
lpp_status lpp_batch_results(lpp_batch_t batch, lpp_result* results);
const char* lpp_batch_last_error(lpp_batch_t batch);
/* Kernels of the batch: *counted = the sum of the mocks' lpp_plan_launch_count figures
 * when the batch was last enqueued or captured; *graph_kernels = the kernel nodes of the
 * captured CUDA graph as the CUDA runtime lists them (-1 without a graph).  Host outputs.
 * LPP_ERR_INVALID_ARG for a null argument, LPP_ERR_CUDA if the graph cannot be read. */
lpp_status lpp_batch_launch_count(lpp_batch_t batch, long long* counted, long long* graph_kernels);

/* ------------------------------------------------------------------ templates
 * Window-convolved theory templates (Sec. 3.2, Eqs. window_convolution_X_hankel and
 * def_of_Q_llp; Appendix D): for every parameter set (A, b_g, sigma_8, tilt, Gamma,
 * shot-noise scale) the LPP_N_MOMENTS native moment slots (the estimator's order; the
 * density quadrupole and hexadecapole are the leakage of the monopole through the window,
 * the mixtures Q^dd_20 = Q_2 and Q^dd_40 = Q_4 of Sec. 4.3, and the minus moments L = 10, 12
 * the leakage of the minus hexadecapole through Q_6 and Q_8)
 *   Pt^(L)_X(k) = H_L[ sum_L' Q^X_LL'(r) xi^(L')_X(r) ](k),  xi^(L')_X = H^-1_L'[P^(L')_X],
 * of the tidal-alignment model (shapes e = -A T_ij, galaxies b_g delta; Eq.
 * power_for_validation scaled): P_dd^(0) = b^2 P, P_gd^(2) = -A b P / 6,
 * P_+^(0,2,4) = A^2 (2/15, -4/21, 2/35) P, P_-^(4) = A^2 P / 420, with a BBKS P(k) of
 * shape Gamma and slope 1 + tilt normalised to sigma_8; the plus monopole also gets the
 * shot-noise scale times shot_plus.  FFTLog Hankel transforms (Hamilton 2000) in FP64 on
 * 2048 log-spaced k in [1e-4, 10] padded to 4096, the input tapered over the outer 10% of
 * ln k; outputs are k^3-weighted averages over the grid k in each shell [e_b, e_b+1). */
typedef struct lpp_template_s* lpp_template_t;

/* Host tables from a window table q[5][n_s] (Q_l at increasing separations s[n_s], l = 0..8
 * even, e.g. from lpp_window_Q; held below s[0], zero beyond s[n_s-1]) and shells. */
lpp_status lpp_template_create(const double* q, const double* s, int n_s, const double* k_edges, int n_bins,
                               double shot_plus, lpp_template_t* tmpl);
void lpp_template_destroy(lpp_template_t tmpl);
lpp_status lpp_template_workspace_size(lpp_template_t tmpl, size_t* bytes);
/* Device buffer (256-byte aligned, caller-owned); uploads the tables on `stream` and synchronises it. */
lpp_status lpp_template_set_workspace(lpp_template_t tmpl, void* device_ptr, size_t bytes, void* stream);
/* Spin-2 local primordial non-Gaussianity (Sec. 5): the shape response P -> [1 + 12 f_nl db_ia /
 * M(k)] P with M(k) = (2/3) k^2 T(k) D (c/H0)^2 / omega_m, T the BBKS transfer function of the
 * template's Gamma and D = 1; the cross spectra carry the factor once, the plus and minus spectra
 * twice (each shape field responds), the density spectrum not.  f_nl = 0 (the default) is the
 * Gaussian template.  LPP_ERR_INVALID_ARG for omega_m <= 0 or a NaN. */
lpp_status lpp_template_set_png(lpp_template_t tmpl, double f_nl, double db_ia, double omega_m);
/* The output slots to compute (bit i: slot i, as in lpp_plan_desc.moments; default all
 * LPP_N_MOMENTS): the others are written as zeros and cost nothing.  lpp_convolve_template_eb
 * needs the nine slots its derived curves read (mask 0x3FE: cross, plus and minus up to L = 8)
 * and returns LPP_ERR_INVALID_ARG without them.  LPP_ERR_INVALID_ARG for bits at or above
 * LPP_N_MOMENTS.  Host-only. */
lpp_status lpp_template_set_slots(lpp_template_t tmpl, unsigned mask);
/* params: device [n_templates][6]; out: device [n_templates][LPP_N_MOMENTS][n_bins].
 * Asynchronous on `stream`. */
lpp_status lpp_convolve_template(lpp_template_t tmpl, const double* params, int n_templates, double* out,
                                 void* stream);
/* As lpp_convolve_template, and also the Legendre multipoles of the derived spectra
 * (gE_0, gE_2, EE_0, EE_2, EE_4, BB_0, BB_2, BB_4; see lpp_derive_eb) standardised as
 * (value - ref) / sigma into eb (device FP32 [n_templates][8][n_bins]); eb_ref and eb_sigma
 * are device [8][n_bins] or NULL (0 and 1). */
lpp_status lpp_convolve_template_eb(lpp_template_t tmpl, const double* params, int n_templates, double* out,
                                    float* eb, const double* eb_ref, const double* eb_sigma, void* stream);

/* ------------------------------------------------------------------ surrogate
 * Template surrogate network (no counterpart in the paper; it emulates the output of
 * lpp_convolve_template): x (6 parameters) -> [Linear 256, GELU] x 4 -> Linear 320, with
 * GELU(z) = z (1 + erf(z/sqrt2)) / 2.  Every matrix product takes BF16 operands (weights,
 * layer inputs, back-propagated gradients) and accumulates in FP32 on the tensor cores;
 * Adam (beta 0.9, 0.999, eps 1e-8, bias-corrected) updates FP32 master weights.
 * Parameters travel as one FP32 host array: for each layer W [out][in] then b [out]
 * (in/out = 6/256, 256/256, 256/256, 256/256, 256/320). */
typedef struct lpp_surrogate_s* lpp_surrogate_t;

/* batch: training minibatch and inference chunk (multiple of 32). */
lpp_status lpp_surrogate_create(int batch, lpp_surrogate_t* net);
void lpp_surrogate_destroy(lpp_surrogate_t net);
lpp_status lpp_surrogate_workspace_size(lpp_surrogate_t net, size_t* bytes);
/* Device workspace (256-byte aligned, caller-owned) and initial host parameters; resets Adam. */
lpp_status lpp_surrogate_set_workspace(lpp_surrogate_t net, void* device_ptr, size_t bytes, const float* params,
                                       void* stream);
lpp_status lpp_surrogate_get_params(lpp_surrogate_t net, float* params, void* stream);
/* Checkpoint of the training state: the Adam step counter, the FP32 master weights and biases
 * and both Adam moments (host buffer of lpp_surrogate_state_size bytes, caller-owned; a
 * 32-byte header with a magic number, a version, the step and an FNV-1a 64-bit checksum of
 * the arrays that follow).  save copies the state out, load copies it in and rebuilds the
 * BF16 copies, so training continues where it stopped.  Synchronous on `stream`; load returns
 * LPP_ERR_INVALID_ARG for a buffer that is too small, carries another magic number or version,
 * or fails its checksum. */
lpp_status lpp_surrogate_state_size(lpp_surrogate_t net, size_t* bytes);
lpp_status lpp_surrogate_save_state(lpp_surrogate_t net, void* host, size_t bytes, void* stream);
lpp_status lpp_surrogate_load_state(lpp_surrogate_t net, const void* host, size_t bytes, void* stream);
/* n_steps Adam steps; step i uses rows schedule[i*batch .. (i+1)*batch) of the device arrays
 * x [n][6] and y [n][320]; losses (device, optional) [n_steps] receive each minibatch's mean
 * squared error before its update.  Asynchronous on `stream`. */
lpp_status lpp_surrogate_train(lpp_surrogate_t net, const float* x, const float* y, const int* schedule,
                               int n_steps, float lr, double* losses, void* stream);
/* Gradients of the mean squared error of one minibatch (rows idx[0..batch) of device x, y)
 * without changing the network: host grads in the parameter layout, host *loss.  Synchronous. */
lpp_status lpp_surrogate_gradients(lpp_surrogate_t net, const float* x, const float* y, const int* idx,
                                   float* grads, double* loss, void* stream);
/* Forward pass: device x [n][6] -> device y [n][320], in chunks of `batch` rows. */
lpp_status lpp_surrogate_infer(lpp_surrogate_t net, const float* x, int n, float* y, void* stream);

/* Map between template parameters and the network (the emulator of lpp_convolve_template_eb
 * built on this network).  Parameters theta = (A, b_g, sigma_8, tilt, Gamma, shot scale).
 * The window-convolved derived curves are exactly
 *     t_j(theta) = pre_c(theta) u_j(tilt, Gamma) + theta_5 s_j,   j = c * 40 + bin,
 * with pre_c = A b_g sigma_8^2 for the gE curves (c = 0, 1) and A^2 sigma_8^2 for the EE/BB
 * curves (c = 2..7): the model multipoles are proportional to b_g^2, A b_g and A^2 times the
 * sigma_8-normalised linear spectrum (Eq. all_convolutions), and the shot-noise term adds to
 * P_+^(0) only.  Inputs x_c = feed_c ? 2 (theta_c - lo_c) / (hi_c - lo_c) - 1 : 0.  The
 * network learns y_j = (u_j - B_j(x)) / sd_j around the baseline
 *     B_j(x) = mu_j + sum_ab l_a(x_p) l_b(x_q) base[a * nodes + b][j],
 * l_a the Lagrange polynomials on the Chebyshev-Lobatto nodes -cos(pi a / (nodes - 1)) and
 * (p, q) = base_in (both fed); base = NULL drops the sum.
 * mu, sd, shot (= s) are device FP64 [320]; base device FP64 [nodes^2][320]; ref and sigma
 * device FP64 [320] or NULL (0, 1) standardise the prediction as (t - ref) / sigma, as
 * lpp_convolve_template_eb does.  The pointers are borrowed and must outlive the surrogate's
 * use of them; the first lpp_surrogate_predict after lpp_surrogate_set_map copies base into
 * the surrogate's workspace as float pairs (hi + lo) for the decoding, which sums the
 * baseline in float-float arithmetic (the FP64 sum to about 2^-44 relative), so a changed
 * base needs lpp_surrogate_set_map again.  nodes in 2..8. */
typedef struct {
    double lo[6], hi[6];
    int feed[6];
    const double* mu;
    const double* sd;
    const double* shot;
    const double* ref;
    const double* sigma;
    const double* base;
    int base_nodes;
    int base_in[2];
} lpp_surrogate_map;

lpp_status lpp_surrogate_set_map(lpp_surrogate_t net, const lpp_surrogate_map* map);
/* Training targets y (device FP32 [n][320]) from device params [n][6] and the native slots
 * that lpp_convolve_template returned for them at unit amplitude and no shot noise
 * (device FP64 [n][LPP_N_MOMENTS][40]). */
lpp_status lpp_surrogate_targets(lpp_surrogate_t net, const double* params, const double* native, int n, float* y,
                                 void* stream);
/* Network inputs for device params [n][6] (FP64) -> device x [n][6] (FP32). */
lpp_status lpp_surrogate_encode(lpp_surrogate_t net, const double* params, int n, float* x, void* stream);
/* Emulated, standardised derived curves: device params [n][6] -> device out [n][320] FP32
 * (the layout of lpp_convolve_template_eb's eb for n_bins = 40).  Requires a map. */
lpp_status lpp_surrogate_predict(lpp_surrogate_t net, const double* params, int n, float* out, void* stream);

/* Gaussian (disconnected, mode-counting) error bars of the derived multipoles, the unit in
 * which the template emulator is trained and checked.  The paper gives no covariance; this
 * is the standard isotropic-Gaussian reading: a shell with N_k = V (k_hi^3 - k_lo^3) / (6 pi^2)
 * Fourier modes (both k and -k counted) and multipole l has
 *   sigma^2(gE_l)    = (2l+1) [(P_gg + N_g)(P_EE + N_e) + P_gE^2] / N_k,
 *   sigma^2(EE/BB_l) = 2 (2l+1) (P_EE/BB + N_e)^2 / N_k,
 * with the monopoles p0 (host [4][n_bins]: P_gg, P_gE, P_EE, P_BB, without shot noise),
 * the galaxy shot noise noise_g and the shot noise of each of E and B, noise_e (half that of
 * P_+).  sigma: host [8][n_bins] in the order gE_0,2, EE_0,2,4, BB_0,2,4.
 * LPP_ERR_INVALID_ARG for an empty or inverted shell, volume <= 0 or negative noise. */
lpp_status lpp_gaussian_sigma(const double* p0, const double* k_edges, int n_bins, double volume, double noise_g,
                              double noise_e, double* sigma);

/* Legendre multipoles of P_gE (l = 0,2), P_EE and P_BB (l = 0,2,4) from normalised
 * native moments p[LPP_N_MOMENTS][n_bins][2] (real parts), by the completeness of
 * {Lm_L/(1-mu^2)^(m/2)} (Sec. 2.4) and P_EE/BB = (P_+ +- P_-)/2 (Eq. relation_pm_EB).
 * Outputs ge[2][n_bins], ee[3][n_bins], bb[3][n_bins].  Host-only arithmetic. */
lpp_status lpp_derive_eb(const double* p, int n_bins, double* ge, double* ee, double* bb);

/* Per-kernel device timing of the last lpp_multipoles call (enabled by
 * lpp_plan_set_timing(plan, 1); events are recorded on the plan's stream).
 * kind: 0 assign, 1 fft, 2 combine, 3 coefficients, 4 partner unpack, 5 other (catalogue
 * sums and the randoms ratio alpha).
 * ms = summed event time, launches = number of launches, bytes = algorithmic DRAM
 * bytes those launches must move. */
lpp_status lpp_plan_set_timing(lpp_plan_t plan, int enable);
lpp_status lpp_plan_kernel_stats(lpp_plan_t plan, int kind, double* ms, long long* launches,
                                 double* bytes);

/* Number of kernels the plan's last estimate enqueued on the device (the last
 * lpp_multipoles call, or the last mock of a batch enqueued or captured on the plan): pencil sorts and scans, reach masks, coefficient and
 * normalisation-sum kernels, fused assignment passes, y/z FFT passes and shell combines
 * (memsets and copies excluded).  Counted with timing on or off.  launches: host output.
 * LPP_ERR_INVALID_ARG for a null plan or pointer. */
lpp_status lpp_plan_launch_count(lpp_plan_t plan, long long* launches);

/* Which forms of the fused assignment + x-FFT pass the last lpp_multipoles call ran (a
 * check for tests and profiles; no counterpart in the paper).  stats[6], host output:
 * [0] one-slot launches, [1] two-slot launches (two channel fields per CTA, FP32 interlaced
 * 256^3 and 512^3 grids), [2] two-slot tiles accumulated in 32-bit fixed point, [3] two-slot
 * tiles accumulated with float atomics, [4] one-slot channel tiles in fixed point, [5] one-slot
 * channel tiles with float atomics (tiles that no particle reaches are not counted).
 * Synchronises the plan's stream.  LPP_ERR_NOT_READY without a workspace. */
lpp_status lpp_plan_path_stats(lpp_plan_t plan, long long* stats);

/* Density monopole P_dd^(0) of a periodic catalogue without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (code running inside another framework's memory pool or under a fixed
 * per-process memory cap, plug-ins handed a stream but no allocator).  It computes the
 * quantity of the LPP_MOM_DD0 slot of lpp_multipoles for a periodic box (I = (sum w)^2/V,
 * shot noise sum w^2 / I always subtracted) by its own simpler path: an unsorted scatter
 * with global atomics into one grid, a full 3D FFT and the partner-mode shell sums, not
 * the fused sorted-tile kernels of lpp_multipoles.  Every intermediate lives in one fixed
 * 40 MiB device array inside the library, which each GPU that loads liblpp holds until
 * the process exits.
 *  - Sizes: grids up to n = 128 in FP32 and in FP64; larger grids return
 *    LPP_ERR_WORKSPACE.  n_bins <= 256.
 *  - pos [3][count] and w [count] (or NULL: unit weights) are device pointers of the given
 *    precision; p_out [n_bins] and n_modes_out [n_bins] (or NULL) are host memory.
 *    count = 0 gives zeros.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    and caches it for the lifetime of the process; after cudaDeviceReset on that device
 *    the cached address is stale, so do not reset a device this entry point has used.
 *  - Each call clears what it accumulates into, copies its results to the host and
 *    synchronises `stream` before returning; it must not be called while `stream` (or the
 *    legacy default stream it may be) is being captured into a CUDA graph.
 *  - All calls share the one array: calls that overlap on the GPU (other streams or
 *    other host threads) race and corrupt each other's results.  Host-side tables are
 *    per thread. */
lpp_status lpp_density_monopole_static(int n, double box, const double* origin, int scheme, int interlace,
                                       int compensate, int precision, const void* pos, const void* w,
                                       long long count, int n_bins, const double* k_edges, double* p_out,
                                       long long* n_modes_out, void* stream);

const char* lpp_status_string(lpp_status status);
/* Last error message recorded on this plan (empty string if none). */
const char* lpp_plan_last_error(lpp_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* LPP_H */
