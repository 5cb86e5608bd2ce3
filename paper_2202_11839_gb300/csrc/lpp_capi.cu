// C ABI of liblpp: plan bookkeeping, workspace layout and the estimate pipeline.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lpp_internal.h"
#include "lpp_kernels.h"
#include <nvtx3/nvToolsExt.h>

using namespace lpp;

namespace {

const double kPi = 3.14159265358979323846;
constexpr int kWindowChannels = 45;   // real harmonics of l = 0, 2, 4, 6, 8

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Catalogue {
    bool set = false;
    long long count = 0;
    int shape_kind = LPP_SHAPE_NONE;
    const void* pos = nullptr;
    const void* w = nullptr;
    const void* nbar = nullptr;
    const void* shape = nullptr;
};

}  // namespace

struct lpp_plan_s {
    lpp_plan_desc d;
    std::vector<double> edges;
    bool fp64 = false;
    size_t es = 4;   // real element size
    int n = 0;
    double box = 0;
    int nb = 0;
    // kept frequency range and geometry
    int nk_pos = 0, nk_neg = 0, nky = 0, nzi = 0;
    FftGeom geom;
    std::vector<int> thr;
    std::vector<int4> items;        // work list of the combine (combine_items)
    std::vector<long long> n_modes;
    std::vector<double> k_mean;
    // channels
    std::vector<Channel> channels;   // tensor channels first, then the density multipole channels
    int n_tensor_ch = 0;             // channels[0 .. n_tensor_ch) read the shape coefficients
    std::vector<CoeffGroup> groups;
    int n_coeff_rows = 2;
    bool need_d = false, need_g = false;
    int batch = 8;
    int batch_ch = 8;
    // host tables
    std::vector<double> polys;
    Quadrature quad[kQuadDegrees];
    KernelPolys kp;
    // workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    size_t ws_need = 0;
    size_t off_sums = 0, off_err = 0, off_out = 0, off_thr = 0, off_tw = 0, off_iw = 0, off_ph = 0;
    size_t off_quad_dirs[kQuadDegrees] = {0}, off_quad_tab[kQuadDegrees] = {0}, off_polys = 0, off_coeff = 0;
    size_t off_partner = 0, off_grids = 0, off_stage[3] = {0, 0, 0};
    // pencil-sorted catalogues: key, cell coordinates, weights, key offsets; shapes permutation
    size_t off_key[3] = {0, 0, 0}, off_su[3] = {0, 0, 0}, off_sw[3] = {0, 0, 0}, off_koff[3] = {0, 0, 0};
    size_t off_perm = 0, off_counts = 0, off_cursor = 0, off_scan = 0;
    size_t off_wout = 0, off_wthr = 0;   // window multipoles: per-channel shell sums, thresholds
    size_t off_pmask = 0;                // [3][n] z planes reached per catalogue role
    size_t off_rmax = 0;                 // [n_coeff_rows][2] max |coefficient|, rms per row (FP32 plans)
    size_t off_rsq = 0;                  // [n_coeff_rows] FP64 sums of squares
    size_t off_trows = 0;                // [2][256] z-tile rows to visit, then [2] counts
    size_t off_plive = 0;                // [3][n*n] bytes: x pencils reached per role
    size_t off_tranges = 0;              // per-tile range records of the two-slot fused passes
    size_t off_work = 0;                 // item counter of the dynamically scheduled fused passes
    size_t off_pstat = 0;                // [4] tile counters of the fused passes (FusedArgs::pstat)
    size_t off_items = 0;                // the combine's work list
    int fty = 4, ftz = 4;
    int n_partner = 0;
    int out_rows = 0;
    bool tables_ready = false;
    cudaStream_t stream = nullptr;
    Catalogue cat[3];
    Timer timer;
    std::string err;
    int n_sm = 152;
    long long n_launch = 0;   // kernels launched by the last estimate
    long long n_fused[2] = {0, 0};   // fused assignment launches of the last estimate: one-slot, two-slot
};

// FP32 interlaced grids of 256^3 or 512^3: channel batches with an even slot count run the
// two-slot fused kernel (with per-tile range records)
static bool two_slot_grid(lpp_plan_t p) {
    return !p->fp64 && p->d.interlace && (p->d.n == 256 || p->d.n == 512) && p->d.n / p->ftz <= 256 &&
           p->d.fused_slots != 1;
}

// Named host ranges around the steps of an estimate (NVTX): a timeline profiler shows each step
// beside the kernels it enqueues; without a tool attached a range costs a few nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    void next(const char* name) {   // end this range and open the next step's
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

static lpp_status fail(lpp_plan_t p, lpp_status s, const std::string& msg) {
    if (p) p->err = msg;
    return s;
}

static lpp_status cuda_fail(lpp_plan_t p, cudaError_t e, const char* where) {
    return fail(p, LPP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LPP_CUDA(call)                                                 \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail(plan, e_, #call);      \
    } while (0)

static double norm_factor(int m, int L) {
    double r = 2.0 * L + 1.0;
    for (int j = L - m + 1; j <= L + m; ++j) r /= j;
    return r;
}

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Integer thresholds on q = |f|^2: a lattice vector f lies in shell b iff
// thr[b] <= q < thr[b+1], the same decision as unit * sqrt(q) in [edge_b, edge_b+1) in FP64.
static void shell_thresholds(int n, double unit, const double* edges, int nb, std::vector<int>& thr) {
    const long long qmax = 3LL * (n / 2) * (n / 2);
    thr.resize(nb + 1);
    for (int b = 0; b <= nb; ++b) {
        const double e = edges[b];
        long long q;
        if (e <= 0) q = 0;
        else {
            const double t = e / unit;
            q = (long long)floor(t * t);
            if (q > qmax + 1) q = qmax + 1;
            while (q > 0 && unit * sqrt((double)(q - 1)) >= e) --q;
            while (q <= qmax && unit * sqrt((double)q) < e) ++q;
        }
        thr[b] = (int)q;
    }
}

// ------------------------------------------------------------------ plan create
extern "C" lpp_status lpp_plan_create(const lpp_plan_desc* desc, lpp_plan_t* out) {
    if (!desc || !out) return LPP_ERR_INVALID_ARG;
    *out = nullptr;
    const lpp_plan_desc& d = *desc;
    if (!is_pow2(d.n) || d.n < 8 || d.n > 1024) return LPP_ERR_UNSUPPORTED;
    if (!(d.box > 0) || d.n_bins < 1 || d.n_bins > 256 || !d.k_edges) return LPP_ERR_INVALID_ARG;
    if (d.scheme != LPP_CIC && d.scheme != LPP_TSC) return LPP_ERR_INVALID_ARG;
    if (d.precision != LPP_FP32 && d.precision != LPP_FP64) return LPP_ERR_INVALID_ARG;
    if ((d.los_proj != LPP_LOS_LOCAL && d.los_proj != LPP_LOS_GLOBAL) ||
        (d.los_est != LPP_LOS_LOCAL && d.los_est != LPP_LOS_GLOBAL))
        return LPP_ERR_INVALID_ARG;
    if ((d.moments & (LPP_WANT_ALL | LPP_WANT_DENSITY)) == 0) return LPP_ERR_INVALID_ARG;
    if (d.max_shapes < 0 || d.max_density < 0 || d.max_randoms < 0) return LPP_ERR_INVALID_ARG;
    if (d.batch < 0 || d.batch > kMaxSlots) return LPP_ERR_INVALID_ARG;
    if (d.fused_slots < 0 || d.fused_slots > 2) return LPP_ERR_INVALID_ARG;
    for (int i = 0; i < d.n_bins; ++i)
        if (!(d.k_edges[i] < d.k_edges[i + 1])) return LPP_ERR_INVALID_ARG;
    const double pn = sqrt(d.pole[0] * d.pole[0] + d.pole[1] * d.pole[1] + d.pole[2] * d.pole[2]);
    if (!(pn > 0)) return LPP_ERR_INVALID_ARG;
    const double gn = sqrt(d.los_global[0] * d.los_global[0] + d.los_global[1] * d.los_global[1] +
                           d.los_global[2] * d.los_global[2]);
    if ((d.los_proj == LPP_LOS_GLOBAL || d.los_est == LPP_LOS_GLOBAL) && !(gn > 0)) return LPP_ERR_INVALID_ARG;

    lpp_plan_t plan = new lpp_plan_s();
    plan->d = d;
    plan->edges.assign(d.k_edges, d.k_edges + d.n_bins + 1);
    plan->d.k_edges = plan->edges.data();
    for (int a = 0; a < 3; ++a) {
        plan->d.pole[a] = d.pole[a] / pn;
        plan->d.los_global[a] = gn > 0 ? d.los_global[a] / gn : 0.0;
    }
    plan->fp64 = d.precision == LPP_FP64;
    plan->es = plan->fp64 ? 8 : 4;
    plan->n = d.n;
    plan->box = d.box;
    plan->nb = d.n_bins;
    const int n = d.n, nb = d.n_bins;

    // thresholds on the integer |f|^2: mode in shell b iff thr[b] <= q < thr[b+1],
    // the same decision as kf*sqrt(q) in [edge_b, edge_b+1) in FP64
    const double kf = 2.0 * kPi / d.box;
    shell_thresholds(n, kf, d.k_edges, nb, plan->thr);
    const int tmax = plan->thr[nb];
    int nk = 0;
    while ((long long)(nk + 1) * (nk + 1) < tmax && nk < n / 2) ++nk;
    plan->nk_pos = std::min(nk, n / 2 - 1);
    plan->nk_neg = std::min(nk, n / 2);
    plan->geom = fft_geometry(n, plan->nk_pos, plan->nk_neg);
    plan->nky = plan->geom.nky;
    plan->nzi = plan->nk_pos + 1 + (plan->nk_neg == n / 2 ? 1 : 0);

    // modes per shell and mean |k| over the kept cube
    plan->n_modes.assign(nb, 0);
    std::vector<double> ksum(nb, 0.0);
    for (int fx = -plan->nk_neg; fx <= plan->nk_pos; ++fx)
        for (int fy = -plan->nk_neg; fy <= plan->nk_pos; ++fy) {
            const long long qxy = (long long)fx * fx + (long long)fy * fy;
            if (qxy >= tmax) continue;
            for (int fz = -plan->nk_neg; fz <= plan->nk_pos; ++fz) {
                const long long q = qxy + (long long)fz * fz;
                if (q == 0 || q < plan->thr[0] || q >= tmax) continue;
                int lo = 0, hi = nb;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) / 2;
                    if (q >= plan->thr[mid]) lo = mid; else hi = mid;
                }
                plan->n_modes[lo] += 1;
                ksum[lo] += kf * sqrt((double)q);
            }
        }
    plan->k_mean.assign(nb, 0.0);
    for (int b = 0; b < nb; ++b) plan->k_mean[b] = plan->n_modes[b] ? ksum[b] / plan->n_modes[b] : 0.0;
    combine_items(n, plan->nk_pos, plan->nk_neg, plan->nky, plan->nzi, tmax, plan->items);

    // kernel polynomials and quadratures
    build_kernel_polys(plan->kp);
    for (int qi = 0; qi < kQuadDegrees; ++qi) build_quadrature(2 * (qi + 1), plan->quad[qi]);

    // channel groups: (kind, L) -> 2L+1 coefficient rows per projected part
    const unsigned m = d.moments;
    const bool cross_b = (m & LPP_WANT_CROSS_B) != 0;
    int row = 2;  // rows 0, 1: w gamma_1, w gamma_2
    auto add_group = [&](int kind, int L, int has_im, const double* poly, int npoly, int slot) {
        CoeffGroup g;
        g.kind = kind;
        g.L = L;
        g.has_im = has_im;
        g.row_re = row;
        row += 2 * L + 1;
        g.row_im = has_im ? row : -1;
        if (has_im) row += 2 * L + 1;
        g.poly = (int)plan->polys.size();
        g.npoly = npoly;
        plan->polys.insert(plan->polys.end(), poly, poly + npoly);
        g.quad = L / 2 - 1;
        plan->groups.push_back(g);
        for (int part = 0; part <= has_im; ++part)
            for (int nn = -L; nn <= L; ++nn) {
                Channel c;
                c.kind = kind;
                c.L = L;
                c.n = nn;
                c.part = part;
                c.moment = slot;
                c.coeff = (part ? g.row_im : g.row_re) + nn + L;
                plan->channels.push_back(c);
            }
    };
    const int crossSlot[3] = {LPP_MOM_CROSS2, LPP_MOM_CROSS4, LPP_MOM_CROSS6};
    for (int i = 0; i < 3; ++i)
        if (m & (1u << crossSlot[i])) add_group(KIND_CROSS, 2 * (i + 1), cross_b ? 1 : 0, plan->kp.cross[i], 2 * i + 1, crossSlot[i]);
    if (m & (1u << LPP_MOM_PLUS2)) add_group(KIND_PLUS, 2, 1, plan->kp.plus[1], 3, LPP_MOM_PLUS2);
    if (m & (1u << LPP_MOM_PLUS4)) add_group(KIND_PLUS, 4, 1, plan->kp.plus[2], 5, LPP_MOM_PLUS4);
    const int minusSlot[5] = {LPP_MOM_MINUS4, LPP_MOM_MINUS6, LPP_MOM_MINUS8, LPP_MOM_MINUS10, LPP_MOM_MINUS12};
    for (int i = 0; i < 5; ++i)
        if (m & (1u << minusSlot[i])) add_group(KIND_MINUS, 4 + 2 * i, 1, plan->kp.minus[i], 2 * i + 1, minusSlot[i]);
    plan->n_coeff_rows = row;
    plan->n_tensor_ch = (int)plan->channels.size();
    // density multipoles (Eqs. lpp_dens_app, delta_ell): by the addition theorem
    // L_l(khat . xhat) = 4 pi / (2l+1) sum_n Y_ln(khat) Y_ln(xhat), 2l+1 real fields
    // FT[w Y_ln(xhat)] of the density catalogue minus alpha times those of the randoms
    for (int l = 2; l <= 4; l += 2) {
        const int slot = l == 2 ? LPP_MOM_DD2 : LPP_MOM_DD4;
        if (!(m & (1u << slot))) continue;
        for (int nn = -l; nn <= l; ++nn) {
            Channel c;
            c.kind = KIND_DENS;
            c.L = l;
            c.n = nn;
            c.part = PART_RE;
            c.moment = slot;
            c.coeff = -1;
            plan->channels.push_back(c);
        }
    }
    plan->need_d = (m & ((1u << LPP_MOM_DD0) | (1u << LPP_MOM_CROSS2) | (1u << LPP_MOM_CROSS4) |
                         (1u << LPP_MOM_CROSS6) | LPP_WANT_DENSITY)) != 0;
    plan->need_g = (m & ((1u << LPP_MOM_PLUS0) | (1u << LPP_MOM_PLUS2) | (1u << LPP_MOM_PLUS4) |
                         (1u << LPP_MOM_MINUS4) | (1u << LPP_MOM_MINUS6) | (1u << LPP_MOM_MINUS8) |
                         LPP_WANT_MINUS_HIGH)) != 0;
    plan->n_partner = (plan->need_d ? 1 : 0) + (plan->need_g ? 2 : 0);
    plan->out_rows = (int)plan->channels.size() + 2;

    // batch: grids per field pass; the partner pass needs up to 3 (interlaced) grids
    int batch = d.batch > 0 ? d.batch : 8;
    const int per_grid = d.interlace ? 1 : 2;
    // shared-memory partials of the combine: channels x bins x 2 <= 8192 values
    int max_ch = std::min(kMaxBatchCh, 4096 / nb);
    if (max_ch < 1) max_ch = 1;
    batch = std::min(batch, std::max(1, max_ch / per_grid));
    const int partner_grids = d.interlace ? plan->n_partner : (plan->need_g ? 1 : 0) + (plan->need_d ? 1 : 0);
    plan->batch = std::max(batch, partner_grids);
    plan->batch_ch = std::min(batch * per_grid, max_ch);

    // workspace layout
    const size_t es = plan->es, cs = 2 * es;
    const size_t n3 = (size_t)n * n * n;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    plan->off_sums = take(SUM_COUNT * sizeof(double));
    plan->off_err = take(sizeof(int));
    plan->off_out = take((size_t)plan->out_rows * nb * 2 * sizeof(double));
    plan->off_thr = take((nb + 1) * sizeof(int));
    plan->off_tw = take(n * cs);
    plan->off_iw = take(n * es);
    plan->off_ph = take(n * cs);
    for (int qi = 0; qi < kQuadDegrees; ++qi) {
        plan->off_quad_dirs[qi] = take(plan->quad[qi].dirs.size() * es);
        plan->off_quad_tab[qi] = take(plan->quad[qi].table.size() * es);
    }
    plan->off_polys = take(std::max<size_t>(1, plan->polys.size()) * es);
    plan->off_coeff = take((size_t)plan->n_coeff_rows * std::max<long long>(1, d.max_shapes) * es);
    {
        int ipt, thr;
        size_t sm;
        fused_geometry(n, es, &plan->fty, &plan->ftz, &ipt, &thr, &sm);
    }
    const long long caps[3] = {std::max<long long>(1, d.max_shapes), std::max<long long>(1, d.max_density),
                               std::max<long long>(1, d.max_randoms)};
    for (int r = 0; r < 3; ++r) {
        plan->off_key[r] = take((size_t)caps[r] * sizeof(int));
        plan->off_su[r] = take((size_t)3 * caps[r] * es);
        plan->off_sw[r] = take((size_t)caps[r] * es);
        plan->off_koff[r] = take(((size_t)n * n + 1) * sizeof(int));
    }
    plan->off_perm = take((size_t)caps[0] * sizeof(int));
    plan->off_counts = take((size_t)n * n * sizeof(int));
    plan->off_cursor = take((size_t)n * n * sizeof(int));
    plan->off_scan = take(1024 * sizeof(int));
    plan->off_pmask = take((size_t)3 * n * sizeof(int));
    plan->off_rmax = take((size_t)std::max(1, plan->n_coeff_rows) * 2 * sizeof(float));
    plan->off_rsq = take((size_t)std::max(1, plan->n_coeff_rows) * sizeof(double));
    plan->off_trows = take((2 * 256 + 2) * sizeof(int));
    plan->off_plive = take((size_t)3 * n * n);
    plan->off_tranges = take(two_slot_grid(plan) ? tile_range_bytes(n, plan->fty, plan->ftz) : sizeof(int));
    plan->off_work = take(sizeof(int));
    plan->off_pstat = take(4 * sizeof(int));
    plan->off_items = take(std::max<size_t>(1, plan->items.size()) * sizeof(int4));
    plan->off_wout = take((size_t)kWindowChannels * 256 * 2 * sizeof(double));
    plan->off_wthr = take(257 * sizeof(int));
    plan->off_partner = take((size_t)std::max(1, plan->n_partner) * n3 * cs);
    plan->off_grids = take((size_t)plan->batch * n3 * cs);
    if (d.host_inputs) {
        plan->off_stage[LPP_SHAPES] = take((size_t)(3 + 1 + 6) * d.max_shapes * es);
        plan->off_stage[LPP_DENSITY] = take((size_t)(3 + 1) * d.max_density * es);
        plan->off_stage[LPP_RANDOMS] = take((size_t)(3 + 1 + 1) * d.max_randoms * es);
    }
    plan->ws_need = off;
    *out = plan;
    return LPP_OK;
}

extern "C" void lpp_plan_destroy(lpp_plan_t plan) {
    if (!plan) return;
    if (plan->timer.created)
        for (int i = 0; i < Timer::kMaxEvents; ++i) cudaEventDestroy(plan->timer.ev[i]);
    delete plan;
}

extern "C" lpp_status lpp_plan_workspace_size(lpp_plan_t plan, size_t* bytes) {
    if (!plan || !bytes) return LPP_ERR_INVALID_ARG;
    *bytes = plan->ws_need;
    return LPP_OK;
}

extern "C" lpp_status lpp_plan_field_count(lpp_plan_t plan, int* n_fields) {
    if (!plan || !n_fields) return LPP_ERR_INVALID_ARG;
    *n_fields = (int)plan->channels.size() + plan->n_partner;
    return LPP_OK;
}

extern "C" lpp_status lpp_plan_set_stream(lpp_plan_t plan, void* stream) {
    if (!plan) return LPP_ERR_INVALID_ARG;
    plan->stream = (cudaStream_t)stream;
    return LPP_OK;
}

template <typename T>
static lpp_status write_tables(lpp_plan_t plan) {
    const int n = plan->n;
    auto put = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
        return cudaMemcpyAsync(plan->ws + off, src, bytes, cudaMemcpyHostToDevice, plan->stream);
    };
    LPP_CUDA(put(plan->off_thr, plan->thr.data(), plan->thr.size() * sizeof(int)));
    if (!plan->items.empty()) LPP_CUDA(put(plan->off_items, plan->items.data(), plan->items.size() * sizeof(int4)));
    // twiddles e^{-2 pi i j / n}
    std::vector<T> tw(2 * n), iw(n), ph(2 * n);
    for (int j = 0; j < n; ++j) {
        tw[2 * j] = (T)cos(2.0 * kPi * j / n);
        tw[2 * j + 1] = (T)(-sin(2.0 * kPi * j / n));
        const int f = j < n / 2 ? j : j - n;
        // assignment window sinc^p(pi f / n) and the half-cell interlacing phase
        const double xarg = kPi * f / n;
        const double sinc = f == 0 ? 1.0 : sin(xarg) / xarg;
        iw[j] = (T)(plan->d.compensate ? 1.0 / pow(sinc, plan->d.scheme) : 1.0);
        ph[2 * j] = (T)cos(xarg);
        ph[2 * j + 1] = (T)(-sin(xarg));
    }
    // host copies stay alive until the stream has consumed them (synchronised below)
    std::vector<std::vector<T>> keep;
    keep.reserve(32);
    keep.push_back(tw);
    keep.push_back(iw);
    keep.push_back(ph);
    LPP_CUDA(put(plan->off_tw, keep[0].data(), keep[0].size() * sizeof(T)));
    LPP_CUDA(put(plan->off_iw, keep[1].data(), keep[1].size() * sizeof(T)));
    LPP_CUDA(put(plan->off_ph, keep[2].data(), keep[2].size() * sizeof(T)));
    for (int qi = 0; qi < kQuadDegrees; ++qi) {
        keep.emplace_back(plan->quad[qi].dirs.begin(), plan->quad[qi].dirs.end());
        LPP_CUDA(put(plan->off_quad_dirs[qi], keep.back().data(), keep.back().size() * sizeof(T)));
        keep.emplace_back(plan->quad[qi].table.begin(), plan->quad[qi].table.end());
        LPP_CUDA(put(plan->off_quad_tab[qi], keep.back().data(), keep.back().size() * sizeof(T)));
    }
    if (!plan->polys.empty()) {
        keep.emplace_back(plan->polys.begin(), plan->polys.end());
        LPP_CUDA(put(plan->off_polys, keep.back().data(), keep.back().size() * sizeof(T)));
    }
    LPP_CUDA(cudaStreamSynchronize(plan->stream));
    plan->tables_ready = true;
    return LPP_OK;
}

extern "C" lpp_status lpp_plan_set_workspace(lpp_plan_t plan, void* device_ptr, size_t bytes) {
    if (!plan || !device_ptr) return LPP_ERR_INVALID_ARG;
    if (((uintptr_t)device_ptr & 255) != 0) return fail(plan, LPP_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (bytes < plan->ws_need) return fail(plan, LPP_ERR_WORKSPACE, "workspace too small");
    plan->ws = (char*)device_ptr;
    plan->ws_bytes = bytes;
    plan->tables_ready = false;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            plan->n_sm = sms;
    }
    return plan->fp64 ? write_tables<double>(plan) : write_tables<float>(plan);
}

extern "C" lpp_status lpp_plan_set_timing(lpp_plan_t plan, int enable) {
    if (!plan) return LPP_ERR_INVALID_ARG;
    if (enable && !plan->timer.created) {
        for (int i = 0; i < Timer::kMaxEvents; ++i) LPP_CUDA(cudaEventCreate(&plan->timer.ev[i]));
        plan->timer.created = true;
    }
    plan->timer.enabled = enable != 0;
    plan->timer.reset();
    return LPP_OK;
}

extern "C" lpp_status lpp_plan_kernel_stats(lpp_plan_t plan, int kind, double* ms, long long* launches,
                                            double* bytes) {
    if (!plan || kind < 0 || kind >= KK_COUNT) return LPP_ERR_INVALID_ARG;
    if (ms) *ms = plan->timer.ms[kind];
    if (launches) *launches = plan->timer.launches[kind];
    if (bytes) *bytes = plan->timer.total_bytes[kind];
    return LPP_OK;
}

// ------------------------------------------------------------------ catalogues
extern "C" lpp_status lpp_assign(lpp_plan_t plan, int role, const lpp_particles* p) {
    if (!plan || !p || role < 0 || role > 2) return LPP_ERR_INVALID_ARG;
    const long long cap = role == LPP_SHAPES ? plan->d.max_shapes
                                             : (role == LPP_DENSITY ? plan->d.max_density : plan->d.max_randoms);
    if (p->count < 0 || p->count > cap) return fail(plan, LPP_ERR_INVALID_ARG, "particle count exceeds the plan capacity");
    if (p->count > 0 && !p->pos) return fail(plan, LPP_ERR_INVALID_ARG, "null positions");
    int sk = role == LPP_SHAPES ? p->shape_kind : LPP_SHAPE_NONE;
    if (sk != LPP_SHAPE_NONE && sk != LPP_SHAPE_GAMMA12 && sk != LPP_SHAPE_TENSOR6)
        return fail(plan, LPP_ERR_INVALID_ARG, "bad shape kind");
    if (role == LPP_SHAPES && plan->need_g + (plan->n_tensor_ch > 0 ? 1 : 0) > 0 && sk == LPP_SHAPE_NONE)
        return fail(plan, LPP_ERR_INVALID_ARG, "the requested moments need shapes");
    if (sk != LPP_SHAPE_NONE && p->count > 0 && !p->shape) return fail(plan, LPP_ERR_INVALID_ARG, "null shapes");
    Catalogue c;
    c.set = true;
    c.count = p->count;
    c.shape_kind = sk;
    if (!p->on_host) {
        c.pos = p->pos;
        c.w = p->w;
        c.nbar = role == LPP_RANDOMS ? p->nbar : nullptr;
        c.shape = sk != LPP_SHAPE_NONE ? p->shape : nullptr;
    } else {
        if (!plan->d.host_inputs) return fail(plan, LPP_ERR_INVALID_ARG, "plan was created without host staging");
        if (!plan->ws) return fail(plan, LPP_ERR_NOT_READY, "workspace not set");
        const size_t es = plan->es;
        const long long cnt = p->count;
        char* base = plan->ws + plan->off_stage[role];
        char* dst = base;
        LPP_CUDA(cudaMemcpyAsync(dst, p->pos, 3 * cnt * es, cudaMemcpyHostToDevice, plan->stream));
        c.pos = dst;
        dst += 3 * cap * es;
        if (p->w) {
            LPP_CUDA(cudaMemcpyAsync(dst, p->w, cnt * es, cudaMemcpyHostToDevice, plan->stream));
            c.w = dst;
        }
        dst += cap * es;
        if (role == LPP_RANDOMS && p->nbar) {
            LPP_CUDA(cudaMemcpyAsync(dst, p->nbar, cnt * es, cudaMemcpyHostToDevice, plan->stream));
            c.nbar = dst;
        }
        if (role == LPP_SHAPES && sk != LPP_SHAPE_NONE) {
            const int comps = sk == LPP_SHAPE_TENSOR6 ? 6 : 2;
            LPP_CUDA(cudaMemcpyAsync(dst, p->shape, comps * cnt * es, cudaMemcpyHostToDevice, plan->stream));
            c.shape = dst;
        }
    }
    plan->cat[role] = c;
    return LPP_OK;
}

extern "C" lpp_status lpp_clear(lpp_plan_t plan, int role) {
    if (!plan || role < 0 || role > 2) return LPP_ERR_INVALID_ARG;
    plan->cat[role] = Catalogue();
    return LPP_OK;
}

// ------------------------------------------------------------------ estimate
// Steps 0-3 of an estimate on the plan's stream, then asynchronous copies of the shell sums,
// the scalar sums and the error flag to host_out [out_rows][nb][2], host_sums [SUM_COUNT] and
// *host_err (pinned memory for a copy that overlaps; the caller synchronises).  No host
// synchronisation, so the whole sequence can be captured into a CUDA graph.
template <typename T>
static lpp_status enqueue(lpp_plan_t plan, double* host_out, double* host_sums, int* host_err) {
    const int n = plan->n, nb = plan->nb;
    const size_t n3 = (size_t)n * n * n;
    cudaStream_t st = plan->stream;
    Timer* tm = plan->timer.enabled ? &plan->timer : nullptr;
    double* sums = (double*)(plan->ws + plan->off_sums);
    int* err = (int*)(plan->ws + plan->off_err);
    double* out = (double*)(plan->ws + plan->off_out);
    c2<T>* grids = (c2<T>*)(plan->ws + plan->off_grids);
    c2<T>* partner = (c2<T>*)(plan->ws + plan->off_partner);
    T* coeff = (T*)(plan->ws + plan->off_coeff);
    float* rmax = (float*)(plan->ws + plan->off_rmax);
    const long long stride = std::max<long long>(1, plan->d.max_shapes);
    const Catalogue& sh = plan->cat[LPP_SHAPES];
    const Catalogue& de = plan->cat[LPP_DENSITY].set ? plan->cat[LPP_DENSITY] : plan->cat[LPP_SHAPES];
    const Catalogue& ra = plan->cat[LPP_RANDOMS];
    const bool has_rand = ra.set;

    LPP_CUDA(cudaMemsetAsync(sums, 0, SUM_COUNT * sizeof(double), st));
    LPP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    LPP_CUDA(cudaMemsetAsync(out, 0, (size_t)plan->out_rows * nb * 2 * sizeof(double), st));
    LPP_CUDA(cudaMemsetAsync(plan->ws + plan->off_pstat, 0, 4 * sizeof(int), st));
    long long& nl = plan->n_launch;
    nl = 0;
    plan->n_fused[0] = plan->n_fused[1] = 0;

    NvtxRange r_est("lpp estimate");
    // 0. pencil sort of every catalogue (cell coordinates and weights in x-pencil key order)
    NvtxRange r_step("lpp 0 sort and reach masks");
    const long long caps[3] = {std::max<long long>(1, plan->d.max_shapes), std::max<long long>(1, plan->d.max_density),
                               std::max<long long>(1, plan->d.max_randoms)};
    int* perm = (int*)(plan->ws + plan->off_perm);
    auto sort_cat = [&](int role, const Catalogue& c) -> lpp_status {
        if (tm) tm->begin(KK_OTHER, st);
        LPP_CUDA(launch_pencil_sort<T>((const T*)c.pos, (const T*)c.w, c.count, caps[role], n, plan->box,
                                       plan->d.origin, (int*)(plan->ws + plan->off_key[role]),
                                       (int*)(plan->ws + plan->off_counts), (int*)(plan->ws + plan->off_koff[role]),
                                       (int*)(plan->ws + plan->off_cursor), (int*)(plan->ws + plan->off_scan),
                                       (T*)(plan->ws + plan->off_su[role]),
                                       (T*)(plan->ws + plan->off_sw[role]), role == LPP_SHAPES ? perm : nullptr, err,
                                       st));
        nl += c.count > 0 ? 5 : 3;
        if (tm) tm->end(KK_OTHER, st, (double)c.count * (plan->es * 8 + 12));
        return LPP_OK;
    };
    { lpp_status s0 = sort_cat(LPP_SHAPES, sh); if (s0 != LPP_OK) return s0; }
    if (plan->cat[LPP_DENSITY].set) { lpp_status s0 = sort_cat(LPP_DENSITY, de); if (s0 != LPP_OK) return s0; }
    if (has_rand) { lpp_status s0 = sort_cat(LPP_RANDOMS, ra); if (s0 != LPP_OK) return s0; }
    int* pmask = (int*)(plan->ws + plan->off_pmask);
    LPP_CUDA(launch_plane_mask((const int*)(plan->ws + plan->off_koff[0]), (const int*)(plan->ws + plan->off_koff[1]),
                               (const int*)(plan->ws + plan->off_koff[2]), 1, plan->cat[LPP_DENSITY].set ? 1 : 0,
                               has_rand ? 1 : 0, n, pmask, st));
    nl += 1;
    // the z-tile rows the fused passes visit: channel slots (shapes) and the partner slots
    int* trows = (int*)(plan->ws + plan->off_trows);
    int* tcount = trows + 512;
    const int part_bits = (1 << LPP_SHAPES) | (plan->cat[LPP_DENSITY].set ? 1 << LPP_DENSITY : 0) |
                          (has_rand ? 1 << LPP_RANDOMS : 0);
    const bool use_rows = n / plan->ftz <= 256;
    if (use_rows) {
        LPP_CUDA(launch_tile_rows(pmask, 1 << LPP_SHAPES, n, plan->ftz, trows, tcount, st));
        LPP_CUDA(launch_tile_rows(pmask, part_bits, n, plan->ftz, trows + 256, tcount + 1, st));
        nl += 2;
    }
    unsigned char* plive = (unsigned char*)(plan->ws + plan->off_plive);
    LPP_CUDA(launch_pencil_live((const int*)(plan->ws + plan->off_koff[0]), (const int*)(plan->ws + plan->off_koff[1]),
                                (const int*)(plan->ws + plan->off_koff[2]), 1, plan->cat[LPP_DENSITY].set ? 1 : 0,
                                has_rand ? 1 : 0, n, plive, st));
    nl += 1;
    // timing only: which planes are reached, for the byte counts of the skipping kernels
    // (one small synchronisation per estimate)
    std::vector<int> hmask;
    std::vector<unsigned char> hlive;
    if (tm) {
        hmask.resize((size_t)3 * n);
        hlive.resize((size_t)3 * n * n);
        LPP_CUDA(cudaMemcpyAsync(hmask.data(), pmask, hmask.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
        LPP_CUDA(cudaMemcpyAsync(hlive.data(), plive, hlive.size(), cudaMemcpyDeviceToHost, st));
        LPP_CUDA(cudaStreamSynchronize(st));
    }
    auto live_at = [&](int bits, size_t zy) {
        int hit = 0;
        for (int r = 0; r < 3; ++r)
            if (bits & (1 << r)) hit |= hlive[(size_t)r * n * n + zy];
        return hit != 0;
    };
    // fraction of x pencils reached, and of fused tiles holding a reached pencil (those store)
    double memo_p[8], memo_t[8];
    for (int b = 0; b < 8; ++b) memo_p[b] = memo_t[b] = -1.0;
    auto pencil_frac = [&](int bits) -> double {
        if (hlive.empty() || bits == 0) return 1.0;
        if (memo_p[bits & 7] >= 0.0) return memo_p[bits & 7];
        long long c = 0;
        for (size_t zy = 0; zy < (size_t)n * n; ++zy) c += live_at(bits, zy);
        return memo_p[bits & 7] = (double)c / ((double)n * n);
    };
    auto tile_frac = [&](int bits) -> double {
        if (hlive.empty() || bits == 0) return 1.0;
        if (memo_t[bits & 7] >= 0.0) return memo_t[bits & 7];
        const int ty = plan->fty, tz = plan->ftz;
        long long c = 0, all = 0;
        for (int z0 = 0; z0 < n; z0 += tz)
            for (int y0 = 0; y0 < n; y0 += ty) {
                bool any = false;
                for (int dz = 0; dz < tz && !any; ++dz)
                    for (int dy = 0; dy < ty && !any; ++dy) any = live_at(bits, (size_t)(z0 + dz) * n + y0 + dy);
                c += any;
                ++all;
            }
        return memo_t[bits & 7] = (double)c / all;
    };
    auto plane_frac = [&](int bits) -> double {
        if (hmask.empty() || bits == 0) return 1.0;
        long long c = 0;
        for (int z = 0; z < n; ++z) {
            int hit = 0;
            for (int r = 0; r < 3; ++r)
                if (bits & (1 << r)) hit |= hmask[(size_t)r * n + z];
            c += hit != 0;
        }
        return (double)c / n;
    };

    r_step.next("lpp 1 harmonic weights");
    // 1. sky frames, shears and harmonic weights of the shape catalogue (in sorted order)
    CoeffArgs<T> ca;
    memset(&ca, 0, sizeof(ca));
    ca.perm = perm;
    ca.pos = (const T*)sh.pos;
    ca.w = (const T*)sh.w;
    ca.shape = (const T*)sh.shape;
    ca.count = sh.count;
    ca.shape_kind = sh.shape_kind;
    for (int a = 0; a < 3; ++a) {
        ca.observer[a] = plan->d.observer[a];
        ca.pole[a] = plan->d.pole[a];
        ca.los_global[a] = plan->d.los_global[a];
    }
    ca.los_proj = plan->d.los_proj;
    ca.los_est = plan->d.los_est;
    ca.coeff = coeff;
    ca.stride = stride;
    ca.n_groups = (int)plan->groups.size();
    for (int g = 0; g < ca.n_groups; ++g) ca.groups[g] = plan->groups[g];
    for (int qi = 0; qi < kQuadDegrees; ++qi) {
        bool used = false;
        for (const CoeffGroup& g : plan->groups) used = used || g.quad == qi;
        ca.quad_dirs[qi] = (const T*)(plan->ws + plan->off_quad_dirs[qi]);
        ca.quad_tab[qi] = (const T*)(plan->ws + plan->off_quad_tab[qi]);
        ca.quad_S[qi] = used ? plan->quad[qi].S : 0;
    }
    ca.polys = (const T*)(plan->ws + plan->off_polys);
    ca.n_polys = (int)plan->polys.size();
    ca.sums = sums;
    ca.err = err;
    if (sh.shape_kind != LPP_SHAPE_NONE) {
        if (tm) tm->begin(KK_COEFF, st);
        LPP_CUDA(launch_coeffs<T>(ca, st));
        nl += sh.count > 0 ? 1 : 0;
        if (tm) tm->end(KK_COEFF, st, (double)sh.count * plan->es * (3 + 1 + 6 + plan->n_coeff_rows));
        if (!plan->fp64) {
            if (tm) tm->begin(KK_OTHER, st);
            LPP_CUDA(launch_rowstat((const float*)coeff, stride, sh.count, plan->n_coeff_rows, rmax,
                                    (double*)(plan->ws + plan->off_rsq), st));
            nl += (sh.count > 0 && plan->n_coeff_rows > 0) ? 2 : 0;
            if (tm) tm->end(KK_OTHER, st, (double)sh.count * plan->n_coeff_rows * sizeof(float));
        }
    } else {
        if (tm) tm->begin(KK_OTHER, st);
        LPP_CUDA(launch_sums<T>((const T*)sh.w, nullptr, sh.count, sums, SUM_W_SHAPES, -1, -1, st));
        nl += sh.count > 0 ? 1 : 0;
        if (tm) tm->end(KK_OTHER, st, (double)sh.count * plan->es);
    }
    if (tm) tm->begin(KK_OTHER, st);
    LPP_CUDA(launch_sums<T>((const T*)de.w, nullptr, de.count, sums, SUM_W_DENS, SUM_W2_DENS, -1, st));
    nl += de.count > 0 ? 1 : 0;
    if (tm) tm->end(KK_OTHER, st, (double)de.count * plan->es);
    if (has_rand) {
        if (tm) tm->begin(KK_OTHER, st);
        LPP_CUDA(launch_sums<T>((const T*)ra.w, (const T*)ra.nbar, ra.count, sums, SUM_W_RAND, SUM_W2_RAND,
                                SUM_NW2_RAND, st));
        nl += ra.count > 0 ? 1 : 0;
        if (tm) tm->end(KK_OTHER, st, (double)ra.count * plan->es * 2);
    }
    if (tm) tm->begin(KK_OTHER, st);
    LPP_CUDA(launch_alpha(sums, has_rand ? 1 : 0, st));
    nl += 1;
    if (tm) tm->end(KK_OTHER, st, 0.0);

    const FftGeom& geom = plan->geom;
    const c2<T>* tw = (const c2<T>*)(plan->ws + plan->off_tw);
    CombineArgs<T> cb;
    memset(&cb, 0, sizeof(cb));
    cb.grids = grids;
    cb.grid_stride = (long long)n3;
    cb.n = n;
    cb.interlace = plan->d.interlace;
    cb.per_grid = plan->d.interlace ? 1 : 2;
    c2<T>* pG1 = partner;
    c2<T>* pG2 = plan->need_g ? partner + n3 : nullptr;
    c2<T>* pD = plan->need_d ? partner + (plan->need_g ? 2 : 0) * n3 : nullptr;
    if (!plan->need_g) pG1 = nullptr;
    cb.pD = pD;
    cb.pG1 = pG1;
    cb.pG2 = pG2;
    cb.inv_w = (const T*)(plan->ws + plan->off_iw);
    cb.phase = (const c2<T>*)(plan->ws + plan->off_ph);
    cb.thr = (const int*)(plan->ws + plan->off_thr);
    cb.nb = nb;
    cb.nk_pos = plan->nk_pos;
    cb.nk_neg = plan->nk_neg;
    cb.nky = plan->nky;
    cb.nzi = plan->nzi;
    cb.out = out;
    cb.err = err;
    cb.items = plan->items.empty() ? nullptr : (const int4*)(plan->ws + plan->off_items);
    cb.n_items = (int)plan->items.size();
    const int n_ch = (int)plan->channels.size();
    cb.row_dd0 = n_ch;
    cb.row_plus0 = n_ch + 1;

    FusedArgs<T> fa;
    memset(&fa, 0, sizeof(fa));
    for (int r = 0; r < 3; ++r) {
        fa.cat[r].su = plan->ws + plan->off_su[r];
        fa.cat[r].sw = plan->ws + plan->off_sw[r];
        fa.cat[r].off = (const int*)(plan->ws + plan->off_koff[r]);
        fa.cat[r].cap = caps[r];
    }
    fa.grids = grids;
    fa.grid_stride = (long long)n3;
    fa.n = n;
    fa.ty = plan->fty;
    fa.tz = plan->ftz;
    fa.scheme = plan->d.scheme;
    fa.interlace = plan->d.interlace;
    fa.nk_pos = plan->nk_pos;
    fa.nk_neg = plan->nk_neg;
    fa.tw = tw;
    fa.sums = sums;
    fa.pmask = pmask;
    fa.skip_empty = 1;
    fa.pstat = (int*)(plan->ws + plan->off_pstat);
    fa.err = err;
    // harmonic weights of the density multipole channels: line of sight from the observer
    // (or the global direction when the estimator uses one)
    for (int a = 0; a < 3; ++a) {
        fa.observer[a] = plan->d.observer[a];
        fa.origin[a] = plan->d.origin[a];
        fa.los_global[a] = plan->d.los_global[a];
    }
    fa.h = plan->box / n;
    fa.ylm_global = plan->d.los_est == LPP_LOS_GLOBAL ? 1 : 0;
    const double xbytes = (double)n * n * plan->nky * sizeof(c2<T>);   // kept x pencils of one grid
    auto slot_bits = [&](const FusedSlot& f) {
        int bits = 0;
        for (int q = 0; q < f.n_src; ++q) bits |= 1 << f.src[q].cat;
        return bits;
    };
    int* work = (int*)(plan->ws + plan->off_work);
    auto assign_fused = [&](long long particles) -> lpp_status {
        // one-slot passes over a tile-row list take (slot, tile) items dynamically
        fa.work = (!fa.dual && fa.trows) ? work : nullptr;
        if (fa.work) LPP_CUDA(cudaMemsetAsync(work, 0, sizeof(int), st));
        if (tm) tm->begin(KK_ASSIGN, st);
        LPP_CUDA(launch_assign_xfft<T>(fa, st));
        nl += fa.n_slots > 0 ? 1 : 0;
        if (fa.n_slots > 0) plan->n_fused[fa.dual ? 1 : 0] += 1;
        if (tm) {
            // kept x pencils are stored on the planes the slot's particles reach
            double wb = 0.0;
            for (int i = 0; i < fa.n_slots; ++i) wb += xbytes * tile_frac(slot_bits(fa.slots[i]));
            tm->end(KK_ASSIGN, st, wb + fa.n_slots * (double)particles * 4 * plan->es);
        }
        return LPP_OK;
    };

    // modes that fall in some shell: what the combine must read per field
    double shell_modes = 0.0;
    for (int b = 0; b < nb; ++b) shell_modes += (double)plan->n_modes[b];

    r_step.next("lpp 2 partner fields");
    // 2. partner fields: G1, G2 (shapes) and D = density - alpha randoms
    const int il = plan->d.interlace;
    const int dens_cat = plan->cat[LPP_DENSITY].set ? LPP_DENSITY : LPP_SHAPES;
    int pgrids = 0;
    {
        fa.n_slots = 0;
        long long parts = 0;
        if (plan->need_g) {
            if (il) {
                FusedSlot g1{};
                g1.n_src = 1;
                g1.src[0] = FusedSrc{LPP_SHAPES, coeff, 0};
                g1.grid = pgrids++;
                fa.slots[fa.n_slots++] = g1;
                FusedSlot g2{};
                g2.n_src = 1;
                g2.src[0] = FusedSrc{LPP_SHAPES, coeff + stride, 0};
                g2.grid = pgrids++;
                fa.slots[fa.n_slots++] = g2;
            } else {
                FusedSlot g{};
                g.n_src = 1;
                g.src[0] = FusedSrc{LPP_SHAPES, coeff, 0};
                g.vals_b = coeff + stride;
                g.grid = pgrids++;
                fa.slots[fa.n_slots++] = g;
            }
            parts += sh.count;
        }
        if (plan->need_d) {
            FusedSlot dsl{};
            dsl.n_src = 1;
            dsl.src[0] = FusedSrc{dens_cat, nullptr, 0};
            if (has_rand) dsl.src[dsl.n_src++] = FusedSrc{LPP_RANDOMS, nullptr, 1};
            // the density field data - alpha randoms accumulates in float atomics: it nearly
            // cancels over large scales, where a fixed-point quantum's rounding bias would show
            dsl.grid = pgrids++;
            fa.slots[fa.n_slots++] = dsl;
            parts += de.count + (has_rand ? ra.count : 0);
        }
        fa.trows = use_rows ? trows + 256 : nullptr;
        fa.trow_count = use_rows ? tcount + 1 : nullptr;
        // the slot with the most particles (D with the randoms) first: its tiles are the
        // first items of the dynamic schedule
        auto weight = [&](const FusedSlot& f) {
            long long w = 0;
            for (int q = 0; q < f.n_src; ++q) w += plan->cat[f.src[q].cat].count;
            return w;
        };
        std::stable_sort(fa.slots, fa.slots + fa.n_slots,
                         [&](const FusedSlot& x, const FusedSlot& y) { return weight(x) > weight(y); });
        { lpp_status s0 = assign_fused(parts); if (s0 != LPP_OK) return s0; }
        FftGeom gp = geom;
        gp.pmask = pmask;
        gp.err = err;
        gp.q_max = plan->thr[nb];
        double fr = 0.0;
        for (int i = 0; i < fa.n_slots; ++i) {
            gp.gmask[fa.slots[i].grid] = slot_bits(fa.slots[i]);
            fr += plane_frac(gp.gmask[fa.slots[i].grid]);
        }
        gp.yread_frac = fa.n_slots ? (float)(fr / fa.n_slots) : 1.0f;
        gp.plive = plive;
        double fl = 0.0;
        for (int i = 0; i < fa.n_slots; ++i) fl += pencil_frac(gp.gmask[fa.slots[i].grid]);
        gp.ylive_frac = fa.n_slots ? (float)(fl / fa.n_slots) : 1.0f;
        LPP_CUDA(fft_yz<T>(grids, pgrids, n, tw, gp, false, st, tm));
        nl += 2;
        cb.partner_mode = 1;
        cb.has_d = plan->need_d;
        cb.has_g = plan->need_g;
        cb.n_ch = 0;
        if (tm) tm->begin(KK_PARTNER, st);
        LPP_CUDA(launch_combine<T>(cb, plan->n_sm, st));
        nl += 1;
        if (tm) tm->end(KK_PARTNER, st, shell_modes * sizeof(c2<T>) * (pgrids + plan->n_partner));
    }

    r_step.next("lpp 3 channel batches");
    // 3. channel fields, a batch of grids at a time: the tensor channels (coefficient rows of
    // the shape catalogue), then the density multipole channels (harmonic weights of the density
    // catalogue and the randoms); a batch never mixes the two
    const int per_grid = il ? 1 : 2;
    cb.partner_mode = 0;
    const int n_tch = plan->n_tensor_ch;
    std::vector<std::pair<int, int>> batches;
    for (int c0 = 0; c0 < n_tch; c0 += plan->batch_ch) batches.push_back({c0, std::min(n_tch, c0 + plan->batch_ch)});
    for (int c0 = n_tch; c0 < n_ch; c0 += plan->batch_ch) batches.push_back({c0, std::min(n_ch, c0 + plan->batch_ch)});
    // range records of the shape tiles, shared by every two-slot channel launch
    int* tranges = nullptr;
    bool any_dual = false;
    for (const auto& bt : batches) any_dual |= bt.first < n_tch && (bt.second - bt.first) % 2 == 0;
    if (two_slot_grid(plan) && use_rows && any_dual) {
        tranges = (int*)(plan->ws + plan->off_tranges);
        FusedArgs<T> fr = fa;
        FusedSlot fs{};
        fs.n_src = 1;
        fs.src[0] = FusedSrc{LPP_SHAPES, nullptr, 0};
        fr.slots[0] = fs;
        fr.n_slots = 1;
        fr.trows = trows;
        fr.trow_count = tcount;
        if (tm) tm->begin(KK_OTHER, st);
        LPP_CUDA(launch_tile_ranges<T>(fr, tranges, st));
        nl += 1;
        if (tm) tm->end(KK_OTHER, st, (double)tile_range_bytes(n, plan->fty, plan->ftz) * tile_frac(1 << LPP_SHAPES));
    }
    for (const auto& bt : batches) {
        const int c0 = bt.first, c1 = bt.second;
        const bool dens = c0 >= n_tch;
        const int nch = c1 - c0;
        const int ngr = (nch + per_grid - 1) / per_grid;
        fa.n_slots = 0;
        cb.n_ch = nch;
        cb.has_d = 0;
        cb.has_g = 0;
        for (int gi = 0; gi < ngr; ++gi) {
            const int ca0 = c0 + gi * per_grid;
            FusedSlot fs{};
            if (dens) {
                fs.n_src = 1;
                fs.src[0] = FusedSrc{dens_cat, nullptr, 0};
                if (has_rand) fs.src[fs.n_src++] = FusedSrc{LPP_RANDOMS, nullptr, 1};
                const Channel& ca = plan->channels[ca0];
                fs.use_ylm = 1;
                fs.yl_a = ca.L;
                fs.yn_a = ca.n;
                fs.ynorm_a = ylm_norm(ca.L, ca.n);
                fs.yl_b = -1;
                if (!il && ca0 + 1 < c1) {
                    const Channel& cbb = plan->channels[ca0 + 1];
                    fs.yl_b = cbb.L;
                    fs.yn_b = cbb.n;
                    fs.ynorm_b = ylm_norm(cbb.L, cbb.n);
                }
            } else {
                fs.n_src = 1;
                fs.src[0] = FusedSrc{LPP_SHAPES, coeff + (long long)plan->channels[ca0].coeff * stride, 0};
                fs.vals_b = (!il && ca0 + 1 < c1) ? coeff + (long long)plan->channels[ca0 + 1].coeff * stride : nullptr;
                if (!plan->fp64) {
                    fs.amax_a = rmax + 2 * plan->channels[ca0].coeff;
                    fs.amax_b = fs.vals_b ? rmax + 2 * plan->channels[ca0 + 1].coeff : nullptr;
                }
            }
            fs.grid = gi;
            fa.slots[fa.n_slots++] = fs;
        }
        for (int ci = 0; ci < nch; ++ci) {
            const Channel& ch = plan->channels[c0 + ci];
            CombineChan& cc = cb.ch[ci];
            cc.slot = ci / per_grid;
            cc.sub = il ? 0 : ci % 2;
            cc.kind = ch.kind;
            cc.L = ch.L;
            cc.n = ch.n;
            cc.part = ch.part;
            cc.out_row = c0 + ci;
            cc.ynorm = ylm_norm_scaled(ch.L, ch.n);
            if (ch.kind == KIND_CROSS || ch.kind == KIND_DENS) cb.has_d = 1; else cb.has_g = 1;
        }
        const int bits = dens ? slot_bits(fa.slots[0]) : 1 << LPP_SHAPES;
        fa.trows = use_rows ? (dens ? trows + 256 : trows) : nullptr;
        fa.trow_count = use_rows ? (dens ? tcount + 1 : tcount) : nullptr;
        fa.dual = (!dens && tranges && fa.n_slots % 2 == 0) ? 1 : 0;
        fa.tranges = fa.dual ? tranges : nullptr;
        { lpp_status s0 = assign_fused(dens ? de.count + (has_rand ? ra.count : 0) : sh.count); if (s0 != LPP_OK) return s0; }
        fa.dual = 0;
        fa.tranges = nullptr;
        FftGeom gc = geom;
        gc.pmask = pmask;
        gc.err = err;
        gc.q_max = plan->thr[nb];
        for (int i = 0; i < ngr; ++i) gc.gmask[i] = bits;
        gc.yread_frac = (float)plane_frac(bits);
        gc.plive = plive;
        gc.ylive_frac = (float)pencil_frac(bits);
        LPP_CUDA(fft_yz<T>(grids, ngr, n, tw, gc, false, st, tm));
        if (tm) tm->begin(KK_COMBINE, st);
        LPP_CUDA(launch_combine<T>(cb, plan->n_sm, st));
        nl += 3;
        if (tm) tm->end(KK_COMBINE, st, shell_modes * sizeof(c2<T>) * (ngr + (cb.has_d ? 1 : 0) + (cb.has_g ? 2 : 0)));
    }

    r_step.next("lpp 4 results");
    // 4. results to the host
    LPP_CUDA(cudaMemcpyAsync(host_out, out, (size_t)plan->out_rows * nb * 2 * sizeof(double), cudaMemcpyDeviceToHost,
                             st));
    LPP_CUDA(cudaMemcpyAsync(host_sums, sums, SUM_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
    LPP_CUDA(cudaMemcpyAsync(host_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    return LPP_OK;
}

// Step 5 on the host from the copied sums (FP64): normalisation, shot noise, moment slots.
static lpp_status finish(lpp_plan_t plan, const double* h_out, const double* h_sums, int h_err, bool has_rand,
                         lpp_result* res) {
    const int nb = plan->nb;
    const int n_ch = (int)plan->channels.size();
    if (h_err & ERRF_BOUNDS)
        return fail(plan, LPP_ERR_BOUNDS, "a device index fell outside its buffer (checking build); access skipped");
    if (h_err) {
        std::string msg = "particle outside the domain:";
        if (h_err & ERRF_DOMAIN) msg += " outside the box";
        if (h_err & ERRF_POLE) msg += " on the frame pole";
        if (h_err & ERRF_OBSERVER) msg += " at the observer";
        return fail(plan, LPP_ERR_DOMAIN, msg);
    }

    // 5. normalisation and shot noise (host, FP64)
    const double vol = plan->box * plan->box * plan->box;
    const double alpha = h_sums[SUM_ALPHA];
    double i_auto, i_cross, i_dd, shot_dd_num;
    if (has_rand) {
        const double I = alpha * h_sums[SUM_NW2_RAND];
        i_auto = i_cross = i_dd = I;
        shot_dd_num = h_sums[SUM_W2_DENS] + alpha * alpha * h_sums[SUM_W2_RAND];
    } else {
        i_auto = h_sums[SUM_W_SHAPES] * h_sums[SUM_W_SHAPES] / vol;
        i_cross = h_sums[SUM_W_SHAPES] * h_sums[SUM_W_DENS] / vol;
        i_dd = h_sums[SUM_W_DENS] * h_sums[SUM_W_DENS] / vol;
        shot_dd_num = h_sums[SUM_W2_DENS];
    }
    if (plan->d.norm_override > 0) i_auto = i_cross = i_dd = plan->d.norm_override;
    const double shot_plus = plan->d.subtract_shot && i_auto != 0 ? h_sums[SUM_W2G2_SHAPES] / i_auto : 0.0;
    const double shot_dd = plan->d.subtract_shot && i_dd != 0 ? shot_dd_num / i_dd : 0.0;

    std::vector<double> mom((size_t)LPP_N_MOMENTS * nb * 2, 0.0);
    for (int c = 0; c < n_ch; ++c) {
        const int slot = plan->channels[c].moment;
        for (int k = 0; k < nb * 2; ++k) mom[(size_t)slot * nb * 2 + k] += h_out[(size_t)c * nb * 2 + k];
    }
    for (int k = 0; k < nb * 2; ++k) {
        mom[(size_t)LPP_MOM_DD0 * nb * 2 + k] = h_out[(size_t)n_ch * nb * 2 + k];
        mom[(size_t)LPP_MOM_PLUS0 * nb * 2 + k] = h_out[(size_t)(n_ch + 1) * nb * 2 + k];
    }
    const unsigned want = plan->d.moments;
    for (int s = 0; s < LPP_N_MOMENTS; ++s) {
        double C = 1.0, I = i_auto, shot = 0.0;
        if (s == LPP_MOM_DD0) { I = i_dd; shot = shot_dd; }
        else if (s == LPP_MOM_DD2 || s == LPP_MOM_DD4) { C = 4.0 * kPi; I = i_dd; }
        else if (s >= LPP_MOM_CROSS2 && s <= LPP_MOM_CROSS6) { C = norm_factor(2, 2 * s); I = i_cross; }
        else if (s >= LPP_MOM_PLUS0 && s <= LPP_MOM_PLUS4) {
            const int l = 2 * (s - LPP_MOM_PLUS0);
            C = 2.0 * l + 1.0;
            if (l == 0) shot = shot_plus;
        } else {
            const int Lm = s == LPP_MOM_MINUS10 ? 10 : s == LPP_MOM_MINUS12 ? 12 : 4 + 2 * (s - LPP_MOM_MINUS4);
            C = norm_factor(4, Lm);
        }
        const bool on = (want & (1u << s)) != 0;
        for (int b = 0; b < nb; ++b) {
            const size_t k = ((size_t)s * nb + b) * 2;
            const double nm = (double)plan->n_modes[b];
            const double rre = on && nm > 0 ? C * mom[k] / nm : 0.0;
            const double rim = on && nm > 0 ? C * mom[k + 1] / nm : 0.0;
            if (res->raw) { res->raw[k] = rre; res->raw[k + 1] = rim; }
            if (res->p) {
                res->p[k] = on && I != 0 ? rre / I - (nm > 0 ? shot : 0.0) : 0.0;
                res->p[k + 1] = on && I != 0 ? rim / I : 0.0;
            }
        }
    }
    if (res->k_mean) for (int b = 0; b < nb; ++b) res->k_mean[b] = plan->k_mean[b];
    if (res->n_modes) for (int b = 0; b < nb; ++b) res->n_modes[b] = plan->n_modes[b];
    res->norm_auto = i_auto;
    res->norm_cross = i_cross;
    res->norm_dd = i_dd;
    res->shot_plus = shot_plus;
    res->shot_dd = shot_dd;
    res->alpha = alpha;
    return LPP_OK;
}

static lpp_status enqueue_any(lpp_plan_t plan, double* host_out, double* host_sums, int* host_err) {
    return plan->fp64 ? enqueue<double>(plan, host_out, host_sums, host_err)
                      : enqueue<float>(plan, host_out, host_sums, host_err);
}

extern "C" lpp_status lpp_multipoles(lpp_plan_t plan, lpp_result* res) {
    if (!plan || !res) return LPP_ERR_INVALID_ARG;
    if (!plan->ws || !plan->tables_ready) return fail(plan, LPP_ERR_NOT_READY, "workspace not set");
    if (!plan->cat[LPP_SHAPES].set) return fail(plan, LPP_ERR_NOT_READY, "no shape catalogue assigned");
    plan->err.clear();
    Timer* tm = plan->timer.enabled ? &plan->timer : nullptr;
    if (tm) tm->reset();
    std::vector<double> h_out((size_t)plan->out_rows * plan->nb * 2);
    double h_sums[SUM_COUNT];
    int h_err = 0;
    lpp_status s = enqueue_any(plan, h_out.data(), h_sums, &h_err);
    if (s != LPP_OK) return s;
    LPP_CUDA(cudaStreamSynchronize(plan->stream));
    if (tm) tm->collect();
    return finish(plan, h_out.data(), h_sums, h_err, plan->cat[LPP_RANDOMS].set, res);
}

// ------------------------------------------------------------------ window multipoles
template <typename T>
static lpp_status run_window(lpp_plan_t plan, int nb, const double* s_edges, double* q, double* s_mean,
                             long long* n_points, double* norm_out) {
    NvtxRange r_win("lpp window multipoles");
    const int n = plan->n;
    const size_t n3 = (size_t)n * n * n;
    const double h = plan->box / n;
    cudaStream_t st = plan->stream;
    std::vector<int> thr;
    shell_thresholds(n, h, s_edges, nb, thr);
    const int tmax = thr[nb];
    int ns = 0;
    while ((long long)(ns + 1) * (ns + 1) < tmax && ns < n / 2) ++ns;
    const int ns_pos = std::min(ns, n / 2 - 1), ns_neg = std::min(ns, n / 2);
    const int nks = ns_pos + 1 + ns_neg;
    // separation points per shell and their mean |s|
    std::vector<long long> npts(nb, 0);
    std::vector<double> ssum(nb, 0.0);
    for (int fx = -ns_neg; fx <= ns_pos; ++fx)
        for (int fy = -ns_neg; fy <= ns_pos; ++fy)
            for (int fz = -ns_neg; fz <= ns_pos; ++fz) {
                const long long qq = (long long)fx * fx + (long long)fy * fy + (long long)fz * fz;
                if (qq == 0 || qq < thr[0] || qq >= tmax) continue;
                int lo = 0, hi = nb;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) / 2;
                    if (qq >= thr[mid]) lo = mid; else hi = mid;
                }
                ++npts[lo];
                ssum[lo] += h * sqrt((double)qq);
            }
    double* sums = (double*)(plan->ws + plan->off_sums);
    int* err = (int*)(plan->ws + plan->off_err);
    double* wout = (double*)(plan->ws + plan->off_wout);
    c2<T>* grids = (c2<T>*)(plan->ws + plan->off_grids);
    c2<T>* pW = (c2<T>*)(plan->ws + plan->off_partner);
    const c2<T>* tw = (const c2<T>*)(plan->ws + plan->off_tw);
    const T* iw = (const T*)(plan->ws + plan->off_iw);
    const Catalogue& ra = plan->cat[LPP_RANDOMS];
    const Catalogue& de = plan->cat[LPP_DENSITY].set ? plan->cat[LPP_DENSITY] : plan->cat[LPP_SHAPES];
    LPP_CUDA(cudaMemsetAsync(sums, 0, SUM_COUNT * sizeof(double), st));
    LPP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    LPP_CUDA(cudaMemsetAsync(wout, 0, (size_t)kWindowChannels * nb * 2 * sizeof(double), st));
    LPP_CUDA(cudaMemcpyAsync(plan->ws + plan->off_wthr, thr.data(), (nb + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    if (de.set) LPP_CUDA(launch_sums<T>((const T*)de.w, nullptr, de.count, sums, SUM_W_DENS, -1, -1, st));
    LPP_CUDA(launch_sums<T>((const T*)ra.w, (const T*)ra.nbar, ra.count, sums, SUM_W_RAND, SUM_W2_RAND, SUM_NW2_RAND, st));
    const long long cap = std::max<long long>(1, plan->d.max_randoms);
    LPP_CUDA(launch_pencil_sort<T>((const T*)ra.pos, (const T*)ra.w, ra.count, cap, n, plan->box, plan->d.origin,
                                   (int*)(plan->ws + plan->off_key[LPP_RANDOMS]), (int*)(plan->ws + plan->off_counts),
                                   (int*)(plan->ws + plan->off_koff[LPP_RANDOMS]),
                                   (int*)(plan->ws + plan->off_cursor), (int*)(plan->ws + plan->off_scan),
                                   (T*)(plan->ws + plan->off_su[LPP_RANDOMS]),
                                   (T*)(plan->ws + plan->off_sw[LPP_RANDOMS]), nullptr, err, st));
    // forward transforms keep every frequency; the inverse keeps the separations of the shells
    FftGeom gfull = fft_geometry(n, n / 2 - 1, n / 2);
    FftGeom gs = fft_geometry(n, ns_pos, ns_neg);
    gfull.err = err;
    gs.err = err;
    FusedArgs<T> fa;
    memset(&fa, 0, sizeof(fa));
    fa.err = err;
    fa.cat[LPP_RANDOMS].su = plan->ws + plan->off_su[LPP_RANDOMS];
    fa.cat[LPP_RANDOMS].sw = plan->ws + plan->off_sw[LPP_RANDOMS];
    fa.cat[LPP_RANDOMS].off = (const int*)(plan->ws + plan->off_koff[LPP_RANDOMS]);
    fa.cat[LPP_RANDOMS].cap = cap;
    fa.grids = grids;
    fa.grid_stride = (long long)n3;
    fa.n = n;
    fa.ty = plan->fty;
    fa.tz = plan->ftz;
    fa.scheme = plan->d.scheme;
    fa.interlace = 0;
    fa.nk_pos = n / 2 - 1;
    fa.nk_neg = n / 2;
    fa.tw = tw;
    fa.sums = sums;
    for (int a = 0; a < 3; ++a) { fa.observer[a] = plan->d.observer[a]; fa.origin[a] = plan->d.origin[a]; }
    fa.h = h;
    // the window field W itself: transformed and deconvolved into the partner array
    fa.n_slots = 1;
    FusedSlot ws{};
    ws.n_src = 1;
    ws.src[0] = FusedSrc{LPP_RANDOMS, nullptr, 0};
    ws.grid = 0;
    ws.yl_a = ws.yl_b = -1;
    fa.slots[0] = ws;
    LPP_CUDA(launch_assign_xfft<T>(fa, st));
    LPP_CUDA(fft_yz<T>(grids, 1, n, tw, gfull, false, st, nullptr));
    LPP_CUDA(launch_window_partner<T>(grids, pW, iw, n, st));
    // channels (l, m), two per grid
    int chl[kWindowChannels], chm[kWindowChannels], nchan = 0;
    for (int l = 0; l <= 8; l += 2)
        for (int m = -l; m <= l; ++m) { chl[nchan] = l; chm[nchan] = m; ++nchan; }
    const int per_batch = std::min(2 * plan->batch, kMaxBatchCh);
    SbinArgs<T> sb;
    memset(&sb, 0, sizeof(sb));
    sb.grids = grids;
    sb.grid_stride = (long long)n3;
    sb.n = n;
    sb.thr = (const int*)(plan->ws + plan->off_wthr);
    sb.nb = nb;
    sb.ns_pos = ns_pos;
    sb.ns_neg = ns_neg;
    sb.nks = nks;
    sb.scale = 1.0 / (double)n3;
    sb.out = wout;
    for (int c0 = 0; c0 < nchan; c0 += per_batch) {
        const int c1 = std::min(nchan, c0 + per_batch);
        const int ngr = (c1 - c0 + 1) / 2;
        fa.n_slots = 0;
        sb.n_ch = 0;
        for (int gi = 0; gi < ngr; ++gi) {
            const int a0 = c0 + 2 * gi, a1 = a0 + 1;
            FusedSlot fs{};
            fs.n_src = 1;
            fs.src[0] = FusedSrc{LPP_RANDOMS, nullptr, 0};
            fs.grid = gi;
            fs.use_ylm = 1;
            fs.yl_a = chl[a0];
            fs.yn_a = chm[a0];
            fs.ynorm_a = ylm_norm(chl[a0], chm[a0]);
            fs.yl_b = a1 < c1 ? chl[a1] : -1;
            fs.yn_b = a1 < c1 ? chm[a1] : 0;
            fs.ynorm_b = a1 < c1 ? ylm_norm(chl[a1], chm[a1]) : 0.0;
            fa.slots[fa.n_slots++] = fs;
            for (int sub = 0; sub < 2; ++sub) {
                const int ci = sub ? a1 : a0;
                if (ci >= c1) continue;
                SbinChan& sc = sb.ch[sb.n_ch++];
                sc.grid = gi;
                sc.sub = sub;
                sc.l = chl[ci];
                sc.m = chm[ci];
                sc.out_row = ci;
                sc.ynorm = ylm_norm(chl[ci], chm[ci]);
            }
        }
        LPP_CUDA(launch_assign_xfft<T>(fa, st));
        LPP_CUDA(fft_yz<T>(grids, ngr, n, tw, gfull, false, st, nullptr));
        LPP_CUDA(launch_window_mult<T>(grids, (long long)n3, ngr, pW, iw, n, st));
        LPP_CUDA(fft3d<T>(grids, ngr, n, tw, gs, true, st, nullptr));
        LPP_CUDA(launch_sbin<T>(sb, plan->n_sm, st));
    }
    std::vector<double> h_out((size_t)kWindowChannels * nb * 2);
    double h_sums[SUM_COUNT];
    int h_err = 0;
    LPP_CUDA(cudaMemcpyAsync(h_out.data(), wout, h_out.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    LPP_CUDA(cudaMemcpyAsync(h_sums, sums, sizeof(h_sums), cudaMemcpyDeviceToHost, st));
    LPP_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LPP_CUDA(cudaStreamSynchronize(st));
    if (h_err & ERRF_BOUNDS)
        return fail(plan, LPP_ERR_BOUNDS, "a device index fell outside its buffer (checking build); access skipped");
    if (h_err) return fail(plan, LPP_ERR_DOMAIN, "random outside the box");
    const double alpha = (de.set && h_sums[SUM_W_RAND] != 0.0) ? h_sums[SUM_W_DENS] / h_sums[SUM_W_RAND] : 1.0;
    const double I = alpha * h_sums[SUM_NW2_RAND];
    const double fac = (I != 0.0) ? 4.0 * kPi * alpha * alpha / (h * h * h * I) : 0.0;
    for (int li = 0; li < 5; ++li)
        for (int b = 0; b < nb; ++b) {
            double v = 0.0;
            for (int ci = 0; ci < nchan; ++ci)
                if (chl[ci] == 2 * li) v += h_out[((size_t)ci * nb + b) * 2];
            q[li * nb + b] = npts[b] > 0 ? fac * v / (double)npts[b] : 0.0;
        }
    for (int b = 0; b < nb; ++b) {
        if (s_mean) s_mean[b] = npts[b] > 0 ? ssum[b] / npts[b] : 0.0;
        if (n_points) n_points[b] = npts[b];
    }
    if (norm_out) *norm_out = I;
    return LPP_OK;
}

extern "C" lpp_status lpp_window_Q(lpp_plan_t plan, int n_s, const double* s_edges, double* q, double* s_mean,
                                   long long* n_points, double* norm) {
    if (!plan || !s_edges || !q || n_s < 1 || n_s > 256) return LPP_ERR_INVALID_ARG;
    for (int i = 0; i < n_s; ++i)
        if (!(s_edges[i] < s_edges[i + 1])) return LPP_ERR_INVALID_ARG;
    if (!plan->ws || !plan->tables_ready) return fail(plan, LPP_ERR_NOT_READY, "workspace not set");
    if (!plan->cat[LPP_RANDOMS].set) return fail(plan, LPP_ERR_NOT_READY, "no randoms assigned");
    plan->err.clear();
    return plan->fp64 ? run_window<double>(plan, n_s, s_edges, q, s_mean, n_points, norm)
                      : run_window<float>(plan, n_s, s_edges, q, s_mean, n_points, norm);
}

extern "C" lpp_status lpp_plan_path_stats(lpp_plan_t plan, long long* stats) {
    if (!plan || !stats) return LPP_ERR_INVALID_ARG;
    if (!plan->ws) return fail(plan, LPP_ERR_NOT_READY, "workspace not set");
    int dev[4] = {0, 0, 0, 0};
    LPP_CUDA(cudaMemcpyAsync(dev, plan->ws + plan->off_pstat, sizeof(dev), cudaMemcpyDeviceToHost, plan->stream));
    LPP_CUDA(cudaStreamSynchronize(plan->stream));
    stats[0] = plan->n_fused[0];
    stats[1] = plan->n_fused[1];
    for (int i = 0; i < 4; ++i) stats[2 + i] = dev[i];
    return LPP_OK;
}

extern "C" const char* lpp_status_string(lpp_status s) {
    switch (s) {
        case LPP_OK: return "ok";
        case LPP_ERR_INVALID_ARG: return "invalid argument";
        case LPP_ERR_CUDA: return "CUDA error";
        case LPP_ERR_NOT_READY: return "not ready";
        case LPP_ERR_WORKSPACE: return "workspace too small";
        case LPP_ERR_UNSUPPORTED: return "unsupported";
        case LPP_ERR_DOMAIN: return "particle outside the domain";
        case LPP_ERR_BOUNDS: return "device index out of bounds (checking build)";
    }
    return "unknown status";
}

extern "C" const char* lpp_plan_last_error(lpp_plan_t plan) { return plan ? plan->err.c_str() : ""; }

// ------------------------------------------------------------------ batches of catalogues
struct lpp_batch_s {
    std::vector<lpp_plan_t> plans;
    std::vector<int> plan_of;
    std::vector<Catalogue> shapes, randoms;
    std::vector<cudaStream_t> streams;       // one per plan (the batch's own)
    std::vector<cudaEvent_t> done;           // one per plan
    cudaEvent_t start = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;   // ordering against the caller's stream
    cudaStream_t root = nullptr;
    double* h_out = nullptr;                 // pinned: per mock [out_rows][nb][2]
    double* h_sums = nullptr;                // pinned: per mock [SUM_COUNT]
    int* h_err = nullptr;                    // pinned: per mock
    std::vector<size_t> out_off;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool launched = false;
    long long n_launch = 0;                  // kernels the mocks' estimates enqueued
    std::string err;
};

static lpp_status batch_fail(lpp_batch_t b, lpp_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}

#define LPP_BCUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return batch_fail(b, LPP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// All mocks, each on its plan's batch stream (mocks of one plan in order, plans concurrently).
static lpp_status batch_enqueue(lpp_batch_t b, cudaStream_t root) {
    NvtxRange r_batch("lpp batch");
    LPP_BCUDA(cudaEventRecord(b->start, root));
    for (size_t p = 0; p < b->plans.size(); ++p) LPP_BCUDA(cudaStreamWaitEvent(b->streams[p], b->start, 0));
    b->n_launch = 0;
    for (size_t j = 0; j < b->plan_of.size(); ++j) {
        const int pi = b->plan_of[j];
        lpp_plan_t plan = b->plans[pi];
        const cudaStream_t keep = plan->stream;
        const bool timing = plan->timer.enabled;
        plan->stream = b->streams[pi];
        plan->timer.enabled = false;
        plan->cat[LPP_SHAPES] = b->shapes[j];
        plan->cat[LPP_DENSITY] = Catalogue();
        plan->cat[LPP_RANDOMS] = b->randoms[j];
        const lpp_status s = enqueue_any(plan, b->h_out + b->out_off[j], b->h_sums + j * SUM_COUNT, b->h_err + j);
        plan->stream = keep;
        plan->timer.enabled = timing;
        if (s != LPP_OK) return batch_fail(b, s, "mock " + std::to_string(j) + ": " + plan->err);
        b->n_launch += plan->n_launch;
    }
    for (size_t p = 0; p < b->plans.size(); ++p) {
        LPP_BCUDA(cudaEventRecord(b->done[p], b->streams[p]));
        LPP_BCUDA(cudaStreamWaitEvent(root, b->done[p], 0));
    }
    return LPP_OK;
}

extern "C" void lpp_batch_destroy(lpp_batch_t b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t s : b->streams) if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->done) if (e) cudaEventDestroy(e);
    if (b->start) cudaEventDestroy(b->start);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->root) cudaStreamDestroy(b->root);
    if (b->h_out) cudaFreeHost(b->h_out);
    if (b->h_sums) cudaFreeHost(b->h_sums);
    if (b->h_err) cudaFreeHost(b->h_err);
    delete b;
}

static bool catalogue_of(lpp_plan_t plan, int role, const lpp_particles* p, Catalogue* c) {
    const long long cap = role == LPP_SHAPES ? plan->d.max_shapes : plan->d.max_randoms;
    if (p->count < 0 || p->count > cap || p->on_host) return false;
    if (p->count > 0 && !p->pos) return false;
    const int sk = role == LPP_SHAPES ? p->shape_kind : LPP_SHAPE_NONE;
    if (role == LPP_SHAPES && (sk != LPP_SHAPE_GAMMA12 && sk != LPP_SHAPE_TENSOR6)) return false;
    if (sk != LPP_SHAPE_NONE && p->count > 0 && !p->shape) return false;
    c->set = true;
    c->count = p->count;
    c->shape_kind = sk;
    c->pos = p->pos;
    c->w = p->w;
    c->nbar = role == LPP_RANDOMS ? p->nbar : nullptr;
    c->shape = sk != LPP_SHAPE_NONE ? p->shape : nullptr;
    return true;
}

extern "C" lpp_status lpp_batch_create(lpp_plan_t* plans, int n_plans, const int* plan_of, const lpp_particles* shapes,
                                       const lpp_particles* randoms, int n_mocks, int use_graph, lpp_batch_t* out) {
    if (!out || !plans || n_plans < 1 || !plan_of || !shapes || n_mocks < 1) return LPP_ERR_INVALID_ARG;
    *out = nullptr;
    for (int p = 0; p < n_plans; ++p) {
        if (!plans[p]) return LPP_ERR_INVALID_ARG;
        if (!plans[p]->ws || !plans[p]->tables_ready) return LPP_ERR_NOT_READY;
        for (int q = 0; q < p; ++q) if (plans[q] == plans[p]) return LPP_ERR_INVALID_ARG;
    }
    lpp_batch_t b = new lpp_batch_s();
    b->plans.assign(plans, plans + n_plans);
    size_t total = 0;
    for (int j = 0; j < n_mocks; ++j) {
        const int pi = plan_of[j];
        if (pi < 0 || pi >= n_plans) { lpp_batch_destroy(b); return LPP_ERR_INVALID_ARG; }
        Catalogue cs, cr;
        if (!catalogue_of(plans[pi], LPP_SHAPES, &shapes[j], &cs) ||
            (randoms && randoms[j].count > 0 && !catalogue_of(plans[pi], LPP_RANDOMS, &randoms[j], &cr))) {
            lpp_batch_destroy(b);
            return LPP_ERR_INVALID_ARG;
        }
        b->plan_of.push_back(pi);
        b->shapes.push_back(cs);
        b->randoms.push_back(cr);
        b->out_off.push_back(total);
        total += (size_t)plans[pi]->out_rows * plans[pi]->nb * 2;
    }
    const lpp_status bad = LPP_ERR_CUDA;
    if (cudaHostAlloc((void**)&b->h_out, total * sizeof(double), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&b->h_sums, (size_t)n_mocks * SUM_COUNT * sizeof(double), cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaHostAlloc((void**)&b->h_err, (size_t)n_mocks * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        lpp_batch_destroy(b);
        return bad;
    }
    b->streams.resize(n_plans, nullptr);
    b->done.resize(n_plans, nullptr);
    bool ok = cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
    for (int p = 0; ok && p < n_plans; ++p)
        ok = cudaStreamCreateWithFlags(&b->streams[p], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->done[p], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { lpp_batch_destroy(b); return bad; }
    if (use_graph) {
        if (cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            lpp_batch_destroy(b);
            return bad;
        }
        const lpp_status s = batch_enqueue(b, b->root);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->root, &g);
        if (s != LPP_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            lpp_batch_destroy(b);
            return s != LPP_OK ? s : bad;
        }
        b->graph = g;
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) { lpp_batch_destroy(b); return bad; }
    }
    *out = b;
    return LPP_OK;
}

extern "C" lpp_status lpp_batch_launch(lpp_batch_t b, void* stream) {
    if (!b) return LPP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // order after the caller's stream, run on the batch's root stream
    LPP_BCUDA(cudaEventRecord(b->ev_in, st));
    LPP_BCUDA(cudaStreamWaitEvent(b->root, b->ev_in, 0));
    if (b->exec) {
        LPP_BCUDA(cudaGraphLaunch(b->exec, b->root));
    } else {
        const lpp_status s = batch_enqueue(b, b->root);
        if (s != LPP_OK) return s;
    }
    LPP_BCUDA(cudaEventRecord(b->ev_out, b->root));
    LPP_BCUDA(cudaStreamWaitEvent(st, b->ev_out, 0));
    b->launched = true;
    return LPP_OK;
}

extern "C" lpp_status lpp_batch_results(lpp_batch_t b, lpp_result* results) {
    if (!b || !results) return LPP_ERR_INVALID_ARG;
    if (!b->launched) return batch_fail(b, LPP_ERR_NOT_READY, "batch not launched");
    LPP_BCUDA(cudaStreamSynchronize(b->root));
    lpp_status first = LPP_OK;
    for (size_t j = 0; j < b->plan_of.size(); ++j) {
        lpp_plan_t plan = b->plans[b->plan_of[j]];
        const lpp_status s = finish(plan, b->h_out + b->out_off[j], b->h_sums + j * SUM_COUNT, b->h_err[j],
                                    b->randoms[j].set, &results[j]);
        if (s != LPP_OK && first == LPP_OK) {
            first = s;
            b->err = "mock " + std::to_string(j) + ": " + plan->err;
        }
    }
    return first;
}

extern "C" const char* lpp_batch_last_error(lpp_batch_t b) { return b ? b->err.c_str() : "null batch"; }

extern "C" lpp_status lpp_plan_launch_count(lpp_plan_t plan, long long* launches) {
    if (!plan || !launches) return LPP_ERR_INVALID_ARG;
    *launches = plan->n_launch;
    return LPP_OK;
}

extern "C" lpp_status lpp_batch_launch_count(lpp_batch_t b, long long* counted, long long* graph_kernels) {
    if (!b || !counted || !graph_kernels) return LPP_ERR_INVALID_ARG;
    *counted = b->n_launch;
    *graph_kernels = -1;
    if (b->graph) {
        size_t num = 0;
        LPP_BCUDA(cudaGraphGetNodes(b->graph, nullptr, &num));
        std::vector<cudaGraphNode_t> nodes(num);
        if (num) LPP_BCUDA(cudaGraphGetNodes(b->graph, nodes.data(), &num));
        long long k = 0;
        for (size_t i = 0; i < num; ++i) {
            cudaGraphNodeType t;
            LPP_BCUDA(cudaGraphNodeGetType(nodes[i], &t));
            if (t == cudaGraphNodeTypeKernel) ++k;
        }
        *graph_kernels = k;
    }
    return LPP_OK;
}
