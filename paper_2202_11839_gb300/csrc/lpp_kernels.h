// Launch interfaces of the liblpp kernels (internal).
#pragma once

#include "lpp_internal.h"

namespace lpp {

// ------------------------------------------------------------------------ timing
// Optional CUDA-event timing of individual launches on the launching stream.
struct Timer {
    static constexpr int kMaxEvents = 2048;
    bool enabled = false;
    int used = 0;
    cudaEvent_t ev[kMaxEvents];
    int kind[kMaxEvents / 2];
    double bytes[kMaxEvents / 2];
    bool created = false;
    double ms[KK_COUNT];
    long long launches[KK_COUNT];
    double total_bytes[KK_COUNT];

    void reset() {
        used = 0;
        for (int k = 0; k < KK_COUNT; ++k) { ms[k] = 0; launches[k] = 0; total_bytes[k] = 0; }
    }
    void begin(int k, cudaStream_t st) {
        if (!enabled || used + 2 > kMaxEvents) return;
        cudaEventRecord(ev[used], st);
        kind[used / 2] = k;
    }
    void end(int k, cudaStream_t st, double b) {
        if (!enabled || used + 2 > kMaxEvents) return;
        cudaEventRecord(ev[used + 1], st);
        bytes[used / 2] = b;
        (void)k;
        used += 2;
    }
    // after the stream is synchronised
    void collect() {
        for (int i = 0; i < used; i += 2) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
            ms[kind[i / 2]] += t;
            launches[kind[i / 2]] += 1;
            total_bytes[kind[i / 2]] += bytes[i / 2];
        }
        used = 0;
    }
};

// ------------------------------------------------------------------------- FFT
struct FftGeom {
    int W;       // pencils per CTA
    int nk_pos;  // kept frequencies 0..nk_pos
    int nk_neg;  // kept frequencies -nk_neg..-1
    int ntx;     // kept x tiles (of W columns)
    int nlo;     // x tiles taken from the low end
    int nky;     // kept y indices
    // optional skipping of empty z planes in the y pass: pmask [3][n] (per catalogue role,
    // nonzero where a particle of that role can reach plane z) and, per grid of the call,
    // the bit set of roles assigned to it (0: never skip)
    const int* pmask = nullptr;
    int gmask[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float yread_frac = 1.0f;   // host bookkeeping: fraction of z planes the y pass writes
    float ylive_frac = 1.0f;   // host bookkeeping: fraction of x pencils the y pass reads
    // z pass: skip (kx, ky) columns whose every mode has |f|^2 >= q_max (beyond the last
    // shell; never read by the combine); 0 transforms every column
    int q_max = 0;
    // optional per-pencil reach [3][n*n] bytes (role, z * n + y): the y pass reads zeros for
    // x pencils that no particle of the grid's roles reaches (the fused pass stores nothing there)
    const unsigned char* plive = nullptr;
    int* err = nullptr;   // ERRF_BOUNDS of LPP_CHECK builds
};

int fft_tile_width(int n);
FftGeom fft_geometry(int n, int nk_pos, int nk_neg);
template <typename T>
cudaError_t fft3d(c2<T>* data, int n_grids, int n, const c2<T>* tw, const FftGeom& g, bool inverse,
                  cudaStream_t st, Timer* timer);
// y and z passes only (the x pass fused into the assignment kernel)
template <typename T>
cudaError_t fft_yz(c2<T>* data, int n_grids, int n, const c2<T>* tw, const FftGeom& g, bool inverse,
                   cudaStream_t st, Timer* timer);

// ---------------------------------------------------------- per-particle weights
constexpr int kMaxGroups = 16;
constexpr int kQuadDegrees = 6;    // harmonic projection quadratures for L = 2, 4, ..., 12
constexpr int kMaxSlots = 8;       // complex grids per batch (FftGeom::gmask has as many)
constexpr int kMaxBatchCh = 16;    // real fields per batch

struct CoeffGroup {
    int kind;    // Kind
    int L;
    int has_im;  // also project the imaginary part of the kernel
    int row_re;  // first coefficient row of the real part (rows row_re + n + L)
    int row_im;  // first row of the imaginary part
    int poly;    // offset of the mu-polynomial in the poly table
    int npoly;   // number of coefficients
    int quad;    // index into the quadrature table list (L/2 - 1)
};

template <typename T>
struct CoeffArgs {
    const int* perm;    // optional: particle i of the output order is input perm[i]
    const T* pos;       // [3][count]
    const T* w;         // [count] or null
    const T* shape;     // [6 or 2][count]
    long long count;
    int shape_kind;
    double observer[3];
    double pole[3];
    double los_global[3];
    int los_proj, los_est;
    T* coeff;           // [rows][stride]
    long long stride;
    int n_groups;
    CoeffGroup groups[kMaxGroups];
    const T* quad_dirs[kQuadDegrees];   // per L = 2,4,...,12: [S][3]
    const T* quad_tab[kQuadDegrees];    // per L: [2L+1][S]
    int quad_S[kQuadDegrees];           // 0 for a degree no group of the plan uses
    const T* polys;          // concatenated mu-polynomial coefficients
    int n_polys;
    double* sums;            // FP64 reductions (see SumSlot)
    int* err;
};

enum SumSlot {
    SUM_W_SHAPES = 0, SUM_W2G2_SHAPES = 1, SUM_W_DENS = 2, SUM_W2_DENS = 3,
    SUM_W_RAND = 4, SUM_NW2_RAND = 5, SUM_W2_RAND = 6, SUM_ALPHA = 7, SUM_COUNT = 8
};

// error flag bits
enum { ERRF_DOMAIN = 1, ERRF_POLE = 2, ERRF_OBSERVER = 4, ERRF_BOUNDS = 8 };

// Bounds checks of LPP_CHECK builds (build.build(check=True), liblpp_check.so): there a false
// condition records ERRF_BOUNDS in *err (the estimate then fails with LPP_ERR_BOUNDS) and the
// caller skips the access instead of faulting; in other builds the condition is not evaluated.
#ifdef LPP_CHECK
__device__ __forceinline__ bool lpp_in_bounds(bool ok, int* err) {
    if (!ok && err) atomicOr(err, (int)ERRF_BOUNDS);
    return ok;
}
#define LPP_IN_BOUNDS(cond, err) ::lpp::lpp_in_bounds((cond), (err))
#else
#define LPP_IN_BOUNDS(cond, err) true
#endif

template <typename T>
cudaError_t launch_coeffs(const CoeffArgs<T>& a, cudaStream_t st);
// rstat[2r] = max_i |coeff[r * stride + i]|, rstat[2r + 1] = rms over i < count, for r < rows
// (rsq: FP64 scratch of rows entries)
cudaError_t launch_rowstat(const float* coeff, long long stride, long long count, int rows, float* rstat,
                           double* rsq, cudaStream_t st);

// plain weight sums of a catalogue: sums[s_w] += w, sums[s_w2] += w^2, sums[s_nw2] += nbar w^2
template <typename T>
cudaError_t launch_sums(const T* w, const T* nbar, long long count, double* sums, int s_w, int s_w2, int s_nw2,
                        cudaStream_t st);
cudaError_t launch_alpha(double* sums, int has_randoms, cudaStream_t st);

// --------------------------------------------------------------------- assignment
struct AssignSlot {
    const void* src_a;   // values for the real part (sub-grid 0), or the field a
    const void* src_b;   // values for the imaginary part when not interlaced (field b), may be null
    int grid;            // grid index in the batch
    int scale_alpha;     // multiply the values by -alpha (randoms into the density field)
    int unit_a;          // src_a is null: value 1 for every particle
};

template <typename T>
struct AssignArgs {
    const T* pos;
    long long count;
    c2<T>* grids;
    long long grid_stride;
    int n;
    double box;
    double origin[3];
    int n_slots;
    AssignSlot slots[kMaxSlots];
    const double* sums;   // for alpha
    int* err;
};

template <typename T>
cudaError_t launch_assign(const AssignArgs<T>& a, int scheme, int interlace, cudaStream_t st);

// ---------------------------------------------------- pencil sort + fused assign/x-FFT
// Catalogue sorted by x-pencil key: cell coordinates su[3][cap], weights sw[cap],
// offsets off[n*n + 1] of every key.
struct PencilCat {
    const void* su;
    const void* sw;
    const int* off;
    long long cap;
};
struct FusedSrc {
    int cat;            // index into FusedArgs::cat
    const void* vals;   // per-particle values in sorted order, or null for the sorted weights
    int neg_alpha;      // multiply by -alpha (randoms into the density field)
};
struct FusedSlot {
    int n_src;
    FusedSrc src[2];
    const void* vals_b;  // non-interlaced: second field (same catalogue as src[0]) in the imaginary part
    int grid;
    // optional real-harmonic weights Y_{l,n}(xhat) of the line of sight for the real-part
    // field and (yl_b >= 0) a second field from the same values (window multipoles);
    // use_ylm = 0 (the value-initialised default) disables both
    int use_ylm;
    int yl_a, yn_a, yl_b, yn_b;
    double ynorm_a, ynorm_b;
    // FP32 channel slots: (max |value|, rms value) of the field a (and b) rows; when set, a
    // tile whose fixed-point unit is fine enough is accumulated in 32-bit fixed point
    // (integer shared-memory atomics) with a per-tile scale that no cell can overflow
    const float* amax_a;
    const float* amax_b;
};
template <typename T>
struct FusedArgs {
    PencilCat cat[3];
    int n_slots;
    FusedSlot slots[kMaxSlots];
    c2<T>* grids;
    long long grid_stride;
    int n, ty, tz, scheme, interlace;
    int nk_pos, nk_neg;
    const c2<T>* tw;
    const double* sums;
    double observer[3], origin[3], h;   // for the harmonic weights
    int ylm_global;                      // 1: harmonic weights of the fixed direction los_global
    double los_global[3];
    const int* pmask;                    // [3][n] planes reached per role, or null (write every pencil)
    const int* trows;                    // z-tile rows to visit (persistent grid), or null (all tiles)
    const int* trow_count;
    int skip_empty;                      // empty tiles store nothing (the y pass fills their zeros)
    int dual;                            // FP32 n = 256/512: two slots per CTA (see k_assign_xfft2)
    const int* tranges;                  // two-slot launches: per-tile range records, or null
    int* work;                           // one-slot launches over trows: item counter, zeroed
                                         // before the launch (dynamic schedule), or null
    int* err;                            // ERRF_BOUNDS of LPP_CHECK builds
    int* pstat;                          // optional tile counters: [0] two-slot fixed-point tiles,
                                         // [1] two-slot float tiles, [2] one-slot fixed-point
                                         // tiles, [3] one-slot float tiles (FP32 channel slots)
};

void fused_geometry(int n, size_t elem_bytes, int* ty, int* tz, int* ipt, int* threads, size_t* smem);
// pmask[r][z] = 1 when a particle of role r (set[r] != 0) sits in a key row f with
// z - 2 <= f <= z + 1 (mod n): the planes its CIC/TSC stencils (interlaced or not) reach.
// rows[0 .. *count) = the z-tile rows (tz planes each) holding a plane reached by a role in
// bits (n / tz <= 256)
cudaError_t launch_tile_rows(const int* pmask, int bits, int n, int tz, int* rows, int* count, cudaStream_t st);
// plive[r][z * n + y] = 1 when a particle of role r (set[r] != 0) sits in a key row
// (fy, fz) with y - 2 <= fy <= y + 1 and z - 2 <= fz <= z + 1 (mod n): the x pencils that
// its CIC/TSC stencils (interlaced or not) reach
cudaError_t launch_pencil_live(const int* off0, const int* off1, const int* off2, int set0, int set1, int set2, int n,
                               unsigned char* plive, cudaStream_t st);
cudaError_t launch_plane_mask(const int* off0, const int* off1, const int* off2, int set0, int set1, int set2, int n,
                              int* pmask, cudaStream_t st);
template <typename T>
cudaError_t launch_pencil_sort(const T* pos, const T* w, long long count, long long cap, int n, double box,
                               const double origin[3], int* key, int* counts, int* off, int* cursor, int* scan_tmp,
                               T* su, T* sw, int* perm, int* err, cudaStream_t st);
template <typename T>
cudaError_t launch_assign_xfft(const FusedArgs<T>& a, cudaStream_t st);
// Range records (particle ranges and fixed-point bound) of every tile of the two-slot
// persistent enumeration over a.trows, for the sources of a.slots[0]; FP32, n = 256 or 512.
// out: tile_range_bytes(n, ty, tz) bytes.  One launch.
template <typename T>
cudaError_t launch_tile_ranges(const FusedArgs<T>& a, int* out, cudaStream_t st);
size_t tile_range_bytes(int n, int ty, int tz);

// --------------------------------------------------------------------- combine
struct CombineChan {
    int slot;      // grid in the batch
    int sub;       // 0: real-part field (or interlaced pair), 1: imaginary-part field
    int kind;      // Kind
    int L, n;      // harmonic
    int part;      // Part: multiply the field by 1 or by i
    int out_row;   // row of the FP64 output [row][bin][2]
    double ynorm;  // normalisation of Y_{L,n} divided by (L - |n|)! (goes with ylm_poly_scaled)
};

template <typename T>
struct CombineArgs {
    const c2<T>* grids;
    long long grid_stride;
    int n;
    int interlace;
    int n_ch;
    int per_grid;          // channels per batch grid: 1 (interlaced) or 2 (two packed fields)
    CombineChan ch[kMaxBatchCh];
    // partner spectra (full n^3 arrays, valid on kept modes); in partner mode a null pD
    // skips storing D (only its shell sums are wanted)
    c2<T>* pD;
    c2<T>* pG1;
    c2<T>* pG2;
    int partner_mode;      // 1: unpack partners (slots hold D, G1, G2) and sum DD0/PLUS0
    int has_d, has_g;      // partner fields present
    int row_dd0, row_plus0;
    const T* inv_w;        // [n] per-index 1/sinc^p (1 without compensation)
    const c2<T>* phase;    // [n] per-index e^{-i pi f/n}
    const int* thr;        // [nb+1] thresholds on n^2
    int nb;
    int nk_pos, nk_neg, nky, nzi;
    double* out;           // [rows][nb][2]
    // optional work list (combine_items): item = {row, first mode, x extent >= 0, x extent < 0}
    // of the modes inside the last shell, 32 at a time; null: one CTA pass per whole row
    const int4* items;
    int n_items;
    int* err;              // ERRF_BOUNDS of LPP_CHECK builds
};

template <typename T>
cudaError_t launch_combine(const CombineArgs<T>& a, int n_sm, cudaStream_t st);
// The work list of the combine for a plan's kept cube: row r = zi * nky + yj (the combine's
// row enumeration) holds the modes fx = 0 .. xp and -1 .. -xn with fx^2 + fy^2 + fz^2 < q_max;
// they are split into items of 32 consecutive modes (fx = 0 .. xp first, then -1 .. -xn).
void combine_items(int n, int nk_pos, int nk_neg, int nky, int nzi, int q_max, std::vector<int4>& items);

// ------------------------------------------------------------------ window multipoles
// pD[m] = Z[m] / W(m) over every mode of grid 0 (the window field alone in the real part)
template <typename T>
cudaError_t launch_window_partner(const c2<T>* grid, c2<T>* pD, const T* inv_w, int n, cudaStream_t st);
// per mode pair, Z <- conj(A/W) pD + i conj(B/W) pD for the two packed fields of every grid
template <typename T>
cudaError_t launch_window_mult(c2<T>* grids, long long grid_stride, int n_grids, const c2<T>* pD, const T* inv_w,
                               int n, cudaStream_t st);
struct SbinChan {
    int grid, sub, l, m, out_row;
    double ynorm;
};
template <typename T>
struct SbinArgs {
    const c2<T>* grids;
    long long grid_stride;
    int n, n_ch;
    SbinChan ch[kMaxBatchCh];
    const int* thr;   // [nb+1] thresholds on the integer |s|^2 / h^2
    int nb;
    int ns_pos, ns_neg, nks;
    double scale;     // 1 / n^3 of the unnormalised inverse FFT
    double* out;      // [rows][nb][2]
};
template <typename T>
cudaError_t launch_sbin(const SbinArgs<T>& a, int n_sm, cudaStream_t st);

}  // namespace lpp
