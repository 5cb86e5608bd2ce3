// Density monopole of a periodic catalogue with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's
// memory pool or under a hard per-process memory cap, plug-ins that are handed a
// stream but no allocator, and paths that must not grow the device footprint after
// start-up.  lpp_density_monopole_static serves them.  It computes the same quantity as
// the P_dd^(0) slot of lpp_multipoles for a periodic box, by its own simpler path: an
// unsorted scatter of the particles into one grid with global atomics (k_assign), a full
// 3D FFT (fft3d, x pass included) and the partner-mode shell sums of the combine kernel.
// Every intermediate lives in one file-scope device array of fixed size, so the library
// itself never allocates device memory on this path.
#include <math.h>
#include <string.h>

#include "lpp_internal.h"
#include "lpp_kernels.h"

using namespace lpp;

namespace {

// Every GPU that loads liblpp holds this array until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)40 << 20;  // 40 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
// Device address of g_static_scratch per device, filled on the first call on that
// device (the host symbol g_static_scratch is only a host-side stand-in).
void* g_scratch_addr[kMaxDevices] = {nullptr};

const double kPi = 3.14159265358979323846;
constexpr int kMaxN = 1024;
constexpr int kMaxBins = 256;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t sums, err, out, thr, tw, iw, ph, grid, total;
};

Layout layout(int n, int nb, size_t es) {
    Layout l;
    const size_t cs = 2 * es, n3 = (size_t)n * n * n;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align256(off + b); return o; };
    l.sums = take(SUM_COUNT * sizeof(double));
    l.err = take(sizeof(int));
    l.out = take((size_t)2 * nb * 2 * sizeof(double));
    l.thr = take((nb + 1) * sizeof(int));
    l.tw = take(n * cs);
    l.iw = take(n * es);
    l.ph = take(n * cs);
    l.grid = take(n3 * cs);
    l.total = off;
    return l;
}

// Host tables live in fixed-size per-thread buffers (no allocation; host threads never
// share them); a pageable copy has consumed its source by the time cudaMemcpyAsync returns.
thread_local int h_thr[kMaxBins + 1];
thread_local long long h_nmodes[kMaxBins];
thread_local double h_out[2 * kMaxBins * 2];
thread_local double h_tab[3 * 2 * kMaxN];

template <typename T>
lpp_status run_static(char* base, const Layout& lay, int n, double box, const double origin[3], int scheme,
                      int interlace, int compensate, const T* pos, const T* w, long long count, int nb,
                      const double* k_edges, double* p_out, long long* n_modes_out, cudaStream_t st) {
    const double kf = 2.0 * kPi / box;
    const long long qmax = 3LL * (n / 2) * (n / 2);
    for (int b = 0; b <= nb; ++b) {
        const double e = k_edges[b];
        long long q = 0;
        if (e > 0) {
            const double t = e / kf;
            q = (long long)floor(t * t);
            if (q > qmax + 1) q = qmax + 1;
            while (q > 0 && kf * sqrt((double)(q - 1)) >= e) --q;
            while (q <= qmax && kf * sqrt((double)q) < e) ++q;
        }
        h_thr[b] = (int)q;
    }
    const int tmax = h_thr[nb];
    int nk = 0;
    while ((long long)(nk + 1) * (nk + 1) < tmax && nk < n / 2) ++nk;
    const int nk_pos = nk < n / 2 - 1 ? nk : n / 2 - 1;
    const int nk_neg = nk < n / 2 ? nk : n / 2;
    for (int b = 0; b < nb; ++b) h_nmodes[b] = 0;
    for (int fx = -nk_neg; fx <= nk_pos; ++fx)
        for (int fy = -nk_neg; fy <= nk_pos; ++fy)
            for (int fz = -nk_neg; fz <= nk_pos; ++fz) {
                const long long q = (long long)fx * fx + (long long)fy * fy + (long long)fz * fz;
                if (q == 0 || q < h_thr[0] || q >= tmax) continue;
                int lo = 0, hi = nb;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) / 2;
                    if (q >= h_thr[mid]) lo = mid; else hi = mid;
                }
                ++h_nmodes[lo];
            }
    cudaError_t e;
#define LPP_STATIC_CUDA(call)                          \
    do {                                               \
        if ((e = (call)) != cudaSuccess) return LPP_ERR_CUDA; \
    } while (0)
    // tables: twiddles, inverse window, interlacing phase (stored as T pairs / T)
    T* tab = reinterpret_cast<T*>(h_tab);
    for (int j = 0; j < n; ++j) {
        tab[2 * j] = (T)cos(2.0 * kPi * j / n);
        tab[2 * j + 1] = (T)(-sin(2.0 * kPi * j / n));
    }
    LPP_STATIC_CUDA(cudaMemcpyAsync(base + lay.tw, tab, 2 * n * sizeof(T), cudaMemcpyHostToDevice, st));
    for (int j = 0; j < n; ++j) {
        const int f = j < n / 2 ? j : j - n;
        const double xa = kPi * f / n;
        const double sinc = f == 0 ? 1.0 : sin(xa) / xa;
        tab[j] = (T)(compensate ? 1.0 / pow(sinc, scheme) : 1.0);
    }
    LPP_STATIC_CUDA(cudaMemcpyAsync(base + lay.iw, tab, n * sizeof(T), cudaMemcpyHostToDevice, st));
    for (int j = 0; j < n; ++j) {
        const int f = j < n / 2 ? j : j - n;
        tab[2 * j] = (T)cos(kPi * f / n);
        tab[2 * j + 1] = (T)(-sin(kPi * f / n));
    }
    LPP_STATIC_CUDA(cudaMemcpyAsync(base + lay.ph, tab, 2 * n * sizeof(T), cudaMemcpyHostToDevice, st));
    LPP_STATIC_CUDA(cudaMemcpyAsync(base + lay.thr, h_thr, (nb + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    // everything the kernels accumulate into starts at zero: the array keeps the last call's contents
    const size_t n3 = (size_t)n * n * n;
    LPP_STATIC_CUDA(cudaMemsetAsync(base + lay.sums, 0, SUM_COUNT * sizeof(double), st));
    LPP_STATIC_CUDA(cudaMemsetAsync(base + lay.err, 0, sizeof(int), st));
    LPP_STATIC_CUDA(cudaMemsetAsync(base + lay.out, 0, (size_t)2 * nb * 2 * sizeof(double), st));
    LPP_STATIC_CUDA(cudaMemsetAsync(base + lay.grid, 0, n3 * 2 * sizeof(T), st));

    double* sums = reinterpret_cast<double*>(base + lay.sums);
    int* err = reinterpret_cast<int*>(base + lay.err);
    c2<T>* grid = reinterpret_cast<c2<T>*>(base + lay.grid);
    LPP_STATIC_CUDA(launch_sums<T>(w, nullptr, count, sums, SUM_W_DENS, SUM_W2_DENS, -1, st));
    LPP_STATIC_CUDA(launch_alpha(sums, 0, st));
    AssignArgs<T> aa;
    memset(&aa, 0, sizeof(aa));
    aa.pos = pos;
    aa.count = count;
    aa.grids = grid;
    aa.grid_stride = (long long)n3;
    aa.n = n;
    aa.box = box;
    for (int a = 0; a < 3; ++a) aa.origin[a] = origin[a];
    aa.n_slots = 1;
    aa.slots[0] = AssignSlot{w, nullptr, 0, 0, w == nullptr};
    aa.sums = sums;
    aa.err = err;
    LPP_STATIC_CUDA(launch_assign<T>(aa, scheme, interlace, st));
    const FftGeom geom = fft_geometry(n, nk_pos, nk_neg);
    LPP_STATIC_CUDA(fft3d<T>(grid, 1, n, reinterpret_cast<const c2<T>*>(base + lay.tw), geom, false, st, nullptr));
    CombineArgs<T> cb;
    memset(&cb, 0, sizeof(cb));
    cb.grids = grid;
    cb.grid_stride = (long long)n3;
    cb.n = n;
    cb.interlace = interlace;
    cb.pD = nullptr;   // only the shell sums of D are wanted
    cb.partner_mode = 1;
    cb.has_d = 1;
    cb.has_g = 0;
    cb.row_dd0 = 0;
    cb.row_plus0 = -1;
    cb.inv_w = reinterpret_cast<const T*>(base + lay.iw);
    cb.phase = reinterpret_cast<const c2<T>*>(base + lay.ph);
    cb.thr = reinterpret_cast<const int*>(base + lay.thr);
    cb.nb = nb;
    cb.nk_pos = nk_pos;
    cb.nk_neg = nk_neg;
    cb.nky = geom.nky;
    cb.nzi = nk_pos + 1 + (nk_neg == n / 2 ? 1 : 0);
    cb.out = reinterpret_cast<double*>(base + lay.out);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    LPP_STATIC_CUDA(launch_combine<T>(cb, sms, st));
    double h_sums[SUM_COUNT];
    int h_err = 0;
    LPP_STATIC_CUDA(cudaMemcpyAsync(h_out, base + lay.out, (size_t)nb * 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    LPP_STATIC_CUDA(cudaMemcpyAsync(h_sums, sums, sizeof(h_sums), cudaMemcpyDeviceToHost, st));
    LPP_STATIC_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LPP_STATIC_CUDA(cudaStreamSynchronize(st));
#undef LPP_STATIC_CUDA
    if (h_err) return LPP_ERR_DOMAIN;
    const double vol = box * box * box;
    const double I = h_sums[SUM_W_DENS] * h_sums[SUM_W_DENS] / vol;
    const double shot = I != 0 ? h_sums[SUM_W2_DENS] / I : 0.0;
    for (int b = 0; b < nb; ++b) {
        const double nm = (double)h_nmodes[b];
        p_out[b] = (nm > 0 && I != 0) ? h_out[2 * b] / nm / I - shot : 0.0;
        if (n_modes_out) n_modes_out[b] = h_nmodes[b];
    }
    return LPP_OK;
}

}  // namespace

extern "C" lpp_status lpp_density_monopole_static(int n, double box, const double* origin, int scheme, int interlace,
                                                  int compensate, int precision, const void* pos, const void* w,
                                                  long long count, int n_bins, const double* k_edges, double* p_out,
                                                  long long* n_modes_out, void* stream) {
    if (n < 8 || n > kMaxN || (n & (n - 1)) != 0) return LPP_ERR_UNSUPPORTED;
    if (!(box > 0) || !origin || !k_edges || !p_out || n_bins < 1 || n_bins > kMaxBins) return LPP_ERR_INVALID_ARG;
    if (scheme != LPP_CIC && scheme != LPP_TSC) return LPP_ERR_INVALID_ARG;
    if (precision != LPP_FP32 && precision != LPP_FP64) return LPP_ERR_INVALID_ARG;
    if (count < 0 || (count > 0 && !pos)) return LPP_ERR_INVALID_ARG;
    for (int i = 0; i < n_bins; ++i)
        if (!(k_edges[i] < k_edges[i + 1])) return LPP_ERR_INVALID_ARG;
    const size_t es = precision == LPP_FP64 ? 8 : 4;
    const Layout lay = layout(n, n_bins, es);
    if (lay.total > kStaticScratchBytes) return LPP_ERR_WORKSPACE;  // grid too large for the fixed array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LPP_ERR_CUDA;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return LPP_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    char* base = static_cast<char*>(g_scratch_addr[dev]);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == LPP_FP64)
        return run_static<double>(base, lay, n, box, origin, scheme, interlace, compensate,
                                  static_cast<const double*>(pos), static_cast<const double*>(w), count, n_bins,
                                  k_edges, p_out, n_modes_out, st);
    return run_static<float>(base, lay, n, box, origin, scheme, interlace, compensate, static_cast<const float*>(pos),
                             static_cast<const float*>(w), count, n_bins, k_edges, p_out, n_modes_out, st);
}
