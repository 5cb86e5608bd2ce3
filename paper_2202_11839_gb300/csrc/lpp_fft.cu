// Batched 3D complex FFT of n^3 grids as three pencil passes (x, y, z).
//
// Each CTA transforms a tile of W pencils (n complex points each) with a mixed-radix
// Stockham FFT (radix 8 stages, one leading radix-2 or -4 stage), every thread holding
// 8 points per stage, and writes the pencils back in place.  Pencils along y and z are
// read as rows of W consecutive x values, so every global access is a contiguous
// W-element segment; the first stage takes its operands straight from those rows and
// the last stage stores straight to them, so shared memory holds only the stages in
// between.  x pencils are transposed into the same column layout in shared memory.
//
// Passes can be pruned to the frequencies the shell binning needs: with a kept
// range f in [-nk_neg, nk_pos] per axis, the x pass writes only kept x, the y pass
// runs only on kept x columns and writes kept y, and the z pass runs only on kept
// (x, y) columns and writes kept z.  Values outside the kept range are left stale.
#include <algorithm>

#include "lpp_internal.h"
#include "lpp_kernels.h"
#include "lpp_fft_dev.cuh"

namespace lpp {

// MODE 0: pencils along x (W consecutive y lines at fixed z)
// MODE 1: pencils along y (W consecutive kept x columns at fixed z)
// MODE 2: pencils along z (W consecutive kept x columns at a fixed kept y)
// Offsets inside one grid fit in 32 bits (n <= 1024); the tile base is a 64-bit pointer.

// Whether z plane `z` of grid `gi` of the call holds anything for the y pass: false when no
// particle of the grid's roles reaches it (neither the fused assignment nor the y pass stores
// it, and the z pass reads zeros there).  CTA-uniform.
__device__ __forceinline__ bool plane_live(const FftGeom& g, int gi, int z, int n) {
    if (!g.pmask || !g.gmask[gi]) return true;
    int hit = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
        if (g.gmask[gi] & (1 << r)) hit |= __ldg(g.pmask + r * n + z);
    return hit != 0;
}

// One y (MODE 1) or z (MODE 2) tile of W pencils of one grid.  twg: with it the twiddles are
// loaded into tw here, after the column test and beside the operand loads (they are first
// read after the first stage's barrier); null when tw already holds them.  Every return is
// CTA-uniform; the tile is free again after the caller's next barrier.
template <typename T, int LOGN, bool INV, int MODE>
__device__ __forceinline__ void pencil_tile(c2<T>* grid, const c2<T>* twg, c2<T>* tw, c2<T>* tile, const FftGeom& g,
                                            int tile_id, int gi) {
    using S = PassShape<LOGN>;
    constexpr int N = S::N, W = S::W, LD = S::LD;
    const int tid = threadIdx.x;
    const unsigned N2 = (unsigned)N * N;
    c2<T>* base = grid;
    const int o = tile_id / g.ntx;
    const int i = tile_id - o * g.ntx;
    const int x0 = (g.ntx == N / W || i < g.nlo) ? i * W : N - (g.ntx - i) * W;
    if (!LPP_IN_BOUNDS(o >= 0 && o < (MODE == 1 ? N : g.nky) && x0 >= 0 && x0 + W <= N, g.err)) return;
    if (MODE == 1) {
        base += (size_t)o * N2 + x0;  // o = z
    } else {
        const int y = (o <= g.nk_pos) ? o : N - (g.nky - o);
        if (g.q_max > 0) {
            // columns outside the last shell in (fx, fy) for every fz: nothing to transform
            const int fy = y < N / 2 ? y : y - N;
            int m2 = 0x7fffffff;
            for (int c = 0; c < W; ++c) {
                const int x = x0 + c;
                const int fx = x < N / 2 ? x : x - N;
                m2 = min(m2, fx * fx);
            }
            if (m2 + fy * fy >= g.q_max) return;
        }
        base += (size_t)y * N + x0;
    }
    // Thread (c, u) owns pencil c (W consecutive x values per row: 128-byte segments in
    // FP32) and butterfly slot u.  The first FFT stage loads its operands straight from
    // the grid and the last stores its results straight back, so the tile holds only the
    // intermediate stages.
    const int c = tid & (W - 1), u = tid >> S::LOGW;
    constexpr unsigned ES = MODE == 1 ? (unsigned)N : (unsigned)N * N;
    c2<T>* gp = base + c;
    static_assert(S::PER == 8 * S::IPT && S::PER <= 32, "one liveness bit per operand");
    // operands on rows that no particle of the grid's roles reaches (y pencils of this z
    // plane for the y pass, z planes for the z pass) are zero and not loaded
    unsigned live = 0xffffffffu;
    const int gm = g.gmask[gi];
    if (gm && (MODE == 1 ? g.plive != nullptr : g.pmask != nullptr)) {
        const int z = o;   // the y pass's plane
        live = 0u;
#pragma unroll
        for (int b = 0; b < S::PER; ++b) {
            const int e = lead_row<LOGN, S::IPT>(u, b);
            int hit = 0;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                if (gm & (1 << r))
                    hit |= MODE == 1 ? __ldg(g.plive + (size_t)r * N * N + (size_t)z * N + e)
                                     : __ldg(g.pmask + r * N + e);
            }
            live |= (hit ? 1u : 0u) << b;
        }
    }
    if (twg)
        for (int k = tid; k < N; k += S::THREADS) tw[k] = twg[k];
    fft_columns_io<T, LOGN, INV, S::IPT, LD>(
        tile, c, u, tw,
        [&](int b, int e) { return ((live >> b) & 1u) ? gp[(size_t)e * ES] : mk<T>((T)0, (T)0); },
        [&](int e, c2<T> v) {
            if (kept(e, N, g.nk_pos, g.nk_neg)) gp[(size_t)e * ES] = v;
        });
}

template <typename T, int LOGN, bool INV, int MODE>
__global__ void __launch_bounds__(PassShape<LOGN>::THREADS, sizeof(T) == 4 ? (LOGN == 9 ? 3 : 2) : 1) k_fft_pass(c2<T>* __restrict__ data,
                                                                      const c2<T>* __restrict__ twg, FftGeom g) {
    using S = PassShape<LOGN>;
    constexpr int N = S::N, W = S::W, LD = S::LD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* tile = tw + N;
    const int tid = threadIdx.x;
    const unsigned N2 = (unsigned)N * N;
    c2<T>* grid = data + (size_t)blockIdx.y * N2 * N;
    const int tile_id = blockIdx.x;
    if constexpr (MODE == 0) {
        for (int i = tid; i < N; i += S::THREADS) tw[i] = twg[i];
        const int ty = tile_id & (N / W - 1);
        const int z = tile_id >> (LOGN - S::LOGW);
        if (!LPP_IN_BOUNDS(z < N, g.err)) return;
        c2<T>* base = grid + (size_t)z * N2 + (size_t)ty * W * N;
#pragma unroll
        for (int k = 0; k < S::PER; ++k) {
            const int idx = tid + k * S::THREADS;
            const int e = idx & (N - 1), c = idx >> LOGN;
            tile[e * LD + c] = base[e + c * N];
        }
        __syncthreads();
        fft_columns<T, LOGN, INV, S::IPT, LD>(tile, tid & (W - 1), tid >> S::LOGW, tw);
#pragma unroll
        for (int k = 0; k < S::PER; ++k) {
            const int idx = tid + k * S::THREADS;
            const int e = idx & (N - 1), c = idx >> LOGN;
            if (kept(e, N, g.nk_pos, g.nk_neg)) base[e + c * N] = tile[e * LD + c];
        }
    } else {
        // a z plane that no particle of the grid's roles reaches: its pencils are zero;
        // neither the fused assignment nor this pass stores it
        if (MODE == 1 && !plane_live(g, blockIdx.y, tile_id / g.ntx, N)) return;
        pencil_tile<T, LOGN, INV, MODE>(grid, twg, tw, tile, g, tile_id, blockIdx.y);
    }
}

// The y pass as a persistent grid over the (grid, plane, x tile) items of the call, for calls
// that skip unreached planes: the items of unreached planes cost a mask test instead of a
// CTA launch (with its shared memory held), and the twiddles are loaded once per CTA.
template <typename T, int LOGN, bool INV>
__global__ void __launch_bounds__(PassShape<LOGN>::THREADS, sizeof(T) == 4 ? (LOGN == 9 ? 3 : 2) : 1) k_fft_ypass(c2<T>* __restrict__ data,
                                                                       const c2<T>* __restrict__ twg, FftGeom g, int n_grids) {
    using S = PassShape<LOGN>;
    constexpr int N = S::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* tile = tw + N;
    for (int i = threadIdx.x; i < N; i += S::THREADS) tw[i] = twg[i];   // first read after a barrier
    const int per_grid = g.ntx * N;
    const int items = per_grid * n_grids;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int gi = it / per_grid, tile_id = it - gi * per_grid;
        if (!plane_live(g, gi, tile_id / g.ntx, N)) continue;
        pencil_tile<T, LOGN, INV, 1>(data + (size_t)gi * N * N * N, nullptr, tw, tile, g, tile_id, gi);
        __syncthreads();   // the next item's first stage rewrites the tile
    }
}

int fft_tile_width(int n) {
    int w = 8192 / n;
    if (w > 32) w = 32;
    if (w > n) w = n;
    return w;
}

FftGeom fft_geometry(int n, int nk_pos, int nk_neg) {
    FftGeom g;
    g.W = fft_tile_width(n);
    g.nk_pos = nk_pos;
    g.nk_neg = nk_neg;
    const int tiles = n / g.W;
    g.nlo = nk_pos / g.W + 1;
    const int nhi = (nk_neg + g.W - 1) / g.W;
    g.ntx = g.nlo + nhi >= tiles ? tiles : g.nlo + nhi;
    if (g.ntx == tiles) g.nlo = tiles;
    g.nky = (nk_pos + 1 + nk_neg >= n) ? n : nk_pos + 1 + nk_neg;
    return g;
}

template <typename T, int LOGN, bool INV>
static cudaError_t launch_passes(c2<T>* data, int n_grids, const c2<T>* tw, const FftGeom& g, bool with_x,
                                 cudaStream_t st, Timer* timer) {
    using S = PassShape<LOGN>;
    constexpr int N = S::N, W = S::W;
    if (g.W != W) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)(N + N * S::LD) * sizeof(c2<T>);
    // the attribute is per device and function: set it on every call (cheap, host-only)
    cudaFuncSetAttribute(k_fft_pass<T, LOGN, INV, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_fft_pass<T, LOGN, INV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_fft_pass<T, LOGN, INV, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const double es = (double)sizeof(c2<T>);
    const double n3 = (double)N * N * N;
    const double keep = (double)(g.nky) / N;               // kept fraction of one axis
    const double xcols = (double)g.ntx * W / N;             // processed fraction of x columns
    if (with_x) {
        if (timer) timer->begin(KK_FFT, st);
        k_fft_pass<T, LOGN, INV, 0><<<dim3((N / W) * N, n_grids), S::THREADS, smem, st>>>(data, tw, g);
        if (timer) timer->end(KK_FFT, st, n_grids * n3 * es * (1.0 + keep));
    }
    if (timer) timer->begin(KK_FFT, st);
    bool skip = false;
    for (int i = 0; i < n_grids && i < 8; ++i) skip = skip || (g.pmask && g.gmask[i]);
    if (skip) {
        // one wave of resident CTAs (the occupancy the launch bounds give), at most one per item
        int dev = 0, sms = 0, ps = 0;
        cudaFuncSetAttribute(k_fft_ypass<T, LOGN, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_fft_ypass<T, LOGN, INV>, S::THREADS, smem);
        if (ps < 1) ps = 1;
        if (sms < 1) sms = 1;
        const long long items = (long long)g.ntx * N * n_grids;
        const int blocks = (int)std::min<long long>(items, (long long)ps * sms);
        k_fft_ypass<T, LOGN, INV><<<blocks, S::THREADS, smem, st>>>(data, tw, g, n_grids);
    } else {
        k_fft_pass<T, LOGN, INV, 1><<<dim3(g.ntx * N, n_grids), S::THREADS, smem, st>>>(data, tw, g);
    }
    // y: only the reached planes are read and written; z: their entries are read, all written
    if (timer)
        timer->end(KK_FFT, st, n_grids * n3 * es * xcols * ((double)g.ylive_frac + (double)g.yread_frac * keep));
    if (timer) timer->begin(KK_FFT, st);
    k_fft_pass<T, LOGN, INV, 2><<<dim3(g.ntx * g.nky, n_grids), S::THREADS, smem, st>>>(data, tw, g);
    if (timer) {
        // the z pass transforms the columns that some shell can use
        double zfrac = 1.0;
        if (g.q_max > 0) {
            long long live = 0, all = 0;
            for (int o = 0; o < g.nky; ++o) {
                const int y = (o <= g.nk_pos) ? o : N - (g.nky - o);
                const int fy = y < N / 2 ? y : y - N;
                for (int i = 0; i < g.ntx; ++i) {
                    const int x0 = (g.ntx == N / W || i < g.nlo) ? i * W : N - (g.ntx - i) * W;
                    int m2 = 0x7fffffff;
                    for (int c = 0; c < W; ++c) {
                        const int fx = (x0 + c) < N / 2 ? x0 + c : x0 + c - N;
                        m2 = std::min(m2, fx * fx);
                    }
                    ++all;
                    live += (m2 + fy * fy < g.q_max);
                }
            }
            zfrac = all ? (double)live / all : 1.0;
        }
        timer->end(KK_FFT, st, n_grids * n3 * es * xcols * keep * zfrac * ((double)g.yread_frac + keep));
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t fft_dispatch(c2<T>* data, int n_grids, int n, const c2<T>* tw, const FftGeom& g, bool inverse,
                                bool with_x, cudaStream_t st, Timer* timer) {
    int logn = 0;
    while ((1 << logn) < n) ++logn;
#define LPP_FFT_CASE(LG)                                                                          \
    case LG:                                                                                      \
        return inverse ? launch_passes<T, LG, true>(data, n_grids, tw, g, with_x, st, timer)     \
                       : launch_passes<T, LG, false>(data, n_grids, tw, g, with_x, st, timer);
    switch (logn) {
        LPP_FFT_CASE(3)
        LPP_FFT_CASE(4)
        LPP_FFT_CASE(5)
        LPP_FFT_CASE(6)
        LPP_FFT_CASE(7)
        LPP_FFT_CASE(8)
        LPP_FFT_CASE(9)
        LPP_FFT_CASE(10)
        default:
            return cudaErrorInvalidValue;
    }
#undef LPP_FFT_CASE
}

template <typename T>
cudaError_t fft3d(c2<T>* data, int n_grids, int n, const c2<T>* tw, const FftGeom& g, bool inverse,
                  cudaStream_t st, Timer* timer) {
    return fft_dispatch<T>(data, n_grids, n, tw, g, inverse, true, st, timer);
}

template <typename T>
cudaError_t fft_yz(c2<T>* data, int n_grids, int n, const c2<T>* tw, const FftGeom& g, bool inverse,
                   cudaStream_t st, Timer* timer) {
    return fft_dispatch<T>(data, n_grids, n, tw, g, inverse, false, st, timer);
}

template cudaError_t fft3d<float>(c2<float>*, int, int, const c2<float>*, const FftGeom&, bool, cudaStream_t, Timer*);
template cudaError_t fft3d<double>(c2<double>*, int, int, const c2<double>*, const FftGeom&, bool, cudaStream_t, Timer*);
template cudaError_t fft_yz<float>(c2<float>*, int, int, const c2<float>*, const FftGeom&, bool, cudaStream_t, Timer*);
template cudaError_t fft_yz<double>(c2<double>*, int, int, const c2<double>*, const FftGeom&, bool, cudaStream_t, Timer*);

}  // namespace lpp
