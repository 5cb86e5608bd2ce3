// Batched 3D complex FFT of n^3 grids as three pencil passes (x, y, z).
//
// Each CTA loads a tile of W pencils (n complex points each) into shared memory,
// runs a mixed-radix Stockham FFT (radix 8 stages, one leading radix-2 or -4 stage)
// with every thread holding 8 points per stage, and writes the pencils back in
// place.  Pencils along y and z are loaded as rows of W consecutive x values, so
// every global access is a contiguous W-element segment; x pencils are transposed
// into the same column layout while loading.
//
// Passes can be pruned to the frequencies the shell binning needs: with a kept
// range f in [-nk_neg, nk_pos] per axis, the x pass writes only kept x, the y pass
// runs only on kept x columns and writes kept y, and the z pass runs only on kept
// (x, y) columns and writes kept z.  Values outside the kept range are left stale.
#include "lpp_internal.h"
#include "lpp_kernels.h"

namespace lpp {

template <typename T, bool INV>
__device__ __forceinline__ void dft4(c2<T>* v) {
    c2<T> a0 = cadd<T>(v[0], v[2]), a1 = csub<T>(v[0], v[2]);
    c2<T> b0 = cadd<T>(v[1], v[3]), b1 = csub<T>(v[1], v[3]);
    b1 = INV ? mk<T>(-b1.y, b1.x) : mk<T>(b1.y, -b1.x);  // * (+i) or * (-i)
    v[0] = cadd<T>(a0, b0);
    v[2] = csub<T>(a0, b0);
    v[1] = cadd<T>(a1, b1);
    v[3] = csub<T>(a1, b1);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft2(c2<T>* v) {
    c2<T> a = v[0];
    v[0] = cadd<T>(a, v[1]);
    v[1] = csub<T>(a, v[1]);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft8(c2<T>* v) {
    c2<T> e[4] = {v[0], v[2], v[4], v[6]};
    c2<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4<T, INV>(e);
    dft4<T, INV>(o);
    const T r = (T)0.70710678118654752440;
    c2<T> t1, t2, t3;
    if (!INV) {
        t1 = mk<T>((o[1].x + o[1].y) * r, (o[1].y - o[1].x) * r);   // * (1 - i)/sqrt2
        t2 = mk<T>(o[2].y, -o[2].x);                               // * (-i)
        t3 = mk<T>((o[3].y - o[3].x) * r, -(o[3].x + o[3].y) * r);  // * (-1 - i)/sqrt2
    } else {
        t1 = mk<T>((o[1].x - o[1].y) * r, (o[1].x + o[1].y) * r);
        t2 = mk<T>(-o[2].y, o[2].x);
        t3 = mk<T>(-(o[3].x + o[3].y) * r, (o[3].x - o[3].y) * r);
    }
    v[0] = cadd<T>(e[0], o[0]);
    v[4] = csub<T>(e[0], o[0]);
    v[1] = cadd<T>(e[1], t1);
    v[5] = csub<T>(e[1], t1);
    v[2] = cadd<T>(e[2], t2);
    v[6] = csub<T>(e[2], t2);
    v[3] = cadd<T>(e[3], t3);
    v[7] = csub<T>(e[3], t3);
}

// One Stockham stage of radix R on every column of the tile.  The thread owns
// column c and butterflies j = u + q N/8 (q < 8/R).
template <typename T, int N, int R, bool INV>
__device__ __forceinline__ void stockham_stage(c2<T>* tile, int ld, int c, int u, int Ns, const c2<T>* tw) {
    constexpr int Q = 8 / R;
    c2<T> v[8];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int j = u + q * (N / 8);
#pragma unroll
        for (int r = 0; r < R; ++r) v[q * R + r] = tile[(j + r * (N / R)) * ld + c];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int j = u + q * (N / 8);
        const int jm = j & (Ns - 1);
        const int step = jm * (N / (Ns * R));
#pragma unroll
        for (int r = 1; r < R; ++r) {
            c2<T> w = tw[step * r];
            if (INV) w.y = -w.y;
            v[q * R + r] = cmul<T>(v[q * R + r], w);
        }
        if (R == 8) dft8<T, INV>(v + q * R);
        else if (R == 4) dft4<T, INV>(v + q * R);
        else dft2<T, INV>(v + q * R);
        const int idxD = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) tile[(idxD + r * Ns) * ld + c] = v[q * R + r];
    }
    __syncthreads();
}

template <typename T, int LOGN, bool INV>
__device__ __forceinline__ void fft_columns(c2<T>* tile, int ld, int c, int u, const c2<T>* tw) {
    constexpr int N = 1 << LOGN;
    constexpr int rem = LOGN % 3;
    int Ns = 1;
    if (rem == 1) { stockham_stage<T, N, 2, INV>(tile, ld, c, u, Ns, tw); Ns = 2; }
    if (rem == 2) { stockham_stage<T, N, 4, INV>(tile, ld, c, u, Ns, tw); Ns = 4; }
#pragma unroll
    for (int s = 0; s < LOGN / 3; ++s) {
        stockham_stage<T, N, 8, INV>(tile, ld, c, u, Ns, tw);
        Ns *= 8;
    }
}

__device__ __forceinline__ bool kept(int e, int n, int nk_pos, int nk_neg) {
    return e <= nk_pos || e >= n - nk_neg;
}

// MODE 0: pencils along x (W consecutive y lines at fixed z)
// MODE 1: pencils along y (W consecutive kept x columns at fixed z)
// MODE 2: pencils along z (W consecutive kept x columns at a fixed kept y)
template <typename T, int LOGN, bool INV, int MODE>
__global__ void __launch_bounds__(1024, 1) k_fft_pass(c2<T>* __restrict__ data, const c2<T>* __restrict__ twg,
                                                      FftGeom g) {
    constexpr int N = 1 << LOGN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* tile = tw + N;
    const int W = g.W;
    const int ld = W + 1;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const long long N2 = (long long)N * N;
    c2<T>* base = data + (long long)blockIdx.y * N2 * N;

    long long off;
    long long es, cs;
    const int tile_id = blockIdx.x;
    if (MODE == 0) {
        const int ty = tile_id % (N / W);
        const int z = tile_id / (N / W);
        off = z * N2 + (long long)ty * W * N;
        es = 1;
        cs = N;
    } else {
        const int i = tile_id % g.ntx;
        const int o = tile_id / g.ntx;
        const int x0 = (g.ntx == N / W || i < g.nlo) ? i * W : N - (g.ntx - i) * W;
        if (MODE == 1) {
            off = o * N2 + x0;  // o = z
            es = N;
        } else {
            const int y = (o <= g.nk_pos) ? o : N - (g.nky - o);
            off = (long long)y * N + x0;
            es = N2;
        }
        cs = 1;
    }
    for (int i = tid; i < N; i += nthr) tw[i] = twg[i];
    const int total = N * W;
#pragma unroll 8
    for (int idx = tid; idx < total; idx += nthr) {
        int e, c;
        if (MODE == 0) { e = idx & (N - 1); c = idx >> LOGN; }
        else { c = idx % W; e = idx / W; }
        tile[e * ld + c] = base[off + e * es + c * cs];
    }
    __syncthreads();
    fft_columns<T, LOGN, INV>(tile, ld, tid % W, tid / W, tw);
#pragma unroll 8
    for (int idx = tid; idx < total; idx += nthr) {
        int e, c;
        if (MODE == 0) { e = idx & (N - 1); c = idx >> LOGN; }
        else { c = idx % W; e = idx / W; }
        if (kept(e, N, g.nk_pos, g.nk_neg)) base[off + e * es + c * cs] = tile[e * ld + c];
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
static cudaError_t launch_passes(c2<T>* data, int n_grids, const c2<T>* tw, const FftGeom& g, cudaStream_t st,
                                 Timer* timer) {
    constexpr int N = 1 << LOGN;
    const int W = g.W;
    const int threads = W * N / 8;
    const size_t smem = (size_t)(N + N * (W + 1)) * sizeof(c2<T>);
    // the attribute is per device and function: set it on every call (cheap, host-only)
    cudaFuncSetAttribute(k_fft_pass<T, LOGN, INV, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_fft_pass<T, LOGN, INV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_fft_pass<T, LOGN, INV, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const double es = (double)sizeof(c2<T>);
    const double n3 = (double)N * N * N;
    const double keep = (double)(g.nky) / N;               // kept fraction of one axis
    const double xcols = (double)g.ntx * W / N;             // processed fraction of x columns
    // x pass
    if (timer) timer->begin(KK_FFT, st);
    k_fft_pass<T, LOGN, INV, 0><<<dim3((N / W) * N, n_grids), threads, smem, st>>>(data, tw, g);
    if (timer) timer->end(KK_FFT, st, n_grids * n3 * es * (1.0 + keep));
    // y pass
    if (timer) timer->begin(KK_FFT, st);
    k_fft_pass<T, LOGN, INV, 1><<<dim3(g.ntx * N, n_grids), threads, smem, st>>>(data, tw, g);
    if (timer) timer->end(KK_FFT, st, n_grids * n3 * es * xcols * (1.0 + keep));
    // z pass
    if (timer) timer->begin(KK_FFT, st);
    k_fft_pass<T, LOGN, INV, 2><<<dim3(g.ntx * g.nky, n_grids), threads, smem, st>>>(data, tw, g);
    if (timer) timer->end(KK_FFT, st, n_grids * n3 * es * xcols * keep * (1.0 + keep));
    return cudaGetLastError();
}

template <typename T>
cudaError_t fft3d(c2<T>* data, int n_grids, int n, const c2<T>* tw, const FftGeom& g, bool inverse,
                  cudaStream_t st, Timer* timer) {
    int logn = 0;
    while ((1 << logn) < n) ++logn;
#define LPP_FFT_CASE(LG)                                                                   \
    case LG:                                                                               \
        return inverse ? launch_passes<T, LG, true>(data, n_grids, tw, g, st, timer)      \
                       : launch_passes<T, LG, false>(data, n_grids, tw, g, st, timer);
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

template cudaError_t fft3d<float>(c2<float>*, int, int, const c2<float>*, const FftGeom&, bool, cudaStream_t, Timer*);
template cudaError_t fft3d<double>(c2<double>*, int, int, const c2<double>*, const FftGeom&, bool, cudaStream_t, Timer*);

}  // namespace lpp
