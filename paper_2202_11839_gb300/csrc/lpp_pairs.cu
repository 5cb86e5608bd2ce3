// Window multipoles by pair counting (Sec. 4.3: the paper measures Q_l(s) from pairs of
// random points in the footprint; Eq. windowQ_ell with the endpoint line of sight).
//
//   Q_l(b) = (2l+1) alpha^2 / (I V_b) sum_{r != r', s_rr' in b} w_r w_r' L_l(shat_rr' . xhat_r)
//
// Every unordered pair {i, j} is visited once and adds w_i w_j [L_l(shat . xhat_i) +
// L_l(shat . xhat_j)] (L_l is even, so the sign of shat does not matter).  A CTA takes a
// tile of 256 points i (one per thread) against a tile of 256 points j staged in shared
// memory; tiles (it, jt) with jt >= it cover the upper triangle, the diagonal tile keeps
// j > i only.  All arithmetic is FP64; the separation that decides the shell is formed with
// explicitly rounded operations (no fused multiply-add), as a plain FP64 evaluation of
// sqrt(dx^2 + dy^2 + dz^2) would, so the shell of every pair is exactly the one of the
// oracle's definition.  Each warp accumulates into its own FP64 shell histogram in shared
// memory; the CTA then adds its histograms to the global sums.
#include <math.h>
#include <string.h>

#include <vector>

#include "lpp_internal.h"

namespace {

constexpr int kTile = 256;
constexpr int kWarps = kTile / 32;
constexpr int kEll = 5;   // l = 0, 2, 4, 6, 8
constexpr int kMaxShells = 256;

struct PairArgs {
    const double* pos;   // [3][n]
    const double* w;     // [n] or null
    long long n;
    int n_tiles;
    double obs[3];
    double box;          // > 0: minimal image in a periodic box of this side
    const double* edges; // [nb + 1]
    int nb;
    double* out;         // [nb][5] pair sums of w w' (L_l(mu_i) + L_l(mu_j))
};

// Legendre polynomials L_0, L_2, ..., L_8 of mu (power-series form)
__device__ __forceinline__ void legendre_even(double mu, double* l) {
    const double m2 = mu * mu;
    l[0] = 1.0;
    l[1] = 0.5 * (3.0 * m2 - 1.0);
    l[2] = (m2 * (35.0 * m2 - 30.0) + 3.0) * 0.125;
    l[3] = (m2 * (m2 * (231.0 * m2 - 315.0) + 105.0) - 5.0) * 0.0625;
    l[4] = (m2 * (m2 * (m2 * (6435.0 * m2 - 12012.0) + 6930.0) - 1260.0) + 35.0) * 0.0078125;
}

__device__ __forceinline__ double min_image(double d, double box) {
    if (box > 0.0) d = __dsub_rn(d, __dmul_rn(box, rint(__ddiv_rn(d, box))));
    return d;
}

// tile pair index -> (it, jt) with jt >= it (row-major over the upper triangle)
__device__ __forceinline__ void tile_pair(long long t, int nt, int& it, int& jt) {
    // rows it = 0 .. nt-1 hold nt - it tiles; find it by stepping (nt is small: n / 256)
    int r = 0;
    long long rem = t;
    while (rem >= nt - r) {
        rem -= nt - r;
        ++r;
    }
    it = r;
    jt = r + (int)rem;
}

__global__ void __launch_bounds__(kTile) k_pair_sums(PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* hist = reinterpret_cast<double*>(smem_raw);            // [kWarps][nb][kEll]
    double* xj = hist + (size_t)kWarps * a.nb * kEll;               // [7][kTile]: x, y, z, w, ux, uy, uz
    double* edges = xj + 7 * kTile;                                 // [nb + 1]
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nb = a.nb;
    for (int i = tid; i < kWarps * nb * kEll; i += kTile) hist[i] = 0.0;
    for (int i = tid; i <= nb; i += kTile) edges[i] = a.edges[i];
    double* h = hist + (size_t)warp * nb * kEll;
    const long long pairs = (long long)a.n_tiles * (a.n_tiles + 1) / 2;
    const long long n = a.n;
    for (long long t = blockIdx.x; t < pairs; t += gridDim.x) {
        int it, jt;
        tile_pair(t, a.n_tiles, it, jt);
        __syncthreads();   // the previous tile's j points are no longer read
        {
            const long long j = (long long)jt * kTile + tid;
            double x = 0, y = 0, z = 0, w = 0, ux = 0, uy = 0, uz = 0;
            if (j < n) {
                x = a.pos[j];
                y = a.pos[n + j];
                z = a.pos[2 * n + j];
                w = a.w ? a.w[j] : 1.0;
                const double px = x - a.obs[0], py = y - a.obs[1], pz = z - a.obs[2];
                const double inv = 1.0 / sqrt(px * px + py * py + pz * pz);
                ux = px * inv;
                uy = py * inv;
                uz = pz * inv;
            }
            xj[tid] = x;
            xj[kTile + tid] = y;
            xj[2 * kTile + tid] = z;
            xj[3 * kTile + tid] = w;
            xj[4 * kTile + tid] = ux;
            xj[5 * kTile + tid] = uy;
            xj[6 * kTile + tid] = uz;
        }
        __syncthreads();
        const long long i = (long long)it * kTile + tid;
        if (i < n) {
            const double x = a.pos[i], y = a.pos[n + i], z = a.pos[2 * n + i];
            const double wi = a.w ? a.w[i] : 1.0;
            const double px = x - a.obs[0], py = y - a.obs[1], pz = z - a.obs[2];
            const double inv = 1.0 / sqrt(px * px + py * py + pz * pz);
            const double ux = px * inv, uy = py * inv, uz = pz * inv;
            const int j0 = (it == jt) ? tid + 1 : 0;
            const long long jn = n - (long long)jt * kTile;
            const int j1 = jn < kTile ? (int)jn : kTile;
            for (int jj = j0; jj < j1; ++jj) {
                const double dx = min_image(__dsub_rn(xj[jj], x), a.box);
                const double dy = min_image(__dsub_rn(xj[kTile + jj], y), a.box);
                const double dz = min_image(__dsub_rn(xj[2 * kTile + jj], z), a.box);
                const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                const double s = __dsqrt_rn(s2);
                if (!(s > 0.0) || s < edges[0] || !(s < edges[nb])) continue;
                int lo = 0, hi = nb;   // edges[lo] <= s < edges[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s >= edges[mid]) lo = mid; else hi = mid;
                }
                const double is = 1.0 / s;
                const double mi = (dx * ux + dy * uy + dz * uz) * is;
                const double mj = (dx * xj[4 * kTile + jj] + dy * xj[5 * kTile + jj] + dz * xj[6 * kTile + jj]) * is;
                double li[kEll], lj[kEll];
                legendre_even(mi, li);
                legendre_even(mj, lj);
                const double ww = wi * xj[3 * kTile + jj];
#pragma unroll
                for (int e = 0; e < kEll; ++e) atomicAdd(h + lo * kEll + e, ww * (li[e] + lj[e]));
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < nb * kEll; i += kTile) {
        double v = 0.0;
        for (int wq = 0; wq < kWarps; ++wq) v += hist[(size_t)wq * nb * kEll + i];
        if (v != 0.0) atomicAdd(a.out + i, v);
    }
}

__global__ void k_nw2_sum(const double* __restrict__ w, const double* __restrict__ nbar, long long n,
                          double* __restrict__ out) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double wi = w ? w[i] : 1.0;
        s += (nbar ? nbar[i] : 1.0) * wi * wi;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" lpp_status lpp_window_Q_pairs_workspace_size(int n_s, size_t* bytes) {
    if (!bytes || n_s < 1 || n_s > kMaxShells) return LPP_ERR_INVALID_ARG;
    *bytes = align256((size_t)n_s * kEll * sizeof(double)) + align256((size_t)(n_s + 1) * sizeof(double)) +
             align256(sizeof(double));
    return LPP_OK;
}

extern "C" lpp_status lpp_window_Q_pairs(const double* pos, const double* w, const double* nbar, long long n,
                                         const double* observer, double box, double alpha, int n_s,
                                         const double* s_edges, double* q, void* workspace, size_t bytes,
                                         void* stream) {
    size_t need = 0;
    if (lpp_window_Q_pairs_workspace_size(n_s, &need) != LPP_OK) return LPP_ERR_INVALID_ARG;
    if (!observer || !s_edges || !q || n < 0 || (n > 0 && !pos) || box < 0.0 || !(alpha > 0.0))
        return LPP_ERR_INVALID_ARG;
    if (!(s_edges[0] >= 0.0)) return LPP_ERR_INVALID_ARG;
    for (int b = 0; b < n_s; ++b)
        if (!(s_edges[b] < s_edges[b + 1])) return LPP_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255) != 0) return LPP_ERR_INVALID_ARG;
    if (bytes < need) return LPP_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = static_cast<char*>(workspace);
    double* d_out = reinterpret_cast<double*>(ws);
    double* d_edges = reinterpret_cast<double*>(ws + align256((size_t)n_s * kEll * sizeof(double)));
    double* d_norm = reinterpret_cast<double*>(ws + align256((size_t)n_s * kEll * sizeof(double)) +
                                               align256((size_t)(n_s + 1) * sizeof(double)));
    if (cudaMemsetAsync(d_out, 0, (size_t)n_s * kEll * sizeof(double), st) != cudaSuccess) return LPP_ERR_CUDA;
    if (cudaMemsetAsync(d_norm, 0, sizeof(double), st) != cudaSuccess) return LPP_ERR_CUDA;
    if (cudaMemcpyAsync(d_edges, s_edges, (size_t)(n_s + 1) * sizeof(double), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return LPP_ERR_CUDA;
    if (n > 0) {
        long long nbk = (n + 255) / 256;
        if (nbk > 152 * 8) nbk = 152 * 8;
        k_nw2_sum<<<(int)nbk, 256, 0, st>>>(w, nbar, n, d_norm);
        PairArgs a;
        memset(&a, 0, sizeof(a));
        a.pos = pos;
        a.w = w;
        a.n = n;
        a.n_tiles = (int)((n + kTile - 1) / kTile);
        for (int k = 0; k < 3; ++k) a.obs[k] = observer[k];
        a.box = box;
        a.edges = d_edges;
        a.nb = n_s;
        a.out = d_out;
        const size_t smem = ((size_t)kWarps * n_s * kEll + 7 * kTile + n_s + 1) * sizeof(double);
        if (cudaFuncSetAttribute(k_pair_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return LPP_ERR_CUDA;
        const long long tp = (long long)a.n_tiles * (a.n_tiles + 1) / 2;
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long grid = tp < (long long)sms * 4 ? tp : (long long)sms * 4;
        k_pair_sums<<<(int)grid, kTile, smem, st>>>(a);
        if (cudaGetLastError() != cudaSuccess) return LPP_ERR_CUDA;
    }
    std::vector<double> h_out((size_t)n_s * kEll);
    double h_norm = 0.0;
    if (cudaMemcpyAsync(h_out.data(), d_out, h_out.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return LPP_ERR_CUDA;
    if (cudaMemcpyAsync(&h_norm, d_norm, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LPP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LPP_ERR_CUDA;
    const double I = alpha * h_norm;
    const double pi = 3.14159265358979323846;
    for (int e = 0; e < kEll; ++e)
        for (int b = 0; b < n_s; ++b) {
            const double vol = 4.0 * pi * (s_edges[b + 1] * s_edges[b + 1] * s_edges[b + 1] -
                                           s_edges[b] * s_edges[b] * s_edges[b]) / 3.0;
            q[e * n_s + b] = I > 0.0 ? (4.0 * e + 1.0) * alpha * alpha * h_out[(size_t)b * kEll + e] / (I * vol) : 0.0;
        }
    return LPP_OK;
}
