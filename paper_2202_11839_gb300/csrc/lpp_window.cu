// Window multipoles Q_l(s) (Eq. windowQ_ell with the endpoint line of sight d = x).
//
// With the addition theorem L_l(s.x) = 4 pi / (2l+1) sum_n Y_{l,n}(s) Y_{l,n}(x) (real
// harmonics), Q_l(s) = 4 pi < sum_n Y_{l,n}(s) C_n(s) >_shell / I with the
// cross-correlations C_n(s) = int_x A_n(x) W(x+s) of A_n = W Y_{l,n}(x) and W.  Each C_n is
// IFFT[conj(A_n(k)) W(k)]; two real fields share one complex grid, so a pass packs
// C_a + i C_b and the inverse transform returns both correlations at once.
#include "lpp_internal.h"
#include "lpp_kernels.h"
#include "lpp_reduce.cuh"

namespace lpp {

template <typename T>
__global__ void k_window_partner(const c2<T>* __restrict__ grid, c2<T>* __restrict__ pD, const T* __restrict__ inv_w,
                                 int n) {
    const long long n3 = (long long)n * n * n;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n3;
         m += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(m % n), y = (int)((m / n) % n), z = (int)(m / ((long long)n * n));
        pD[m] = cscale<T>(grid[m], inv_w[x] * inv_w[y] * inv_w[z]);
    }
}

template <typename T>
cudaError_t launch_window_partner(const c2<T>* grid, c2<T>* pD, const T* inv_w, int n, cudaStream_t st) {
    k_window_partner<T><<<152 * 8, 256, 0, st>>>(grid, pD, inv_w, n);
    return cudaGetLastError();
}

// One thread per mode pair (m, -m): rows (z, y) with z in [0, n/2]; in the self-conjugate
// planes z = 0 and z = n/2 the pair is taken from its lexicographically smaller member.
template <typename T>
__global__ void k_window_mult(c2<T>* __restrict__ grids, long long grid_stride, const c2<T>* __restrict__ pD,
                              const T* __restrict__ inv_w, int n) {
    c2<T>* g = grids + (long long)blockIdx.y * grid_stride;
    const int rows = (n / 2 + 1) * n;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int z = row / n, y = row - z * n;
        const int zp = (n - z) & (n - 1), yp = (n - y) & (n - 1);
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            const int xp = (n - x) & (n - 1);
            if (z == zp && (y > yp || (y == yp && x > xp))) continue;
            const long long im = ((long long)z * n + y) * n + x;
            const long long ip = ((long long)zp * n + yp) * n + xp;
            const c2<T> zm = g[im], zq = g[ip];
            const T h = (T)0.5;
            const c2<T> A = mk<T>(h * (zm.x + zq.x), h * (zm.y - zq.y));        // (Z(m) + conj Z(-m)) / 2
            const c2<T> B = mk<T>(h * (zm.y + zq.y), -h * (zm.x - zq.x));       // -i (Z(m) - conj Z(-m)) / 2
            const T wm = inv_w[x] * inv_w[y] * inv_w[z];
            const T wp = inv_w[xp] * inv_w[yp] * inv_w[zp];
            const c2<T> Pm = pD[im], Pp = pD[ip];
            // conj(F/W) P at m; the fields at -m are conj A, conj B
            const c2<T> ca = cmul<T>(cconj<T>(cscale<T>(A, wm)), Pm);
            const c2<T> cb = cmul<T>(cconj<T>(cscale<T>(B, wm)), Pm);
            g[im] = mk<T>(ca.x - cb.y, ca.y + cb.x);                            // Ca + i Cb
            if (ip != im) {
                const c2<T> da = cmul<T>(cscale<T>(A, wp), Pp);
                const c2<T> db = cmul<T>(cscale<T>(B, wp), Pp);
                g[ip] = mk<T>(da.x - db.y, da.y + db.x);
            }
        }
    }
}

template <typename T>
cudaError_t launch_window_mult(c2<T>* grids, long long grid_stride, int n_grids, const c2<T>* pD, const T* inv_w,
                               int n, cudaStream_t st) {
    const int rows = (n / 2 + 1) * n;
    int bx = rows < 152 * 8 ? rows : 152 * 8;
    const int threads = n < 256 ? n : 256;
    k_window_mult<T><<<dim3(bx, n_grids), threads, 0, st>>>(grids, grid_stride, pD, inv_w, n);
    return cudaGetLastError();
}

// Shell sums over separations: rows (sz, sy) of the kept cube; lanes cover sx >= 0 and
// sx < 0 in two halves so that |s| grows monotonically along each warp.
template <typename T>
__global__ void __launch_bounds__(1024) k_sbin(SbinArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, nb = a.nb;
    const int E = a.n_ch * nb * 2;
    T* acc = reinterpret_cast<T*>(smem_raw);
    T* own = acc + E;
    int* thr = reinterpret_cast<int*>(own + E * Owned<T>::words);
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < E; i += nthr) acc[i] = (T)0;
    for (int i = tid; i < E * Owned<T>::words; i += nthr) own[i] = (T)0;
    for (int i = tid; i <= nb; i += nthr) thr[i] = a.thr[i];
    __syncthreads();
    const int P = nthr / 2;
    const int fx = tid < P ? tid : -1 - (tid - P);
    const bool xvalid = tid < P ? (fx <= a.ns_pos) : (-fx <= a.ns_neg);
    const int x = fx >= 0 ? fx : n + fx;
    const int rows = a.nks * a.nks;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int zj = row / a.nks, yj = row - zj * a.nks;
        const int z = zj <= a.ns_pos ? zj : n - (a.nks - zj);
        const int y = yj <= a.ns_pos ? yj : n - (a.nks - yj);
        const int fz = z < n / 2 ? z : z - n, fy = y < n / 2 ? y : y - n;
        const int q2 = fx * fx + fy * fy + fz * fz;
        int bin = -1;
        if (xvalid && q2 > 0 && q2 >= thr[0] && q2 < thr[nb]) {
            int lo = 0, hi = nb;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (q2 >= thr[mid]) lo = mid; else hi = mid;
            }
            bin = lo;
        }
        T sxh = 0, syh = 0, szh = 0;
        long long idx = 0;
        if (bin >= 0) {
            const T inv = (T)1 / sqrt((T)q2);
            sxh = fx * inv;
            syh = fy * inv;
            szh = fz * inv;
            idx = ((long long)z * n + y) * n + x;
        }
        for (int ci = 0; ci < a.n_ch; ++ci) {
            const SbinChan& ch = a.ch[ci];
            T v = 0;
            if (bin >= 0) {
                const c2<T> c = a.grids[(long long)ch.grid * a.grid_stride + idx];
                const T corr = (ch.sub ? c.y : c.x) * (T)a.scale;
                v = (T)ch.ynorm * ylm_poly<T>(ch.l, ch.m, sxh, syh, szh) * corr;
            }
            warp_bin_add<T>(v, (T)0, bin, acc + ci * 2 * nb);
        }
        __syncthreads();
        for (int i = tid; i < E; i += nthr) {
            const T v = acc[i];
            if (v != (T)0) {
                Owned<T>::add(own + i, own + E + i, v);
                acc[i] = (T)0;
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < E; i += nthr) {
        const double v = Owned<T>::value(own + i, own + E + i);
        if (v != 0.0) {
            const int ci = i / (2 * nb);
            atomicAdd(a.out + (long long)a.ch[ci].out_row * 2 * nb + (i - ci * 2 * nb), v);
        }
    }
}

template <typename T>
cudaError_t launch_sbin(const SbinArgs<T>& a, int n_sm, cudaStream_t st) {
    const int P = ((a.ns_pos + 1) + 31) / 32 * 32;
    const int threads = 2 * P;
    const int E = a.n_ch * a.nb * 2;
    const size_t smem = (size_t)E * sizeof(T) * (1 + Owned<T>::words) + (size_t)(a.nb + 1) * sizeof(int);
    cudaFuncSetAttribute(k_sbin<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int rows = a.nks * a.nks;
    int blocks = n_sm * (threads <= 256 ? 8 : (threads <= 512 ? 4 : 2));
    if (blocks > rows) blocks = rows;
    k_sbin<T><<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_window_partner<float>(const c2<float>*, c2<float>*, const float*, int, cudaStream_t);
template cudaError_t launch_window_partner<double>(const c2<double>*, c2<double>*, const double*, int, cudaStream_t);
template cudaError_t launch_window_mult<float>(c2<float>*, long long, int, const c2<float>*, const float*, int,
                                               cudaStream_t);
template cudaError_t launch_window_mult<double>(c2<double>*, long long, int, const c2<double>*, const double*, int,
                                                cudaStream_t);
template cudaError_t launch_sbin<float>(const SbinArgs<float>&, int, cudaStream_t);
template cudaError_t launch_sbin<double>(const SbinArgs<double>&, int, cudaStream_t);

}  // namespace lpp
