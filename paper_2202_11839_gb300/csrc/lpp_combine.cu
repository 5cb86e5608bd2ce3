// k-space combination and FP64 shell sums (Sec. 3.1.2 estimators).
//
// A batch grid Z holds two real fields packed as Z = a + i b: either the two
// interlaced sub-grids of one field, or two different fields.  Their DFTs are
// recovered exactly from the pair of modes (m, -m):
//   A(m) = (Z(m) + conj Z(-m)) / 2,   B(m) = -i (Z(m) - conj Z(-m)) / 2,
//   A(-m) = conj A(m),  B(-m) = conj B(m).
// Interlaced fields become F = (A + e^{-i pi (fx+fy+fz)/n} B) / 2, and every field is
// divided by the assignment window prod_a sinc^p(pi f_a / n) when compensation is on.
//
// One CTA walks rows (fz, fy) of kept modes; its lanes cover fx >= 0 (first half)
// and fx < 0 (second half), so |k| grows monotonically along each warp and equal
// shells form contiguous lane runs.  Per-mode products are reduced within a warp by a
// segmented scan, added to FP32 shared-memory partials per row, and folded after every
// row into compensated (two-float) or FP64 accumulators that the CTA flushes to the
// global FP64 shell sums once at the end.
#include "lpp_internal.h"
#include "lpp_kernels.h"
#include "lpp_reduce.cuh"

namespace lpp {

template <typename T>
struct ModeCtx {
    c2<T> ph_m, ph_p;   // interlace phases at m and -m
    T iw_m, iw_p;       // inverse windows
    long long im, ip;   // linear indices of m and of its mirror
    bool self;          // m == -m (index-wise)
};

// DFTs of the two packed fields at m; the values at the mirror are their conjugates.
template <typename T>
__device__ __forceinline__ void unpack(const c2<T>* g, const ModeCtx<T>& c, c2<T>& A, c2<T>& B) {
    const c2<T> zm = g[c.im];
    const c2<T> zp = g[c.ip];
    const T h = (T)0.5;
    A = mk<T>(h * (zm.x + zp.x), h * (zm.y - zp.y));
    // B = -i (zm - conj zp) / 2
    const T dr = zm.x - zp.x, di = zm.y + zp.y;
    B = mk<T>(h * di, -h * dr);
}

// k-space field at m and -m for sub-field `sub` of a slot, from its packed values.
template <typename T>
__device__ __forceinline__ void field_of(c2<T> zm, c2<T> zp, int sub, int interlace, const ModeCtx<T>& c, c2<T>& Fm,
                                         c2<T>& Fp) {
    const T h = (T)0.5;
    const c2<T> A = mk<T>(h * (zm.x + zp.x), h * (zm.y - zp.y));
    const c2<T> B = mk<T>(h * (zm.y + zp.y), -h * (zm.x - zp.x));   // -i (zm - conj zp) / 2
    if (interlace) {
        Fm = cscale<T>(cadd<T>(A, cmul<T>(c.ph_m, B)), h * c.iw_m);
        Fp = cscale<T>(cadd<T>(cconj<T>(A), cmul<T>(c.ph_p, cconj<T>(B))), h * c.iw_p);
    } else {
        const c2<T> X = sub ? B : A;
        Fm = cscale<T>(X, c.iw_m);
        Fp = cscale<T>(cconj<T>(X), c.iw_p);
    }
}

// k-space field at m and -m for sub-field `sub` of a slot.
template <typename T>
__device__ __forceinline__ void field_at(const c2<T>* g, int sub, int interlace, const ModeCtx<T>& c, c2<T>& Fm,
                                         c2<T>& Fp) {
    field_of<T>(g[c.im], g[c.ip], sub, interlace, c, Fm, Fp);
}

// ylm_poly_scaled(L, +-M, x, y, z) with L and M known at compile time: the same recurrence
// with constant coefficients and no loops; use_im selects the sine part (n < 0).
template <typename T, int L, int M>
__device__ __forceinline__ T ylm_fixed(T x, T y, T z, bool use_im) {
    T qmm = (T)1;
#pragma unroll
    for (int i = 1; i <= M; ++i) qmm *= (T)(2 * i - 1);
    T q = qmm;
    if constexpr (L > M) {
        T q0 = qmm, q1 = (T)(2 * M + 1) * z * qmm;
#pragma unroll
        for (int l = M + 2; l <= L; ++l) {
            const T q2 = (T)(2 * l - 1) * z * q1 - (T)((l + M - 1) * (l - M - 1)) * q0;
            q0 = q1;
            q1 = q2;
        }
        q = q1;
    }
    if constexpr (M == 0) {
        return q;
    } else {
        T re = x, im = y;
#pragma unroll
        for (int i = 1; i < M; ++i) {
            const T t = re * x - im * y;
            im = re * y + im * x;
            re = t;
        }
        return q * (use_im ? im : re);
    }
}

// The channel's harmonic (warp-uniform L, n): the estimators' even degrees up to 8 by a
// compile-time case, anything else by the general recurrence.
template <typename T>
__device__ __forceinline__ T ylm_channel(int L, int n, T x, T y, T z) {
    const int m = n < 0 ? -n : n;
    const bool use_im = n < 0;
    switch (L * 16 + m) {
#define LPP_YCASE(LL, MM) \
    case LL * 16 + MM:    \
        return ylm_fixed<T, LL, MM>(x, y, z, use_im);
        LPP_YCASE(0, 0)
        LPP_YCASE(2, 0) LPP_YCASE(2, 1) LPP_YCASE(2, 2)
        LPP_YCASE(4, 0) LPP_YCASE(4, 1) LPP_YCASE(4, 2) LPP_YCASE(4, 3) LPP_YCASE(4, 4)
        LPP_YCASE(6, 0) LPP_YCASE(6, 1) LPP_YCASE(6, 2) LPP_YCASE(6, 3) LPP_YCASE(6, 4) LPP_YCASE(6, 5)
        LPP_YCASE(6, 6)
        LPP_YCASE(8, 0) LPP_YCASE(8, 1) LPP_YCASE(8, 2) LPP_YCASE(8, 3) LPP_YCASE(8, 4) LPP_YCASE(8, 5)
        LPP_YCASE(8, 6) LPP_YCASE(8, 7) LPP_YCASE(8, 8)
#undef LPP_YCASE
        default:
            return ylm_poly_scaled<T>(L, n, x, y, z);
    }
}

// COMPACT: walk the work list (a.items, 256 threads, three CTAs per SM); otherwise one pass
// per whole row (up to 1024 threads)
template <typename T, bool COMPACT>
__global__ void __launch_bounds__(COMPACT ? 256 : 1024, COMPACT ? 3 : 1) k_combine(CombineArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n;
    const int nb = a.nb;
    const int nacc = a.partner_mode ? 2 : a.n_ch;
    const int E = nacc * nb * 2;
    T* acc = reinterpret_cast<T*>(smem_raw);                       // [nacc][nb][2] per-row partials
    T* own = acc + E;                                              // [E][words] owned accumulators
    T* iw = own + E * Owned<T>::words;                             // [n]
    c2<T>* ph = reinterpret_cast<c2<T>*>(iw + n + (n & 1));        // [n]
    int* thr = reinterpret_cast<int*>(ph + n);                     // [nb+1]

    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    for (int i = tid; i < E; i += nthr) acc[i] = (T)0;
    for (int i = tid; i < E * Owned<T>::words; i += nthr) own[i] = (T)0;
    for (int i = tid; i < n; i += nthr) { iw[i] = a.inv_w[i]; ph[i] = a.phase[i]; }
    for (int i = tid; i <= nb; i += nthr) thr[i] = a.thr[i];
    __syncthreads();

    auto fold = [&]() {
        __syncthreads();
        for (int i = tid; i < E; i += nthr) {
            const T v = acc[i];
            if (v != (T)0) {
                Owned<T>::add(own + i, own + E + i, v);
                acc[i] = (T)0;
            }
        }
        __syncthreads();
    };
    // The work of one mode pair (m, -m) with m = (fx, y, z) (grid indices y, z); xvalid: the
    // lane has a mode; half: 0 for fx >= 0, 1 for fx < 0 (shell labels are monotone within a
    // half, so (half, bin) keys the lane's segment in the warp-segmented sums).  Every lane of
    // the warp calls it (the shell sums are warp-collective).
    auto mode_work = [&](bool xvalid, int fx, int z, int y, int half) {
        // shell label (contiguous along the warp) and whether this lane owns the pair
        const int x = fx >= 0 ? fx : n + fx;
        const int xp = (n - x) & (n - 1);
        const int fxp = freq_of<T>(xp, n);
        const int zp = (n - z) & (n - 1);
        const int yp = (n - y) & (n - 1);
        const int fz = freq_of<T>(z, n), fy = freq_of<T>(y, n);
        const int fzp = freq_of<T>(zp, n), fyp = freq_of<T>(yp, n);
        const int q2 = fx * fx + fy * fy + fz * fz;
        int bin = -1;
        if (xvalid && q2 > 0 && q2 >= thr[0] && q2 < thr[nb]) {
            int lo = 0, hi = nb;  // thr[lo] <= q2 < thr[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (q2 >= thr[mid]) lo = mid; else hi = mid;
            }
            bin = lo;
        }
        bool own_pair = bin >= 0;
        ModeCtx<T> c;
        c.self = false;
        if (own_pair && z == zp) {
            // self-conjugate plane: take each pair once, from its lexicographically smaller member
            if (y > yp || (y == yp && x > xp)) own_pair = false;
            c.self = (y == yp && x == xp);
        }
        T kx = 0, ky = 0, kz = 0, kxp = 0, kyp = 0, kzp = 0;
        if (own_pair) {
            c.im = ((long long)z * n + y) * n + x;
            c.ip = ((long long)zp * n + yp) * n + xp;
            const long long n3 = (long long)n * n * n;
            if (!LPP_IN_BOUNDS(c.im >= 0 && c.im < n3 && c.ip >= 0 && c.ip < n3 && bin < nb, a.err)) own_pair = false;
        }
        if (own_pair) {
            c.iw_m = iw[x] * iw[y] * iw[z];
            c.iw_p = iw[xp] * iw[yp] * iw[zp];
            c.ph_m = cmul<T>(cmul<T>(ph[x], ph[y]), ph[z]);
            c.ph_p = cmul<T>(cmul<T>(ph[xp], ph[yp]), ph[zp]);
            const T inv = (T)1 / sqrt((T)q2);
            kx = fx * inv; ky = fy * inv; kz = fz * inv;
            kxp = fxp * inv; kyp = fyp * inv; kzp = fzp * inv;
        }
        if (a.partner_mode) {
            T dd = 0, gg = 0;
            if (own_pair) {
                // partner grids: interlaced -> G1 | G2 | D one field per grid;
                // otherwise (G1, G2) packed in one grid, then (D, -)
                const c2<T>* g0 = a.grids;
                int slot = 0;
                c2<T> Dm = mk<T>(0, 0), Dp = Dm, G1m = Dm, G1p = Dm, G2m = Dm, G2p = Dm;
                if (a.interlace) {
                    if (a.has_g) {
                        field_at<T>(g0 + (slot++) * a.grid_stride, 0, 1, c, G1m, G1p);
                        field_at<T>(g0 + (slot++) * a.grid_stride, 0, 1, c, G2m, G2p);
                    }
                    if (a.has_d) field_at<T>(g0 + slot * a.grid_stride, 0, 1, c, Dm, Dp);
                } else {
                    if (a.has_g) {
                        field_at<T>(g0, 0, 0, c, G1m, G1p);
                        field_at<T>(g0, 1, 0, c, G2m, G2p);
                        ++slot;
                    }
                    if (a.has_d) field_at<T>(g0 + slot * a.grid_stride, 0, 0, c, Dm, Dp);
                }
                if (a.has_d) {
                    if (a.pD) {   // null: the caller wants only the shell sums
                        a.pD[c.im] = Dm;
                        a.pD[c.ip] = Dp;
                    }
                    dd = Dm.x * Dm.x + Dm.y * Dm.y;
                    if (!c.self) dd += Dp.x * Dp.x + Dp.y * Dp.y;
                }
                if (a.has_g) {
                    a.pG1[c.im] = G1m;
                    a.pG1[c.ip] = G1p;
                    a.pG2[c.im] = G2m;
                    a.pG2[c.ip] = G2p;
                    // G = G1 + i G2: the transform of the complex shear field
                    const T gr = G1m.x - G2m.y, gi = G1m.y + G2m.x;
                    gg = gr * gr + gi * gi;
                    if (!c.self) {
                        const T hr = G1p.x - G2p.y, hi2 = G1p.y + G2p.x;
                        gg += hr * hr + hi2 * hi2;
                    }
                }
            }
            const int key = bin >= 0 ? bin + half * 65536 : -1;
            warp_bin_add<T>(dd, (T)0, bin, acc, key);
            warp_bin_add<T>(gg, (T)0, bin, acc + 2 * nb, key);
        } else {
            c2<T> Dm = mk<T>(0, 0), Dp = Dm, G1m = Dm, G1p = Dm, G2m = Dm, G2p = Dm;
            if (own_pair) {
                if (a.has_d) { Dm = a.pD[c.im]; Dp = a.pD[c.ip]; }
                if (a.has_g) { G1m = a.pG1[c.im]; G1p = a.pG1[c.ip]; G2m = a.pG2[c.im]; G2p = a.pG2[c.ip]; }
            }
            // the mirror is exactly -k unless an index sits at the Nyquist frequency; then an
            // even-degree harmonic takes the same value at both members of the pair
            const bool mirror_neg = (fxp == -fx) && (fyp == -fy) && (fzp == -fz);
            // a warp none of whose lanes owns a mode pair (rows near the last shell) has
            // nothing to add: it skips the channels (warp-uniform)
            const bool warp_live = __any_sync(0xffffffffu, own_pair);
            const SegMask segm = seg_mask(bin >= 0 ? bin + half * 65536 : -1);
            const int n_slots = warp_live ? (a.n_ch + a.per_grid - 1) / a.per_grid : 0;
            // four slots at a time: their packed values at m and -m are loaded together
            for (int s0 = 0; s0 < n_slots; s0 += 4) {
                c2<T> zm[4], zp[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    zm[k] = zp[k] = mk<T>(0, 0);
                    if (own_pair && s0 + k < n_slots) {
                        const c2<T>* g = a.grids + (long long)(s0 + k) * a.grid_stride;
                        zm[k] = g[c.im];
                        zp[k] = g[c.ip];
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (s0 + k >= n_slots) break;
                    for (int sub = 0; sub < a.per_grid; ++sub) {
                        const int ci = (s0 + k) * a.per_grid + sub;
                        if (ci >= a.n_ch) break;
                        const CombineChan& ch = a.ch[ci];
                        T tre = 0, tim = 0;
                        if (own_pair) {
                            c2<T> Fm, Fp;
                            field_of<T>(zm[k], zp[k], ch.sub, a.interlace, c, Fm, Fp);
                            if (ch.part == PART_IM) {
                                Fm = mk<T>(-Fm.y, Fm.x);
                                Fp = mk<T>(-Fp.y, Fp.x);
                            }
                            // partner: delta(-k) = conj D; gamma*(-k) = conj G1 - i conj G2;
                            // gamma(-k) = conj G1 + i conj G2
                            c2<T> Pm, Pp;
                            if (ch.kind == KIND_CROSS || ch.kind == KIND_DENS) {
                                Pm = cconj<T>(Dm);
                                Pp = cconj<T>(Dp);
                            } else {
                                const T s = ch.kind == KIND_PLUS ? (T)-1 : (T)1;
                                // conj(G1) + s i conj(G2)
                                Pm = mk<T>(G1m.x + s * G2m.y, -G1m.y + s * G2m.x);
                                Pp = mk<T>(G1p.x + s * G2p.y, -G1p.y + s * G2p.x);
                            }
                            const T yn = (T)ch.ynorm;
                            const T ym = yn * ylm_channel<T>(ch.L, ch.n, kx, ky, kz);
                            c2<T> t = cscale<T>(cmul<T>(Fm, Pm), ym);
                            if (!c.self) {
                                const T yp2 = (mirror_neg && (ch.L & 1) == 0)
                                                  ? ym
                                                  : yn * ylm_channel<T>(ch.L, ch.n, kxp, kyp, kzp);
                                t = cadd<T>(t, cscale<T>(cmul<T>(Fp, Pp), yp2));
                            }
                            tre = t.x;
                            tim = t.y;
                        }
                        warp_bin_add_seg<T>(tre, tim, bin, segm, acc + ci * 2 * nb);
                    }
                }
            }
        }
    };

    if constexpr (!COMPACT) {
        // one pass per row (fz, fy) of the kept cube; lanes cover fx >= 0 (first half) and
        // fx < 0 (second half)
        const int P = nthr / 2;
        const int fx = tid < P ? tid : -1 - (tid - P);
        const bool xvalid = tid < P ? (fx <= a.nk_pos) : (-fx <= a.nk_neg);
        const int rows = a.nzi * a.nky;
        int nrow = 0;
        for (int row = blockIdx.x; row < rows; row += gridDim.x) {
            const int zi = row / a.nky;
            const int yj = row - zi * a.nky;
            const int z = zi <= a.nk_pos ? zi : n / 2;
            const int y = yj <= a.nk_pos ? yj : n - (a.nky - yj);
            const int fz = freq_of<T>(z, n), fy = freq_of<T>(y, n);
            if (fy * fy + fz * fz >= thr[nb]) continue;   // no mode of this row lies in a shell (CTA-uniform)
            mode_work(xvalid, fx, z, y, tid < P ? 0 : 1);
            // fold the partials into the compensated accumulators every second row (a row pair
            // adds at most 2 x 16 warp segments per shell to an FP32 partial)
            if ((++nrow & 1) == 0) fold();
        }
        if (nrow & 1) fold();
    } else {
        // the work list: each warp takes one item (32 consecutive modes of a row inside the
        // last shell) per round; the partials are folded after every round
        const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
        for (int base = blockIdx.x * nw; base < a.n_items; base += gridDim.x * nw) {
            const int it = base + warp;
            bool xvalid = false;
            int fx = 0, z = 0, y = 0, half = 0;
            if (it < a.n_items) {
                const int4 item = a.items[it];
                const int zi = item.x / a.nky;
                const int yj = item.x - zi * a.nky;
                z = zi <= a.nk_pos ? zi : n / 2;
                y = yj <= a.nk_pos ? yj : n - (a.nky - yj);
                const int t = item.y + lane;
                xvalid = t <= item.z + item.w;
                half = t > item.z ? 1 : 0;
                fx = half ? -(t - item.z) : t;
            }
            mode_work(xvalid, fx, z, y, half);
            fold();
        }
    }
    for (int i = tid; i < E; i += nthr) {
        const double v = Owned<T>::value(own + i, own + E + i);
        if (v != 0.0) {
            const int ci = i / (2 * nb);
            const int rem = i - ci * 2 * nb;
            const int row_out = a.partner_mode ? (ci == 0 ? a.row_dd0 : a.row_plus0) : a.ch[ci].out_row;
            if (row_out >= 0) atomicAdd(a.out + (long long)row_out * 2 * nb + rem, v);
        }
    }
}

template <typename T>
cudaError_t launch_combine(const CombineArgs<T>& a, int n_sm, cudaStream_t st) {
    const int nacc = a.partner_mode ? 2 : a.n_ch;
    const int E = nacc * a.nb * 2;
    size_t smem = (size_t)E * sizeof(T) * (1 + Owned<T>::words) + (size_t)(a.n + (a.n & 1)) * sizeof(T) +
                  (size_t)a.n * sizeof(c2<T>) + (size_t)(a.nb + 1) * sizeof(int);
    if (a.items != nullptr) {
        // 8 warps per CTA, three CTAs per SM
        cudaFuncSetAttribute(k_combine<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int threads = 256;
        int blocks = n_sm * 3;
        const int rounds = (a.n_items + 7) / 8;
        if (blocks > rounds) blocks = rounds > 0 ? rounds : 1;
        k_combine<T, true><<<blocks, threads, smem, st>>>(a);
        return cudaGetLastError();
    }
    cudaFuncSetAttribute(k_combine<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int P = ((a.nk_pos + 1) + 31) / 32 * 32;
    const int threads = 2 * P;
    const int rows = a.nzi * a.nky;
    int blocks = n_sm * (threads <= 256 ? 8 : (threads <= 512 ? 4 : 2));
    if (blocks > rows) blocks = rows;
    k_combine<T, false><<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

void combine_items(int n, int nk_pos, int nk_neg, int nky, int nzi, int q_max, std::vector<int4>& items) {
    items.clear();
    for (int zi = 0; zi < nzi; ++zi) {
        const int z = zi <= nk_pos ? zi : n / 2;
        const int fz = z < n / 2 ? z : z - n;
        for (int yj = 0; yj < nky; ++yj) {
            const int y = yj <= nk_pos ? yj : n - (nky - yj);
            const int fy = y < n / 2 ? y : y - n;
            const long long rem = (long long)q_max - (long long)fy * fy - (long long)fz * fz;
            if (rem <= 0) continue;
            // |fx| <= xr with fx^2 < rem
            int xr = 0;
            while ((long long)(xr + 1) * (xr + 1) < rem) ++xr;
            const int xp = xr < nk_pos ? xr : nk_pos;
            const int xn = xr < nk_neg ? xr : nk_neg;
            const int m = xp + 1 + xn;
            for (int t0 = 0; t0 < m; t0 += 32) items.push_back(make_int4(zi * nky + yj, t0, xp, xn));
        }
    }
}

template cudaError_t launch_combine<float>(const CombineArgs<float>&, int, cudaStream_t);
template cudaError_t launch_combine<double>(const CombineArgs<double>&, int, cudaStream_t);

}  // namespace lpp
