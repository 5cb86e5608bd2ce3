// Device-side building blocks of the shared-memory pencil FFT (internal).
//
// A tile holds W pencils of N complex points in shared memory as tile[e * ld + c]
// (point e of pencil c, ld >= W).  Every thread owns IPT pencils c, c + W/IPT, ...
// and, in each Stockham stage, the 8 points of one radix-8 butterfly (or two radix-4 /
// four radix-2 butterflies) of each of them.  Consecutive threads own consecutive
// pencils, so shared-memory accesses of a warp are contiguous.
#pragma once

#include "lpp_internal.h"

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

// One Stockham stage of radix R on every pencil of the tile.  The thread owns pencil c
// and the butterfly slots u + s US (s < IPT, US = N / (8 IPT)), each slot being one
// radix-8 butterfly or 8/R radix-R ones (j = slot + q N/8).  Consecutive threads own
// consecutive pencils at the same slot, so with an odd LD the 16 threads of a half warp
// touch 16 different banks pairs (no conflicts) and read the same twiddle (a broadcast).
// LD and the stage's sub-transform length NS are compile-time, so every address is a
// per-thread base plus an immediate offset; the first stage (NS = 1) has no twiddles.
template <typename T, int N, int R, bool INV, int IPT, int LD, int NS>
__device__ __forceinline__ void stockham_stage(c2<T>* tile, int c, int u, const c2<T>* tw) {
    constexpr int Q = 8 / R;
    constexpr int US = N / (8 * IPT);
    c2<T> v[IPT][8];
    const c2<T>* src = tile + u * LD + c;
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[s][q * R + r] = src[(s * US + q * (N / 8) + r * (N / R)) * LD];
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int j = u + s * US + q * (N / 8);
            const int jm = j & (NS - 1);
            if (NS > 1) {
                const int step = jm * (N / (NS * R));
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    c2<T> w = tw[step * r];
                    if (INV) w.y = -w.y;
                    v[s][q * R + r] = cmul<T>(v[s][q * R + r], w);
                }
            }
            if (R == 8) dft8<T, INV>(v[s] + q * R);
            else if (R == 4) dft4<T, INV>(v[s] + q * R);
            else dft2<T, INV>(v[s] + q * R);
            c2<T>* dst = tile + ((j - jm) * R + jm) * LD + c;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[r * NS * LD] = v[s][q * R + r];
        }
    }
    __syncthreads();
}

template <typename T, int N, bool INV, int IPT, int LD, int NS>
__device__ __forceinline__ void radix8_stages(c2<T>* tile, int c, int u, const c2<T>* tw) {
    if constexpr (NS < N) {
        stockham_stage<T, N, 8, INV, IPT, LD, NS>(tile, c, u, tw);
        radix8_stages<T, N, INV, IPT, LD, NS * 8>(tile, c, u, tw);
    }
}

// Forward (or inverse, unnormalised) FFT of length N = 2^LOGN along every pencil: one
// radix-2 or radix-4 stage when LOGN is not a multiple of 3, then radix-8 stages.
// c = the thread's pencil, u = its first butterfly slot (0 .. N / (8 IPT) - 1).
template <typename T, int LOGN, bool INV, int IPT, int LD>
__device__ __forceinline__ void fft_columns(c2<T>* tile, int c, int u, const c2<T>* tw) {
    constexpr int N = 1 << LOGN;
    constexpr int rem = LOGN % 3;
    if constexpr (rem == 1) {
        stockham_stage<T, N, 2, INV, IPT, LD, 1>(tile, c, u, tw);
        radix8_stages<T, N, INV, IPT, LD, 2>(tile, c, u, tw);
    } else if constexpr (rem == 2) {
        stockham_stage<T, N, 4, INV, IPT, LD, 1>(tile, c, u, tw);
        radix8_stages<T, N, INV, IPT, LD, 4>(tile, c, u, tw);
    } else {
        radix8_stages<T, N, INV, IPT, LD, 1>(tile, c, u, tw);
    }
}

// ---- stages with their operands outside the tile ----------------------------------------
// Radix of the leading stage for N = 2^LOGN (2 or 4 when LOGN is not a multiple of 3).
template <int LOGN>
struct LeadRadix {
    static constexpr int R = LOGN % 3 == 1 ? 2 : (LOGN % 3 == 2 ? 4 : 8);
};

// Point of the thread's pencil that operand b (= s 8 + q R + r) of the leading stage
// reads: butterfly slot u + s US + q N/8, leg r.
template <int LOGN, int IPT>
__device__ __forceinline__ int lead_row(int u, int b) {
    constexpr int N = 1 << LOGN, R = LeadRadix<LOGN>::R, US = N / (8 * IPT);
    const int s = b >> 3, q = (b & 7) / R, r = (b & 7) % R;
    return u + s * US + q * (N / 8) + r * (N / R);
}

// Leading stage (NS = 1, no twiddles) with operand b of point e from load(b, e); results
// to the tile.  INPLACE: load reads the tile itself (a barrier separates the reads from
// the writes).  Ends with a barrier.
template <typename T, int LOGN, bool INV, int IPT, int LD, bool INPLACE, class Load>
__device__ __forceinline__ void lead_stage(c2<T>* tile, int c, int u, Load&& load) {
    constexpr int N = 1 << LOGN, R = LeadRadix<LOGN>::R, Q = 8 / R, US = N / (8 * IPT);
    c2<T> v[IPT][8];
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[s][k] = load(s * 8 + k, lead_row<LOGN, IPT>(u, s * 8 + k));
    }
    if (INPLACE) __syncthreads();
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int j = u + s * US + q * (N / 8);
            if (R == 8) dft8<T, INV>(v[s] + q * R);
            else if (R == 4) dft4<T, INV>(v[s] + q * R);
            else dft2<T, INV>(v[s] + q * R);
            c2<T>* dst = tile + j * R * LD + c;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[r * LD] = v[s][q * R + r];
        }
    }
    __syncthreads();
}

template <typename T, int N, bool INV, int IPT, int LD, int NS, int NS_END>
__device__ __forceinline__ void radix8_until(c2<T>* tile, int c, int u, const c2<T>* tw) {
    if constexpr (NS < NS_END) {
        stockham_stage<T, N, 8, INV, IPT, LD, NS>(tile, c, u, tw);
        radix8_until<T, N, INV, IPT, LD, NS * 8, NS_END>(tile, c, u, tw);
    }
}

// Last radix-8 stage (NS = N/8) from the tile, results to store(e, value): the butterfly
// at slot j writes points j + r N/8.  No barrier at the end.
template <typename T, int N, bool INV, int IPT, int LD, class Store>
__device__ __forceinline__ void last_stage(const c2<T>* tile, int c, int u, const c2<T>* tw, Store&& store) {
    constexpr int US = N / (8 * IPT);
    c2<T> v[IPT][8];
    const c2<T>* src = tile + u * LD + c;
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[s][r] = src[(s * US + r * (N / 8)) * LD];
    }
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
        const int j = u + s * US;
#pragma unroll
        for (int r = 1; r < 8; ++r) {
            c2<T> w = tw[j * r];
            if (INV) w.y = -w.y;
            v[s][r] = cmul<T>(v[s][r], w);
        }
        dft8<T, INV>(v[s]);
#pragma unroll
        for (int r = 0; r < 8; ++r) store(j + r * (N / 8), v[s][r]);
    }
}

// Last radix-8 stage (NS = N/8) with one warp per pencil: lane l of the warp for pencil c
// takes the butterflies at slots j = l + 32 s (s < IPT), so the points j + r N/8 that it
// hands to store(e, value) are consecutive across the warp (a coalesced store along the
// pencil).  twr holds each leg's twiddles by slot, twr[(r - 1) N/8 + j] = w^(j r), so the
// lanes read consecutive words.  No barrier at the end.
template <typename T, int N, bool INV, int IPT, int LD, class Store>
__device__ __forceinline__ void last_stage_warp(const c2<T>* tile, int c, int l, const c2<T>* twr, Store&& store) {
    static_assert(N / 8 == 32 * IPT, "one warp covers the N/8 butterfly slots of a pencil");
    c2<T> v[IPT][8];
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[s][r] = tile[(l + 32 * s + r * (N / 8)) * LD + c];
    }
#pragma unroll
    for (int s = 0; s < IPT; ++s) {
        const int j = l + 32 * s;
#pragma unroll
        for (int r = 1; r < 8; ++r) {
            c2<T> w = twr[(r - 1) * (N / 8) + j];
            if (INV) w.y = -w.y;
            v[s][r] = cmul<T>(v[s][r], w);
        }
        dft8<T, INV>(v[s]);
#pragma unroll
        for (int r = 0; r < 8; ++r) store(j + r * (N / 8), v[s][r]);
    }
}

// FFT of one pencil (column c of the tile; N = 64 R1 points, R1 = 4 or 8) by the 32 lanes
// of one warp, with __syncwarp between the passes and no block barrier.  With
// n = n0 + 8 n1 + 64 n2 and k = k0 + R1 k1 + 8 R1 k2:
//   pass 1: y1[m, k0] = w^(m k0) DFT_R1 over n2 of x[m + 64 n2]   (m = n0 + 8 n1)
//   pass 2: y2[n0, k0, k1] = w^(R1 n0 k1) DFT_8 over n1 of y1[n0 + 8 n1, k0]
//   pass 3: X[k0 + R1 k1 + 8 R1 k2] = DFT_8 over n0 of y2[n0, k0, k1]
// y1 sits at row 64 k0 + (m + 8 k0) % 64 and y2 at row 8 R1 n0 + (k0 + R1 k1 + 2 n0) % (8 R1),
// so that with an odd LD the 16 lanes of every half-warp access 16 different bank pairs in
// each pass.  load(e): point e of the input; store(k, value): output k (consecutive lanes
// store consecutive k).  t1[(k0 - 1) 64 + m] = w^(m k0) and t2[(k1 - 1) 8 + n0] = w^(R1 n0 k1)
// (forward twiddles; conjugated for INV).
template <typename T, int LOGN, bool INV, int LD, bool ZERO = false, class Load, class Store>
__device__ __forceinline__ void fft_pencil_warp(c2<T>* tile, int c, int lane, const c2<T>* t1, const c2<T>* t2,
                                                Load&& load, Store&& store) {
    constexpr int N = 1 << LOGN, R1 = N / 64, Q = 8 * R1, B = R1 / 4;
    static_assert(R1 == 4 || R1 == 8, "N = 256 or 512");
    c2<T>* col = tile + c;
    {
        c2<T> v[2][R1];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int n2 = 0; n2 < R1; ++n2) v[h][n2] = load(lane + 32 * h + 64 * n2);
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = lane + 32 * h;
            if (R1 == 8) dft8<T, INV>(v[h]);
            else dft4<T, INV>(v[h]);
#pragma unroll
            for (int k0 = 1; k0 < R1; ++k0) {
                c2<T> w = t1[(k0 - 1) * 64 + m];
                if (INV) w.y = -w.y;
                v[h][k0] = cmul<T>(v[h][k0], w);
            }
#pragma unroll
            for (int k0 = 0; k0 < R1; ++k0) col[(64 * k0 + ((m + 8 * k0) & 63)) * LD] = v[h][k0];
        }
        __syncwarp();
    }
    c2<T> v[B][8];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int m2 = lane + 32 * b, n0 = m2 & 7, k0 = m2 >> 3;
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) v[b][n1] = col[(64 * k0 + ((n0 + 8 * n1 + 8 * k0) & 63)) * LD];
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int m2 = lane + 32 * b, n0 = m2 & 7, k0 = m2 >> 3;
        dft8<T, INV>(v[b]);
#pragma unroll
        for (int k1 = 1; k1 < 8; ++k1) {
            c2<T> w = t2[(k1 - 1) * 8 + n0];
            if (INV) w.y = -w.y;
            v[b][k1] = cmul<T>(v[b][k1], w);
        }
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) col[(Q * n0 + ((k0 + R1 * k1 + 2 * n0) & (Q - 1))) * LD] = v[b][k1];
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int q = lane + 32 * b;
#pragma unroll
        for (int n0 = 0; n0 < 8; ++n0) v[b][n0] = col[(Q * n0 + ((q + 2 * n0) & (Q - 1))) * LD];
    }
    if constexpr (ZERO) {
        // every row of the column was read exactly once by this pass: leave the column zeroed
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int q = lane + 32 * b;
#pragma unroll
            for (int n0 = 0; n0 < 8; ++n0) col[(Q * n0 + ((q + 2 * n0) & (Q - 1))) * LD] = mk<T>((T)0, (T)0);
        }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int q = lane + 32 * b;
        dft8<T, INV>(v[b]);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) store(q + Q * k2, v[b][k2]);
    }
}

// Entries of the twiddle tables t1, t2 of fft_pencil_warp for N = 2^LOGN (t2 follows t1).
template <int LOGN>
struct PencilWarpTw {
    static constexpr int R1 = (1 << LOGN) / 64;
    static constexpr int T1 = (R1 - 1) * 64, T2 = 56, SIZE = T1 + T2;
};

// fft_columns with the input read by load(b, e) (b as in lead_row) inside the first stage
// and the output handed to store(e, value) by the last: the tile holds only the
// intermediate stages, so a pass moves each point through shared memory twice (not four
// times) for N = 512.  The caller reuses the tile only after a barrier.
template <typename T, int LOGN, bool INV, int IPT, int LD, class Load, class Store>
__device__ __forceinline__ void fft_columns_io(c2<T>* tile, int c, int u, const c2<T>* tw, Load&& load,
                                               Store&& store) {
    constexpr int N = 1 << LOGN;
    if constexpr (N == 8) {
        c2<T> v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = load(k, k);
        dft8<T, INV>(v);
#pragma unroll
        for (int k = 0; k < 8; ++k) store(k, v[k]);
    } else {
        lead_stage<T, LOGN, INV, IPT, LD, false>(tile, c, u, load);
        radix8_until<T, N, INV, IPT, LD, LeadRadix<LOGN>::R, N / 8>(tile, c, u, tw);
        last_stage<T, N, INV, IPT, LD>(tile, c, u, tw, store);
    }
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// Shape of the pencil passes for n = 2^LOGN: W pencils per CTA (W n / 8 <= 1024 butterfly
// slots, segments of up to 32 complex), IPT pencils per thread, THREADS per CTA.
template <int LOGN>
struct PassShape {
    static constexpr int N = 1 << LOGN;
    static constexpr int W0 = (8192 >> LOGN) > 32 ? 32 : (8192 >> LOGN);
    static constexpr int W = W0 > N ? N : W0;
    static constexpr int LOGW = ilog2(W);
    static constexpr int IPT = LOGN == 9 ? 4 : (LOGN >= 8 ? 2 : 1);
    static constexpr int THREADS = W * N / (8 * IPT);
    static constexpr int LD = W + 1;
    static constexpr int PER = N * W / THREADS;   // tile elements per thread
};

// Frequency index e is kept when f(e) lies in [-nk_neg, nk_pos].
__device__ __forceinline__ bool kept(int e, int n, int nk_pos, int nk_neg) {
    return e <= nk_pos || e >= n - nk_neg;
}

}  // namespace lpp
