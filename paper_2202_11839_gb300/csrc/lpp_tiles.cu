// Pencil sort of the catalogues and the fused assignment + x-FFT kernel.
//
// Sort.  Every particle gets the key iz * n + iy of the x pencil of the cell holding it
// (iy = floor(u_y) mod n, u = (x - origin) n / L); a counting sort (histogram, scan,
// scatter) stores the cell coordinates u and the weight of each particle in key order.
//
// Fused kernel.  One CTA owns a tile of TY x TZ x-pencils (all n points along x) of one
// batch grid.  CIC and TSC stencils, on the grid and on the half-cell shifted grid,
// reach the rows floor(u) - 1 .. floor(u) + 2, so the particles that touch the tile are
// exactly those with keys in rows [y0 - 2, y0 + TY] x [z0 - 2, z0 + TZ]: TZ + 3
// contiguous key ranges of the sorted arrays.  The CTA scatters them into the tile with
// shared-memory atomics (sub-grid 0 into the real part and the shifted sub-grid into the
// imaginary part, or two fields), runs the x-FFT of its pencils in place and writes only
// the kept x frequencies.  The grid is never zeroed, never touched by global atomics and
// never read back for an x pass.
#include <string.h>

#include <algorithm>

#include "lpp_internal.h"
#include "lpp_kernels.h"
#include "lpp_fft_dev.cuh"

namespace lpp {

// 16-byte global -> shared copy that does not hold registers while in flight (cp.async;
// both addresses 16-byte aligned), and the wait for this thread's copies.
__device__ __forceinline__ void copy16_async(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T>
__global__ void __launch_bounds__(256) k_pencil_count(const T* __restrict__ pos, long long count, int n, T ih,
                                                      T ox, T oy, T oz, int* __restrict__ key,
                                                      int* __restrict__ counts, int* err) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const T u0 = (pos[i] - ox) * ih;
        const T u1 = (pos[count + i] - oy) * ih;
        const T u2 = (pos[2 * count + i] - oz) * ih;
        int k = 0;
        if (!(u0 >= (T)0 && u0 <= (T)n && u1 >= (T)0 && u1 <= (T)n && u2 >= (T)0 && u2 <= (T)n)) {
            // flagged (the estimate is rejected) but still sorted, under key 0, so that
            // the sorted arrays and the permutation cover every particle
            atomicOr(err, ERRF_DOMAIN);
        } else {
            const int iy = ((int)floor(u1)) & (n - 1);
            const int iz = ((int)floor(u2)) & (n - 1);
            k = iz * n + iy;
        }
        key[i] = k;
        atomicAdd(counts + k, 1);
    }
}

// Exclusive scan of counts[0..nk) into off[0..nk] and cursor[0..nk) in three steps:
// segments of 2048 keys per CTA (local exclusive prefix and the segment total), one CTA's
// scan of the segment totals (at most 512 of them for n <= 1024), and the add.
constexpr int kScanSeg = 2048;   // keys per CTA (256 threads x 8)

__global__ void __launch_bounds__(256) k_scan_part(const int* __restrict__ counts, int nk, int* __restrict__ off,
                                                   int* __restrict__ bsum) {
    __shared__ int wsum[8];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int base = blockIdx.x * kScanSeg + t * 8;
    int v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = base + k < nk ? counts[base + k] : 0;
        s += v[k];
    }
    int inc = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += wsum[w];
    int run = wpre + inc - s;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (base + k < nk) off[base + k] = run;
        run += v[k];
    }
    if (t == 255) bsum[blockIdx.x] = wpre + inc;
}

__global__ void __launch_bounds__(1024) k_scan_top(int* __restrict__ bsum, int nb, int* __restrict__ total) {
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int s = t < nb ? bsum[t] : 0;
    int inc = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += wsum[w];
    if (t < nb) bsum[t] = wpre + inc - s;
    if (t == 1023) *total = wpre + inc;
}

__global__ void __launch_bounds__(256) k_scan_add(const int* __restrict__ bsum, int nk, int* __restrict__ off,
                                                  int* __restrict__ cursor) {
    const int add = bsum[blockIdx.x];
    const int base = blockIdx.x * kScanSeg;
    for (int k = threadIdx.x; k < kScanSeg; k += 256) {
        const int i = base + k;
        if (i < nk) {
            const int o = off[i] + add;
            off[i] = o;
            cursor[i] = o;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pencil_scatter(const T* __restrict__ pos, const T* __restrict__ w,
                                                        long long count, long long cap, T ih, T ox, T oy, T oz,
                                                        const int* __restrict__ key, int* __restrict__ cursor,
                                                        T* __restrict__ su, T* __restrict__ sw,
                                                        int* __restrict__ perm, int* err) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = key[i];
        const int j = atomicAdd(cursor + k, 1);
        if (!LPP_IN_BOUNDS(j >= 0 && j < cap, err)) continue;
        su[j] = (pos[i] - ox) * ih;
        su[cap + j] = (pos[count + i] - oy) * ih;
        su[2 * cap + j] = (pos[2 * count + i] - oz) * ih;
        sw[j] = w ? w[i] : (T)1;
        if (perm) perm[j] = (int)i;
    }
}

template <typename T>
cudaError_t launch_pencil_sort(const T* pos, const T* w, long long count, long long cap, int n, double box,
                               const double origin[3], int* key, int* counts, int* off, int* cursor, int* scan_tmp,
                               T* su, T* sw, int* perm, int* err, cudaStream_t st) {
    const int nk = n * n;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)nk * sizeof(int), st);
    if (e != cudaSuccess) return e;
    const T ih = (T)((double)n / box);
    const T ox = (T)origin[0], oy = (T)origin[1], oz = (T)origin[2];
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (count > 0) k_pencil_count<T><<<(int)blocks, 256, 0, st>>>(pos, count, n, ih, ox, oy, oz, key, counts, err);
    // segment totals in scan_tmp (at most 1024 entries: nk <= 1024^2 = 512 segments)
    const int nb = (nk + kScanSeg - 1) / kScanSeg;
    int* bsum = scan_tmp;
    k_scan_part<<<nb, 256, 0, st>>>(counts, nk, off, bsum);
    k_scan_top<<<1, 1024, 0, st>>>(bsum, nb, off + nk);
    k_scan_add<<<nb, 256, 0, st>>>(bsum, nk, off, cursor);
    if (count > 0)
        k_pencil_scatter<T><<<(int)blocks, 256, 0, st>>>(pos, w, count, cap, ih, ox, oy, oz, key, cursor, su, sw,
                                                         perm, err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fused kernel
template <typename T>
__device__ __forceinline__ void stencil1(T u, int n, int P, int cells[3], T w[3]) {
    if (P == 2) {
        const T fl = floor(u);
        const T f = u - fl;
        const int i0 = (int)fl;
        w[0] = (T)1 - f;
        w[1] = f;
        w[2] = (T)0;
        cells[0] = i0;
        cells[1] = i0 + 1;
        cells[2] = i0 + 1;
    } else {
        const T ic = floor(u + (T)0.5);
        const T d = u - ic;
        const int c = (int)ic;
        const T hm = (T)0.5 - d, hp = (T)0.5 + d;
        w[0] = (T)0.5 * hm * hm;
        w[1] = (T)0.75 - d * d;
        w[2] = (T)0.5 * hp * hp;
        cells[0] = c - 1;
        cells[1] = c;
        cells[2] = c + 1;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) cells[k] &= (n - 1);   // periodic wrap (n is a power of two)
}

// Fixed-point tiles: the units below keep every contribution within |x| <= 2^21 (a cell's
// window bound is taken as at least kMinWindow particles), where adding 1.5 x 2^23 in FP32
// leaves round-to-nearest-even(x) in the low mantissa bits.  fixed_round(a, b) is that
// integer for the exact product a b: one FFMA and one integer subtraction, against the
// quarter-rate conversion instruction.
constexpr int kMinWindow = 512;
__device__ __forceinline__ int fixed_round(float a, float b) {
    return __float_as_int(fmaf(a, b, 12582912.0f)) - 0x4B400000;
}

// Scatter one particle's weights (stencil at offset `shift` cells) into the tile part `im`.
// The loops run to the fixed bound 3 with a guard on P so the stencil stays in registers.
template <typename T, bool FIXED>
__device__ __forceinline__ void scatter_one(T* tilef, int ld, int n, int P, T ux, T uy, T uz, T shift, int y0,
                                            int z0, int ty, int tz, T va, T vb, bool two_fields, int im,
                                            int* err = nullptr) {
    int cx[3], cy[3], cz[3];
    T wx[3], wy[3], wz[3];
    stencil1<T>(ux - shift, n, P, cx, wx);
    stencil1<T>(uy - shift, n, P, cy, wy);
    stencil1<T>(uz - shift, n, P, cz, wz);
#pragma unroll
    for (int kz = 0; kz < 3; ++kz) {
        const int lz = (cz[kz] - z0) & (n - 1);
        if (kz >= P || lz >= tz) continue;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int ly = (cy[ky] - y0) & (n - 1);
            if (ky >= P || ly >= ty) continue;
            const int line = lz * ty + ly;
            const T wyz = wz[kz] * wy[ky];
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                if (kx >= P) continue;
                const int idx = 2 * (cx[kx] * ld + line);
                if (!LPP_IN_BOUNDS(cx[kx] >= 0 && cx[kx] < n && line >= 0 && line < ty * tz, err)) continue;
                const T ww = wyz * wx[kx];
                if constexpr (FIXED) {
                    // va, vb arrive pre-scaled to the tile's fixed-point unit
                    int* ti = reinterpret_cast<int*>(tilef);
                    atomicAdd(ti + idx + im, fixed_round((float)va, (float)ww));
                    if (two_fields) atomicAdd(ti + idx + 1, fixed_round((float)vb, (float)ww));
                } else {
                    atomicAdd(tilef + idx + im, va * ww);
                    if (two_fields) atomicAdd(tilef + idx + 1, vb * ww);
                }
            }
        }
    }
}

// Two channel slots of the same particles: the stencil is evaluated once and each weight
// is added to both tiles (values v0, v1 already in the tiles' units).
template <typename T, bool FIXED>
__device__ __forceinline__ void scatter_two(T* t0, T* t1, int ld, int n, int P, T ux, T uy, T uz, T shift, int y0,
                                            int z0, int ty, int tz, T v0, T v1, int im, int* err = nullptr) {
    int cx[3], cy[3], cz[3];
    T wx[3], wy[3], wz[3];
    stencil1<T>(ux - shift, n, P, cx, wx);
    stencil1<T>(uy - shift, n, P, cy, wy);
    stencil1<T>(uz - shift, n, P, cz, wz);
#pragma unroll
    for (int kz = 0; kz < 3; ++kz) {
        const int lz = (cz[kz] - z0) & (n - 1);
        if (kz >= P || lz >= tz) continue;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int ly = (cy[ky] - y0) & (n - 1);
            if (ky >= P || ly >= ty) continue;
            const int line = lz * ty + ly;
            const T wyz = wz[kz] * wy[ky];
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                if (kx >= P) continue;
                const int idx = 2 * (cx[kx] * ld + line) + im;
                if (!LPP_IN_BOUNDS(cx[kx] >= 0 && cx[kx] < n && line >= 0 && line < ty * tz, err)) continue;
                const T ww = wyz * wx[kx];
                if constexpr (FIXED) {
                    atomicAdd(reinterpret_cast<int*>(t0) + idx, fixed_round((float)v0, (float)ww));
                    atomicAdd(reinterpret_cast<int*>(t1) + idx, fixed_round((float)v1, (float)ww));
                } else {
                    atomicAdd(t0 + idx, v0 * ww);
                    atomicAdd(t1 + idx, v1 * ww);
                }
            }
        }
    }
}

// Tile of TY x TZ pencils: TY = 4 (TY = 2 when the FP64 1024-point tile would not fit).
template <typename T, int LOGN>
struct FusedShape {
    static constexpr int N = 1 << LOGN;
    static constexpr int TY = (sizeof(T) == 8 && LOGN >= 10) ? 2 : 4;
    static constexpr int TZ = 4;
    static constexpr int W = TY * TZ;
    static constexpr int LD = W + 1;
    static constexpr int IPT = (W * N / 8) <= 512 ? 1 : ((W * N / 8) <= 1024 ? 2 : 4);
    static constexpr int THREADS = W * N / (8 * IPT);
    static constexpr int MAXR = 2 * 2 * (TZ + 3);   // key ranges: sources x z rows x (1 or 2)
    // resident CTAs per SM the register budget is sized for (shared memory allows 3 at
    // n = 512 in FP32)
    static constexpr int MINB = (sizeof(T) == 4 && (LOGN == 9 || LOGN == 8)) ? 2 : 1;
    // the last x stage runs one warp per pencil and stores straight to the grid when a
    // warp's 32 lanes cover the N/8 butterfly slots (N >= 256); it reads the per-leg
    // twiddle table of TWR entries after the tiles
    static constexpr bool WARP_OUT = (N / 8 == 32 * IPT) && (THREADS == 32 * W);
    // n = 256, 512: the whole x transform of a pencil by one warp (fft_pencil_warp), with
    // its twiddle tables in the TWR entries
    static constexpr bool WARP_FFT = WARP_OUT && (N == 256 || N == 512);
    static constexpr int TWR = WARP_FFT ? PencilWarpTw<LOGN>::SIZE : (WARP_OUT ? 7 * (N / 8) : 0);
};

// The per-leg twiddles after the tiles: fft_pencil_warp's t1, t2 (WARP_FFT), else the last
// stage's twr[(r - 1) N/8 + j] = w^(j r).  Threads `first`, first + step, ... fill them.
template <typename T, int LOGN>
__device__ __forceinline__ void fill_twr(const c2<T>* tw, c2<T>* twr, int first, int step) {
    using S = FusedShape<T, LOGN>;
    constexpr int N = S::N;
    if constexpr (S::WARP_FFT) {
        using P = PencilWarpTw<LOGN>;
        for (int i = first; i < P::SIZE; i += step) {
            if (i < P::T1) {
                const int k0 = i / 64 + 1, m = i - (k0 - 1) * 64;
                twr[i] = tw[m * k0];
            } else {
                const int k1 = (i - P::T1) / 8 + 1, n0 = (i - P::T1) - (k1 - 1) * 8;
                twr[i] = tw[P::R1 * n0 * k1];
            }
        }
    } else if constexpr (S::TWR > 0) {
        for (int i = first; i < S::TWR; i += step) {
            const int r = i / (N / 8) + 1, j = i - (r - 1) * (N / 8);
            twr[i] = tw[j * r];
        }
    }
}

// The particle ranges of the tile at (y0, z0) for the sources of slot `sl`, found by one
// warp (all 32 lanes): TZ+3 z rows of keys y0-2 .. y0+TY per source, one or two contiguous
// ranges each (the y window may wrap).  Lane l takes row l (source l / (TZ+3)); a warp scan
// places the ranges.  With want_wmax, also the largest 4 x 4 key-row window count of source
// 0 (the fixed-point bound).  rcount: the warp's scratch.
template <typename T, int LOGN>
__device__ __forceinline__ void warp_ranges(const FusedArgs<T>& a, const FusedSlot& sl, int y0, int z0, int lane,
                                            int* r_begin, int* r_pref, int* r_src, int& n_ranges,
                                            int (*rcount)[FusedShape<T, LOGN>::TY + 3], int& wmax, bool want_wmax) {
    using S = FusedShape<T, LOGN>;
    constexpr int N = S::N, TY = S::TY, TZ = S::TZ;
    int bb[2] = {0, 0}, ee[2] = {0, 0}, m = 0, s_idx = 0;
    if (lane < sl.n_src * (TZ + 3)) {
        s_idx = lane / (TZ + 3);
        const int dz = lane - s_idx * (TZ + 3);
        const int* off = a.cat[sl.src[s_idx].cat].off;
        const int zr = (z0 - 2 + dz) & (N - 1);
        const int ylo = y0 - 2, yhi = y0 + TY;   // inclusive
        bb[m] = off[zr * N + (ylo < 0 ? 0 : ylo)];
        ee[m++] = off[zr * N + (yhi >= N ? N - 1 : yhi) + 1];
        if (ylo < 0) { bb[m] = off[zr * N + N + ylo]; ee[m++] = off[zr * N + N]; }
        if (yhi >= N) { bb[m] = off[zr * N]; ee[m++] = off[zr * N + (yhi - N) + 1]; }
    }
    int nr_l = 0, cnt_l = 0;
    for (int q = 0; q < m; ++q)
        if (ee[q] > bb[q]) { ++nr_l; cnt_l += ee[q] - bb[q]; }
    int nr_inc = nr_l, cnt_inc = cnt_l;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int a1 = __shfl_up_sync(0xffffffffu, nr_inc, d);
        const int a2 = __shfl_up_sync(0xffffffffu, cnt_inc, d);
        if (lane >= d) { nr_inc += a1; cnt_inc += a2; }
    }
    int nr = nr_inc - nr_l, acc = cnt_inc - cnt_l;
    for (int q = 0; q < m; ++q) {
        if (ee[q] <= bb[q]) continue;
        r_begin[nr] = bb[q];
        r_src[nr] = s_idx;
        r_pref[nr] = acc;
        acc += ee[q] - bb[q];
        ++nr;
    }
    if (lane == 31) {
        r_pref[nr_inc] = cnt_inc;
        n_ranges = nr_inc;
    }
    if (want_wmax) {
        // a cell (y, z) of the tile receives only from the key rows y-2..y+1, z-2..z+1:
        // the largest such 4 x 4 window sum bounds the contributions of any one cell
        if (lane < TZ + 3) {
            const int* off = a.cat[sl.src[0].cat].off;
            const int zr = (z0 - 2 + lane) & (N - 1);
#pragma unroll
            for (int dy = 0; dy < TY + 3; ++dy) {
                const int yr = (y0 - 2 + dy) & (N - 1);
                rcount[lane][dy] = off[zr * N + yr + 1] - off[zr * N + yr];
            }
        }
        __syncwarp();
        int wsum = 0;
        if (lane < TY * TZ) {
            const int ly = lane % TY, lz = lane / TY;   // cell (y0 + ly, z0 + lz): rows ly..ly+3
#pragma unroll
            for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
                for (int b2 = 0; b2 < 4; ++b2) wsum += rcount[lz + a2][ly + b2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wsum = max(wsum, __shfl_down_sync(0xffffffffu, wsum, o));
        if (lane == 0) wmax = wsum;
    }
}

// Set-up of one tile (shared by the one- and two-slot tiles): warp 0 finds the particle
// ranges (warp_ranges; the fixed-point bound for fixed-point slots) while the other warps
// clear `tile_elems` elements of the tiles and load the twiddles.  NT: threads of the CTA.
template <typename T, int LOGN, int NT>
__device__ __forceinline__ void tile_setup(const FusedArgs<T>& a, const FusedSlot& sl, int y0, int z0, c2<T>* tw,
                                           c2<T>* twr, c2<T>* tiles, int tile_elems, int* r_begin, int* r_pref,
                                           int* r_src, int& n_ranges, int (*rcount)[FusedShape<T, LOGN>::TY + 3],
                                           int& wmax) {
    using S = FusedShape<T, LOGN>;
    constexpr int N = S::N, TY = S::TY, TZ = S::TZ;
    const int tid = threadIdx.x;
    if (NT < 64) {
        // tiny tiles (n <= 16): one thread finds the ranges, everybody clears the tile
        if (tid == 0) {
            int nr = 0, acc = 0;
            for (int sidx = 0; sidx < sl.n_src; ++sidx) {
                const int* off = a.cat[sl.src[sidx].cat].off;
                for (int dz = 0; dz < TZ + 3; ++dz) {
                    const int zr = (z0 - 2 + dz) & (N - 1);
                    const int ylo = y0 - 2, yhi = y0 + TY;
                    int bb[2], ee[2], m = 0;
                    bb[m] = off[zr * N + (ylo < 0 ? 0 : ylo)];
                    ee[m++] = off[zr * N + (yhi >= N ? N - 1 : yhi) + 1];
                    if (ylo < 0) { bb[m] = off[zr * N + N + ylo]; ee[m++] = off[zr * N + N]; }
                    if (yhi >= N) { bb[m] = off[zr * N]; ee[m++] = off[zr * N + (yhi - N) + 1]; }
                    for (int q = 0; q < m; ++q) {
                        if (ee[q] <= bb[q]) continue;
                        r_begin[nr] = bb[q];
                        r_src[nr] = sidx;
                        r_pref[nr] = acc;
                        acc += ee[q] - bb[q];
                        ++nr;
                    }
                }
            }
            r_pref[nr] = acc;
            n_ranges = nr;
            wmax = acc;   // every particle of the tile: a looser but valid per-cell bound
        }
        for (int i = tid; i < N; i += NT) tw[i] = a.tw[i];
        for (int i = tid; i < tile_elems; i += NT) tiles[i] = mk<T>((T)0, (T)0);
    } else if (tid < 32) {
        warp_ranges<T, LOGN>(a, sl, y0, z0, tid, r_begin, r_pref, r_src, n_ranges, rcount, wmax,
                             sl.amax_a != nullptr);
    } else {
        for (int i = tid - 32; i < N; i += NT - 32) tw[i] = a.tw[i];
        fill_twr<T, LOGN>(a.tw, twr, tid - 32, NT - 32);
        for (int i = tid - 32; i < tile_elems; i += NT - 32) tiles[i] = mk<T>((T)0, (T)0);
    }
}

// Forward x transform of the tile's pencils after the scatter, and the store of the kept x
// frequencies to the grid (out: the tile's first pencil; pencil c = lz TY + ly at
// out + (lz n + ly) n).  A fixed-point tile is converted back to floating point (value =
// integer x unit) inside the first FFT stage.  t: the thread's index among the S::THREADS
// that transform this tile; fixed is CTA-uniform.
template <typename T, int LOGN, bool ZERO = false>
__device__ __forceinline__ void x_transform(c2<T>* tile, int t, const c2<T>* tw, const c2<T>* twr, bool fixed,
                                            float unit, c2<T>* out, int nk_pos, int nk_neg) {
    static_assert(!ZERO || FusedShape<T, LOGN>::WARP_FFT, "zeroing needs the warp-per-pencil transform");
    using S = FusedShape<T, LOGN>;
    constexpr int N = S::N, W = S::W, LD = S::LD, IPT = S::IPT, TY = S::TY, R0 = LeadRadix<LOGN>::R;
    if constexpr (S::WARP_FFT) {
        // one warp per pencil
        const int pc = t >> 5, lane = t & 31;
        c2<T>* po = out + ((size_t)(pc / TY) * N + (pc & (TY - 1))) * N;
        auto store = [&](int e, c2<T> v) {
            if (kept(e, N, nk_pos, nk_neg)) po[e] = v;
        };
        constexpr int T1 = PencilWarpTw<LOGN>::T1;
        if constexpr (sizeof(T) == 4) {
            if (fixed) {
                const int2* ti = reinterpret_cast<const int2*>(tile) + pc;
                fft_pencil_warp<T, LOGN, false, LD, ZERO>(tile, pc, lane, twr, twr + T1, [&](int e) {
                    const int2 q = ti[e * LD];
                    return mk<T>((T)((float)q.x * unit), (T)((float)q.y * unit));
                }, store);
                return;
            }
        }
        const c2<T>* col = tile + pc;
        fft_pencil_warp<T, LOGN, false, LD, ZERO>(tile, pc, lane, twr, twr + T1, [&](int e) { return col[e * LD]; },
                                                  store);
    } else {
        const int c = t & (W - 1), u = t >> ilog2(W);
        bool converted = false;
        if constexpr (sizeof(T) == 4) {
            if (fixed) {
                const int2* ti = reinterpret_cast<const int2*>(tile) + c;
                lead_stage<T, LOGN, false, IPT, LD, true>(tile, c, u, [&](int, int e) {
                    const int2 q = ti[e * LD];
                    return mk<T>((T)((float)q.x * unit), (T)((float)q.y * unit));
                });
                converted = true;
            }
        }
        if (!converted) stockham_stage<T, N, R0, false, IPT, LD, 1>(tile, c, u, tw);
        if constexpr (S::WARP_OUT) {
            radix8_until<T, N, false, IPT, LD, R0, N / 8>(tile, c, u, tw);
            const int pc = t >> 5;
            c2<T>* po = out + ((size_t)(pc / TY) * N + (pc & (TY - 1))) * N;
            last_stage_warp<T, N, false, IPT, LD>(tile, pc, t & 31, twr, [&](int e, c2<T> v) {
                if (kept(e, N, nk_pos, nk_neg)) po[e] = v;
            });
        } else {
            radix8_until<T, N, false, IPT, LD, R0, N>(tile, c, u, tw);
            // LPL consecutive threads store one pencil (coalesced along x)
            constexpr int LPL = S::THREADS / W;
            const int cw = t / LPL;
            const int nkept = nk_pos + 1 + nk_neg;
            for (int k = t & (LPL - 1); k < nkept; k += LPL) {
                const int e = k <= nk_pos ? k : N - nkept + k;
                out[((cw / TY) * N + (cw & (TY - 1))) * N + e] = tile[e * LD + cw];
            }
        }
    }
}

// One tile (tile_y, tile_z) of TY x TZ pencils of slot `slot`: particle ranges,
// scatter, x transform, store of the kept x frequencies.  Every return is CTA-uniform.
template <typename T, int LOGN>
__device__ __forceinline__ void fused_tile(const FusedArgs<T>& a, int slot, int tile_y, int tile_z) {
    using S = FusedShape<T, LOGN>;
    constexpr int N = S::N, TY = S::TY, TZ = S::TZ, W = S::W, LD = S::LD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int r_begin[S::MAXR], r_pref[S::MAXR + 1], r_src[S::MAXR];
    __shared__ int n_ranges;
    // particles per key row around the tile (fixed-point bound; rows of source 0)
    __shared__ int rcount[TZ + 3][TY + 3];
    __shared__ int wmax;
    c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* tile = tw + N;
    c2<T>* twr = tile + N * LD;
    T* tilef = reinterpret_cast<T*>(tile);
    const int tid = threadIdx.x;
    const int y0 = tile_y * TY;
    const int z0 = tile_z * TZ;
    const FusedSlot& sl = a.slots[slot];
    c2<T>* out = a.grids + (size_t)sl.grid * a.grid_stride + ((size_t)z0 * N + y0) * N;

    tile_setup<T, LOGN, S::THREADS>(a, sl, y0, z0, tw, twr, tile, N * LD, r_begin, r_pref, r_src, n_ranges, rcount,
                                    wmax);
    __syncthreads();
    const int nr = n_ranges;
    if (!LPP_IN_BOUNDS(nr >= 0 && nr <= S::MAXR && tile_y >= 0 && tile_y < N / TY && tile_z >= 0 && tile_z < N / TZ,
                       a.err))
        return;   // CTA-uniform
    const int total = r_pref[nr];
    // kept x frequencies of a pencil: indices 0..nk_pos and n-nk_neg..n-1; LPL consecutive
    // threads write one pencil (coalesced along x)
    const int nkept = a.nk_pos + 1 + a.nk_neg;
    constexpr int LPL = S::THREADS / W;
    const int cw = tid / LPL;
    if (total == 0) {
        // no particle reaches these pencils: their transform is zero.  Planes that no
        // particle of the slot's roles reaches are skipped by the y pass, which writes
        // their zeros itself: nothing to store for those.
        if (a.skip_empty) return;   // the y pass reads zeros for every pencil of this tile
        bool write = true;
        if (a.pmask) {
            const int z = z0 + cw / TY;
            write = false;
            for (int sidx = 0; sidx < sl.n_src; ++sidx) write |= a.pmask[sl.src[sidx].cat * N + z] != 0;
        }
        if (write) {
            for (int k = tid & (LPL - 1); k < nkept; k += LPL) {
                const int e = k <= a.nk_pos ? k : N - nkept + k;
                out[((cw / TY) * N + (cw & (TY - 1))) * N + e] = mk<T>((T)0, (T)0);
            }
        }
        return;
    }
    const T alpha = (T)a.sums[SUM_ALPHA];
    const int P = a.scheme;
    const T* vb_ptr = (!a.interlace && sl.vals_b) ? static_cast<const T*>(sl.vals_b) : nullptr;
    // fixed-point accumulation (FP32 channel slots): a cell sums at most wmax contributions
    // (particles of its 4 x 4 key-row window) of magnitude <= amax (the TSC/CIC weights are
    // <= 1), so 2^30 / (max(wmax, kMinWindow) amax) units keep every cell and its rounding
    // (<= wmax units, two sub-grid stencils) inside int32 and every contribution within
    // 2^21 units (fixed_round).  The tile takes it only
    // when that unit is at most 2^-16 of the rows' rms value, so that rounding each
    // contribution to the unit costs no more than the FP32 sums it replaces; otherwise float
    // atomics.
    bool fixed = false;
    float fscale = 1.f, finv = 1.f;
    if (sizeof(T) == 4 && sl.amax_a != nullptr) {
        float am = sl.amax_a[0], rms = sl.amax_a[1];
        if (sl.amax_b) {
            am = fmaxf(am, sl.amax_b[0]);
            rms = fminf(rms, sl.amax_b[1]);
        }
        const float bound = (float)max(wmax, kMinWindow) * am;
        if (bound == 0.f) {
            fixed = true;                        // every value is zero
        } else if (bound * (1.f / 1073741824.f) <= rms * (1.f / 65536.f)) {
            fixed = true;
            fscale = 1073741824.f / bound;
            finv = bound / 1073741824.f;
        }
        if (a.pstat && tid == 0) atomicAdd(a.pstat + (fixed ? 2 : 3), 1);
    }
    int r = 0;
    for (int t = tid; t < total; t += S::THREADS) {
        while (r + 1 < nr && r_pref[r + 1] <= t) ++r;   // t increases, so the range index only grows
        const int j = r_begin[r] + (t - r_pref[r]);
        const FusedSrc& src = sl.src[r_src[r]];
        const PencilCat& cat = a.cat[src.cat];
        const T* su = static_cast<const T*>(cat.su);
        const T* vals = src.vals ? static_cast<const T*>(src.vals) : static_cast<const T*>(cat.sw);
        const long long cap = cat.cap;
        if (!LPP_IN_BOUNDS(j >= 0 && j < cap, a.err)) continue;
        const T ux = su[j], uy = su[cap + j], uz = su[2 * cap + j];
        const T base = vals[j];
        T va = base;
        if (src.neg_alpha) va *= -alpha;
        bool two = vb_ptr != nullptr && r_src[r] == 0;
        T vb = two ? vb_ptr[j] : (T)0;
        if (sl.use_ylm) {
            // line of sight of the particle from its cell coordinates (or the fixed direction)
            T px, py, pz;
            if (a.ylm_global) {
                px = (T)a.los_global[0];
                py = (T)a.los_global[1];
                pz = (T)a.los_global[2];
            } else {
                px = (T)a.origin[0] + ux * (T)a.h - (T)a.observer[0];
                py = (T)a.origin[1] + uy * (T)a.h - (T)a.observer[1];
                pz = (T)a.origin[2] + uz * (T)a.h - (T)a.observer[2];
            }
            const T inv = (T)1 / sqrt(px * px + py * py + pz * pz);
            va *= (T)sl.ynorm_a * ylm_poly<T>(sl.yl_a, sl.yn_a, px * inv, py * inv, pz * inv);
            if (sl.yl_b >= 0) {
                const T sb = src.neg_alpha ? base * -alpha : base;
                vb = sb * (T)sl.ynorm_b * ylm_poly<T>(sl.yl_b, sl.yn_b, px * inv, py * inv, pz * inv);
                two = true;
            }
        }
        if (a.interlace) {
            // both sub-grids; odd lanes take the shifted one (the imaginary words) first, so that
            // each atomic instruction spreads over the even and the odd banks
            const int odd = tid & 1;
            const T sh0 = odd ? (T)0.5 : (T)0, sh1 = odd ? (T)0 : (T)0.5;
            if (fixed) {
                va *= fscale;
                scatter_one<T, true>(tilef, LD, N, P, ux, uy, uz, sh0, y0, z0, TY, TZ, va, (T)0, false, odd, a.err);
                scatter_one<T, true>(tilef, LD, N, P, ux, uy, uz, sh1, y0, z0, TY, TZ, va, (T)0, false, 1 - odd, a.err);
            } else {
                scatter_one<T, false>(tilef, LD, N, P, ux, uy, uz, sh0, y0, z0, TY, TZ, va, (T)0, false, odd, a.err);
                scatter_one<T, false>(tilef, LD, N, P, ux, uy, uz, sh1, y0, z0, TY, TZ, va, (T)0, false, 1 - odd, a.err);
            }
        } else if (fixed) {
            va *= fscale;
            vb *= fscale;
            scatter_one<T, true>(tilef, LD, N, P, ux, uy, uz, (T)0, y0, z0, TY, TZ, va, vb, two, 0, a.err);
        } else {
            scatter_one<T, false>(tilef, LD, N, P, ux, uy, uz, (T)0, y0, z0, TY, TZ, va, vb, two, 0, a.err);
        }
    }
    __syncthreads();
    x_transform<T, LOGN>(tile, tid, tw, twr, fixed, finv, out, a.nk_pos, a.nk_neg);
}

__global__ void k_plane_mask(const int* __restrict__ off0, const int* __restrict__ off1, const int* __restrict__ off2,
                             int set0, int set1, int set2, int n, int* __restrict__ pmask) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int r = i / n, z = i - r * n;
    const int* off = r == 0 ? off0 : (r == 1 ? off1 : off2);
    const int set = r == 0 ? set0 : (r == 1 ? set1 : set2);
    int hit = 0;
    if (set) {
        for (int d = -2; d <= 1; ++d) {
            const int f = (z + d) & (n - 1);
            hit |= off[(size_t)(f + 1) * n] > off[(size_t)f * n];
        }
    }
    pmask[i] = hit;
}

__global__ void k_pencil_live(const int* __restrict__ off0, const int* __restrict__ off1,
                              const int* __restrict__ off2, int set0, int set1, int set2, int n,
                              unsigned char* __restrict__ plive) {
    const long long nn = (long long)n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * nn;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / nn);
        const int zy = (int)(i - r * nn);
        const int z = zy / n, y = zy - z * n;
        const int* off = r == 0 ? off0 : (r == 1 ? off1 : off2);
        const int set = r == 0 ? set0 : (r == 1 ? set1 : set2);
        int hit = 0;
        if (set) {
            for (int dz = -2; dz <= 1 && !hit; ++dz) {
                const int fz = (z + dz) & (n - 1);
                for (int dy = -2; dy <= 1; ++dy) {
                    const int key = fz * n + ((y + dy) & (n - 1));
                    if (off[key + 1] > off[key]) { hit = 1; break; }
                }
            }
        }
        plive[i] = (unsigned char)hit;
    }
}

cudaError_t launch_pencil_live(const int* off0, const int* off1, const int* off2, int set0, int set1, int set2, int n,
                               unsigned char* plive, cudaStream_t st) {
    const long long total = 3LL * n * n;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_pencil_live<<<(int)blocks, 256, 0, st>>>(off0, off1, off2, set0, set1, set2, n, plive);
    return cudaGetLastError();
}

cudaError_t launch_plane_mask(const int* off0, const int* off1, const int* off2, int set0, int set1, int set2, int n,
                              int* pmask, cudaStream_t st) {
    k_plane_mask<<<(3 * n + 255) / 256, 256, 0, st>>>(off0, off1, off2, set0, set1, set2, n, pmask);
    return cudaGetLastError();
}

// Tile shape (TY, TZ), pencils per thread, threads and shared memory of the fused kernel
// (mirrors FusedShape).
void fused_geometry(int n, size_t elem_bytes, int* ty, int* tz, int* ipt, int* threads, size_t* smem) {
    *ty = (elem_bytes == 8 && n >= 1024) ? 2 : 4;
    *tz = 4;
    const int w = *ty * *tz;
    const int t1 = w * n / 8;
    *ipt = t1 <= 512 ? 1 : (t1 <= 1024 ? 2 : 4);
    *threads = t1 / *ipt;
    const bool warp_out = n / 8 == 32 * *ipt && *threads == 32 * w;
    const bool warp_fft = warp_out && (n == 256 || n == 512);
    // PencilWarpTw<LOGN>::SIZE: two-pass tables at n = 512, three-pass at n = 256
    const int twr = warp_fft ? (n / 64 - 1) * 64 + 56 : (warp_out ? 7 * (n / 8) : 0);
    *smem = (size_t)(n + n * (w + 1) + twr) * 2 * elem_bytes;
}

// Tile range records (k_tile_ranges): per tile of the persistent enumeration, kRec ints:
// [0] range count, [1] fixed-point bound wmax, [kRecBegin..) first particle of each range,
// [kRecPref..) running particle count before each range (and the total), [kRecSrc..) source.
constexpr int kRec = 96, kRecBegin = 2, kRecPref = 32, kRecSrc = 64;

// Tiles of a two-slot launch with range records: cleared tiles only (16-byte stores; the
// ranges come from a record and the kernel loads the twiddles once, before its tile loop).
template <typename T, int LOGN, int NT>
__device__ __forceinline__ void tile_clear(c2<T>* tiles, int tile_elems) {
    static_assert(sizeof(c2<T>) == 8 || sizeof(c2<T>) == 16, "complex float or double");
    float4* t4 = reinterpret_cast<float4*>(tiles);
    const int n4 = tile_elems * (int)sizeof(c2<T>) / 16;   // tile_elems even for complex float
    for (int i = threadIdx.x; i < n4; i += NT) t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Twiddles of a tile's x transform in shared memory: the N-entry table (unless every pencil
// is transformed by fft_pencil_warp, which reads only the per-leg tables) and the per-leg
// tables after the tiles.
template <typename T, int LOGN, int NT>
__device__ __forceinline__ void load_twiddles(const FusedArgs<T>& a, c2<T>* tw, c2<T>* twr) {
    using S = FusedShape<T, LOGN>;
    if constexpr (!S::WARP_FFT) {
        for (int i = threadIdx.x; i < S::N; i += NT) tw[i] = a.tw[i];
    }
    fill_twr<T, LOGN>(a.tw, twr, threadIdx.x, NT);
}

// Two interlaced channel slots (2 blockIdx.y, 2 blockIdx.y + 1: single-source coefficient
// rows of the same catalogue) in one CTA of 2 x THREADS threads: one set-up, every particle
// visit computes its stencils once for both tiles; the halves of the CTA transform and store
// one tile each.  The tiles use fixed point only when both slots' units pass the guard.
// With range records (rec) the tiles arrive zeroed: the kernel clears them once and every x
// transform leaves its column zeroed; bnd[2 q], bnd[2 q + 1] are slot q's coefficient bounds
// (max |c|, rms c), in shared memory.
template <typename T, int LOGN>
__device__ __forceinline__ void fused_tile2(const FusedArgs<T>& a, int tile_y, int tile_z, const int* rec,
                                            const float* bnd) {
    using S = FusedShape<T, LOGN>;
    constexpr int N = S::N, TY = S::TY, TZ = S::TZ, W = S::W, LD = S::LD;
    constexpr int NT = 2 * S::THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int r_begin_s[S::MAXR], r_pref_s[S::MAXR + 1], r_src_s[S::MAXR];
    __shared__ int n_ranges_s;
    __shared__ int rcount[TZ + 3][TY + 3];
    __shared__ int wmax_s;
    c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* tile0 = tw + N;
    c2<T>* tile1 = tile0 + N * LD;
    c2<T>* twr = tile1 + N * LD;
    const int tid = threadIdx.x;
    const int y0 = tile_y * TY, z0 = tile_z * TZ;
    const FusedSlot& s0 = a.slots[2 * blockIdx.y];
    const FusedSlot& s1 = a.slots[2 * blockIdx.y + 1];
    if (!rec) {
        tile_setup<T, LOGN, NT>(a, s0, y0, z0, tw, twr, tile0, 2 * N * LD, r_begin_s, r_pref_s, r_src_s,
                                n_ranges_s, rcount, wmax_s);
        __syncthreads();
    }
    const int* r_begin = rec ? rec + kRecBegin : r_begin_s;
    const int* r_pref = rec ? rec + kRecPref : r_pref_s;
    const int nr = rec ? rec[0] : n_ranges_s;
    const int wmax = rec ? rec[1] : wmax_s;
    if (!LPP_IN_BOUNDS(nr >= 0 && nr <= S::MAXR && tile_y >= 0 && tile_y < N / TY && tile_z >= 0 && tile_z < N / TZ,
                       a.err))
        return;   // CTA-uniform; the tiles stay as they are (zero)
    const int total = r_pref[nr];
    const int half = tid / S::THREADS, th = tid - half * S::THREADS;
    const FusedSlot& sh = half ? s1 : s0;
    c2<T>* out = a.grids + (size_t)sh.grid * a.grid_stride + ((size_t)z0 * N + y0) * N;
    const int nkept = a.nk_pos + 1 + a.nk_neg;
    constexpr int LPL = S::THREADS / W;
    const int cw = th / LPL;
    if (total == 0) {
        if (a.skip_empty) return;
        bool write = true;
        if (a.pmask) write = a.pmask[sh.src[0].cat * N + z0 + cw / TY] != 0;
        if (write) {
            for (int k = th & (LPL - 1); k < nkept; k += LPL) {
                const int e = k <= a.nk_pos ? k : N - nkept + k;
                out[((cw / TY) * N + (cw & (TY - 1))) * N + e] = mk<T>((T)0, (T)0);
            }
        }
        return;
    }
    // fixed point as in fused_tile, with one unit per slot
    bool fixed = sizeof(T) == 4;
    float fs[2] = {1.f, 1.f}, fi[2] = {1.f, 1.f};
    for (int q = 0; q < 2 && fixed; ++q) {
        const float bound = (float)max(wmax, kMinWindow) * bnd[2 * q];
        if (bound == 0.f) continue;
        if (bound * (1.f / 1073741824.f) <= bnd[2 * q + 1] * (1.f / 65536.f)) {
            fs[q] = 1073741824.f / bound;
            fi[q] = bound / 1073741824.f;
        } else {
            fixed = false;
        }
    }
    if (a.pstat && tid == 0) atomicAdd(a.pstat + (fixed ? 0 : 1), 1);
    const int P = a.scheme;
    const PencilCat& cat = a.cat[s0.src[0].cat];
    const T* su = static_cast<const T*>(cat.su);
    const T* vals0 = static_cast<const T*>(s0.src[0].vals);
    const T* vals1 = static_cast<const T*>(s1.src[0].vals);
    const long long cap = cat.cap;
    T* t0 = reinterpret_cast<T*>(tile0);
    T* t1 = reinterpret_cast<T*>(tile1);
    // odd lanes scatter the shifted sub-grid (the imaginary words) first: every atomic
    // instruction then spreads over the even and the odd banks
    const int odd = tid & 1;
    const T sh0 = odd ? (T)0.5 : (T)0, sh1 = odd ? (T)0 : (T)0.5;
    int r = 0;
    for (int t = tid; t < total; t += NT) {
        while (r + 1 < nr && r_pref[r + 1] <= t) ++r;
        const int j = r_begin[r] + (t - r_pref[r]);
        if (!LPP_IN_BOUNDS(j >= 0 && j < cap, a.err)) continue;
        const T ux = su[j], uy = su[cap + j], uz = su[2 * cap + j];
        T v0 = vals0[j], v1 = vals1[j];
        if (fixed) {
            v0 *= fs[0];
            v1 *= fs[1];
            scatter_two<T, true>(t0, t1, LD, N, P, ux, uy, uz, sh0, y0, z0, TY, TZ, v0, v1, odd, a.err);
            scatter_two<T, true>(t0, t1, LD, N, P, ux, uy, uz, sh1, y0, z0, TY, TZ, v0, v1, 1 - odd, a.err);
        } else {
            scatter_two<T, false>(t0, t1, LD, N, P, ux, uy, uz, sh0, y0, z0, TY, TZ, v0, v1, odd, a.err);
            scatter_two<T, false>(t0, t1, LD, N, P, ux, uy, uz, sh1, y0, z0, TY, TZ, v0, v1, 1 - odd, a.err);
        }
    }
    __syncthreads();
    c2<T>* tile = half ? tile1 : tile0;
    if constexpr (S::WARP_FFT) {
        if (rec) {
            x_transform<T, LOGN, true>(tile, th, tw, twr, fixed, fi[half], out, a.nk_pos, a.nk_neg);
            return;
        }
    }
    x_transform<T, LOGN>(tile, th, tw, twr, fixed, fi[half], out, a.nk_pos, a.nk_neg);
}

// With range records (a.tranges) warp 0 loads the next tile's record into registers while
// the CTA works on the current tile and stores it into the other record buffer at the end.
template <typename T, int LOGN>
__global__ void __launch_bounds__(2 * FusedShape<T, LOGN>::THREADS, 1) k_assign_xfft2(FusedArgs<T> a) {
    using S = FusedShape<T, LOGN>;
    static_assert(S::MAXR <= kRecPref - kRecBegin && S::MAXR + 1 <= kRecSrc - kRecPref && S::MAXR <= kRec - kRecSrc,
                  "range record layout");
    constexpr int NTY = S::N / S::TY;
    __shared__ __align__(16) int recs[2][kRec];
    // the slots' coefficient bounds (max |c|, rms) for the fixed-point units, once per CTA
    __shared__ float bnd[4];
    const int total = *a.trow_count * NTY;
    const int tid = threadIdx.x;
    if (tid < 4) bnd[tid] = sizeof(T) == 4 ? a.slots[2 * blockIdx.y + (tid >> 1)].amax_a[tid & 1] : 0.f;
    if (a.tranges == nullptr) {
        __syncthreads();
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            fused_tile2<T, LOGN>(a, t % NTY, a.trows[t / NTY], nullptr, bnd);
            __syncthreads();
        }
        return;
    }
    static_assert(kRec % 4 == 0 && kRec / 4 <= 32, "a record is copied by one warp in 16-byte pieces");
    if (tid < kRec / 4 && (int)blockIdx.x < total) copy16_async(&recs[0][4 * tid], a.tranges + (size_t)blockIdx.x * kRec + 4 * tid);
    cp_async_wait_all();
    {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        c2<T>* tw = reinterpret_cast<c2<T>*>(smem_raw);
        load_twiddles<T, LOGN, 2 * S::THREADS>(a, tw, tw + S::N + 2 * S::N * S::LD);
        // both tiles start zeroed; afterwards each x transform leaves its columns zeroed
        tile_clear<T, LOGN, 2 * S::THREADS>(tw + S::N, 2 * S::N * S::LD);
    }
    __syncthreads();
    int buf = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int tn = t + gridDim.x;
        // the next tile's record streams into the other buffer while this tile is worked on
        if (tid < kRec / 4 && tn < total) copy16_async(&recs[buf ^ 1][4 * tid], a.tranges + (size_t)tn * kRec + 4 * tid);
        fused_tile2<T, LOGN>(a, t % NTY, a.trows[t / NTY], recs[buf], bnd);
        cp_async_wait_all();
        __syncthreads();
        buf ^= 1;
    }
}

// Range records of every tile of the persistent enumeration (tile t: y index t % (n/TY),
// z-tile row trows[t / (n/TY)]) for the sources of slots[0], with the fixed-point bound:
// one warp per tile, 8 per CTA.
template <typename T, int LOGN>
__global__ void __launch_bounds__(256) k_tile_ranges(FusedArgs<T> a, int* __restrict__ out) {
    using S = FusedShape<T, LOGN>;
    constexpr int NTY = S::N / S::TY;
    __shared__ int rec[8][kRec];
    __shared__ int rcount[8][S::TZ + 3][S::TY + 3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = *a.trow_count * NTY;
    for (int t = blockIdx.x * 8 + w; t < total; t += gridDim.x * 8) {
        const int y0 = (t % NTY) * S::TY, z0 = a.trows[t / NTY] * S::TZ;
        warp_ranges<T, LOGN>(a, a.slots[0], y0, z0, lane, rec[w] + kRecBegin, rec[w] + kRecPref,
                             rec[w] + kRecSrc, rec[w][0], rcount[w], rec[w][1], true);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kRec / 32; ++k) out[(size_t)t * kRec + lane + 32 * k] = rec[w][lane + 32 * k];
        __syncwarp();
    }
}

// Without a tile-row list one CTA per tile; with one (trows: z-tile rows that contain a
// plane some particle reaches, *trow_count of them) a persistent grid walks those rows' tiles.
template <typename T, int LOGN>
__global__ void __launch_bounds__(FusedShape<T, LOGN>::THREADS, FusedShape<T, LOGN>::MINB)
k_assign_xfft(FusedArgs<T> a) {
    using S = FusedShape<T, LOGN>;
    constexpr int NTY = S::N / S::TY;
    if (a.trows == nullptr) {
        fused_tile<T, LOGN>(a, blockIdx.y, blockIdx.x % NTY, blockIdx.x / NTY);
        return;
    }
    const int total = *a.trow_count * NTY;
    if (a.work) {
        // dynamic: every CTA takes the next (slot, tile) item, slot-major, until none is left
        // (slots of very different particle counts share the SMs evenly)
        __shared__ int item;
        const int items = total * a.n_slots;
        for (;;) {
            if (threadIdx.x == 0) item = atomicAdd(a.work, 1);
            __syncthreads();
            const int it = item;
            if (it >= items) break;
            const int sl = it / total, t = it - sl * total;
            fused_tile<T, LOGN>(a, sl, t % NTY, a.trows[t / NTY]);
            __syncthreads();   // the tile's shared memory and `item` are reused by the next one
        }
        return;
    }
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        fused_tile<T, LOGN>(a, blockIdx.y, t % NTY, a.trows[t / NTY]);
        __syncthreads();   // the tile's shared memory is reused by the next one
    }
}

// Tile rows (of tz planes) that contain a plane reached by a role in `bits`; one CTA.
__global__ void __launch_bounds__(256) k_tile_rows(const int* __restrict__ pmask, int bits, int n, int tz,
                                                   int* __restrict__ rows, int* __restrict__ count) {
    __shared__ int woff[8];
    const int r = threadIdx.x, lane = r & 31, wid = r >> 5;
    int live = 0;
    if (r < n / tz) {
        for (int z = r * tz; z < r * tz + tz; ++z)
            for (int q = 0; q < 3; ++q)
                if (bits & (1 << q)) live |= pmask[q * n + z];
    }
    const unsigned b = __ballot_sync(0xffffffffu, live != 0);
    if (lane == 0) woff[wid] = __popc(b);
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; ++w) base += woff[w];
    if (live) rows[base + __popc(b & ((1u << lane) - 1u))] = r;
    if (r == 255) *count = base + __popc(b);
}

template <typename T>
cudaError_t launch_tile_ranges(const FusedArgs<T>& a, int* out, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (a.trows == nullptr || a.trow_count == nullptr) return cudaErrorInvalidValue;
        if (a.n == 256 || a.n == 512) {
            const int tiles = (a.n / a.ty) * (a.n / a.tz);
            const int blocks = std::max(1, std::min((tiles + 7) / 8, 152 * 8));
            if (a.n == 256) k_tile_ranges<T, 8><<<blocks, 256, 0, st>>>(a, out);
            else k_tile_ranges<T, 9><<<blocks, 256, 0, st>>>(a, out);
            return cudaGetLastError();
        }
    }
    return cudaErrorInvalidValue;
}

size_t tile_range_bytes(int n, int ty, int tz) { return (size_t)(n / ty) * (n / tz) * kRec * sizeof(int); }

cudaError_t launch_tile_rows(const int* pmask, int bits, int n, int tz, int* rows, int* count, cudaStream_t st) {
    if (n / tz > 256) return cudaErrorInvalidValue;
    k_tile_rows<<<1, 256, 0, st>>>(pmask, bits, n, tz, rows, count);
    return cudaGetLastError();
}

template <typename T, int LOGN>
static cudaError_t launch_fused_n(const FusedArgs<T>& a, int n_tiles, cudaStream_t st) {
    using S = FusedShape<T, LOGN>;
    if (a.ty != S::TY || a.tz != S::TZ) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)(S::N + S::N * S::LD + S::TWR) * sizeof(c2<T>);
    cudaFuncSetAttribute(k_assign_xfft<T, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if constexpr (sizeof(T) == 4 && (LOGN == 8 || LOGN == 9)) {
        if (a.dual) {
            // two slots per CTA (FusedArgs::dual: even slot count, interlaced single-source
            // coefficient slots, a tile-row list)
            const size_t smem2 = (size_t)(S::N + 2 * S::N * S::LD + S::TWR) * sizeof(c2<T>);
            cudaFuncSetAttribute(k_assign_xfft2<T, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
            int dev = 0, sms = 152;
            if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int pairs = a.n_slots / 2;
            const int g2 = std::max(1, std::min(n_tiles, 2 * sms / pairs));
            k_assign_xfft2<T, LOGN><<<dim3(g2, pairs), 2 * S::THREADS, smem2, st>>>(a);
            return cudaGetLastError();
        }
    }
    int grid = n_tiles, slots_y = a.n_slots;
    if (a.trows) {
        // persistent: about two resident waves over all slots (dynamic: one resident wave
        // that takes items until none is left)
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = std::max(1, (int)((227 * 1024) / (smem + 1024)));
        if (a.work) {
            grid = std::max(1, std::min(n_tiles * a.n_slots, sms * per_sm));
            slots_y = 1;
        } else {
            grid = std::max(1, std::min(n_tiles, 2 * sms * per_sm / std::max(1, a.n_slots)));
        }
    }
    k_assign_xfft<T, LOGN><<<dim3(grid, slots_y), S::THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_assign_xfft(const FusedArgs<T>& a, cudaStream_t st) {
    if (a.n_slots == 0) return cudaSuccess;
    const int n_tiles = (a.n / a.ty) * (a.n / a.tz);
    switch (a.n) {
        case 8: return launch_fused_n<T, 3>(a, n_tiles, st);
        case 16: return launch_fused_n<T, 4>(a, n_tiles, st);
        case 32: return launch_fused_n<T, 5>(a, n_tiles, st);
        case 64: return launch_fused_n<T, 6>(a, n_tiles, st);
        case 128: return launch_fused_n<T, 7>(a, n_tiles, st);
        case 256: return launch_fused_n<T, 8>(a, n_tiles, st);
        case 512: return launch_fused_n<T, 9>(a, n_tiles, st);
        case 1024: return launch_fused_n<T, 10>(a, n_tiles, st);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_pencil_sort<float>(const float*, const float*, long long, long long, int, double,
                                               const double*, int*, int*, int*, int*, int*, float*, float*, int*, int*,
                                               cudaStream_t);
template cudaError_t launch_pencil_sort<double>(const double*, const double*, long long, long long, int, double,
                                                const double*, int*, int*, int*, int*, int*, double*, double*, int*, int*,
                                                cudaStream_t);
template cudaError_t launch_tile_ranges<float>(const FusedArgs<float>&, int*, cudaStream_t);
template cudaError_t launch_tile_ranges<double>(const FusedArgs<double>&, int*, cudaStream_t);
template cudaError_t launch_assign_xfft<float>(const FusedArgs<float>&, cudaStream_t);
template cudaError_t launch_assign_xfft<double>(const FusedArgs<double>&, cudaStream_t);

}  // namespace lpp
