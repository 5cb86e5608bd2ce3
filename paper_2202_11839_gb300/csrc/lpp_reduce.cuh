// Warp-segmented shell reduction and compensated accumulators (internal).
#pragma once

#include "lpp_internal.h"

namespace lpp {

template <typename T> struct Owned;
template <> struct Owned<float> {
    // compensated sum (Knuth two-sum) in two floats
    static __device__ __forceinline__ void add(float* hi, float* lo, float v) {
        const float s = *hi + v;
        const float bp = s - *hi;
        const float err = (*hi - (s - bp)) + (v - bp);
        *hi = s;
        *lo += err;
    }
    static __device__ __forceinline__ double value(const float* hi, const float* lo) {
        return (double)*hi + (double)*lo;
    }
    static constexpr int words = 2;
};
template <> struct Owned<double> {
    static __device__ __forceinline__ void add(double* hi, double*, double v) { *hi += v; }
    static __device__ __forceinline__ double value(const double* hi, const double*) { return *hi; }
    static constexpr int words = 1;
};

template <typename T>
__device__ __forceinline__ int freq_of(int i, int n) { return i < n / 2 ? i : i - n; }

// segmented inclusive scan of (re, im) over lanes with equal segment keys, the keys monotone
// along the warp (equal keys form one contiguous run); the last lane of each run adds the run
// total to acc[bin][2].  key = bin when the shell labels themselves are monotone.
template <typename T>
__device__ __forceinline__ void warp_bin_add(T re, T im, int bin, T* acc, int key) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int ok = __shfl_up_sync(full, key, d);
        const T ore = __shfl_up_sync(full, re, d);
        const T oim = __shfl_up_sync(full, im, d);
        if (lane >= d && ok == key) {
            re += ore;
            im += oim;
        }
    }
    const int nk = __shfl_down_sync(full, key, 1);
    const bool last = (lane == 31) || (nk != key);
    if (last && bin >= 0) {
        atomicAdd(acc + 2 * bin, re);
        atomicAdd(acc + 2 * bin + 1, im);
    }
}
template <typename T>
__device__ __forceinline__ void warp_bin_add(T re, T im, int bin, T* acc) {
    warp_bin_add<T>(re, im, bin, acc, bin);
}

// The shell labels of a row are the same for every channel: the steps of the segmented scan
// that add (bit s: lane >= 2^s and the lane 2^s below is in the same shell) and whether the
// lane ends its segment are computed once per row.
struct SegMask {
    unsigned add;   // bit s set: add the value shuffled up by 2^s
    bool last;      // the lane holds its segment's sum after the scan
};

// key: the lane's segment (equal keys contiguous along the warp), e.g. its shell label
__device__ __forceinline__ SegMask seg_mask(int key) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    SegMask m;
    m.add = 0u;
#pragma unroll
    for (int s = 0, d = 1; d < 32; d <<= 1, ++s) {
        const int ok = __shfl_up_sync(full, key, d);
        if (lane >= d && ok == key) m.add |= 1u << s;
    }
    const int nk = __shfl_down_sync(full, key, 1);
    m.last = (lane == 31) || (nk != key);
    return m;
}

// warp_bin_add with the row's precomputed segment structure
template <typename T>
__device__ __forceinline__ void warp_bin_add_seg(T re, T im, int bin, const SegMask& m, T* acc) {
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int s = 0, d = 1; d < 32; d <<= 1, ++s) {
        const T ore = __shfl_up_sync(full, re, d);
        const T oim = __shfl_up_sync(full, im, d);
        if ((m.add >> s) & 1u) {
            re += ore;
            im += oim;
        }
    }
    if (m.last && bin >= 0) {
        atomicAdd(acc + 2 * bin, re);
        atomicAdd(acc + 2 * bin + 1, im);
    }
}

}  // namespace lpp
