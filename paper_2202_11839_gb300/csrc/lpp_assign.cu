// Per-particle harmonic weights, catalogue sums and CIC/TSC mass assignment.
//
// Harmonic weights.  For a galaxy at xhat with shear gamma, every LPP kernel is a
// pure degree-L spherical harmonic of khat (Y_L^m(S^-1(x) k) = N Lm_L(k.x) e^{im phi},
// Appendix C):
//   cross: gamma (2 e*_ij k_i k_j) Lm2_L(mu)/(1-mu^2)       (Eq. def_of_Xiij)
//   plus : gamma L_l(mu)                                    (Eq. lpp_estimator_auto_+)
//   minus: gamma (2 e*_ij k_i k_j)^2 Lm4_L(mu)/(1-mu^2)^2   (Eq. def_of_Xiijkl)
// with 2 e*_ij k_i k_j = (k.e_theta - i k.e_phi)^2.  Its 2L+1 real-harmonic
// coefficients are obtained exactly by a Gauss-Legendre (L+1 nodes in cos theta) x
// trapezoid (2L+1 azimuths) quadrature of K(khat) Y_{L,n}(khat), which integrates the
// degree-2L integrand without error.  One field per coefficient then carries the
// kernel to the grid: F(k) = sum_n Y_{L,n}(khat) FT[sum_g w_g c_n(g) delta_D](k).
#include "lpp_internal.h"
#include "lpp_kernels.h"

namespace lpp {

// Sky frame about the pole p: e_phi = unit(p x xhat), e_theta = e_phi x xhat.
template <typename T>
__device__ __forceinline__ void sky_frame(const T xh[3], const double pole[3], T et[3], T ep[3], int* err) {
    const T p0 = (T)pole[0], p1 = (T)pole[1], p2 = (T)pole[2];
    T c0 = p1 * xh[2] - p2 * xh[1];
    T c1 = p2 * xh[0] - p0 * xh[2];
    T c2v = p0 * xh[1] - p1 * xh[0];
    T nrm = sqrt(c0 * c0 + c1 * c1 + c2v * c2v);
    if (!(nrm >= (T)1e-6)) {
        atomicOr(err, ERRF_POLE);
        nrm = (T)1;
    }
    ep[0] = c0 / nrm;
    ep[1] = c1 / nrm;
    ep[2] = c2v / nrm;
    et[0] = ep[1] * xh[2] - ep[2] * xh[1];
    et[1] = ep[2] * xh[0] - ep[0] * xh[2];
    et[2] = ep[0] * xh[1] - ep[1] * xh[0];
}

// Shared-memory layout of the quadrature for degree L = 2 (q + 1): directions as [S][4]
// (x, y, z, 0) and the table transposed to [S][NHP] (NHP = 2L + 1 rounded up to a multiple
// of 4), so that a quadrature point reads its direction and its 2L + 1 table entries in
// 16-byte words; every thread of a block reads the same entries at the same time
// (broadcast).  The blocks of L = 2, 4, ..., 12 follow one another, then the polynomials; a
// degree that no group of the plan uses has S = 0 and takes no space.
__host__ __device__ constexpr int quad_nhp(int q) { return (2 * (2 * (q + 1)) + 1 + 3) & ~3; }

template <typename T>
__host__ __device__ inline int quad_block_words(const CoeffArgs<T>& a, int q) { return a.quad_S[q] * (4 + quad_nhp(q)); }

// sm: the block's shared copy of the quadrature directions, tables and polynomials
template <typename T, int L, bool HAS_IM>
__device__ __forceinline__ void project_group(const CoeffArgs<T>& a, const CoeffGroup& g, long long i, T wgt,
                                              T gre, T gim, const T et[3], const T ep[3], const T xh[3],
                                              const T* sm) {
    constexpr int NH = 2 * L + 1;
    constexpr int q = L / 2 - 1;
    constexpr int NHP = quad_nhp(q);
    int o = 0;
#pragma unroll
    for (int qq = 0; qq < q; ++qq) o += quad_block_words(a, qq);
    const int S = a.quad_S[q];
    const T* dirs = sm + o;
    const T* tab = dirs + 4 * S;
    int op = 0;
#pragma unroll
    for (int qq = 0; qq < kQuadDegrees; ++qq) op += quad_block_words(a, qq);
    const T* poly = sm + op + g.poly;
    // the kernel polynomial in registers, zero-padded to NPC coefficients (the leading zeros
    // leave Horner's scheme exact); the minus kernel of L = 12 has degree 8
    constexpr int NPC = L > 10 ? 9 : 8;
    T pc[NPC];
#pragma unroll
    for (int k = 0; k < NPC; ++k) pc[k] = k < g.npoly ? poly[k] : (T)0;
    T accr[NH], acci[NH];
#pragma unroll
    for (int n = 0; n < NH; ++n) { accr[n] = (T)0; acci[n] = (T)0; }
    for (int s = 0; s < S; ++s) {
        T kx, ky, kz;
        T t[NHP];
        if constexpr (sizeof(T) == 4) {
            const float4 d = reinterpret_cast<const float4*>(dirs)[s];
            kx = d.x;
            ky = d.y;
            kz = d.z;
            const float4* tv = reinterpret_cast<const float4*>(tab + s * NHP);
#pragma unroll
            for (int j = 0; j < NHP / 4; ++j) {
                const float4 v = tv[j];
                t[4 * j] = v.x;
                t[4 * j + 1] = v.y;
                t[4 * j + 2] = v.z;
                t[4 * j + 3] = v.w;
            }
        } else {
            kx = dirs[4 * s];
            ky = dirs[4 * s + 1];
            kz = dirs[4 * s + 2];
#pragma unroll
            for (int n = 0; n < NH; ++n) t[n] = tab[s * NHP + n];
        }
        const T mu = kx * xh[0] + ky * xh[1] + kz * xh[2];
        T pm = (T)0;
#pragma unroll
        for (int k = NPC - 1; k >= 0; --k) pm = pm * mu + pc[k];
        T kre, kim;
        if (g.kind == KIND_PLUS) {
            kre = gre * pm;
            kim = gim * pm;
        } else {
            const T ca = kx * et[0] + ky * et[1] + kz * et[2];
            const T cb = kx * ep[0] + ky * ep[1] + kz * ep[2];
            T zr = ca * ca - cb * cb, zi = (T)-2 * ca * cb;  // (a - i b)^2
            if (g.kind == KIND_MINUS) {
                const T tt = zr * zr - zi * zi;
                zi = (T)2 * zr * zi;
                zr = tt;
            }
            zr *= pm;
            zi *= pm;
            kre = gre * zr - gim * zi;
            kim = gre * zi + gim * zr;
        }
#pragma unroll
        for (int n = 0; n < NH; ++n) {
            accr[n] += t[n] * kre;
            if (HAS_IM) acci[n] += t[n] * kim;
        }
    }
#pragma unroll
    for (int n = 0; n < NH; ++n) {
        a.coeff[(long long)(g.row_re + n) * a.stride + i] = wgt * accr[n];
        if (HAS_IM) a.coeff[(long long)(g.row_im + n) * a.stride + i] = wgt * acci[n];
    }
}

template <typename T>
__device__ __forceinline__ void unit_los(const T* pos, long long count, long long i, const double obs[3], T xh[3],
                                         int* err) {
    T r0 = pos[i] - (T)obs[0];
    T r1 = pos[count + i] - (T)obs[1];
    T r2 = pos[2 * count + i] - (T)obs[2];
    T nrm = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
    if (!(nrm > (T)0)) {
        atomicOr(err, ERRF_OBSERVER);
        nrm = (T)1;
    }
    xh[0] = r0 / nrm;
    xh[1] = r1 / nrm;
    xh[2] = r2 / nrm;
}

template <typename T>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_add(double v, double* dst) {
    __shared__ double part[32];
    v = warp_sum<double>(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) part[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
        v = warp_sum<double>(v);
        if (lane == 0 && v != 0.0) atomicAdd(dst, v);
    }
}

// Shared-memory words for the quadrature directions and tables (L = 2, 4, ..., 12, laid out
// as in project_group) and the polynomials.
template <typename T>
__host__ __device__ inline int coeff_smem_words(const CoeffArgs<T>& a) {
    int w = a.n_polys;
    for (int q = 0; q < kQuadDegrees; ++q) w += quad_block_words(a, q);
    return w;
}

// HIGH: the plan has groups of degree 10 or 12 (the minus moments beyond L = 8), a separate
// instantiation so that their register arrays leave the usual one unchanged
template <typename T, bool HIGH>
__global__ void __launch_bounds__(256) k_coeffs(CoeffArgs<T> a) {
    extern __shared__ __align__(16) unsigned char coeff_smem[];
    T* sm = reinterpret_cast<T*>(coeff_smem);
    {
        int o = 0;
        for (int q = 0; q < kQuadDegrees; ++q) {
            const int S = a.quad_S[q], nh = 2 * (2 * (q + 1)) + 1, nhp = quad_nhp(q);
            // directions [S][3] -> [S][4]; table [nh][S] -> [S][nhp] (zero padding)
            for (int i = threadIdx.x; i < 4 * S; i += blockDim.x)
                sm[o + i] = (i & 3) < 3 ? a.quad_dirs[q][(i >> 2) * 3 + (i & 3)] : (T)0;
            o += 4 * S;
            for (int i = threadIdx.x; i < nhp * S; i += blockDim.x) {
                const int si = i / nhp, n = i - si * nhp;
                sm[o + i] = n < nh ? a.quad_tab[q][n * S + si] : (T)0;
            }
            o += nhp * S;
        }
        for (int i = threadIdx.x; i < a.n_polys; i += blockDim.x) sm[o + i] = a.polys[i];
        __syncthreads();
    }
    double sw = 0.0, sg = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.count;
         i += (long long)gridDim.x * blockDim.x) {
        const long long si = a.perm ? (long long)a.perm[i] : i;  // input index of output particle i
        if (!LPP_IN_BOUNDS(si >= 0 && si < a.count, a.err)) continue;
        T xl[3];
        unit_los(a.pos, a.count, si, a.observer, xl, a.err);
        T xg[3] = {(T)a.los_global[0], (T)a.los_global[1], (T)a.los_global[2]};
        const T* xp = a.los_proj == LPP_LOS_GLOBAL ? xg : xl;
        const T* xe = a.los_est == LPP_LOS_GLOBAL ? xg : xl;
        T etp[3], epp[3], ete[3], epe[3];
        sky_frame(xp, a.pole, etp, epp, a.err);
        if (a.los_proj == a.los_est) {
            for (int d = 0; d < 3; ++d) { ete[d] = etp[d]; epe[d] = epp[d]; }
        } else {
            sky_frame(xe, a.pole, ete, epe, a.err);
        }
        T g1, g2;
        if (a.shape_kind == LPP_SHAPE_TENSOR6) {
            const T* s = a.shape;
            const long long c = a.count;
            const T sxx = s[si], syy = s[c + si], szz = s[2 * c + si], sxy = s[3 * c + si], sxz = s[4 * c + si],
                    syz = s[5 * c + si];
            const T st0 = sxx * etp[0] + sxy * etp[1] + sxz * etp[2];
            const T st1 = sxy * etp[0] + syy * etp[1] + syz * etp[2];
            const T st2 = sxz * etp[0] + syz * etp[1] + szz * etp[2];
            const T sp0 = sxx * epp[0] + sxy * epp[1] + sxz * epp[2];
            const T sp1 = sxy * epp[0] + syy * epp[1] + syz * epp[2];
            const T sp2 = sxz * epp[0] + syz * epp[1] + szz * epp[2];
            const T stt = etp[0] * st0 + etp[1] * st1 + etp[2] * st2;
            const T spp = epp[0] * sp0 + epp[1] * sp1 + epp[2] * sp2;
            const T stp = etp[0] * sp0 + etp[1] * sp1 + etp[2] * sp2;
            g1 = (T)0.5 * (stt - spp);  // gamma = e_ij s_ij (Eq. gamma_def)
            g2 = stp;
        } else {
            g1 = a.shape[si];
            g2 = a.shape[a.count + si];
        }
        const T w = a.w ? a.w[si] : (T)1;
        a.coeff[i] = w * g1;              // row 0: w gamma_1
        a.coeff[a.stride + i] = w * g2;   // row 1: w gamma_2
        sw += (double)w;
        sg += (double)w * (double)w * ((double)g1 * g1 + (double)g2 * g2);
        for (int gi = 0; gi < a.n_groups; ++gi) {
            const CoeffGroup& g = a.groups[gi];
            if (g.L == 2) {
                if (g.has_im) project_group<T, 2, true>(a, g, i, w, g1, g2, ete, epe, xe, sm);
                else project_group<T, 2, false>(a, g, i, w, g1, g2, ete, epe, xe, sm);
            } else if (g.L == 4) {
                if (g.has_im) project_group<T, 4, true>(a, g, i, w, g1, g2, ete, epe, xe, sm);
                else project_group<T, 4, false>(a, g, i, w, g1, g2, ete, epe, xe, sm);
            } else if (g.L == 6) {
                if (g.has_im) project_group<T, 6, true>(a, g, i, w, g1, g2, ete, epe, xe, sm);
                else project_group<T, 6, false>(a, g, i, w, g1, g2, ete, epe, xe, sm);
            } else if (g.L == 8) {
                project_group<T, 8, true>(a, g, i, w, g1, g2, ete, epe, xe, sm);
            } else if constexpr (HIGH) {
                if (g.L == 10) project_group<T, 10, true>(a, g, i, w, g1, g2, ete, epe, xe, sm);
                else if (g.L == 12) project_group<T, 12, true>(a, g, i, w, g1, g2, ete, epe, xe, sm);
            }
        }
    }
    block_add(sw, a.sums + SUM_W_SHAPES);
    block_add(sg, a.sums + SUM_W2G2_SHAPES);
}

template <typename T>
cudaError_t launch_coeffs(const CoeffArgs<T>& a, cudaStream_t st) {
    if (a.count == 0) return cudaSuccess;
    long long blocks = (a.count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const size_t smem = (size_t)coeff_smem_words(a) * sizeof(T);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    bool high = false;
    for (int g = 0; g < a.n_groups; ++g) high = high || a.groups[g].L > 8;
    if (high) {
        cudaFuncSetAttribute(k_coeffs<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_coeffs<T, true><<<(int)blocks, 256, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(k_coeffs<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_coeffs<T, false><<<(int)blocks, 256, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_sums(const T* w, const T* nbar, long long count, double* sums, int s_w,
                                              int s_w2, int s_nw2) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const double wi = w ? (double)w[i] : 1.0;
        const double ni = nbar ? (double)nbar[i] : 1.0;
        a += wi;
        b += wi * wi;
        c += ni * wi * wi;
    }
    if (s_w >= 0) block_add(a, sums + s_w);
    if (s_w2 >= 0) block_add(b, sums + s_w2);
    if (s_nw2 >= 0) block_add(c, sums + s_nw2);
}

template <typename T>
cudaError_t launch_sums(const T* w, const T* nbar, long long count, double* sums, int s_w, int s_w2, int s_nw2,
                        cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_sums<T><<<(int)blocks, 256, 0, st>>>(w, nbar, count, sums, s_w, s_w2, s_nw2);
    return cudaGetLastError();
}

__global__ void k_alpha(double* sums, int has_randoms) {
    sums[SUM_ALPHA] = (has_randoms && sums[SUM_W_RAND] != 0.0) ? sums[SUM_W_DENS] / sums[SUM_W_RAND] : 0.0;
}

cudaError_t launch_alpha(double* sums, int has_randoms, cudaStream_t st) {
    k_alpha<<<1, 1, 0, st>>>(sums, has_randoms);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ assignment
// Node i of sub-grid s sits at origin + (i + s/2) H.  CIC (P = 2): w(d) = 1 - |d|;
// TSC (P = 3): w(d) = 3/4 - d^2 for |d| <= 1/2, (3/2 - |d|)^2 / 2 for 1/2 <= |d| < 3/2.
template <typename T, int P>
__device__ __forceinline__ void stencil(T u, int n, int cells[P], T w[P]) {
    if (P == 2) {
        const T fl = floor(u);
        const T f = u - fl;
        int i0 = (int)fl;
        w[0] = (T)1 - f;
        w[1] = f;
        cells[0] = i0;
        cells[1] = i0 + 1;
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
    for (int k = 0; k < P; ++k) {
        int c = cells[k];
        c = c < 0 ? c + n : (c >= n ? c - n : c);
        cells[k] = c;
    }
}

template <typename T, int P, bool IL>
__global__ void __launch_bounds__(256) k_assign(AssignArgs<T> a) {
    const int n = a.n;
    const T ih = (T)((double)n / a.box);
    const T ox = (T)a.origin[0], oy = (T)a.origin[1], oz = (T)a.origin[2];
    const T alpha = (T)a.sums[SUM_ALPHA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.count;
         i += (long long)gridDim.x * blockDim.x) {
        const T u0 = (a.pos[i] - ox) * ih;
        const T u1 = (a.pos[a.count + i] - oy) * ih;
        const T u2 = (a.pos[2 * a.count + i] - oz) * ih;
        if (!(u0 >= (T)0 && u0 <= (T)n && u1 >= (T)0 && u1 <= (T)n && u2 >= (T)0 && u2 <= (T)n)) {
            atomicOr(a.err, ERRF_DOMAIN);
            continue;
        }
        int cx[P], cy[P], cz[P];
        T wx[P], wy[P], wz[P];
        stencil<T, P>(u0, n, cx, wx);
        stencil<T, P>(u1, n, cy, wy);
        stencil<T, P>(u2, n, cz, wz);
        int dx[P], dy[P], dz[P];
        T vx[P], vy[P], vz[P];
        if (IL) {
            stencil<T, P>(u0 - (T)0.5, n, dx, vx);
            stencil<T, P>(u1 - (T)0.5, n, dy, vy);
            stencil<T, P>(u2 - (T)0.5, n, dz, vz);
        }
        for (int s = 0; s < a.n_slots; ++s) {
            const AssignSlot& sl = a.slots[s];
            T va = sl.unit_a ? (T)1 : static_cast<const T*>(sl.src_a)[i];
            if (sl.scale_alpha) va *= -alpha;
            const bool has_b = !IL && sl.src_b != nullptr;
            const T vb = has_b ? static_cast<const T*>(sl.src_b)[i] : (T)0;
            T* g = reinterpret_cast<T*>(a.grids + sl.grid * a.grid_stride);
#pragma unroll
            for (int kz = 0; kz < P; ++kz)
#pragma unroll
                for (int ky = 0; ky < P; ++ky) {
                    const long long row = ((long long)cz[kz] * n + cy[ky]) * n;
                    const T wzy = wz[kz] * wy[ky];
#pragma unroll
                    for (int kx = 0; kx < P; ++kx) {
                        const long long idx = 2 * (row + cx[kx]);
                        const T ww = wzy * wx[kx];
                        atomicAdd(g + idx, va * ww);
                        if (has_b) atomicAdd(g + idx + 1, vb * ww);
                    }
                }
            if (IL) {
#pragma unroll
                for (int kz = 0; kz < P; ++kz)
#pragma unroll
                    for (int ky = 0; ky < P; ++ky) {
                        const long long row = ((long long)dz[kz] * n + dy[ky]) * n;
                        const T wzy = vz[kz] * vy[ky];
#pragma unroll
                        for (int kx = 0; kx < P; ++kx) atomicAdd(g + 2 * (row + dx[kx]) + 1, va * (wzy * vx[kx]));
                    }
            }
        }
    }
}

template <typename T>
cudaError_t launch_assign(const AssignArgs<T>& a, int scheme, int interlace, cudaStream_t st) {
    if (a.count == 0 || a.n_slots == 0) return cudaSuccess;
    long long blocks = (a.count + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    const int b = (int)blocks;
    if (scheme == LPP_CIC) {
        if (interlace) k_assign<T, 2, true><<<b, 256, 0, st>>>(a);
        else k_assign<T, 2, false><<<b, 256, 0, st>>>(a);
    } else {
        if (interlace) k_assign<T, 3, true><<<b, 256, 0, st>>>(a);
        else k_assign<T, 3, false><<<b, 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

// Per-row statistics of the coefficients: rstat[2r] = max |c| (atomicMax on the float's
// bits: non-negative floats order like ints) and rstat[2r + 1] = rms c, from a grid-stride
// loop per row (blockIdx.y), warp reductions and FP64 sums of squares in rsq.
__global__ void __launch_bounds__(256) k_rowstat(const float* __restrict__ coeff, long long stride, long long count,
                                                 float* __restrict__ rstat, double* __restrict__ rsq) {
    const float* row = coeff + (long long)blockIdx.y * stride;
    float m = 0.f, qf = 0.f;   // per-thread sums cover count / (64 * 256) values: FP32 is plenty
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = row[i];
        m = fmaxf(m, fabsf(v));
        qf = fmaf(v, v, qf);
    }
    double q = (double)qf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
        q += __shfl_down_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (m > 0.f) atomicMax(reinterpret_cast<int*>(rstat) + 2 * blockIdx.y, __float_as_int(m));
        if (q > 0.0) atomicAdd(rsq + blockIdx.y, q);
    }
}

__global__ void k_rowrms(const double* __restrict__ rsq, long long count, int rows, float* __restrict__ rstat) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) rstat[2 * r + 1] = count > 0 ? (float)sqrt(rsq[r] / (double)count) : 0.f;
}

cudaError_t launch_rowstat(const float* coeff, long long stride, long long count, int rows, float* rstat,
                           double* rsq, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(rstat, 0, (size_t)rows * 2 * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rsq, 0, (size_t)rows * sizeof(double), st);
    if (e != cudaSuccess || count == 0 || rows == 0) return e;
    long long bx = (count + 255) / 256;
    if (bx > 64) bx = 64;
    k_rowstat<<<dim3((unsigned)bx, (unsigned)rows), 256, 0, st>>>(coeff, stride, count, rstat, rsq);
    k_rowrms<<<(rows + 127) / 128, 128, 0, st>>>(rsq, count, rows, rstat);
    return cudaGetLastError();
}

template cudaError_t launch_coeffs<float>(const CoeffArgs<float>&, cudaStream_t);
template cudaError_t launch_coeffs<double>(const CoeffArgs<double>&, cudaStream_t);
template cudaError_t launch_sums<float>(const float*, const float*, long long, double*, int, int, int, cudaStream_t);
template cudaError_t launch_sums<double>(const double*, const double*, long long, double*, int, int, int,
                                         cudaStream_t);
template cudaError_t launch_assign<float>(const AssignArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_assign<double>(const AssignArgs<double>&, int, int, cudaStream_t);

}  // namespace lpp
