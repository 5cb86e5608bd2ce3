// Template surrogate network: 6 -> [256, GELU] x 4 -> 320, BF16 operands, FP32 accumulation.
//
// Every matrix product C = A B^T (A [M x K], B [N x K], both BF16 with K contiguous) runs on
// the tensor cores (mma.m16n8k16, BF16 in, FP32 accumulate) in 64 x 64 CTA tiles with fused
// epilogues: bias + GELU for hidden layers (the BF16 activation and, when training, its
// transpose), bias for the output, plain FP32 for weight gradients, and the GELU derivative
// for back-propagated gradients.  Adam keeps FP32 master weights and refreshes their BF16
// copies (and transposes) after every step.  The training loop is native: one call runs all
// steps of a schedule of minibatch indices.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <utility>
#include <vector>

#include "lpp_internal.h"

namespace {

using bf16 = __nv_bfloat16;
constexpr int kLayers = 5;
constexpr int kIn[kLayers] = {6, 256, 256, 256, 256};
constexpr int kInPad[kLayers] = {16, 256, 256, 256, 256};
constexpr int kOut[kLayers] = {256, 256, 256, 256, 320};
constexpr int kNout = 320;
constexpr int kNin = 6;

enum Epi { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_DW = 2, EPI_DA_GELU = 3 };

struct GemmArgs {
    const bf16* A;
    int lda;
    const bf16* B;
    int ldb;
    int M, N, K;
    int epi;
    const float* bias;
    float* z;          // hidden: pre-activation; out: output; dW: gradient
    int ldz;
    bf16* a16;         // hidden: BF16 GELU(z); da: BF16 gradient
    int ld16;
    bf16* a16t;        // transposed BF16 copy (optional)
    int ld16t;
    const float* zprev;   // da: pre-activation of the layer below
    int ldzp;
    float* g32;           // da: FP32 gradient
    int ldg;
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

constexpr int BM = 64, BN = 64, BK = 32, LDS = BK + 8;

__global__ void __launch_bounds__(128) k_gemm(GemmArgs a) {
    __shared__ __align__(16) bf16 As[BM][LDS];
    __shared__ __align__(16) bf16 Bs[BN][LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    for (int k0 = 0; k0 < a.K; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = tid + i * 128;   // 256 chunks of 8 BF16 per tile
            const int row = c >> 2, col = (c & 3) * 8;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + row < a.M && k0 + col < a.K)
                va = *reinterpret_cast<const uint4*>(a.A + (size_t)(m0 + row) * a.lda + k0 + col);
            if (n0 + row < a.N && k0 + col < a.K)
                vb = *reinterpret_cast<const uint4*>(a.B + (size_t)(n0 + row) * a.ldb + k0 + col);
            *reinterpret_cast<uint4*>(&As[row][col]) = va;
            *reinterpret_cast<uint4*>(&Bs[row][col]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm * 32 + mi * 16 + g;
                af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t]);
                af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t]);
                af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t + 8]);
                af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int n = wn * 32 + ni * 8 + g;
                bfr[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 2 * t]);
                bfr[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
                        : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bfr[ni][0]),
                          "r"(bfr[ni][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm * 32 + mi * 16 + g + (r >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + ni * 8 + 2 * t + (r & 1);
                if (row >= a.M || col >= a.N) continue;
                const float v = acc[mi][ni][r];
                if (a.epi == EPI_HIDDEN) {
                    const float z = v + a.bias[col];
                    a.z[(size_t)row * a.ldz + col] = z;
                    const bf16 h = __float2bfloat16_rn(gelu(z));
                    a.a16[(size_t)row * a.ld16 + col] = h;
                    if (a.a16t) a.a16t[(size_t)col * a.ld16t + row] = h;
                } else if (a.epi == EPI_OUT) {
                    a.z[(size_t)row * a.ldz + col] = v + a.bias[col];
                } else if (a.epi == EPI_DW) {
                    a.z[(size_t)row * a.ldz + col] = v;
                } else {
                    const float gv = v * gelu_grad(a.zprev[(size_t)row * a.ldzp + col]);
                    a.g32[(size_t)row * a.ldg + col] = gv;
                    const bf16 h = __float2bfloat16_rn(gv);
                    a.a16[(size_t)row * a.ld16 + col] = h;
                    a.a16t[(size_t)col * a.ld16t + row] = h;
                }
            }
}

cudaError_t gemm(const GemmArgs& a, cudaStream_t st) {
    dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM);
    k_gemm<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// inputs x [m][6] FP32 -> BF16 [m][16] (zero padded) and, when training, its transpose [16][ld]
__global__ void k_input(const float* __restrict__ x, const int* __restrict__ idx, int m, bf16* a0, bf16* a0t,
                        int ldt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m * 16; i += gridDim.x * blockDim.x) {
        const int r = i / 16, c = i % 16;
        const int src = idx ? idx[r] : r;
        const float v = c < kNin ? x[(size_t)src * kNin + c] : 0.f;
        const bf16 h = __float2bfloat16_rn(v);
        a0[i] = h;
        if (a0t) a0t[(size_t)c * ldt + r] = h;
    }
}

// dL/d out = 2 (out - y) / (m * 320); loss sum of squares into loss (FP64)
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ y, const int* __restrict__ idx, int m,
                       float* g32, bf16* g16, bf16* g16t, int ldt, double* loss) {
    double part = 0.0;
    const float sc = 2.0f / (float)(m * kNout);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m * kNout; i += gridDim.x * blockDim.x) {
        const int r = i / kNout, c = i % kNout;
        const int src = idx ? idx[r] : r;
        const float d = out[i] - y[(size_t)src * kNout + c];
        part += (double)d * d;
        const float gv = sc * d;
        g32[i] = gv;
        const bf16 h = __float2bfloat16_rn(gv);
        g16[i] = h;
        g16t[(size_t)c * ldt + r] = h;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(loss, part / (double)(m * kNout));
}

// db[n] = sum over rows of g[m][n]
// db[c] = sum_r g[r][c]: 32 columns per CTA (a warp reads 32 consecutive columns of a row),
// eight warps each over every eighth row, then the eight partial sums in a fixed order
__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ g, int m, int n, float* db) {
    __shared__ float part[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (c < n)
        for (int r = w; r < m; r += 8) s += g[(size_t)r * n + c];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && c < n) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += part[k][lane];
        db[c] = t;
    }
}

struct AdamLayer {
    float *w, *b, *mw, *vw, *mb, *vb, *dw, *db;
    bf16 *w16, *w16t;
    int out, in, inp;
};
struct AdamArgs {
    AdamLayer L[kLayers];
    float lr, b1, b2, eps, bc1, bc2;
};

__global__ void k_adam(AdamArgs a) {
    const int layer = blockIdx.y;
    const AdamLayer& L = a.L[layer];
    const int nw = L.out * L.inp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + L.out; i += gridDim.x * blockDim.x) {
        float *p, *m, *v;
        float gr;
        if (i < nw) {
            const int c = i % L.inp;
            if (c >= L.in) continue;   // padded input columns stay zero
            p = L.w + i;
            m = L.mw + i;
            v = L.vw + i;
            gr = L.dw[i];
        } else {
            const int j = i - nw;
            p = L.b + j;
            m = L.mb + j;
            v = L.vb + j;
            gr = L.db[j];
        }
        const float mm = a.b1 * *m + (1.f - a.b1) * gr;
        const float vv = a.b2 * *v + (1.f - a.b2) * gr * gr;
        *m = mm;
        *v = vv;
        const float upd = a.lr * (mm / a.bc1) / (sqrtf(vv / a.bc2) + a.eps);
        const float nwv = *p - upd;
        *p = nwv;
        if (i < nw) {
            const int r = i / L.inp, c = i % L.inp;
            const bf16 h = __float2bfloat16_rn(nwv);
            L.w16[i] = h;
            L.w16t[(size_t)c * L.out + r] = h;
        }
    }
}

// BF16 copies of the master weights (after loading parameters)
__global__ void k_refresh(AdamArgs a) {
    const int layer = blockIdx.y;
    const AdamLayer& L = a.L[layer];
    const int nw = L.out * L.inp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        const int r = i / L.inp, c = i % L.inp;
        const bf16 h = __float2bfloat16_rn(L.w[i]);
        L.w16[i] = h;
        L.w16t[(size_t)c * L.out + r] = h;
    }
}

// parameters -> network inputs and network outputs -> curves (see lpp_surrogate_map)
constexpr int kMaxNodes = 8;
struct MapArgs {
    float scale[kNin], shift[kNin];   // x_c = theta_c * scale_c + shift_c (0, 0 when not fed)
    double dscale[kNin], dshift[kNin];
    const double* mu;
    const double* sd;
    const double* shot;
    const double* ref;
    const double* sigma;
    const double* base;               // [nodes^2][320] or null
    int nodes, base_in[2];
    double N[2][3], M[3][3];          // native moments -> derived multipoles
    // the decoding's copy of base as float pairs (hi + lo = base to 2^-48), and the Lobatto
    // nodes with the Lagrange normalisations 1 / prod_{j != i} (x_i - x_j), for k_decode
    const float* base_hi;
    const float* base_lo;
    double xs[kMaxNodes], cw[kMaxNodes];
};

__global__ void k_encode(const double* __restrict__ theta, int n, float* __restrict__ x, MapArgs m) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * kNin; i += gridDim.x * blockDim.x) {
        const int c = i % kNin;
        x[i] = (float)(theta[i] * (double)m.scale[c] + (double)m.shift[c]);
    }
}

// Lagrange basis at the Chebyshev-Lobatto nodes x_i = -cos(pi i / (n - 1)), evaluated at x
__device__ void lobatto_basis(double x, int n, double* l) {
    double xs[kMaxNodes];
    for (int i = 0; i < n; ++i) xs[i] = -cospi((double)i / (double)(n - 1));
    for (int i = 0; i < n; ++i) {
        double v = 1.0;
        for (int j = 0; j < n; ++j)
            if (j != i) v *= (x - xs[j]) / (xs[i] - xs[j]);
        l[i] = v;
    }
}

// The same Lagrange basis from the map's nodes and normalisations: products only.
__device__ __forceinline__ void lobatto_basis_fast(double x, const MapArgs& a, double* l) {
    for (int i = 0; i < a.nodes; ++i) {
        double v = a.cw[i];
        for (int j = 0; j < a.nodes; ++j)
            if (j != i) v *= x - a.xs[j];
        l[i] = v;
    }
}

// base -> (hi, lo) float pairs, hi = rn(b), lo = rn(b - hi)
__global__ void k_split_base(const double* __restrict__ base, int count, float* __restrict__ hi,
                             float* __restrict__ lo) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const double b = base[i];
        const float h = (float)b;
        hi[i] = h;
        lo[i] = (float)(b - (double)h);
    }
}

// baseline mu_j + sum_ab l_a(x_p) l_b(x_q) base[a n + b][j] for one parameter row
__device__ double baseline(const MapArgs& a, const double* t, int j) {
    double u = a.mu[j];
    if (a.base) {
        double la[kMaxNodes], lb[kMaxNodes];
        lobatto_basis(t[a.base_in[0]] * a.dscale[a.base_in[0]] + a.dshift[a.base_in[0]], a.nodes, la);
        lobatto_basis(t[a.base_in[1]] * a.dscale[a.base_in[1]] + a.dshift[a.base_in[1]], a.nodes, lb);
        for (int p = 0; p < a.nodes; ++p)
            for (int q = 0; q < a.nodes; ++q) u += la[p] * lb[q] * a.base[(size_t)(p * a.nodes + q) * kNout + j];
    }
    return u;
}

// network outputs y [m][320] -> standardised curves (pre_c (baseline + sd y) + theta_5 s - ref) / sigma.
// One CTA of kNout threads per kDecodeRows parameter rows at a time: the rows' Lagrange weights
// l_a(x_p) l_b(x_q) are formed once in FP64 in shared memory and split into float pairs; thread
// j loads its base column once for the rows and sums each row's baseline output in float-float
// arithmetic (error-free products and sums, Dekker and Knuth): the FP64 sum of baseline() to
// about 2^-44 relative, on the FP32 pipes (GB300 runs FP64 at a small fraction of the FP32 rate).
constexpr int kDecodeRows = 4;
__global__ void __launch_bounds__(kNout) k_decode(const double* __restrict__ theta, int m, const float* __restrict__ y,
                                                  float* __restrict__ out, MapArgs a) {
    constexpr int nb = kNout / 8, R = kDecodeRows;
    __shared__ double la[R][kMaxNodes], lb[R][kMaxNodes];
    __shared__ float whi[R][kMaxNodes * kMaxNodes], wlo[R][kMaxNodes * kMaxNodes];
    const int j = threadIdx.x;
    const int nn = a.base ? a.nodes * a.nodes : 0;
    for (int r0 = blockIdx.x * R; r0 < m; r0 += gridDim.x * R) {
        const int nr = m - r0 < R ? m - r0 : R;
        if (a.base) {
            if (j < 2 * R && (j >> 1) < nr) {
                const int rr = j >> 1, c = a.base_in[j & 1];
                const double* t = theta + (size_t)(r0 + rr) * kNin;
                lobatto_basis_fast(t[c] * a.dscale[c] + a.dshift[c], a, (j & 1) ? lb[rr] : la[rr]);
            }
            __syncthreads();
            for (int q = j; q < R * nn; q += blockDim.x) {
                const int rr = q / nn, qq = q - rr * nn;
                float h = 0.f, l = 0.f;
                if (rr < nr) {
                    const double w = la[rr][qq / a.nodes] * lb[rr][qq % a.nodes];
                    h = (float)w;
                    l = (float)(w - (double)h);
                }
                whi[rr][qq] = h;
                wlo[rr][qq] = l;
            }
            __syncthreads();
        }
        float s_hi[R], s_lo[R];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) s_hi[rr] = s_lo[rr] = 0.f;
        for (int q = 0; q < nn; ++q) {
            const float bh = a.base_hi[(size_t)q * kNout + j], bl = a.base_lo[(size_t)q * kNout + j];
#pragma unroll
            for (int rr = 0; rr < R; ++rr) {
                const float wh = whi[rr][q], wl = wlo[rr][q];
                // the _rn intrinsics are never contracted into FMAs, which the exact
                // transformations need
                const float p = __fmul_rn(wh, bh);
                float e = fmaf(wh, bh, -p);              // wh bh = p + e exactly
                e += fmaf(wh, bl, wl * bh);              // the cross terms (wl bl is below 2^-48)
                const float s = __fadd_rn(s_hi[rr], p);  // s_hi + p = s + err exactly
                const float bb = __fsub_rn(s, s_hi[rr]);
                const float err = __fadd_rn(__fsub_rn(s_hi[rr], __fsub_rn(s, bb)), __fsub_rn(p, bb));
                s_hi[rr] = s;
                s_lo[rr] += err + e;
            }
        }
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
            if (rr >= nr) break;
            const int r = r0 + rr;
            const double* t = theta + (size_t)r * kNin;
            const double u = a.mu[j] + ((double)s_hi[rr] + (double)s_lo[rr]);
            const size_t i = (size_t)r * kNout + j;
            const double amp = t[2] * t[2] * ((j / nb) < 2 ? t[0] * t[1] : t[0] * t[0]);
            double v = amp * (u + a.sd[j] * (double)y[i]) + t[5] * a.shot[j];
            if (a.ref) v -= a.ref[j];
            if (a.sigma) v /= a.sigma[j];
            out[i] = (float)v;
        }
        __syncthreads();   // la, lb, whi, wlo are rewritten for the next rows
    }
}

// training targets: derived curves u of native template slots [n][LPP_N_MOMENTS][40] (FP64, unit
// amplitude, no shot noise), y = (u - baseline) / sd
__global__ void k_targets(const double* __restrict__ theta, const double* __restrict__ native, int n,
                          float* __restrict__ y, MapArgs a) {
    constexpr int nb = kNout / 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * kNout; i += gridDim.x * blockDim.x) {
        const int r = i / kNout, j = i % kNout, c = j / nb, b = j % nb;
        const double* o = native + (size_t)r * LPP_N_MOMENTS * nb;
        double u;
        if (c < 2) {
            u = a.N[c][0] * o[1 * nb + b] + a.N[c][1] * o[2 * nb + b] + a.N[c][2] * o[3 * nb + b];
        } else {
            const int li = (c - 2) % 3;
            const double mm = a.M[li][0] * o[7 * nb + b] + a.M[li][1] * o[8 * nb + b] + a.M[li][2] * o[9 * nb + b];
            u = 0.5 * (o[(4 + li) * nb + b] + (c < 5 ? mm : -mm));
        }
        y[i] = (float)((u - baseline(a, theta + (size_t)r * kNin, j)) / a.sd[j]);
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct lpp_surrogate_s {
    int batch = 0;
    long long step = 0;
    char* ws = nullptr;
    size_t need = 0;
    // offsets
    size_t w[kLayers], b[kLayers], mw[kLayers], vw[kLayers], mb[kLayers], vb[kLayers], dw[kLayers], db[kLayers];
    size_t w16[kLayers], w16t[kLayers], act[kLayers + 1], actt[kLayers], z[kLayers];
    size_t g32[2], g16[2], g16t[2], loss, xin;
    size_t base_hi, base_lo;          // the decoding's float-pair copy of the map's base
    bool has_map = false;
    bool base_split = false;          // base_hi/base_lo hold the current map's base
    MapArgs map;
};

extern "C" lpp_status lpp_surrogate_create(int batch, lpp_surrogate_t* out) {
    if (!out || batch < 32 || batch % 32 != 0 || batch > (1 << 20)) return LPP_ERR_INVALID_ARG;
    lpp_surrogate_t s = new lpp_surrogate_s();
    s->batch = batch;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = (size_t)kOut[l] * kInPad[l];
        s->w[l] = take(nw * 4);
        s->mw[l] = take(nw * 4);
        s->vw[l] = take(nw * 4);
        s->dw[l] = take(nw * 4);
        s->b[l] = take(kOut[l] * 4);
        s->mb[l] = take(kOut[l] * 4);
        s->vb[l] = take(kOut[l] * 4);
        s->db[l] = take(kOut[l] * 4);
        s->w16[l] = take(nw * 2);
        s->w16t[l] = take(nw * 2);
        s->act[l] = take((size_t)batch * kInPad[l] * 2);
        s->actt[l] = take((size_t)batch * kInPad[l] * 2);
        s->z[l] = take((size_t)batch * kOut[l] * 4);
    }
    s->act[kLayers] = 0;
    for (int i = 0; i < 2; ++i) {
        s->g32[i] = take((size_t)batch * kNout * 4);
        s->g16[i] = take((size_t)batch * kNout * 2);
        s->g16t[i] = take((size_t)batch * kNout * 2);
    }
    s->loss = take(8);
    s->xin = take((size_t)batch * kNin * 4);
    s->base_hi = take((size_t)kMaxNodes * kMaxNodes * kNout * 4);
    s->base_lo = take((size_t)kMaxNodes * kMaxNodes * kNout * 4);
    s->need = off;
    *out = s;
    return LPP_OK;
}

extern "C" void lpp_surrogate_destroy(lpp_surrogate_t s) { delete s; }

extern "C" lpp_status lpp_surrogate_workspace_size(lpp_surrogate_t s, size_t* bytes) {
    if (!s || !bytes) return LPP_ERR_INVALID_ARG;
    *bytes = s->need;
    return LPP_OK;
}

static AdamArgs adam_args(lpp_surrogate_t s) {
    AdamArgs a;
    memset(&a, 0, sizeof(a));
    for (int l = 0; l < kLayers; ++l) {
        AdamLayer& L = a.L[l];
        L.w = (float*)(s->ws + s->w[l]);
        L.b = (float*)(s->ws + s->b[l]);
        L.mw = (float*)(s->ws + s->mw[l]);
        L.vw = (float*)(s->ws + s->vw[l]);
        L.mb = (float*)(s->ws + s->mb[l]);
        L.vb = (float*)(s->ws + s->vb[l]);
        L.dw = (float*)(s->ws + s->dw[l]);
        L.db = (float*)(s->ws + s->db[l]);
        L.w16 = (bf16*)(s->ws + s->w16[l]);
        L.w16t = (bf16*)(s->ws + s->w16t[l]);
        L.out = kOut[l];
        L.in = kIn[l];
        L.inp = kInPad[l];
    }
    return a;
}

// Host params: for every layer W [out][in] then b [out], FP32, unpadded.
extern "C" lpp_status lpp_surrogate_set_workspace(lpp_surrogate_t s, void* dev, size_t bytes, const float* params,
                                                  void* stream) {
    if (!s || !dev || !params) return LPP_ERR_INVALID_ARG;
    if (((uintptr_t)dev & 255) != 0) return LPP_ERR_INVALID_ARG;
    if (bytes < s->need) return LPP_ERR_WORKSPACE;
    s->ws = (char*)dev;
    s->step = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(s->ws, 0, s->need, st) != cudaSuccess) return LPP_ERR_CUDA;
    std::vector<float> wpad;
    size_t p = 0;
    for (int l = 0; l < kLayers; ++l) {
        wpad.assign((size_t)kOut[l] * kInPad[l], 0.f);
        for (int r = 0; r < kOut[l]; ++r)
            for (int c = 0; c < kIn[l]; ++c) wpad[(size_t)r * kInPad[l] + c] = params[p++];
        if (cudaMemcpyAsync(s->ws + s->w[l], wpad.data(), wpad.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return LPP_ERR_CUDA;
        if (cudaMemcpyAsync(s->ws + s->b[l], params + p, kOut[l] * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return LPP_ERR_CUDA;
        p += kOut[l];
        if (cudaStreamSynchronize(st) != cudaSuccess) return LPP_ERR_CUDA;
    }
    AdamArgs a = adam_args(s);
    k_refresh<<<dim3(64, kLayers), 256, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return LPP_ERR_CUDA;
    return LPP_OK;
}

// Training state (checkpoint): a 32-byte header (magic, version, Adam step, FNV-1a 64-bit
// checksum of the rest, 8 reserved bytes), then per layer the FP32 master W (rows padded to
// kInPad, the device layout), its Adam moments m and v, the bias and its m and v.  The BF16
// copies are derived and rebuilt on load.
constexpr unsigned kStateMagic = 0x5350504Cu;   // "LPPS"
constexpr unsigned kStateVersion = 2u;
constexpr size_t kStateHeader = 32;

static unsigned long long fnv1a64(const unsigned char* p, size_t n) {
    unsigned long long h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

static size_t state_bytes() {
    size_t b = kStateHeader;
    for (int l = 0; l < kLayers; ++l) b += (size_t)3 * ((size_t)kOut[l] * kInPad[l] + kOut[l]) * 4;
    return b;
}

extern "C" lpp_status lpp_surrogate_state_size(lpp_surrogate_t s, size_t* bytes) {
    if (!s || !bytes) return LPP_ERR_INVALID_ARG;
    *bytes = state_bytes();
    return LPP_OK;
}

// The state's device arrays in file order: {offset, bytes} per layer.
static void state_parts(lpp_surrogate_t s, std::vector<std::pair<size_t, size_t>>& parts) {
    parts.clear();
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = (size_t)kOut[l] * kInPad[l] * 4, nb = (size_t)kOut[l] * 4;
        parts.push_back({s->w[l], nw});
        parts.push_back({s->mw[l], nw});
        parts.push_back({s->vw[l], nw});
        parts.push_back({s->b[l], nb});
        parts.push_back({s->mb[l], nb});
        parts.push_back({s->vb[l], nb});
    }
}

extern "C" lpp_status lpp_surrogate_save_state(lpp_surrogate_t s, void* host, size_t bytes, void* stream) {
    if (!s || !s->ws || !host || bytes < state_bytes()) return LPP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* p = (unsigned char*)host;
    const unsigned hdr[2] = {kStateMagic, kStateVersion};
    memcpy(p, hdr, 8);
    const long long step = s->step;
    memcpy(p + 8, &step, 8);
    memset(p + 16, 0, 16);
    size_t o = kStateHeader;
    std::vector<std::pair<size_t, size_t>> parts;
    state_parts(s, parts);
    for (const auto& q : parts) {
        if (cudaMemcpyAsync(p + o, s->ws + q.first, q.second, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return LPP_ERR_CUDA;
        o += q.second;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return LPP_ERR_CUDA;
    const unsigned long long sum = fnv1a64(p + kStateHeader, state_bytes() - kStateHeader);
    memcpy(p + 16, &sum, 8);
    return LPP_OK;
}

extern "C" lpp_status lpp_surrogate_load_state(lpp_surrogate_t s, const void* host, size_t bytes, void* stream) {
    if (!s || !s->ws || !host || bytes < state_bytes()) return LPP_ERR_INVALID_ARG;
    const unsigned char* p = (const unsigned char*)host;
    unsigned hdr[2];
    memcpy(hdr, p, 8);
    if (hdr[0] != kStateMagic || hdr[1] != kStateVersion) return LPP_ERR_INVALID_ARG;
    long long step = 0;
    memcpy(&step, p + 8, 8);
    if (step < 0) return LPP_ERR_INVALID_ARG;
    unsigned long long sum = 0;
    memcpy(&sum, p + 16, 8);
    if (sum != fnv1a64(p + kStateHeader, state_bytes() - kStateHeader)) return LPP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    size_t o = kStateHeader;
    std::vector<std::pair<size_t, size_t>> parts;
    state_parts(s, parts);
    for (const auto& q : parts) {
        if (cudaMemcpyAsync(s->ws + q.first, p + o, q.second, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return LPP_ERR_CUDA;
        o += q.second;
    }
    AdamArgs a = adam_args(s);
    k_refresh<<<dim3(64, kLayers), 256, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return LPP_ERR_CUDA;
    s->step = step;
    return LPP_OK;
}

extern "C" lpp_status lpp_surrogate_get_params(lpp_surrogate_t s, float* params, void* stream) {
    if (!s || !s->ws || !params) return LPP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<float> wpad;
    size_t p = 0;
    for (int l = 0; l < kLayers; ++l) {
        wpad.resize((size_t)kOut[l] * kInPad[l]);
        if (cudaMemcpyAsync(wpad.data(), s->ws + s->w[l], wpad.size() * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return LPP_ERR_CUDA;
        if (cudaMemcpyAsync(params + p + (size_t)kOut[l] * kIn[l], s->ws + s->b[l], kOut[l] * 4,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return LPP_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return LPP_ERR_CUDA;
        for (int r = 0; r < kOut[l]; ++r)
            for (int c = 0; c < kIn[l]; ++c) params[p++] = wpad[(size_t)r * kInPad[l] + c];
        p += kOut[l];
    }
    return LPP_OK;
}

// forward pass of m <= batch rows (inputs gathered through idx when given)
static cudaError_t forward(lpp_surrogate_t s, const float* x, const int* idx, int m, bool train, float* out_final,
                           cudaStream_t st) {
    const int B = s->batch;
    bf16* a0 = (bf16*)(s->ws + s->act[0]);
    k_input<<<(m * 16 + 255) / 256, 256, 0, st>>>(x, idx, m, a0, train ? (bf16*)(s->ws + s->actt[0]) : nullptr, B);
    for (int l = 0; l < kLayers; ++l) {
        GemmArgs g;
        memset(&g, 0, sizeof(g));
        g.A = (const bf16*)(s->ws + s->act[l]);
        g.lda = kInPad[l];
        g.B = (const bf16*)(s->ws + s->w16[l]);
        g.ldb = kInPad[l];
        g.M = m;
        g.N = kOut[l];
        g.K = kInPad[l];
        g.bias = (const float*)(s->ws + s->b[l]);
        if (l < kLayers - 1) {
            g.epi = EPI_HIDDEN;
            g.z = (float*)(s->ws + s->z[l]);
            g.ldz = kOut[l];
            g.a16 = (bf16*)(s->ws + s->act[l + 1]);
            g.ld16 = kInPad[l + 1];
            g.a16t = train ? (bf16*)(s->ws + s->actt[l + 1]) : nullptr;
            g.ld16t = B;
        } else {
            g.epi = EPI_OUT;
            g.z = out_final ? out_final : (float*)(s->ws + s->z[l]);
            g.ldz = kOut[l];
        }
        cudaError_t e = gemm(g, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

extern "C" lpp_status lpp_surrogate_infer(lpp_surrogate_t s, const float* x, int n, float* y, void* stream) {
    if (!s || !s->ws || n < 0 || (n > 0 && (!x || !y))) return LPP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    for (int r0 = 0; r0 < n; r0 += s->batch) {
        const int m = n - r0 < s->batch ? n - r0 : s->batch;
        if (forward(s, x + (size_t)r0 * kNin, nullptr, m, false, y + (size_t)r0 * kNout, st) != cudaSuccess)
            return LPP_ERR_CUDA;
    }
    return LPP_OK;
}

extern "C" lpp_status lpp_surrogate_set_map(lpp_surrogate_t s, const lpp_surrogate_map* m) {
    if (!s || !m || !m->mu || !m->sd || !m->shot) return LPP_ERR_INVALID_ARG;
    MapArgs a;
    memset(&a, 0, sizeof(a));
    for (int c = 0; c < kNin; ++c) {
        if (!m->feed[c]) continue;
        if (!(m->hi[c] > m->lo[c])) return LPP_ERR_INVALID_ARG;
        const double sc = 2.0 / (m->hi[c] - m->lo[c]);
        a.dscale[c] = sc;
        a.dshift[c] = -1.0 - m->lo[c] * sc;
        a.scale[c] = (float)a.dscale[c];
        a.shift[c] = (float)a.dshift[c];
    }
    if (m->base) {
        if (m->base_nodes < 2 || m->base_nodes > kMaxNodes) return LPP_ERR_INVALID_ARG;
        for (int d = 0; d < 2; ++d)
            if (m->base_in[d] < 0 || m->base_in[d] >= kNin || !m->feed[m->base_in[d]]) return LPP_ERR_INVALID_ARG;
        a.base = m->base;
        a.nodes = m->base_nodes;
        a.base_in[0] = m->base_in[0];
        a.base_in[1] = m->base_in[1];
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < a.nodes; ++i) a.xs[i] = -cos(pi * i / (a.nodes - 1));
        for (int i = 0; i < a.nodes; ++i) {
            double d = 1.0;
            for (int k = 0; k < a.nodes; ++k)
                if (k != i) d *= a.xs[i] - a.xs[k];
            a.cw[i] = 1.0 / d;
        }
    }
    a.mu = m->mu;
    a.sd = m->sd;
    a.shot = m->shot;
    a.ref = m->ref;
    a.sigma = m->sigma;
    lpp::eb_matrices(a.N, a.M);
    s->map = a;
    s->has_map = true;
    s->base_split = false;
    return LPP_OK;
}

extern "C" lpp_status lpp_surrogate_targets(lpp_surrogate_t s, const double* theta, const double* native, int n,
                                            float* y, void* stream) {
    if (!s || !s->has_map || n < 0 || (n > 0 && (!theta || !native || !y))) return LPP_ERR_INVALID_ARG;
    if (n == 0) return LPP_OK;
    const long long total = (long long)n * kNout;
    const int blocks = (int)((total + 255) / 256 < 65535 * 8 ? (total + 255) / 256 : 65535 * 8);
    k_targets<<<blocks, 256, 0, (cudaStream_t)stream>>>(theta, native, n, y, s->map);
    return cudaGetLastError() == cudaSuccess ? LPP_OK : LPP_ERR_CUDA;
}

extern "C" lpp_status lpp_surrogate_encode(lpp_surrogate_t s, const double* theta, int n, float* x, void* stream) {
    if (!s || !s->has_map || n < 0 || (n > 0 && (!theta || !x))) return LPP_ERR_INVALID_ARG;
    if (n == 0) return LPP_OK;
    k_encode<<<(n * kNin + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, n, x, s->map);
    return cudaGetLastError() == cudaSuccess ? LPP_OK : LPP_ERR_CUDA;
}

extern "C" lpp_status lpp_surrogate_predict(lpp_surrogate_t s, const double* theta, int n, float* out, void* stream) {
    if (!s || !s->ws || !s->has_map || n < 0 || (n > 0 && (!theta || !out))) return LPP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float* x = (float*)(s->ws + s->xin);
    if (s->map.base) {
        s->map.base_hi = (const float*)(s->ws + s->base_hi);
        s->map.base_lo = (const float*)(s->ws + s->base_lo);
        if (!s->base_split) {
            const int count = s->map.nodes * s->map.nodes * kNout;
            k_split_base<<<(count + 255) / 256, 256, 0, st>>>(s->map.base, count, (float*)(s->ws + s->base_hi),
                                                             (float*)(s->ws + s->base_lo));
            if (cudaGetLastError() != cudaSuccess) return LPP_ERR_CUDA;
            s->base_split = true;
        }
    }
    for (int r0 = 0; r0 < n; r0 += s->batch) {
        const int m = n - r0 < s->batch ? n - r0 : s->batch;
        const double* th = theta + (size_t)r0 * kNin;
        k_encode<<<(m * kNin + 255) / 256, 256, 0, st>>>(th, m, x, s->map);
        float* y = out + (size_t)r0 * kNout;
        if (forward(s, x, nullptr, m, false, y, st) != cudaSuccess) return LPP_ERR_CUDA;
        {
            int dev = 0, sms = 152;
            if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int groups = (m + kDecodeRows - 1) / kDecodeRows;
            const int blocks = groups < sms * 6 ? (groups > 0 ? groups : 1) : sms * 6;
            k_decode<<<blocks, kNout, 0, st>>>(th, m, y, y, s->map);
        }
    }
    return cudaGetLastError() == cudaSuccess ? LPP_OK : LPP_ERR_CUDA;
}

// One Adam step on the minibatch rows idx[0..batch) of (x, y); the mean squared error of the
// minibatch (before the step) is added to *loss_out (device).
static cudaError_t train_step(lpp_surrogate_t s, const float* x, const float* y, const int* idx, float lr,
                              double* loss_out, cudaStream_t st) {
    const int B = s->batch;
    cudaError_t e = forward(s, x, idx, B, true, nullptr, st);
    if (e != cudaSuccess) return e;
    int cur = 0;
    k_loss<<<(B * kNout + 255) / 256, 256, 0, st>>>((const float*)(s->ws + s->z[kLayers - 1]), y, idx, B,
                                                    (float*)(s->ws + s->g32[cur]), (bf16*)(s->ws + s->g16[cur]),
                                                    (bf16*)(s->ws + s->g16t[cur]), B, loss_out);
    for (int l = kLayers - 1; l >= 0; --l) {
        // dW_l = g^T a_l : [out x inp] = [out x B] . [inp x B]^T
        GemmArgs gw;
        memset(&gw, 0, sizeof(gw));
        gw.A = (const bf16*)(s->ws + s->g16t[cur]);
        gw.lda = B;
        gw.B = (const bf16*)(s->ws + s->actt[l]);
        gw.ldb = B;
        gw.M = kOut[l];
        gw.N = kInPad[l];
        gw.K = B;
        gw.epi = EPI_DW;
        gw.z = (float*)(s->ws + s->dw[l]);
        gw.ldz = kInPad[l];
        if ((e = gemm(gw, st)) != cudaSuccess) return e;
        k_bias_grad<<<(kOut[l] + 31) / 32, 256, 0, st>>>((const float*)(s->ws + s->g32[cur]), B, kOut[l],
                                                           (float*)(s->ws + s->db[l]));
        if (l > 0) {
            // g_{l-1} = (g_l W_l) * GELU'(z_{l-1}) : [B x inp] = [B x out] . [inp x out]^T
            GemmArgs gd;
            memset(&gd, 0, sizeof(gd));
            gd.A = (const bf16*)(s->ws + s->g16[cur]);
            gd.lda = kOut[l];
            gd.B = (const bf16*)(s->ws + s->w16t[l]);
            gd.ldb = kOut[l];
            gd.M = B;
            gd.N = kInPad[l];
            gd.K = kOut[l];
            gd.epi = EPI_DA_GELU;
            gd.zprev = (const float*)(s->ws + s->z[l - 1]);
            gd.ldzp = kOut[l - 1];
            gd.g32 = (float*)(s->ws + s->g32[1 - cur]);
            gd.ldg = kInPad[l];
            gd.a16 = (bf16*)(s->ws + s->g16[1 - cur]);
            gd.ld16 = kInPad[l];
            gd.a16t = (bf16*)(s->ws + s->g16t[1 - cur]);
            gd.ld16t = B;
            if ((e = gemm(gd, st)) != cudaSuccess) return e;
            cur = 1 - cur;
        }
    }
    s->step += 1;
    AdamArgs a = adam_args(s);
    a.lr = lr;
    a.b1 = 0.9f;
    a.b2 = 0.999f;
    a.eps = 1e-8f;
    a.bc1 = (float)(1.0 - pow(0.9, (double)s->step));
    a.bc2 = (float)(1.0 - pow(0.999, (double)s->step));
    k_adam<<<dim3(128, kLayers), 256, 0, st>>>(a);
    return cudaGetLastError();
}

extern "C" lpp_status lpp_surrogate_train(lpp_surrogate_t s, const float* x, const float* y, const int* schedule,
                                          int n_steps, float lr, double* losses, void* stream) {
    if (!s || !s->ws || !x || !y || !schedule || n_steps < 0) return LPP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (losses && cudaMemsetAsync(losses, 0, (size_t)n_steps * sizeof(double), st) != cudaSuccess) return LPP_ERR_CUDA;
    double* scratch = (double*)(s->ws + s->loss);
    for (int i = 0; i < n_steps; ++i) {
        double* lo = losses ? losses + i : scratch;
        if (train_step(s, x, y, schedule + (size_t)i * s->batch, lr, lo, st) != cudaSuccess) return LPP_ERR_CUDA;
    }
    return LPP_OK;
}

// Gradients of the loss of one minibatch without an update (for checks): host dW [out][in], db [out].
extern "C" lpp_status lpp_surrogate_gradients(lpp_surrogate_t s, const float* x, const float* y, const int* idx,
                                              float* grads, double* loss, void* stream) {
    if (!s || !s->ws || !x || !y || !idx || !grads) return LPP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long saved = s->step;
    double* lo = (double*)(s->ws + s->loss);
    if (cudaMemsetAsync(lo, 0, 8, st) != cudaSuccess) return LPP_ERR_CUDA;
    // run the step with lr = 0 so that only the gradients are formed (Adam moments are restored below)
    std::vector<char> mom;
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = (size_t)kOut[l] * kInPad[l] * 4;
        const size_t off0 = mom.size();
        mom.resize(off0 + 2 * nw + 2 * kOut[l] * 4);
        cudaMemcpyAsync(mom.data() + off0, s->ws + s->mw[l], nw, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(mom.data() + off0 + nw, s->ws + s->vw[l], nw, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(mom.data() + off0 + 2 * nw, s->ws + s->mb[l], kOut[l] * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(mom.data() + off0 + 2 * nw + kOut[l] * 4, s->ws + s->vb[l], kOut[l] * 4,
                        cudaMemcpyDeviceToHost, st);
    }
    if (train_step(s, x, y, idx, 0.0f, lo, st) != cudaSuccess) return LPP_ERR_CUDA;
    size_t p = 0, mo = 0;
    std::vector<float> dw;
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = (size_t)kOut[l] * kInPad[l];
        dw.resize(nw);
        cudaMemcpyAsync(dw.data(), s->ws + s->dw[l], nw * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(grads + p + (size_t)kOut[l] * kIn[l], s->ws + s->db[l], kOut[l] * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(s->ws + s->mw[l], mom.data() + mo, nw * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(s->ws + s->vw[l], mom.data() + mo + nw * 4, nw * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(s->ws + s->mb[l], mom.data() + mo + 2 * nw * 4, kOut[l] * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(s->ws + s->vb[l], mom.data() + mo + 2 * nw * 4 + kOut[l] * 4, kOut[l] * 4,
                        cudaMemcpyHostToDevice, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return LPP_ERR_CUDA;
        for (int r = 0; r < kOut[l]; ++r)
            for (int c = 0; c < kIn[l]; ++c) grads[p++] = dw[(size_t)r * kInPad[l] + c];
        p += kOut[l];
        mo += 2 * nw * 4 + 2 * kOut[l] * 4;
    }
    s->step = saved;
    if (loss && cudaMemcpyAsync(loss, lo, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LPP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LPP_ERR_CUDA;
    return LPP_OK;
}
