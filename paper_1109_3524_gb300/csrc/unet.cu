// U-Net of the learned warm start for the Poisson solve (not part of the
// paper): BF16 activations and weights on the tensor cores, FP32 gradients,
// master weights and Adam.  The forward 3x3 convolutions run on tcgen05 with
// the accumulator in tensor memory (k_conv_tc.cu); the 1x1 output layer, the
// backward passes and IBM_CNN_NO_TC=1 use the mma.sync m16n8k16 implicit GEMM
// below (FP32 accumulation in both).
//
// Network (NHWC): levels L, channels base*2^l.  Encoder level l: two 3x3 convs
// + ReLU, then 2x2 average pooling (not after the bottleneck).  Decoder stage
// l = L-2..0: nearest 2x upsampling, concatenation with the encoder output of
// level l, two 3x3 convs + ReLU.  Output: 1x1 conv to one channel.
//
// Every convolution is an implicit GEMM on one tiled kernel:
//   forward      C[pixel, cout] = sum_k A[pixel, (ky,kx,cin)] W[(ky,kx,cin), cout]
//   backward x   C[pixel, cin]  = sum_k G[pixel+shift, cout] W[flip(ky,kx), cin, cout]
//   backward W   C[(ky,kx,cin)|bias, cout] = sum_pixels A[pixel+shift, cin] G[pixel, cout]
//                (split over pixel chunks, the slices summed in order)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ibm.h"
#include "conv_tc.h"
#include "device.cuh"

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 64, BN = 32, BK = 32, GT = 128;   // GEMM tile and threads
constexpr int SK = BK + 8;                            // padded smem row (bf16)

union Pack8 {      // 8 BF16 values moved as one 16-byte word
    uint4 u;
    bf16 h[8];
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct Geo {
    int B, H, W;      // spatial size of the layer (same padding)
    int Cin, Cout, ks;
    int K;            // ks*ks*Cin
};

// ---- loaders: 8 consecutive K entries of one row (A) / column (B) -----------------
// A of the forward conv: input pixels shifted by (ky,kx), channels ci..ci+7
struct LoadFwdA {
    const bf16* x;
    Geo g;
    __device__ __forceinline__ void load8(int m, int k, bf16* dst) const {
        const int HW = g.H * g.W;
        if (m >= g.B * HW || k >= g.K) {
            for (int i = 0; i < 8; ++i) dst[i] = __float2bfloat16(0.f);
            return;
        }
        const int b = m / HW, r = m - b * HW, y = r / g.W, xx = r - y * g.W;
        if ((g.Cin & 7) == 0) {
            const int kk = k / g.Cin, ci = k - kk * g.Cin;
            const int ky = kk / g.ks, kx = kk - ky * g.ks, p = g.ks / 2;
            const int yy = y + ky - p, xs = xx + kx - p;
            if (yy < 0 || yy >= g.H || xs < 0 || xs >= g.W) {
                for (int i = 0; i < 8; ++i) dst[i] = __float2bfloat16(0.f);
                return;
            }
            *reinterpret_cast<uint4*>(dst) =
                *reinterpret_cast<const uint4*>(x + ((long long)(b * g.H + yy) * g.W + xs) * g.Cin + ci);
            return;
        }
        for (int i = 0; i < 8; ++i) {
            const int kq = k + i;
            bf16 v = __float2bfloat16(0.f);
            if (kq < g.K) {
                const int kk = kq / g.Cin, ci = kq - kk * g.Cin;
                const int ky = kk / g.ks, kx = kk - ky * g.ks, p = g.ks / 2;
                const int yy = y + ky - p, xs = xx + kx - p;
                if (yy >= 0 && yy < g.H && xs >= 0 && xs < g.W)
                    v = x[((long long)(b * g.H + yy) * g.W + xs) * g.Cin + ci];
            }
            dst[i] = v;
        }
    }
};
// B of the forward conv: Wt[cout][k] (k contiguous)
struct LoadFwdB {
    const bf16* wt;
    Geo g;
    __device__ __forceinline__ void load8(int n, int k, bf16* dst) const {
        if (n >= g.Cout || k >= g.K) {
            for (int i = 0; i < 8; ++i) dst[i] = __float2bfloat16(0.f);
            return;
        }
        if ((g.K & 7) == 0) {
            *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(wt + (long long)n * g.K + k);
            return;
        }
        for (int i = 0; i < 8; ++i) dst[i] = (k + i < g.K) ? wt[(long long)n * g.K + k + i] : __float2bfloat16(0.f);
    }
};
// A of backward-data: gradient (pre-activation) at pixel+shift, channels of cout;
// k = (ky, kx, cout)
struct LoadBwdA {
    const bf16* gz;
    Geo g;
    __device__ __forceinline__ void load8(int m, int k, bf16* dst) const {
        const int HW = g.H * g.W, Kb = g.ks * g.ks * g.Cout;
        if (m >= g.B * HW || k >= Kb) {
            for (int i = 0; i < 8; ++i) dst[i] = __float2bfloat16(0.f);
            return;
        }
        const int b = m / HW, r = m - b * HW, y = r / g.W, xx = r - y * g.W, p = g.ks / 2;
        for (int i = 0; i < 8; ++i) {
            const int kq = k + i;
            bf16 v = __float2bfloat16(0.f);
            if (kq < Kb) {
                const int kk = kq / g.Cout, co = kq - kk * g.Cout;
                const int ky = kk / g.ks, kx = kk - ky * g.ks;
                const int yy = y + ky - p, xs = xx + kx - p;
                if (yy >= 0 && yy < g.H && xs >= 0 && xs < g.W)
                    v = gz[((long long)(b * g.H + yy) * g.W + xs) * g.Cout + co];
            }
            dst[i] = v;
        }
    }
};
// B of backward-data: W[flip(ky,kx), ci = n, co] from Wt[co][(ky,kx,ci)]
struct LoadBwdB {
    const bf16* wt;
    Geo g;
    __device__ __forceinline__ void load8(int n, int k, bf16* dst) const {
        const int Kb = g.ks * g.ks * g.Cout;
        for (int i = 0; i < 8; ++i) {
            const int kq = k + i;
            bf16 v = __float2bfloat16(0.f);
            if (n < g.Cin && kq < Kb) {
                const int kk = kq / g.Cout, co = kq - kk * g.Cout;
                const int ky = kk / g.ks, kx = kk - ky * g.ks;
                const int kf = ((g.ks - 1 - ky) * g.ks + (g.ks - 1 - kx)) * g.Cin + n;
                v = wt[(long long)co * g.K + kf];
            }
            dst[i] = v;
        }
    }
};
// A of backward-weight: row m = (ky,kx,ci) or the bias row (m = K), column = pixel
struct LoadWgtA {
    const bf16* x;
    Geo g;
    __device__ __forceinline__ void load8(int m, int k, bf16* dst) const {
        const int HW = g.H * g.W, P = g.B * HW;
        if (m > g.K) {
            for (int i = 0; i < 8; ++i) dst[i] = __float2bfloat16(0.f);
            return;
        }
        if (m == g.K) {
            for (int i = 0; i < 8; ++i) dst[i] = __float2bfloat16(k + i < P ? 1.f : 0.f);
            return;
        }
        const int kk = m / g.Cin, ci = m - kk * g.Cin;
        const int ky = kk / g.ks, kx = kk - ky * g.ks, p = g.ks / 2;
        for (int i = 0; i < 8; ++i) {
            const int pix = k + i;
            bf16 v = __float2bfloat16(0.f);
            if (pix < P) {
                const int b = pix / HW, r = pix - b * HW, y = r / g.W, xx = r - y * g.W;
                const int yy = y + ky - p, xs = xx + kx - p;
                if (yy >= 0 && yy < g.H && xs >= 0 && xs < g.W)
                    v = x[((long long)(b * g.H + yy) * g.W + xs) * g.Cin + ci];
            }
            dst[i] = v;
        }
    }
};
// B of backward-weight: gradient at pixel k (rows), channel n
struct LoadWgtB {
    const bf16* gz;
    Geo g;
    __device__ __forceinline__ void load8(int n, int k, bf16* dst) const {
        const int P = g.B * g.H * g.W;
        for (int i = 0; i < 8; ++i)
            dst[i] = (n < g.Cout && k + i < P) ? gz[(long long)(k + i) * g.Cout + n] : __float2bfloat16(0.f);
    }
};

// ---- epilogues -------------------------------------------------------------------------
struct EpiFwd {            // out = act(acc + bias): BF16 (hidden) or FP32 (output layer)
    bf16* y16;
    float* y32;
    const float* bias;
    int N, M, relu;
    __device__ __forceinline__ void operator()(int m, int n, float v) const {
        if (m >= M || n >= N) return;
        v += bias[n];
        if (relu) v = fmaxf(v, 0.f);
        if (y16) y16[(long long)m * N + n] = __float2bfloat16(v);
        else y32[(long long)m * N + n] = v;
    }
};
struct EpiStore32 {        // plain FP32 store
    float* y;
    int N, M;
    __device__ __forceinline__ void operator()(int m, int n, float v) const {
        if (m < M && n < N) y[(long long)m * N + n] = v;
    }
};
struct EpiSlice32 {        // split-K: slice blockIdx.z of the partial products
    float* ws;
    int N, M;
    __device__ __forceinline__ void operator()(int m, int n, float v) const {
        if (m < M && n < N) ws[(long long)blockIdx.z * M * N + (long long)m * N + n] = v;
    }
};

// y += the sum over the sz slices of ws, in slice order (deterministic)
__global__ void k_slice_sum(long long mn, int sz, const float* __restrict__ ws, float* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < mn; i += (long long)gridDim.x * blockDim.x) {
        float a = y[i];
        for (int z = 0; z < sz; ++z) a += ws[(long long)z * mn + i];
        y[i] = a;
    }
}

// C[M x N] (+)= A[M x K] B[K x N] over K range [kb, ke) of this block's z-slice
template <class LA, class LB, class EP>
__global__ void __launch_bounds__(GT) k_gemm(int M, int N, int K, int kchunk, LA la, LB lb, EP ep) {
    __shared__ __align__(16) bf16 As[BM][SK];
    __shared__ __align__(16) bf16 Bs[BN][SK];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += BK) {
        // A: 64 x 32 = 256 chunks of 8; B: 32 x 32 = 128 chunks of 8
        for (int c = tid; c < BM * (BK / 8); c += GT) {
            const int mm = c / (BK / 8), kk = (c % (BK / 8)) * 8;
            Pack8 t;
            if (k0 + kk < ke) la.load8(m0 + mm, k0 + kk, t.h);
            else
                for (int i = 0; i < 8; ++i) t.h[i] = __float2bfloat16(0.f);
            // entries beyond this slice's K end belong to another slice
            for (int i = 0; i < 8; ++i)
                if (k0 + kk + i >= ke) t.h[i] = __float2bfloat16(0.f);
            *reinterpret_cast<uint4*>(&As[mm][kk]) = t.u;
        }
        for (int c = tid; c < BN * (BK / 8); c += GT) {
            const int nn = c / (BK / 8), kk = (c % (BK / 8)) * 8;
            Pack8 t;
            if (k0 + kk < ke) lb.load8(n0 + nn, k0 + kk, t.h);
            else
                for (int i = 0; i < 8; ++i) t.h[i] = __float2bfloat16(0.f);
            for (int i = 0; i < 8; ++i)
                if (k0 + kk + i >= ke) t.h[i] = __float2bfloat16(0.f);
            *reinterpret_cast<uint4*>(&Bs[nn][kk]) = t.u;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            const int r0 = warp * 16 + gq;
            const uint32_t a0 = *reinterpret_cast<const uint32_t*>(&As[r0][ks + 2 * tq]);
            const uint32_t a1 = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][ks + 2 * tq]);
            const uint32_t a2 = *reinterpret_cast<const uint32_t*>(&As[r0][ks + 2 * tq + 8]);
            const uint32_t a3 = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][ks + 2 * tq + 8]);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[nt * 8 + gq][ks + 2 * tq]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[nt * 8 + gq][ks + 2 * tq + 8]);
                mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
            }
        }
        __syncthreads();
    }
    const int r0 = m0 + warp * 16 + gq;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int c0 = n0 + nt * 8 + 2 * tq;
        ep(r0, c0, acc[nt][0]);
        ep(r0, c0 + 1, acc[nt][1]);
        ep(r0 + 8, c0, acc[nt][2]);
        ep(r0 + 8, c0 + 1, acc[nt][3]);
    }
}

// returns the number of K slices launched
template <class LA, class LB, class EP>
int gemm(int M, int N, int K, int splits, LA la, LB lb, EP ep, cudaStream_t st) {
    int kchunk = (K + splits - 1) / splits;
    kchunk = ((kchunk + BK - 1) / BK) * BK;
    const int sz = std::max(1, (K + kchunk - 1) / kchunk);
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, sz);
    k_gemm<LA, LB, EP><<<grid, GT, 0, st>>>(M, N, K, kchunk, la, lb, ep);
    return sz;
}

// ---- elementwise / layout kernels ----------------------------------------------------------
__global__ void k_to_bf16(long long n, const float* __restrict__ x, bf16* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}
// 3-channel NHWC input padded to 8 channels (16-byte pixels)
__global__ void k_pad8(long long P, const bf16* __restrict__ x, bf16* __restrict__ y) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        Pack8 v;
        v.u = make_uint4(0u, 0u, 0u, 0u);
        v.h[0] = x[3 * p];
        v.h[1] = x[3 * p + 1];
        v.h[2] = x[3 * p + 2];
        reinterpret_cast<uint4*>(y)[p] = v.u;
    }
}
// 2x2 average pooling, NHWC BF16
__global__ void k_pool(int B, int H, int W, int C, const bf16* __restrict__ x, bf16* __restrict__ y) {
    const int Ho = H / 2, Wo = W / 2;
    const long long n = (long long)B * Ho * Wo * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        long long r = i / C;
        const int xo = int(r % Wo);
        r /= Wo;
        const int yo = int(r % Ho);
        const int b = int(r / Ho);
        const long long base = ((long long)(b * H + 2 * yo) * W + 2 * xo) * C + c;
        const float s = __bfloat162float(x[base]) + __bfloat162float(x[base + C]) +
                        __bfloat162float(x[base + (long long)W * C]) + __bfloat162float(x[base + (long long)W * C + C]);
        y[i] = __float2bfloat16(0.25f * s);
    }
}
// concat(up2(a), s): a (B, H/2, W/2, Ca), s (B, H, W, Cs) -> y (B, H, W, Ca+Cs)
__global__ void k_upcat(int B, int H, int W, int Ca, int Cs, const bf16* __restrict__ a, const bf16* __restrict__ s,
                        bf16* __restrict__ y) {
    const int C = Ca + Cs;
    const long long n = (long long)B * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long pix = i / C;
        const int xx = int(pix % W);
        const long long r = pix / W;
        const int yy = int(r % H);
        const int b = int(r / H);
        y[i] = (c < Ca) ? a[((long long)(b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * Ca + c]
                        : s[pix * Cs + (c - Ca)];
    }
}
// gradient through ReLU: gz = g * (act > 0), BF16 out
__global__ void k_relu_bwd(long long n, const float* __restrict__ g, const bf16* __restrict__ act, bf16* __restrict__ gz) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        gz[i] = __float2bfloat16(__bfloat162float(act[i]) > 0.f ? g[i] : 0.f);
}
// split the gradient of concat(up2(a), s): ga (B,H/2,W/2,Ca) = sum over 2x2; gs += rest
__global__ void k_upcat_bwd(int B, int H, int W, int Ca, int Cs, const float* __restrict__ gy, float* __restrict__ ga,
                            float* __restrict__ gs) {
    const int C = Ca + Cs, Ho = H / 2, Wo = W / 2;
    const long long na = (long long)B * Ho * Wo * Ca, ns = (long long)B * H * W * Cs;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < na + ns; i += (long long)gridDim.x * blockDim.x) {
        if (i < na) {
            const int c = int(i % Ca);
            long long r = i / Ca;
            const int xo = int(r % Wo);
            r /= Wo;
            const int yo = int(r % Ho);
            const int b = int(r / Ho);
            const long long p = (long long)(b * H + 2 * yo) * W + 2 * xo;
            ga[i] = gy[p * C + c] + gy[(p + 1) * C + c] + gy[(p + W) * C + c] + gy[(p + W + 1) * C + c];
        } else {
            const long long j = i - na;
            const int c = int(j % Cs);
            const long long pix = j / Cs;
            gs[j] += gy[pix * C + Ca + c];
        }
    }
}
// gradient of 2x2 average pooling into an existing gradient: gx += 0.25 gy (upsampled)
__global__ void k_pool_bwd_add(int B, int H, int W, int C, const float* __restrict__ gy, float* __restrict__ gx) {
    const long long n = (long long)B * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long pix = i / C;
        const int xx = int(pix % W);
        const long long r = pix / W;
        const int yy = int(r % H);
        const int b = int(r / H);
        gx[i] += 0.25f * gy[((long long)(b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c];
    }
}
// MSE: loss partials and gradient 2 (out - t) / n
// per-block sums of NV values into part[k * gridDim.x + block] (256 threads)
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* part) {
    __shared__ double sh[NV][8];
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][threadIdx.x >> 5] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double a = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) a += sh[threadIdx.x][w];
        part[threadIdx.x * gridDim.x + blockIdx.x] = a;
    }
}
// acc[k] = sum of the nb partials of value k, in block order (one block)
__global__ void k_part_sum(int nv, int nb, const double* __restrict__ part, double* __restrict__ acc) {
    __shared__ double sh[8];
    for (int k = 0; k < nv; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[k * nb + b];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[w];
            acc[k] = t;
        }
        __syncthreads();
    }
}
// MSE: loss partials and gradient 2 (out - t) / n
__global__ void k_mse(long long n, const float* __restrict__ out, const float* __restrict__ t, float* __restrict__ g,
                      double* __restrict__ part) {
    double s[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - t[i];
        g[i] = 2.f * d / float(n);
        s[0] += double(d) * d;
    }
    block_partials<1>(s, part);
}
// Adam on FP32 master parameters (weights [K][Cout] then bias), BF16 transposed copy
__global__ void k_adam(int K, int Cout, float* __restrict__ w, float* __restrict__ b, float* __restrict__ m,
                       float* __restrict__ v, const float* __restrict__ g, bf16* __restrict__ wt,
                       bf16* __restrict__ wtc, int cin, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int n = (K + 1) * Cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float step = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        const int r = i / Cout, co = i - r * Cout;
        if (r < K) {
            const float nw = w[i] - step;
            w[i] = nw;
            wt[(long long)co * K + r] = __float2bfloat16(nw);
            if (wtc) {   // [tap][cin block][cout][8]
                const int t = r / cin, ci = r - t * cin, cbt = (cin + 15) / 16 * 2;
                wtc[((long long)(t * cbt + ci / 8) * Cout + co) * 8 + (ci & 7)] = __float2bfloat16(nw);
            }
        } else {
            b[co] -= step;
        }
    }
}
// BF16 copies of the master weights: transposed [cout][K] and, for the
// tcgen05 convolution, [tap][cin block of 8][cout][8] (channels >= cin stay 0)
__global__ void k_wt(int K, int Cout, int cin, const float* __restrict__ w, bf16* __restrict__ wt,
                     bf16* __restrict__ wtc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * Cout; i += gridDim.x * blockDim.x) {
        const int r = i / Cout, co = i - r * Cout;
        wt[(long long)co * K + r] = __float2bfloat16(w[i]);
        if (wtc) {
            const int t = r / cin, ci = r - t * cin, cbt = (cin + 15) / 16 * 2;
            wtc[((long long)(t * cbt + ci / 8) * Cout + co) * 8 + (ci & 7)] = __float2bfloat16(w[i]);
        }
    }
}

// ---- standardised inputs from solver fields ----------------------------------------------
// sums over the pressure cells: [d.d, r.r, a.a] with d = phi_n - phi_nm1 and
// a = 2 phi_n - phi_nm1 (the extrapolated warm start), r its residual
__global__ void k_in_sums(long long nc, const double* __restrict__ pn, const double* __restrict__ pm,
                          const double* __restrict__ bb, double* __restrict__ part) {
    double s[3] = {0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x) {
        const double d = pn[i] - pm[i];
        const double a = pn[i] + d;
        s[0] += d * d;
        s[1] += bb[i] * bb[i];
        s[2] += a * a;
    }
    block_partials<3>(s, part);
}
// crops of the three channels [d/s_d, r/s_r, a/s_a] and of the target
// (phi_np1 - a)/s_d, d = phi_n - phi_nm1, a = phi_n + d; crops (x0, y0)
__global__ void k_in_crops(int nx, int ny, long long nc, const double* __restrict__ pn, const double* __restrict__ pm,
                           const double* __restrict__ bb, const double* __restrict__ pp, const double* __restrict__ acc,
                           int ncrop, const int* __restrict__ xy, int ch, int cw, float* __restrict__ in,
                           float* __restrict__ tgt) {
    const double sd = sqrt(acc[0] / double(nc)) + 1e-300, sb = sqrt(acc[1] / double(nc)) + 1e-300,
                 sp = sqrt(acc[2] / double(nc)) + 1e-300;
    const long long n = (long long)ncrop * ch * cw;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i / ((long long)ch * cw));
        const long long r = i - (long long)c * ch * cw;
        const int y = int(r / cw), x = int(r - (long long)y * cw);
        const long long k = (long long)(xy[2 * c + 1] + y) * nx + (xy[2 * c] + x);
        const double d = pn[k] - pm[k];
        const double a = pn[k] + d;
        in[3 * i] = float(d / sd);
        in[3 * i + 1] = float(bb[k] / sb);
        in[3 * i + 2] = float(a / sp);
        if (tgt) tgt[i] = float((pp[k] - a) / sd);
    }
}
// warm start: lambda0 = 2 lambda^n - lambda^{n-1} + s_d * out (pressure part),
// extrapolation only on the force part; lambda^{n-1} <- lambda^n
__global__ void k_cnn_apply(long long nc, long long nl, double* __restrict__ lam, double* __restrict__ prev,
                            const float* __restrict__ out, const double* __restrict__ acc) {
    const double sd = sqrt(acc[0] / double(nc));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nl; i += (long long)gridDim.x * blockDim.x) {
        const double t = lam[i];
        double g = 2.0 * t - prev[i];
        if (i < nc) g += sd * double(out[i]);
        lam[i] = g;
        prev[i] = t;
    }
}

// the same with the correction confined to a window of w x h cells at (x0, y0)
__global__ void k_cnn_apply_win(long long nc, long long nl, int nx, int x0, int y0, int w, int h,
                                double* __restrict__ lam, double* __restrict__ prev, const float* __restrict__ out,
                                const double* __restrict__ acc) {
    const double sd = sqrt(acc[0] / double(nc));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nl; i += (long long)gridDim.x * blockDim.x) {
        const double t = lam[i];
        double g = 2.0 * t - prev[i];
        if (i < nc) {
            const int x = int(i % nx) - x0, y = int(i / nx) - y0;
            if (x >= 0 && x < w && y >= 0 && y < h) g += sd * double(out[(long long)y * w + x]);
        }
        lam[i] = g;
        prev[i] = t;
    }
}

// out = 2 lam - prev (the extrapolated guess, without touching lam, prev)
__global__ void k_extrap_to(long long n, const double* __restrict__ lam, const double* __restrict__ prev,
                            double* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = 2.0 * lam[i] - prev[i];
}

inline int grid1(long long n) { return int(std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096))); }
constexpr int kWgtSplits = 64;   // most K slices of a weight-gradient GEMM

}  // namespace

// =====================================================================================
struct ibm_cnn {
    int base = 16, levels = 4;
    long long max_pix = 0;
    struct Layer {
        int cin, cout, ks, K;
        size_t w_off, b_off;        // in the flat parameter vector
        float *w = nullptr, *b = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // FP32 master, Adam, grad
        bf16* wt = nullptr;         // BF16 [cout][K]
        bf16* wtc = nullptr;        // BF16 [tap][cin block][cout][8] (tcgen05 convolutions)
        bool tc = false;            // forward on tcgen05
        int ck = 0;                 // input channels per staged chunk of the tcgen05 convolution
    };
    std::vector<Layer> L;
    long long nparam = 0;
    int adam_t = 0;
    // activations (BF16): per conv its output; per decoder stage the concat input;
    // pooled tensors; gradient scratch (FP32) sized for the largest tensor
    std::vector<bf16*> act;         // output of conv i
    std::vector<bf16*> cat;         // decoder concat inputs
    std::vector<bf16*> pooled;      // pooled encoder outputs
    bf16* x16 = nullptr;            // network input BF16
    bf16* x16p = nullptr;           // the same, 8 channels (zero-padded) for the tcgen05 first layer
    float* out32 = nullptr;         // network output FP32
    float *g0 = nullptr, *g1 = nullptr, *gcat = nullptr;   // FP32 gradient buffers
    std::vector<float*> gskip;      // accumulated gradients of the skip tensors
    bf16* gz = nullptr;             // BF16 pre-activation gradient
    float* gout = nullptr;          // loss gradient
    double* dacc = nullptr;         // small FP64 accumulators
    double* dpart = nullptr;        // per-block partial sums (3 x 4096)
    float* gws = nullptr;           // K slices of a weight gradient (kWgtSplits x max (K + 1) cout)
    float* fin = nullptr;           // standardised input (FP32) and target for inference/prepare
    float* ftgt = nullptr;
    int* dxy = nullptr;
    int* tc_err = nullptr;          // set by a tcgen05 convolution whose barrier wait gave up
    bool use_tc = true;             // forward 3x3 convolutions on tcgen05
    int win[4] = {0, 0, 0, 0};      // inference window x0, y0, w, h of the warm start (w = 0: whole grid)
    size_t ws_bytes = 0;
    char* ws = nullptr;
    cudaStream_t st = nullptr;
    bool bound = false;
    std::string err;
};

namespace ibm {
int cnn_tc_check(ibm_cnn* c, std::string* err);
}

namespace {

struct CnnCarver {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += std::max<size_t>(n, 1) * sizeof(T);
        return p;
    }
};

void cnn_specs(ibm_cnn* c) {
    c->L.clear();
    std::vector<int> ch(c->levels);
    for (int l = 0; l < c->levels; ++l) ch[l] = c->base << l;
    int cin = 3;
    auto add = [&](int ci, int co, int ks) {
        ibm_cnn::Layer ly;
        ly.cin = ci;
        ly.cout = co;
        ly.ks = ks;
        ly.K = ks * ks * ci;
        c->L.push_back(ly);
    };
    for (int l = 0; l < c->levels; ++l) {
        add(cin, ch[l], 3);
        add(ch[l], ch[l], 3);
        cin = ch[l];
    }
    for (int l = c->levels - 2; l >= 0; --l) {
        add(cin + ch[l], ch[l], 3);
        add(ch[l], ch[l], 3);
        cin = ch[l];
    }
    add(cin, 1, 1);
    size_t o = 0;
    for (auto& ly : c->L) {
        ly.w_off = o;
        o += size_t(ly.K) * ly.cout;
        ly.b_off = o;
        o += ly.cout;
    }
    c->nparam = (long long)o;
}

// spatial size (relative to the input) of conv i's output: encoder level l convs at
// 1/2^l, decoder convs at the stage's level, output conv at full size
int conv_level(const ibm_cnn* c, int i) {
    const int ne = 2 * c->levels;
    if (i < ne) return i / 2;
    if (i < int(c->L.size()) - 1) return (c->levels - 2) - (i - ne) / 2;
    return 0;
}

size_t cnn_layout(ibm_cnn* c, CnnCarver& cv) {
    const long long P = c->max_pix;
    for (auto& ly : c->L) {
        const size_t nw = size_t(ly.K) * ly.cout;
        ly.w = cv.take<float>(nw);
        ly.b = cv.take<float>(ly.cout);
        ly.m = cv.take<float>(nw + ly.cout);
        ly.v = cv.take<float>(nw + ly.cout);
        ly.g = cv.take<float>(nw + ly.cout);
        ly.wt = cv.take<bf16>(nw);
        ly.wtc = nullptr;
        ly.tc = c->use_tc && ly.ks == 3 && ibm::conv_tc_shape_ok(ly.cin, ly.cout) && (ly.cin % 8 == 0 || ly.cin < 8);
        if (ly.tc) {
            ly.wtc = cv.take<bf16>(size_t(9) * ibm::conv_tc_cinp(ly.cin) * ly.cout);
            ly.ck = ibm::conv_tc_chunk(ly.cin, ly.cout, 100 * 1024);
        }
    }
    c->act.assign(c->L.size(), nullptr);
    for (size_t i = 0; i < c->L.size() - 1; ++i) {
        const int lv = conv_level(c, int(i));
        c->act[i] = cv.take<bf16>(size_t(P >> (2 * lv)) * c->L[i].cout);
    }
    c->cat.assign(c->levels, nullptr);
    c->pooled.assign(c->levels, nullptr);
    c->gskip.assign(c->levels, nullptr);
    size_t maxe = size_t(P) * 3;
    for (size_t i = 0; i < c->L.size(); ++i) {
        const auto& ly = c->L[i];
        maxe = std::max(maxe, size_t(P >> (2 * conv_level(c, int(i)))) * std::max(ly.cin, ly.cout));
    }
    for (int l = 0; l < c->levels - 1; ++l) {
        const int chl = c->base << l;
        const int chn = c->base << (l + 1);
        c->cat[l] = cv.take<bf16>(size_t(P >> (2 * l)) * (chn + chl));
        c->pooled[l + 1] = cv.take<bf16>(size_t(P >> (2 * (l + 1))) * chl);
        c->gskip[l] = cv.take<float>(size_t(P >> (2 * l)) * chl);
    }
    c->x16 = cv.take<bf16>(size_t(P) * 3);
    // (the sizing pass runs with a null base: test the flag, not the pointer)
    c->x16p = c->L[0].tc ? cv.take<bf16>(size_t(P) * 8) : nullptr;
    c->out32 = cv.take<float>(size_t(P));
    c->g0 = cv.take<float>(maxe);
    c->g1 = cv.take<float>(maxe);
    c->gcat = cv.take<float>(maxe);
    c->gz = cv.take<bf16>(maxe);
    c->gout = cv.take<float>(size_t(P));
    c->dacc = cv.take<double>(8);
    c->dpart = cv.take<double>(3 * 4096);
    size_t maxkc = 0;
    for (const auto& ly : c->L) maxkc = std::max(maxkc, (size_t(ly.K) + 1) * ly.cout);
    c->gws = cv.take<float>(size_t(kWgtSplits) * maxkc);
    c->fin = cv.take<float>(size_t(P) * 3);
    c->ftgt = cv.take<float>(size_t(P));
    c->dxy = cv.take<int>(4096);
    c->tc_err = cv.take<int>(1);
    return cv.off;
}

int cfail(ibm_cnn* c, int code, const std::string& m) {
    c->err = m;
    return code;
}
#define CCUDA(call)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return cfail(c, IBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

Geo geo_of(const ibm_cnn* c, int i, int B, int H, int W) {
    const int lv = conv_level(c, i);
    const auto& ly = c->L[i];
    return Geo{B, H >> lv, W >> lv, ly.cin, ly.cout, ly.ks, ly.K};
}

// input tensor of conv i during the forward pass
const bf16* conv_input(const ibm_cnn* c, int i) {
    const int ne = 2 * c->levels, nl = int(c->L.size());
    if (i == 0) return c->x16;
    if (i < ne) {
        if (i % 2 == 1) return c->act[i - 1];
        return c->pooled[i / 2];          // first conv of encoder level i/2
    }
    if (i < nl - 1) {
        const int st = (i - ne) / 2, lv = (c->levels - 2) - st;
        return (i - ne) % 2 == 0 ? c->cat[lv] : c->act[i - 1];
    }
    return c->act[i - 1];
}

// ev (nullable): two events per convolution, recorded around its launch
void run_forward(ibm_cnn* c, int B, int H, int W, cudaEvent_t* ev = nullptr) {
    const int ne = 2 * c->levels, nl = int(c->L.size());
    const long long P = (long long)B * H * W;
    for (int i = 0; i < nl; ++i) {
        // producers of this conv's input
        if (i < ne && i % 2 == 0 && i > 0) {
            const int lv = i / 2;   // pool encoder output of level lv-1
            const int Hs = H >> (lv - 1), Ws = W >> (lv - 1);
            const long long n = (long long)B * (Hs / 2) * (Ws / 2) * (c->base << (lv - 1));
            k_pool<<<grid1(n), 256, 0, c->st>>>(B, Hs, Ws, c->base << (lv - 1), c->act[i - 1], c->pooled[lv]);
        }
        if (i >= ne && i < nl - 1 && (i - ne) % 2 == 0) {
            const int lv = (c->levels - 2) - (i - ne) / 2;
            const int Hs = H >> lv, Ws = W >> lv;
            const int Ca = c->L[i - 1].cout, Cs = c->base << lv;
            const long long n = (long long)B * Hs * Ws * (Ca + Cs);
            k_upcat<<<grid1(n), 256, 0, c->st>>>(B, Hs, Ws, Ca, Cs, c->act[i - 1], c->act[2 * lv + 1], c->cat[lv]);
        }
        const Geo g = geo_of(c, i, B, H, W);
        const auto& ly = c->L[i];
        const int M = g.B * g.H * g.W;
        if (ev) cudaEventRecord(ev[2 * i], c->st);
        if (ly.tc && i < nl - 1) {
            const bool pad = (ly.cin & 7) != 0;   // the network input: its 8-channel copy
            if (pad) k_pad8<<<grid1(M), 256, 0, c->st>>>(M, conv_input(c, i), c->x16p);
            const int cin = pad ? 8 : ly.cin;
            // fewer tiles than two per SM: one CTA per SM, so a larger chunk
            // (fewer serial load-and-multiply rounds)
            const long long tiles = (long long)g.B * ((g.W + 7) / 8) * ((g.H + 15) / 16);
            const int ck = tiles < 2 * 152 ? ibm::conv_tc_chunk(cin, ly.cout, 200 * 1024) : ly.ck;
            const ibm::ConvTcArgs a{pad ? c->x16p : conv_input(c, i), ly.wtc, ly.b, c->act[i], g.B, g.H, g.W,
                                    cin, ibm::conv_tc_cinp(cin), ly.cout, ck, 1, c->tc_err};
            ibm::launch_conv3x3_tc(a, ibm::conv_tc_smem(ck, ly.cout), c->st);
        } else {
            EpiFwd ep{i < nl - 1 ? c->act[i] : nullptr, i < nl - 1 ? nullptr : c->out32, ly.b, ly.cout, M,
                      i < nl - 1};
            gemm(M, ly.cout, ly.K, 1, LoadFwdA{conv_input(c, i), g}, LoadFwdB{ly.wt, g}, ep, c->st);
        }
        if (ev) cudaEventRecord(ev[2 * i + 1], c->st);
    }
    (void)P;
}

// backward pass from the loss gradient c->gout; accumulates layer gradients
void run_backward(ibm_cnn* c, int B, int H, int W) {
    const int ne = 2 * c->levels, nl = int(c->L.size());
    for (int l = 0; l < c->levels - 1; ++l) {
        const long long n = (long long)B * (H >> l) * (W >> l) * (c->base << l);
        cudaMemsetAsync(c->gskip[l], 0, n * sizeof(float), c->st);
    }
    // gradient w.r.t. the current conv's output (FP32), starting at the output layer
    float* gcur = c->gout;
    for (int i = nl - 1; i >= 0; --i) {
        const Geo g = geo_of(c, i, B, H, W);
        const auto& ly = c->L[i];
        const long long M = (long long)g.B * g.H * g.W;
        const bf16* gz;
        if (i == nl - 1) {
            // linear output layer: pre-activation gradient = gout
            k_to_bf16<<<grid1(M), 256, 0, c->st>>>(M, gcur, c->gz);
        } else {
            k_relu_bwd<<<grid1(M * ly.cout), 256, 0, c->st>>>(M * ly.cout, gcur, c->act[i], c->gz);
        }
        gz = c->gz;
        // weight and bias gradient (split over pixel chunks, slices summed in
        // order afterwards: the same gradient on every run)
        const int splits = int(std::max<long long>(1, std::min<long long>(kWgtSplits, M / 4096)));
        const int sz = gemm(ly.K + 1, ly.cout, int(M), splits, LoadWgtA{conv_input(c, i), g}, LoadWgtB{gz, g},
                            EpiSlice32{c->gws, ly.cout, ly.K + 1}, c->st);
        const long long mn = (long long)(ly.K + 1) * ly.cout;
        k_slice_sum<<<grid1(mn), 256, 0, c->st>>>(mn, sz, c->gws, ly.g);
        if (i == 0) break;
        // input gradient
        float* gin = (gcur == c->g0) ? c->g1 : c->g0;
        const bool dec_first = (i >= ne && i < nl - 1 && (i - ne) % 2 == 0);
        float* gdst = dec_first ? c->gcat : gin;
        gemm(int(M), ly.cin, ly.ks * ly.ks * ly.cout, 1, LoadBwdA{gz, g}, LoadBwdB{ly.wt, g},
             EpiStore32{gdst, ly.cin, int(M)}, c->st);
        if (dec_first) {
            // split concat(up(prev), skip)
            const int lv = (c->levels - 2) - (i - ne) / 2;
            const int Ca = c->L[i - 1].cout, Cs = c->base << lv;
            const long long nt = (long long)B * (H >> (lv + 1)) * (W >> (lv + 1)) * Ca + (long long)B * (H >> lv) * (W >> lv) * Cs;
            k_upcat_bwd<<<grid1(nt), 256, 0, c->st>>>(B, H >> lv, W >> lv, Ca, Cs, c->gcat, gin, c->gskip[lv]);
        } else if (i < ne && i % 2 == 0) {
            // first conv of encoder level lv = i/2: its input is the pooled output of level lv-1
            const int lv = i / 2;
            const int Hs = H >> (lv - 1), Ws = W >> (lv - 1), C = c->base << (lv - 1);
            // gradient of level lv-1's output = skip gradient + pooled-path gradient
            k_pool_bwd_add<<<grid1((long long)B * Hs * Ws * C), 256, 0, c->st>>>(B, Hs, Ws, C, gin, c->gskip[lv - 1]);
            gin = c->gskip[lv - 1];
        }
        gcur = gin;
    }
}

}  // namespace

extern "C" {

int ibm_cnn_create(int32_t base, int32_t levels, int64_t max_pixels, ibm_cnn** out) {
    if (!out || base < 1 || levels < 2 || levels > 6 || max_pixels < 1) return IBM_ERR_ARG;
    ibm_cnn* c = new (std::nothrow) ibm_cnn();
    if (!c) return IBM_ERR_NO_MEM;
    c->base = base;
    c->levels = levels;
    c->max_pix = max_pixels;
    c->use_tc = std::getenv("IBM_CNN_NO_TC") == nullptr;
    cnn_specs(c);
    CnnCarver cv{nullptr};
    c->ws_bytes = cnn_layout(c, cv) + 256;
    // the layout must not depend on the base address (a stand-in base, never
    // dereferenced; ibm_cnn_bind lays the workspace out again)
    CnnCarver probe{reinterpret_cast<char*>(uintptr_t(1) << 20)};
    if (cnn_layout(c, probe) + 256 != c->ws_bytes) {
        delete c;
        return IBM_ERR_STATE;
    }
    *out = c;
    return IBM_OK;
}

void ibm_cnn_destroy(ibm_cnn* c) { delete c; }
const char* ibm_cnn_last_error(const ibm_cnn* c) { return c ? c->err.c_str() : "null network"; }

int ibm_cnn_set_window(ibm_cnn* c, int32_t x0, int32_t y0, int32_t w, int32_t h) {
    if (!c) return IBM_ERR_ARG;
    const int d = 1 << (c->levels - 1);
    if (w == 0 && h == 0) {
        c->win[0] = c->win[1] = c->win[2] = c->win[3] = 0;
        return IBM_OK;
    }
    if (x0 < 0 || y0 < 0 || w < d || h < d || w % d || h % d)
        return cfail(c, IBM_ERR_ARG, "window: non-negative origin, sides positive multiples of 2^(levels-1)");
    if ((long long)w * h > c->max_pix) return cfail(c, IBM_ERR_ARG, "window exceeds the network's pixel capacity");
    c->win[0] = x0;
    c->win[1] = y0;
    c->win[2] = w;
    c->win[3] = h;
    return IBM_OK;
}

int ibm_cnn_param_count(const ibm_cnn* c, int64_t* n) {
    if (!c || !n) return IBM_ERR_ARG;
    *n = c->nparam;
    return IBM_OK;
}

int ibm_cnn_workspace_bytes(const ibm_cnn* c, size_t* bytes) {
    if (!c || !bytes) return IBM_ERR_ARG;
    *bytes = c->ws_bytes;
    return IBM_OK;
}

int ibm_cnn_bind(ibm_cnn* c, void* dev_ws, size_t bytes, void* stream) {
    if (!c || !dev_ws) return IBM_ERR_ARG;
    if (bytes < c->ws_bytes) return cfail(c, IBM_ERR_NO_MEM, "network workspace too small");
    if (reinterpret_cast<uintptr_t>(dev_ws) % 256) return cfail(c, IBM_ERR_ARG, "workspace must be 256-byte aligned");
    c->ws = static_cast<char*>(dev_ws);
    c->st = static_cast<cudaStream_t>(stream);
    CnnCarver cv{c->ws};
    if (cnn_layout(c, cv) + 256 > c->ws_bytes) return cfail(c, IBM_ERR_STATE, "network layout outgrew its workspace");
    CCUDA(cudaMemsetAsync(c->ws, 0, c->ws_bytes - 256, c->st));
    c->bound = true;
    return IBM_OK;
}

int ibm_cnn_set_params(ibm_cnn* c, const double* host, int64_t n) {
    if (!c || !host || n != c->nparam) return IBM_ERR_ARG;
    if (!c->bound) return cfail(c, IBM_ERR_STATE, "network not bound");
    for (auto& ly : c->L) {
        const size_t nw = size_t(ly.K) * ly.cout;
        std::vector<float> w(host + ly.w_off, host + ly.w_off + nw), b(host + ly.b_off, host + ly.b_off + ly.cout);
        CCUDA(cudaMemcpyAsync(ly.w, w.data(), nw * sizeof(float), cudaMemcpyHostToDevice, c->st));
        CCUDA(cudaMemcpyAsync(ly.b, b.data(), ly.cout * sizeof(float), cudaMemcpyHostToDevice, c->st));
        CCUDA(cudaMemsetAsync(ly.m, 0, (nw + ly.cout) * sizeof(float), c->st));
        CCUDA(cudaMemsetAsync(ly.v, 0, (nw + ly.cout) * sizeof(float), c->st));
        k_wt<<<grid1(nw), 256, 0, c->st>>>(ly.K, ly.cout, ly.cin, ly.w, ly.wt, ly.wtc);
        CCUDA(cudaStreamSynchronize(c->st));
    }
    c->adam_t = 0;
    return IBM_OK;
}

int ibm_cnn_get_params(ibm_cnn* c, double* host, int64_t n) {
    if (!c || !host || n != c->nparam) return IBM_ERR_ARG;
    if (!c->bound) return cfail(c, IBM_ERR_STATE, "network not bound");
    for (auto& ly : c->L) {
        const size_t nw = size_t(ly.K) * ly.cout;
        std::vector<float> w(nw), b(ly.cout);
        CCUDA(cudaMemcpyAsync(w.data(), ly.w, nw * sizeof(float), cudaMemcpyDeviceToHost, c->st));
        CCUDA(cudaMemcpyAsync(b.data(), ly.b, ly.cout * sizeof(float), cudaMemcpyDeviceToHost, c->st));
        CCUDA(cudaStreamSynchronize(c->st));
        std::copy(w.begin(), w.end(), host + ly.w_off);
        std::copy(b.begin(), b.end(), host + ly.b_off);
    }
    return IBM_OK;
}

static int check_dims(ibm_cnn* c, int B, int H, int W) {
    if (!c->bound) return cfail(c, IBM_ERR_STATE, "network not bound");
    const int d = 1 << (c->levels - 1);
    if (B < 1 || H < d || W < d || H % d || W % d)
        return cfail(c, IBM_ERR_ARG, "height and width must be positive multiples of 2^(levels-1)");
    if ((long long)B * H * W > c->max_pix) return cfail(c, IBM_ERR_ARG, "batch exceeds the network's pixel capacity");
    return IBM_OK;
}

int ibm_cnn_forward(ibm_cnn* c, int32_t B, int32_t H, int32_t W, const float* d_in, float* d_out) {
    if (!c || !d_in || !d_out) return IBM_ERR_ARG;
    int rc = check_dims(c, B, H, W);
    if (rc) return rc;
    const long long P = (long long)B * H * W;
    k_to_bf16<<<grid1(P * 3), 256, 0, c->st>>>(P * 3, d_in, c->x16);
    run_forward(c, B, H, W);
    CCUDA(cudaMemcpyAsync(d_out, c->out32, P * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    CCUDA(cudaGetLastError());
    std::string e;
    if (int rc2 = ibm::cnn_tc_check(c, &e)) return cfail(c, rc2, e);
    return IBM_OK;
}

int ibm_cnn_loss_grad(ibm_cnn* c, int32_t B, int32_t H, int32_t W, const float* d_in, const float* d_target,
                      double* loss, double* host_grad) {
    if (!c || !d_in || !d_target) return IBM_ERR_ARG;
    int rc = check_dims(c, B, H, W);
    if (rc) return rc;
    const long long P = (long long)B * H * W;
    for (auto& ly : c->L) CCUDA(cudaMemsetAsync(ly.g, 0, (size_t(ly.K) + 1) * ly.cout * sizeof(float), c->st));
    k_to_bf16<<<grid1(P * 3), 256, 0, c->st>>>(P * 3, d_in, c->x16);
    run_forward(c, B, H, W);
    CCUDA(cudaMemsetAsync(c->dacc, 0, sizeof(double), c->st));
    k_mse<<<grid1(P), 256, 0, c->st>>>(P, c->out32, d_target, c->gout, c->dpart);
    k_part_sum<<<1, 256, 0, c->st>>>(1, grid1(P), c->dpart, c->dacc);
    run_backward(c, B, H, W);
    double h = 0.0;
    CCUDA(cudaMemcpyAsync(&h, c->dacc, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CCUDA(cudaStreamSynchronize(c->st));
    CCUDA(cudaGetLastError());
    {
        std::string e;
        if (int rc2 = ibm::cnn_tc_check(c, &e)) return cfail(c, rc2, e);
    }
    if (loss) *loss = h / double(P);
    if (host_grad) {
        for (auto& ly : c->L) {
            // device layout [K+1][cout]: weights rows then the bias row
            std::vector<float> g((size_t(ly.K) + 1) * ly.cout);
            CCUDA(cudaMemcpy(g.data(), ly.g, g.size() * sizeof(float), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < size_t(ly.K) * ly.cout; ++i) host_grad[ly.w_off + i] = g[i];
            for (int k = 0; k < ly.cout; ++k) host_grad[ly.b_off + k] = g[size_t(ly.K) * ly.cout + k];
        }
    }
    return IBM_OK;
}

int ibm_cnn_adam_step(ibm_cnn* c, double lr, double beta1, double beta2, double eps) {
    if (!c) return IBM_ERR_ARG;
    if (!c->bound) return cfail(c, IBM_ERR_STATE, "network not bound");
    c->adam_t++;
    const float c1 = float(1.0 - std::pow(beta1, c->adam_t)), c2 = float(1.0 - std::pow(beta2, c->adam_t));
    for (auto& ly : c->L) {
        const int n = (ly.K + 1) * ly.cout;
        k_adam<<<grid1(n), 256, 0, c->st>>>(ly.K, ly.cout, ly.w, ly.b, ly.m, ly.v, ly.g, ly.wt, ly.wtc, ly.cin,
                                           float(lr), float(beta1), float(beta2), float(eps), c1, c2);
    }
    CCUDA(cudaGetLastError());
    return IBM_OK;
}

int ibm_cnn_time_forward(ibm_cnn* c, int32_t B, int32_t H, int32_t W, int32_t reps, double* ms, int32_t n) {
    if (!c || !ms || reps < 1 || n != int32_t(c->L.size())) return IBM_ERR_ARG;
    int rc = check_dims(c, B, H, W);
    if (rc) return rc;
    std::vector<cudaEvent_t> ev(2 * size_t(n));
    for (auto& e : ev) CCUDA(cudaEventCreate(&e));
    std::vector<double> acc(n, 0.0);
    run_forward(c, B, H, W);
    int failed = 0;
    for (int r = 0; r < reps && !failed; ++r) {
        run_forward(c, B, H, W, ev.data());
        if (cudaStreamSynchronize(c->st) != cudaSuccess) failed = 1;
        for (int i = 0; i < n && !failed; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) failed = 1;
            acc[i] += t;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (failed) return cfail(c, IBM_ERR_CUDA, "timing the forward pass failed");
    std::string e;
    if (int rc2 = ibm::cnn_tc_check(c, &e)) return cfail(c, rc2, e);
    for (int i = 0; i < n; ++i) ms[i] = acc[i] / reps;
    return IBM_OK;
}

int ibm_cnn_layer_info(const ibm_cnn* c, int32_t i, int32_t* cin, int32_t* cout, int32_t* ks, int32_t* level,
                       int32_t* tc) {
    if (!c || i < 0 || i >= int32_t(c->L.size())) return IBM_ERR_ARG;
    const auto& ly = c->L[i];
    if (cin) *cin = ly.cin;
    if (cout) *cout = ly.cout;
    if (ks) *ks = ly.ks;
    if (level) *level = conv_level(c, i);
    if (tc) *tc = (ly.tc && i + 1 < int32_t(c->L.size())) ? 1 : 0;
    return IBM_OK;
}

int ibm_cnn_prepare(ibm_cnn* c, int32_t nx, int32_t ny, const double* d_phi_n, const double* d_phi_nm1,
                    const double* d_b_phi, const double* d_phi_np1, int32_t ncrop, const int32_t* h_crop_xy,
                    int32_t crop_h, int32_t crop_w, float* d_in, float* d_target) {
    if (!c || !d_phi_n || !d_phi_nm1 || !d_b_phi || !h_crop_xy || !d_in || ncrop < 1 || ncrop > 2048)
        return IBM_ERR_ARG;
    if (!c->bound) return cfail(c, IBM_ERR_STATE, "network not bound");
    for (int k = 0; k < ncrop; ++k)
        if (h_crop_xy[2 * k] < 0 || h_crop_xy[2 * k + 1] < 0 || h_crop_xy[2 * k] + crop_w > nx ||
            h_crop_xy[2 * k + 1] + crop_h > ny)
            return cfail(c, IBM_ERR_ARG, "crop outside the grid");
    if (d_target && !d_phi_np1) return IBM_ERR_ARG;
    const long long nc = (long long)nx * ny;
    CCUDA(cudaMemcpyAsync(c->dxy, h_crop_xy, 2 * ncrop * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CCUDA(cudaMemsetAsync(c->dacc, 0, 3 * sizeof(double), c->st));
    k_in_sums<<<grid1(nc), 256, 0, c->st>>>(nc, d_phi_n, d_phi_nm1, d_b_phi, c->dpart);
    k_part_sum<<<1, 256, 0, c->st>>>(3, grid1(nc), c->dpart, c->dacc);
    const long long n = (long long)ncrop * crop_h * crop_w;
    k_in_crops<<<grid1(n), 256, 0, c->st>>>(nx, ny, nc, d_phi_n, d_phi_nm1, d_b_phi, d_phi_np1, c->dacc, ncrop,
                                            c->dxy, crop_h, crop_w, d_in, d_target);
    CCUDA(cudaStreamSynchronize(c->st));
    CCUDA(cudaGetLastError());
    return IBM_OK;
}

}  // extern "C"

// Learned warm start inside a time step: lambda (= lambda^n on entry) becomes
// 2 lambda^n - lambda^{n-1} + s_d * UNet(...) on the pressure cells; r0 is the
// residual of the extrapolated guess (see cnn_extrapolated).
namespace ibm {
// reads (and clears) the flag a tcgen05 convolution sets when one of its
// bounded barrier waits gives up; synchronises the network's stream
int cnn_tc_check(ibm_cnn* c, std::string* err) {
    if (!c->tc_err) return IBM_OK;
    int h = 0;
    if (cudaMemcpyAsync(&h, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess) {
        *err = "warm-start network: reading the convolution status failed";
        return IBM_ERR_CUDA;
    }
    if (h) {
        cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->st);
        *err = "warm-start network: a tensor-core convolution gave up waiting on its barrier";
        return IBM_ERR_CUDA;
    }
    return IBM_OK;
}
void cnn_extrapolated(ibm_cnn* c, long long nl, const double* lam, const double* prev, double* out) {
    k_extrap_to<<<grid1(nl), 256, 0, c->st>>>(nl, lam, prev, out);
}
int cnn_warm_start(ibm_cnn* c, int nx, int ny, double* lam, double* lam_prev, const double* b_phi, long long nl,
                   std::string* err, int64_t* launches) {
    const bool win = c->win[2] > 0;
    const int x0 = win ? c->win[0] : 0, y0 = win ? c->win[1] : 0;
    const int w = win ? c->win[2] : nx, h = win ? c->win[3] : ny;
    if (win && (x0 < 0 || y0 < 0 || x0 + w > nx || y0 + h > ny)) {
        *err = "warm-start network: the inference window leaves the grid";
        return IBM_ERR_ARG;
    }
    const int rcd = check_dims(c, 1, h, w);
    if (rcd) {
        *err = c->err;
        return rcd;
    }
    const long long nc = (long long)nx * ny, nw = (long long)w * h;
    cudaMemsetAsync(c->dacc, 0, 3 * sizeof(double), c->st);
    k_in_sums<<<grid1(nc), 256, 0, c->st>>>(nc, lam, lam_prev, b_phi, c->dpart);
    k_part_sum<<<1, 256, 0, c->st>>>(3, grid1(nc), c->dpart, c->dacc);
    const int xy0[2] = {x0, y0};
    cudaMemcpyAsync(c->dxy, xy0, sizeof(xy0), cudaMemcpyHostToDevice, c->st);
    k_in_crops<<<grid1(nw), 256, 0, c->st>>>(nx, ny, nc, lam, lam_prev, b_phi, nullptr, c->dacc, 1, c->dxy, h, w,
                                             c->fin, nullptr);
    k_to_bf16<<<grid1(nw * 3), 256, 0, c->st>>>(nw * 3, c->fin, c->x16);
    run_forward(c, 1, h, w);
    if (win)
        k_cnn_apply_win<<<grid1(nl), 256, 0, c->st>>>(nc, nl, nx, x0, y0, w, h, lam, lam_prev, c->out32, c->dacc);
    else
        k_cnn_apply<<<grid1(nl), 256, 0, c->st>>>(nc, nl, lam, lam_prev, c->out32, c->dacc);
    *launches += 4 + 2 * int64_t(c->L.size()) + 2 * (c->levels - 1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("warm-start network: ") + cudaGetErrorString(e);
        return IBM_ERR_CUDA;
    }
    return IBM_OK;
}
cudaStream_t cnn_stream(ibm_cnn* c) { return c->st; }
}  // namespace ibm
