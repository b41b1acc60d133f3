// 3x3 convolution (same padding, NHWC, BF16 operands, FP32 accumulation) on
// the fifth-generation tensor cores: an implicit GEMM whose accumulator lives
// in tensor memory.
//
// One CTA of 128 threads computes a tile of 8 x 16 output pixels (M = 128)
// and all Cout (N = 16 .. 128) of one image.  For each chunk of CK input
// channels it stages
//   the input patch   (10 x 18 pixels, tile plus a one-pixel halo) as
//                     [channel block of 8][patch pixel][8] BF16, by 16-byte
//                     cp.async copies (zero fill outside the image), and
//   the weights       [tap][channel block][cout][8] BF16, by bulk copies
//                     (cp.async.bulk, completion on an mbarrier),
// then one thread issues, per tap (ky, kx) and per 16 channels, one
// tcgen05.mma of 128 x N x 16.  Both operands are K-major without swizzle:
// a core matrix is 8 rows x 16 bytes, contiguous.  In the patch, the 8 rows
// of a core matrix are 8 neighbouring pixels of one tile row, so the tap's
// operand is the patch shifted by (ky * 10 + kx) pixels: the leading-dimension
// offset (next 8 channels) is one patch plane, the stride offset (next tile
// row) is one patch row.  The epilogue reads the accumulator with tcgen05.ld
// (warp w owns lanes 32w .. 32w + 31, one output pixel per lane), adds the
// bias, applies the ReLU and stores BF16.
//
// Launched with programmatic stream serialisation: the tensor-memory
// allocation, the barrier set-up and the first chunk's weights (which no
// earlier kernel of the forward pass writes) overlap the previous layer;
// griddepcontrol.wait comes before the first read of the input.
//
// Every wait is bounded: a barrier that does not complete sets *err, the
// CTA skips the remaining work, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "conv_tc.h"
#include "kernels.h"

namespace ibm {
namespace {

constexpr int kTW = 8, kTH = 16;                 // output tile (x, y)
constexpr int kPW = kTW + 2, kPH = kTH + 2;      // patch with halo
constexpr int kPP = kPW * kPH;                   // patch pixels
constexpr int kThreadsTc = 128;
constexpr long long kWaitLimit = 1LL << 21;      // polls of one barrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;   // descriptor version of the fifth-generation tensor cores
    return d;
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t phase) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        if (bar_try(bar, phase)) return true;
        if (i > 32) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

union Pack16 {
    uint4 u;
    __nv_bfloat16 h[8];
};

__global__ void __launch_bounds__(kThreadsTc) k_conv3x3_tc(ConvTcArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int CKB = a.ck / 8;                        // channel blocks per chunk
    const int CBt = a.cinp / 8;                      // channel blocks in all
    const int nchunk = a.cinp / a.ck;
    unsigned char* patch = smem;                                    // CKB * kPP * 16 B
    unsigned char* wsm = smem + size_t(CKB) * kPP * 16;             // 9 * CKB * Cout * 16 B
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + size_t(9) * CKB * a.cout * 16);   // [0] weights, [1] mma
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2);
    const uint32_t bar_w = smem_u32(&bars[0]), bar_m = smem_u32(&bars[1]);
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH, b = blockIdx.z;
    const uint32_t ncols = a.cout < 32 ? 32u : uint32_t(a.cout);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_w) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *slot;
    const uint32_t idesc = idesc_bf16(128, a.cout);
    const uint32_t wbytes = uint32_t(CKB) * uint32_t(a.cout) * 16u;   // one tap of one chunk
    auto issue_weights = [&](int c0) {   // thread 0: the nine taps of one chunk
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar_w), "r"(9u * wbytes)
                     : "memory");
        for (int t = 0; t < 9; ++t) {
            const __nv_bfloat16* src = a.wtc + (size_t(t) * CBt + c0 / 8) * a.cout * 8;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                    smem_u32(wsm + size_t(t) * wbytes)),
                "l"(src), "r"(wbytes), "r"(bar_w)
                : "memory");
        }
    };
    if (tid == 0) issue_weights(0);
    bool ok = true;
    int issued = 0, wissued = 1;   // MMA groups committed, weight batches requested
    // the input is the previous kernel's output
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    for (int k = 0; k < nchunk && ok; ++k) {
        const int c0 = k * a.ck;
        if (k > 0) {   // the previous chunk's MMAs have read the staging buffers
            const bool w = bar_wait(bar_m, uint32_t(k - 1) & 1u);
            ok = __syncthreads_and(w);
            if (!ok) break;
            if (tid == 0) issue_weights(c0);
            wissued = k + 1;
        }
        // input patch of this chunk: one 16-byte copy per (pixel, channel block),
        // all in flight together; zero fill outside the image and past cin
        for (int idx = tid; idx < kPP * CKB; idx += kThreadsTc) {
            const int p = idx / CKB, cb = idx - p * CKB;
            const int py = p / kPW, px = p - py * kPW;
            const int gy = y0 - 1 + py, gx = x0 - 1 + px, ch = c0 + cb * 8;
            const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W && ch < a.cin;
            const __nv_bfloat16* src = in ? a.x + ((size_t(b) * a.H + gy) * a.W + gx) * a.cin + ch : a.x;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                             smem_u32(patch + (size_t(cb) * kPP + p) * 16)),
                         "l"(src), "r"(in ? 16u : 0u)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        {
            const bool w = bar_wait(bar_w, uint32_t(k) & 1u);
            ok = __syncthreads_and(w);
            if (!ok) break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t pa = smem_u32(patch), pw = smem_u32(wsm);
            for (int t = 0; t < 9; ++t) {
                const int ky = t / 3, kx = t - ky * 3;
                for (int j = 0; j < CKB; j += 2) {
                    const uint64_t da = sdesc(pa + uint32_t((ky * kPW + kx) + j * kPP) * 16u, kPP * 16, kPW * 16);
                    const uint64_t db = sdesc(pw + uint32_t((t * CKB + j) * a.cout) * 16u, a.cout * 16, 128);
                    mma_bf16_tc(tmem, da, db, idesc, (k | t | j) != 0);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_m)
                         : "memory");
        }
        issued = k + 1;
    }
    if (ok && issued == nchunk) {
        const bool w = bar_wait(bar_m, uint32_t(nchunk - 1) & 1u);
        ok = __syncthreads_and(w);
    } else {
        ok = false;
    }
    if (!ok) {
        if (tid == 0) atomicExch(a.err, 1);
        // let the work already issued drain before the buffers go away (bounded)
        if (issued > 0) bar_wait(bar_m, uint32_t(issued - 1) & 1u);
        if (wissued > 0) bar_wait(bar_w, uint32_t(wissued - 1) & 1u);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int m = warp * 32 + lane;
        const int gy = y0 + m / kTW, gx = x0 + m % kTW;
        const bool store = gy < a.H && gx < a.W;
        __nv_bfloat16* dst = a.y + ((size_t(b) * a.H + gy) * a.W + gx) * a.cout;
        for (int c = 0; c < a.cout; c += 16) {
            float v[16];
            tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c), v);
            if (store) {
                Pack16 o[2];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float t = v[i] + a.bias[c + i];
                    if (a.relu) t = fmaxf(t, 0.f);
                    o[i >> 3].h[i & 7] = __float2bfloat16(t);
                }
                *reinterpret_cast<uint4*>(dst + c) = o[0].u;
                *reinterpret_cast<uint4*>(dst + c + 8) = o[1].u;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

bool conv_tc_shape_ok(int cin, int cout) {
    return cin >= 1 && (cout == 16 || cout == 32 || cout == 64 || cout == 128);
}

int conv_tc_cinp(int cin) { return (cin + 15) / 16 * 16; }

size_t conv_tc_smem(int ck, int cout) {
    return size_t(ck / 8) * kPP * 16 + size_t(9) * (ck / 8) * cout * 16 + 2 * sizeof(uint64_t) + 16;
}

int conv_tc_chunk(int cin, int cout, size_t budget) {
    const int cinp = conv_tc_cinp(cin);
    for (int ck = cinp; ck >= 16; ck -= 16)
        if (cinp % ck == 0 && conv_tc_smem(ck, cout) <= budget) return ck;
    return 16;
}

cudaError_t launch_conv3x3_tc(const ConvTcArgs& a, size_t smem_bytes, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (smem_bytes < conv_tc_smem(a.ck, a.cout)) return cudaErrorInvalidValue;
    if (!conv_tc_shape_ok(a.cin, a.cout) || a.cin % 8 || a.cinp != conv_tc_cinp(a.cin) || a.ck < 16 || a.ck % 16 ||
        a.cinp % a.ck || a.B < 1 || a.H < 1 || a.W < 1 || !a.err)
        return cudaErrorInvalidValue;
    // at most 512 / ncols CTAs per SM: their tensor memory always fits
    const size_t ncols = a.cout < 32 ? 32 : size_t(a.cout);
    const size_t share = size_t(228 * 1024) * ncols / 512;
    if (smem_bytes < share - 1024) smem_bytes = share - 1024;
    if (smem_bytes > size_t(227 * 1024)) return cudaErrorInvalidValue;
    const dim3 grid((a.W + kTW - 1) / kTW, (a.H + kTH - 1) / kTH, a.B);
    return launch_k(k_conv3x3_tc, grid, kThreadsTc, smem_bytes, st, a);
}

}  // namespace ibm
