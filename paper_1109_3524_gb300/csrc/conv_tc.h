// 3x3 convolution on the fifth-generation tensor cores (k_conv_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace ibm {

struct ConvTcArgs {
    const __nv_bfloat16* x;     // input, NHWC [B][H][W][cin]
    const __nv_bfloat16* wtc;   // weights [9 taps][cinp / 8][cout][8], zero for channels >= cin
    const float* bias;          // [cout]
    __nv_bfloat16* y;           // output, NHWC [B][H][W][cout]
    int B, H, W;
    int cin, cinp, cout;        // cinp: cin rounded up to 16
    int ck;                     // input channels per staged chunk (multiple of 16 dividing cinp)
    int relu;
    int* err;                   // set to 1 when a barrier wait gives up
};

bool conv_tc_shape_ok(int cin, int cout);
int conv_tc_cinp(int cin);
size_t conv_tc_smem(int ck, int cout);
// largest chunk whose staging fits `budget` bytes of shared memory
int conv_tc_chunk(int cin, int cout, size_t budget);
// smem_bytes: at least conv_tc_smem(ck, cout); the launch takes more when
// needed so that the CTAs resident on one SM fit its tensor memory
cudaError_t launch_conv3x3_tc(const ConvTcArgs& a, size_t smem_bytes, cudaStream_t st);

}  // namespace ibm
