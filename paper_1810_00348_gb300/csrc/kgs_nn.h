// kgs_nn.h -- internal declarations shared by the network kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace kgs {
namespace nn {

struct ConvDims {
    int B, D, H, W;  // batch and volume (channels-last tensors [B][D][H][W][C])
    int cin_p, cout_p;
};

// 3x3x3 convolution with zero padding on the tensor cores (tcgen05, bf16
// operands, FP32 accumulator in tensor memory), output channels <= 112.
//   mode 0: out = relu(acc + bias) as bf16
//   mode 1: out = acc + bias as FP32
//   mode 2: out = acc * (gate > 0) as bf16 (gate: bf16, same layout as out)
// w: [27][cout_p][cin_p] bf16; wpk: scratch of the same size that receives
// the weights repacked for the kernel.  err: device word set to 1 if a
// bounded wait inside the kernel gave up (the output is then incomplete).
cudaError_t conv_tc(int mode, const __nv_bfloat16 *in, const __nv_bfloat16 *w, __nv_bfloat16 *wpk, const float *bias,
                    void *out, const __nv_bfloat16 *gate, ConvDims dm, int *err, cudaStream_t s);

// Weight gradient of the same convolution on the tensor cores:
// part[b][chunk][t][co][ci] (FP32, wgrad_chunks(dm) chunks of voxels per
// sample) = sum over the chunk's voxels v of dy[v][co] in[v + off(t)][ci];
// the caller sums the partials over samples and chunks in a fixed order.
int wgrad_chunks(const ConvDims &dm);
cudaError_t wgrad_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *dy, float *part, ConvDims dm, int *err,
                     cudaStream_t s);

}  // namespace nn
}  // namespace kgs
