// Launchers of the U-Net kernels (k_nn.cu, k_conv_tc.cu).  Activations are BF16 NHWC; a
// view of an activation is (buffer, channels per pixel ld, first channel off).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ibm {
namespace nn {

using bf16 = __nv_bfloat16;

// Y = act(conv3x3(X, W) + bias), zero padding, on the tcgen05 tensor cores
// (k_conv_tc.cu); Cin, Cout % 16 == 0, ldx, offx, ldy, offy % 8 == 0; wpk:
// the weights packed by pack_conv_weights; yf: optional dense FP32 copy of the
// output [H][W][Cout].  Returns 0, or -1 with ibm_last_error set.
int conv3x3(cudaStream_t s, int H, int W, int Cin, int Cout, const bf16* X, int ldx, int offx, const bf16* wpk,
            const float* bias, bf16* Y, int ldy, int offy, bool relu, float* yf);
// elements of the packed weights of a convolution with Cin inputs and Cout
// outputs, and the packing of w[Cout][9][Cin] (flip: of the data-gradient
// operator of a layer with weights w[Cin][9][Cout], W'[co][tap][ci] =
// w[ci][8 - tap][co])
size_t packed_conv_weights(int Cin, int Cout);
struct PackJob {
  int cin, cout, nt, ntiles, flip;
  const bf16* w;
  bf16* wpk;
};
PackJob pack_job(int Cin, int Cout, const bf16* w, bf16* wpk, bool flip);
// every job of the device array jobs_dev in one launch; max_elems: the
// largest job's packed_conv_weights
void pack_conv_weights(cudaStream_t s, const PackJob* jobs_dev, int njobs, long max_elems);
// true once a convolution kernel has given up a bounded wait
bool conv_tc_failed();
// dW[co][tap][ci] += sum_p G[p][co] X[p + shift(tap)][ci] on the tcgen05 tensor
// cores (k_conv_tc.cu); Cout <= 128; returns 0, or -1 with ibm_last_error set
int conv3x3_wgrad(cudaStream_t s, int H, int W, int Cin, int Cout, const bf16* G, int ldg, int offg, const bf16* X,
                   int ldx, int offx, float* dW);
void relu_grad(cudaStream_t s, long npix, int C, bf16* G, int ldg, int offg, const bf16* Y, int ldy, int offy);
void avgpool(cudaStream_t s, int H, int W, int C, const bf16* X, int ldx, int offx, bf16* Y, int ldy, int offy);
void avgpool_grad(cudaStream_t s, int H, int W, int C, const bf16* dY, int ldy, int offy, bf16* dX, int ldx, int offx,
                  bool acc);
void upsample(cudaStream_t s, int H, int W, int C, const bf16* X, int ldx, int offx, bf16* Y, int ldy, int offy);
void upsample_grad(cudaStream_t s, int H, int W, int C, const bf16* dY, int ldy, int offy, bf16* dX, int ldx, int offx,
                   bool acc);
void bias_grad(cudaStream_t s, long npix, int C, const bf16* G, int ldg, int offg, float* db);
void mse(cudaStream_t s, long npix, const float* out, int ldo, const float* target, const float* mask, float inv_count,
         bf16* dout, int ldd, double* loss);
void adam(cudaStream_t s, long n, float* w, const float* g, float* m, float* v, bf16* wb, float lr, float b1, float b2,
          float eps, float c1, float c2);
void to_bf16(cudaStream_t s, long n, const float* a, bf16* b);
void pack_input(cudaStream_t s, long npix, int cin, int cpad, const float* f, bf16* x);

}  // namespace nn
}  // namespace ibm
