// Kernels of the learned warm start: a 4-level convolutional U-Net with BF16
// weights and activations and FP32 accumulation, trained on the GPU.
//
// Layout: activations NHWC (channels contiguous), BF16; a layer may read or
// write a channel slice of a wider buffer (ld = channels per pixel of the
// buffer, off = first channel), which is how the decoder's concatenations
// are formed without copies.  Weights of a 3x3 convolution are [Cout][9][Cin]
// (tap = 3*(dy+1) + (dx+1)), i.e. K-contiguous columns of the GEMM operand B.
//
// The convolutions (forward, data gradient, weight gradient) run on the
// tcgen05 tensor cores (k_conv_tc.cu); this file holds the element-wise
// kernels around them.
#include <cuda_bf16.h>
#include <stdint.h>

#include "ibm_internal.h"

namespace ibm {
namespace nn {

using bf16 = __nv_bfloat16;

namespace {

// Kernels of the forward pass are programmatic dependent launches: each
// waits for the previous kernel on the stream to complete (and its writes to
// be visible) before touching global memory, then lets the next one start.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*k)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(block);
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaLaunchKernelEx(&lc, k, static_cast<KArgs>(args)...);
}

// 8 BF16 channels (16 bytes) to FP32
__device__ inline void bf16x8_to_float(const uint4& u, float (&f)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 t = __bfloat1622float2(h[j]);
    f[2 * j] = t.x;
    f[2 * j + 1] = t.y;
  }
}

// FP32 to 8 BF16 channels (16 bytes), round to nearest
__device__ inline uint4 bf16x8_to(const float (&f)[8]) {
  uint4 o;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
  for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
  return o;
}

// ---------------------------------------------------------- elementwise

// G[p][c] (a slice) *= (Y[p][c] > 0): gradient through ReLU, in place; one
// thread per pixel and 8 channels (C, the slices' ld and off are multiples
// of 8: 16-byte loads and stores)
__global__ void k_relu_grad(long npix, int C, bf16* __restrict__ G, int ldg, int offg, const bf16* __restrict__ Y,
                            int ldy, int offy) {
  const int Gc = C / 8;
  const long n = npix * Gc;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const long p = k / Gc;
    const int c0 = (int)(k % Gc) * 8;
    uint4* gp = reinterpret_cast<uint4*>(G + p * ldg + offg + c0);
    float g[8], y[8];
    bf16x8_to_float(*gp, g);
    bf16x8_to_float(*reinterpret_cast<const uint4*>(Y + p * ldy + offy + c0), y);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (!(y[j] > 0.f)) g[j] = 0.f;
    *gp = bf16x8_to(g);
  }
}

// 2x2 average pool (H, W even): out[y][x][c] = mean of the 2x2 block; one
// thread per output pixel and 8 channels (C, the slices' ld and off are
// multiples of 8: 16-byte loads and stores)
__global__ void k_avgpool(int H, int W, int C, const bf16* __restrict__ X, int ldx, int offx, bf16* __restrict__ Y,
                          int ldy, int offy) {
  pdl_enter();
  const int H2 = H / 2, W2 = W / 2, G = C / 8;
  const int n = H2 * W2 * G;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int g = k % G, p = k / G, x = p % W2, y = p / W2;
    auto at = [&](int yy, int xx) {
      return *reinterpret_cast<const uint4*>(X + ((size_t)yy * W + xx) * ldx + offx + 8 * g);
    };
    float a[8], b[8], c[8], d[8];
    bf16x8_to_float(at(2 * y, 2 * x), a);
    bf16x8_to_float(at(2 * y, 2 * x + 1), b);
    bf16x8_to_float(at(2 * y + 1, 2 * x), c);
    bf16x8_to_float(at(2 * y + 1, 2 * x + 1), d);
    uint4 o;
    __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      oh[j] = __floats2bfloat162_rn(0.25f * (a[2 * j] + b[2 * j] + c[2 * j] + d[2 * j]),
                                    0.25f * (a[2 * j + 1] + b[2 * j + 1] + c[2 * j + 1] + d[2 * j + 1]));
    *reinterpret_cast<uint4*>(Y + (size_t)p * ldy + offy + 8 * g) = o;
  }
}

// gradient of the average pool: dX[2y+a][2x+b][c] (+)= dY[y][x][c] / 4; one
// thread per fine pixel and 8 channels
__global__ void k_avgpool_grad(int H, int W, int C, const bf16* __restrict__ dY, int ldy, int offy,
                               bf16* __restrict__ dX, int ldx, int offx, int accumulate) {
  const int Gc = C / 8, n = H * W * Gc;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int c0 = (k % Gc) * 8, p = k / Gc, x = p % W, y = p / W;
    float g[8], d[8];
    bf16x8_to_float(*reinterpret_cast<const uint4*>(dY + ((size_t)(y / 2) * (W / 2) + x / 2) * ldy + offy + c0), g);
    uint4* dp = reinterpret_cast<uint4*>(dX + (size_t)p * ldx + offx + c0);
    if (accumulate) bf16x8_to_float(*dp, d);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float gj = 0.25f * g[j];
      d[j] = accumulate ? d[j] + gj : gj;
    }
    *dp = bf16x8_to(d);
  }
}

// nearest 2x upsampling of a (H/2 x W/2) map into a (H x W) channel slice;
// one thread per output pixel and 8 channels
__global__ void k_upsample(int H, int W, int C, const bf16* __restrict__ X, int ldx, int offx, bf16* __restrict__ Y,
                           int ldy, int offy) {
  pdl_enter();
  const int G = C / 8, n = H * W * G;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int g = k % G, p = k / G, x = p % W, y = p / W;
    *reinterpret_cast<uint4*>(Y + (size_t)p * ldy + offy + 8 * g) =
        *reinterpret_cast<const uint4*>(X + ((size_t)(y / 2) * (W / 2) + x / 2) * ldx + offx + 8 * g);
  }
}

// gradient of the upsampling: dX[y][x][c] (+)= sum of the 2x2 block of dY;
// one thread per coarse pixel and 8 channels
__global__ void k_upsample_grad(int H, int W, int C, const bf16* __restrict__ dY, int ldy, int offy,
                                bf16* __restrict__ dX, int ldx, int offx, int accumulate) {
  const int H2 = H / 2, W2 = W / 2, Gc = C / 8, n = H2 * W2 * Gc;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int c0 = (k % Gc) * 8, p = k / Gc, x = p % W2, y = p / W2;
    auto at = [&](int yy, int xx, float (&f)[8]) {
      bf16x8_to_float(*reinterpret_cast<const uint4*>(dY + ((size_t)yy * W + xx) * ldy + offy + c0), f);
    };
    float a[8], b[8], c[8], e[8], d[8];
    at(2 * y, 2 * x, a);
    at(2 * y, 2 * x + 1, b);
    at(2 * y + 1, 2 * x, c);
    at(2 * y + 1, 2 * x + 1, e);
    uint4* dp = reinterpret_cast<uint4*>(dX + (size_t)p * ldx + offx + c0);
    if (accumulate) bf16x8_to_float(*dp, d);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float g = a[j] + b[j] + c[j] + e[j];
      d[j] = accumulate ? d[j] + g : g;
    }
    *dp = bf16x8_to(d);
  }
}

// bias gradient: db[c] += sum_p G[p][c].  A block of 256 threads reads 256 /
// (C / 8) pixels at a time, each thread 8 channels of one pixel (16 bytes),
// sums over its pixels, then the block sums its threads' partials per channel
// in shared memory and adds them to db (C <= 256).
__global__ void k_bias_grad(long npix, int C, const bf16* __restrict__ G, int ldg, int offg, float* __restrict__ db) {
  __shared__ float part[256][9];  // [thread][8 channels], padded against bank conflicts
  const int Gc = C / 8, rows = blockDim.x / Gc;
  const int g = threadIdx.x % Gc, r = threadIdx.x / Gc;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (r < rows) {
    for (long p = (long)blockIdx.x * rows + r; p < npix; p += (long)gridDim.x * rows) {
      float v[8];
      bf16x8_to_float(*reinterpret_cast<const uint4*>(G + p * ldg + offg + 8 * g), v);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += v[j];
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) part[threadIdx.x][j] = acc[j];
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int cg = c / 8, j = c % 8;
    float sum = 0.f;
    for (int rr = 0; rr < rows; ++rr) sum += part[rr * Gc + cg][j];
    atomicAdd(&db[c], sum);
  }
}

// loss = mean over masked pixels of (out[p][0] - target[p])^2 ; dOut = 2 (out - target) / count
__global__ void k_mse(long npix, const float* __restrict__ out, int ldo, const float* __restrict__ target,
                      const float* __restrict__ mask, float inv_count, bf16* __restrict__ dout, int ldd,
                      double* __restrict__ loss) {
  double s = 0.0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < npix; p += (long)gridDim.x * blockDim.x) {
    float m = mask ? mask[p] : 1.f;
    float d = (out[p * ldo] - target[p]) * m;
    s += (double)d * d;
    dout[p * ldd] = __float2bfloat16_rn(2.f * d * inv_count);
    for (int c = 1; c < ldd; ++c) dout[p * ldd + c] = __float2bfloat16_rn(0.f);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_count);
}

// Adam on FP32 master weights, BF16 copy for the kernels
__global__ void k_adam(long n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ wb, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    float gk = g[k];
    float mk = b1 * m[k] + (1.f - b1) * gk, vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    float wk = w[k] - lr * (mk * c1) / (sqrtf(vk * c2) + eps);
    w[k] = wk;
    if (wb) wb[k] = __float2bfloat16_rn(wk);
  }
}

__global__ void k_to_bf16(long n, const float* __restrict__ a, bf16* __restrict__ b) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    b[k] = __float2bfloat16_rn(a[k]);
}

// FP32 [H][W][cin] features -> BF16 [H][W][cpad] (zero padded channels;
// cpad a multiple of 8); one thread per pixel and 8 channels
__global__ void k_pack_input(long npix, int cin, int cpad, const float* __restrict__ f, bf16* __restrict__ x) {
  pdl_enter();
  const int G = cpad / 8;
  const long n = npix * G;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const long p = k / G;
    const int c0 = (int)(k % G) * 8;
    uint4 o;
    __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 2 * j;
      oh[j] = __floats2bfloat162_rn(c < cin ? f[p * cin + c] : 0.f, c + 1 < cin ? f[p * cin + c + 1] : 0.f);
    }
    *reinterpret_cast<uint4*>(x + p * cpad + c0) = o;
  }
}

inline int grid1(long n) {
  long b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace

void relu_grad(cudaStream_t s, long npix, int C, bf16* G, int ldg, int offg, const bf16* Y, int ldy, int offy) {
  k_relu_grad<<<grid1(npix * C / 8), 256, 0, s>>>(npix, C, G, ldg, offg, Y, ldy, offy);
}
void avgpool(cudaStream_t s, int H, int W, int C, const bf16* X, int ldx, int offx, bf16* Y, int ldy, int offy) {
  launch_pdl(k_avgpool, grid1((long)H * W * C / 32), 256, s, H, W, C, X, ldx, offx, Y, ldy, offy);
}
void avgpool_grad(cudaStream_t s, int H, int W, int C, const bf16* dY, int ldy, int offy, bf16* dX, int ldx, int offx,
                  bool acc) {
  k_avgpool_grad<<<grid1((long)H * W * C / 8), 256, 0, s>>>(H, W, C, dY, ldy, offy, dX, ldx, offx, acc ? 1 : 0);
}
void upsample(cudaStream_t s, int H, int W, int C, const bf16* X, int ldx, int offx, bf16* Y, int ldy, int offy) {
  launch_pdl(k_upsample, grid1((long)H * W * C / 8), 256, s, H, W, C, X, ldx, offx, Y, ldy, offy);
}
void upsample_grad(cudaStream_t s, int H, int W, int C, const bf16* dY, int ldy, int offy, bf16* dX, int ldx, int offx,
                   bool acc) {
  k_upsample_grad<<<grid1((long)H * W * C / 32), 256, 0, s>>>(H, W, C, dY, ldy, offy, dX, ldx, offx, acc ? 1 : 0);
}
void bias_grad(cudaStream_t s, long npix, int C, const bf16* G, int ldg, int offg, float* db) {
  const long rows = 256 / (C / 8);
  long blocks = (npix + rows * 8 - 1) / (rows * 8);  // at least 8 pixels per thread
  if (blocks > 608) blocks = 608;
  if (blocks < 1) blocks = 1;
  k_bias_grad<<<(int)blocks, 256, 0, s>>>(npix, C, G, ldg, offg, db);
}
void mse(cudaStream_t s, long npix, const float* out, int ldo, const float* target, const float* mask, float inv_count,
         bf16* dout, int ldd, double* loss) {
  k_mse<<<grid1(npix), 256, 0, s>>>(npix, out, ldo, target, mask, inv_count, dout, ldd, loss);
}
void adam(cudaStream_t s, long n, float* w, const float* g, float* m, float* v, bf16* wb, float lr, float b1, float b2,
          float eps, float c1, float c2) {
  k_adam<<<grid1(n), 256, 0, s>>>(n, w, g, m, v, wb, lr, b1, b2, eps, c1, c2);
}
void to_bf16(cudaStream_t s, long n, const float* a, bf16* b) { k_to_bf16<<<grid1(n), 256, 0, s>>>(n, a, b); }
void pack_input(cudaStream_t s, long npix, int cin, int cpad, const float* f, bf16* x) {
  launch_pdl(k_pack_input, grid1(npix * cpad / 8), 256, s, npix, cin, cpad, f, x);
}

}  // namespace nn
}  // namespace ibm
