// U-Net of the learned warm start: architecture, parameters, forward,
// backward and Adam, on the kernels of k_nn.cu.
//
// Architecture (widths w0..w3, every convolution 3x3 with zero padding):
//   level 0:  conv(16 -> w0) relu, conv(w0 -> w0) relu            = e0
//   level l:  pool(e_{l-1}), conv(. -> w_l) relu, conv relu       = e_l (l = 1, 2, 3)
//   decoder l = 2, 1, 0:  [up(d_{l+1} or e3), e_l] -> conv relu, conv relu = d_l
//   head:     conv(w0 -> 16), channel 0 is the output, no activation
// The four input features are zero-padded to 16 channels; H and W must be
// multiples of 8.  Activations are BF16; weights are kept as FP32 master
// copies (Adam) and BF16 working copies (tensor-core kernels).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/ibm.h"
#include "ibm_internal.h"
#include "nn_internal.h"

using namespace ibm;
using namespace ibm::nn;

namespace {

struct Conv {
  int cin, cout;
  bool relu;
  size_t w, b;     // offsets of weights [cout][9][cin] and bias [cout] in the parameter vector
  size_t pk, pkf;  // offsets of the packed forward and data-gradient weights
};

// a view of an activation: buffer, channels per pixel, first channel, channels
struct Act {
  bf16* p = nullptr;
  int ld = 0, off = 0, c = 0;
};

struct Level {
  int H = 0, W = 0;
  bf16 *in = nullptr, *a = nullptr, *cat = nullptr, *bb = nullptr, *d = nullptr;  // activations
  bf16 *gin = nullptr, *ga = nullptr, *gcat = nullptr, *gbb = nullptr, *gd = nullptr;  // their gradients
  int cin = 0, cup = 0;  // input channels of the first conv; channels of the upsampled part of cat
};

}  // namespace

struct ibm_unet {
  int w[4];
  std::vector<Conv> conv;
  size_t nparam = 0;
  float *pw = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, gradient, Adam moments
  bf16* wb = nullptr;                                                  // BF16 weights
  bf16 *wpk = nullptr, *wpkf = nullptr;  // packed for the tensor-core convolutions: forward, data gradient
  size_t npk = 0, npkf = 0;
  bool wdirty = true;  // wb changed since the packed copies were made
  PackJob* pack_jobs = nullptr;  // device: one forward and one data-gradient job per convolution
  int npack = 0;
  long pack_max = 0;
  long long adam_t = 0;
  // activations for the current size
  int H = 0, W = 0;
  Level lv[4];
  bf16 *e3 = nullptr, *ge3 = nullptr, *out = nullptr, *gout = nullptr;
  float *outf = nullptr;
  double* loss_d = nullptr;
  std::vector<void*> act_allocs;

  ~ibm_unet() {
    free_acts();
    void* ps[] = {pw, grad, m, v, wb, wpk, wpkf, loss_d, pack_jobs};
    for (void* p : ps)
      if (p) cudaFree(p);
  }
  void free_acts() {
    for (void* p : act_allocs) cudaFree(p);
    act_allocs.clear();
    H = W = 0;
  }
};

namespace {

thread_local std::string g_unet_err;

int ufail(int code, const char* msg) {
  ibm::set_last_error(msg);
  return code;
}

#define UCUDA(expr)                                                   \
  do {                                                                \
    cudaError_t e_ = (expr);                                          \
    if (e_ != cudaSuccess) return ufail(IBM_E_CUDA, cudaGetErrorString(e_)); \
  } while (0)

int dalloc(ibm_unet* n, void** p, size_t bytes) {
  UCUDA(cudaMalloc(p, bytes ? bytes : 16));
  UCUDA(cudaMemset(*p, 0, bytes ? bytes : 16));
  n->act_allocs.push_back(*p);
  return IBM_OK;
}

// buffers for an H x W input
int ensure_acts(ibm_unet* n, int H, int W) {
  if (n->H == H && n->W == W) return IBM_OK;
  n->free_acts();
  int rc = 0;
  auto B = [&](bf16** p, size_t px, int c) { rc |= dalloc(n, (void**)p, px * c * sizeof(bf16)); };
  const int* w = n->w;
  for (int l = 0; l < 4; ++l) {
    Level& L = n->lv[l];
    L.H = H >> l;
    L.W = W >> l;
    size_t px = (size_t)L.H * L.W;
    L.cin = l == 0 ? 16 : w[l - 1];
    L.cup = l < 3 ? (l == 2 ? w[3] : w[l + 1]) : 0;
    B(&L.in, px, L.cin);
    B(&L.gin, px, L.cin);
    B(&L.a, px, w[l]);
    B(&L.ga, px, w[l]);
    if (l < 3) {
      B(&L.cat, px, L.cup + w[l]);
      B(&L.gcat, px, L.cup + w[l]);
      B(&L.bb, px, w[l]);
      B(&L.gbb, px, w[l]);
      B(&L.d, px, w[l]);
      B(&L.gd, px, w[l]);
    }
  }
  size_t px3 = (size_t)n->lv[3].H * n->lv[3].W, px0 = (size_t)H * W;
  B(&n->e3, px3, w[3]);
  B(&n->ge3, px3, w[3]);
  B(&n->out, px0, 16);
  B(&n->gout, px0, 16);
  rc |= dalloc(n, (void**)&n->outf, px0 * 16 * sizeof(float));
  if (rc) return IBM_E_CUDA;
  n->H = H;
  n->W = W;
  return IBM_OK;
}

// conv index, its input and its output (views into the level buffers)
struct Edge {
  int conv;
  Act x, y;
};

std::vector<Edge> edges(ibm_unet* n) {
  std::vector<Edge> e;
  const int* w = n->w;
  for (int l = 0; l < 4; ++l) {
    Level& L = n->lv[l];
    Act in{L.in, L.cin, 0, L.cin}, a{L.a, w[l], 0, w[l]};
    Act el = l < 3 ? Act{L.cat, L.cup + w[l], L.cup, w[l]} : Act{n->e3, w[3], 0, w[3]};
    e.push_back({2 * l, in, a});
    e.push_back({2 * l + 1, a, el});
  }
  for (int l = 2, k = 8; l >= 0; --l, k += 2) {
    Level& L = n->lv[l];
    Act cat{L.cat, L.cup + w[l], 0, L.cup + w[l]}, bb{L.bb, w[l], 0, w[l]}, d{L.d, w[l], 0, w[l]};
    e.push_back({k, cat, bb});
    e.push_back({k + 1, bb, d});
  }
  e.push_back({14, Act{n->lv[0].d, w[0], 0, w[0]}, Act{n->out, 16, 0, 16}});
  return e;
}

// gradient view matching an activation view
Act grad_of(ibm_unet* n, const Act& a) {
  for (int l = 0; l < 4; ++l) {
    Level& L = n->lv[l];
    bf16* pairs[][2] = {{L.in, L.gin}, {L.a, L.ga}, {L.cat, L.gcat}, {L.bb, L.gbb}, {L.d, L.gd}};
    for (auto& pr : pairs)
      if (pr[0] == a.p) return Act{pr[1], a.ld, a.off, a.c};
  }
  if (a.p == n->e3) return Act{n->ge3, a.ld, a.off, a.c};
  if (a.p == n->out) return Act{n->gout, a.ld, a.off, a.c};
  return Act{};
}

int level_of(ibm_unet* n, const Act& a) {
  for (int l = 0; l < 4; ++l) {
    Level& L = n->lv[l];
    if (a.p == L.in || a.p == L.a || a.p == L.cat || a.p == L.bb || a.p == L.d) return l;
  }
  return a.p == n->e3 ? 3 : 0;
}

// packed copies of the BF16 weights for the convolution kernels, after the
// weights changed (creation, new parameters, an Adam step)
void ensure_packed(ibm_unet* n, cudaStream_t s) {
  if (!n->wdirty) return;
  pack_conv_weights(s, n->pack_jobs, n->npack, n->pack_max);
  n->wdirty = false;
}

int forward(ibm_unet* n, cudaStream_t s) {
  const int* w = n->w;
  std::vector<Edge> E = edges(n);
  ensure_packed(n, s);
  int rc = 0;
  auto run = [&](const Edge& e) {
    const Conv& c = n->conv[e.conv];
    Level& L = n->lv[level_of(n, e.x)];
    rc |= conv3x3(s, L.H, L.W, c.cin, c.cout, e.x.p, e.x.ld, e.x.off, n->wpk + c.pk, n->pw + c.b, e.y.p, e.y.ld,
                  e.y.off, c.relu, e.conv == 14 ? n->outf : nullptr);
  };
  // encoder
  for (int l = 0; l < 4; ++l) {
    if (l > 0) {
      Level& P = n->lv[l - 1];
      avgpool(s, P.H, P.W, w[l - 1], P.cat, P.cup + w[l - 1], P.cup, n->lv[l].in, w[l - 1], 0);
    }
    run(E[2 * l]);
    run(E[2 * l + 1]);
  }
  // decoder
  for (int l = 2, k = 8; l >= 0; --l, k += 2) {
    Level& L = n->lv[l];
    const bf16* src = l == 2 ? n->e3 : n->lv[l + 1].d;
    upsample(s, L.H, L.W, L.cup, src, L.cup, 0, L.cat, L.cup + w[l], 0);
    run(E[k]);
    run(E[k + 1]);
  }
  run(E[14]);
  return rc;
}

// one conv's backward: mask the output gradient, accumulate dW and db, and
// write the input gradient (unless it is the network input)
int conv_backward(ibm_unet* n, const Edge& e, cudaStream_t s, bool need_dx) {
  const Conv& c = n->conv[e.conv];
  Level& L = n->lv[level_of(n, e.x)];
  Act gy = grad_of(n, e.y), gx = grad_of(n, e.x);
  const long npix = (long)L.H * L.W;
  if (c.relu) relu_grad(s, npix, c.cout, gy.p, gy.ld, gy.off, e.y.p, e.y.ld, e.y.off);
  if (conv3x3_wgrad(s, L.H, L.W, c.cin, c.cout, gy.p, gy.ld, gy.off, e.x.p, e.x.ld, e.x.off, n->grad + c.w)) return -1;
  bias_grad(s, npix, c.cout, gy.p, gy.ld, gy.off, n->grad + c.b);
  if (need_dx)
    return conv3x3(s, L.H, L.W, c.cout, c.cin, gy.p, gy.ld, gy.off, n->wpkf + c.pkf, nullptr, gx.p, gx.ld, gx.off,
                   false, nullptr);
  return 0;
}

int backward(ibm_unet* n, cudaStream_t s) {
  const int* w = n->w;
  std::vector<Edge> E = edges(n);
  int rc = conv_backward(n, E[14], s, true);  // head -> d(d0)
  for (int l = 0, k = 12; l <= 2; ++l, k -= 2) {
    Level& L = n->lv[l];
    rc |= conv_backward(n, E[k + 1], s, true);  // d(d_l) -> d(bb_l)
    rc |= conv_backward(n, E[k], s, true);      // d(bb_l) -> d(cat_l), both parts
    // the upsampled part of cat_l comes from d_{l+1} (or e3)
    if (l < 2)
      upsample_grad(s, L.H, L.W, L.cup, L.gcat, L.cup + w[l], 0, n->lv[l + 1].gd, L.cup, 0, false);
    else
      upsample_grad(s, L.H, L.W, L.cup, L.gcat, L.cup + w[l], 0, n->ge3, L.cup, 0, false);
  }
  // encoder, from the bottom: e_l's gradient is in the skip slice of gcat_l
  // (decoder path) plus the pooling path of level l+1
  for (int l = 3; l >= 0; --l) {
    rc |= conv_backward(n, E[2 * l + 1], s, true);  // d(e_l) -> d(a_l)
    rc |= conv_backward(n, E[2 * l], s, l > 0);      // d(a_l) -> d(in_l)
    if (l > 0) {
      Level& P = n->lv[l - 1];
      avgpool_grad(s, P.H, P.W, w[l - 1], n->lv[l].gin, w[l - 1], 0, P.gcat, P.cup + w[l - 1], P.cup, true);
    }
  }
  return rc;
}

}  // namespace

extern "C" {

int ibm_unet_create(const int widths[4], unsigned long long seed, ibm_unet** out) {
  if (!widths || !out) return ufail(IBM_E_INVAL, "null argument");
  for (int l = 0; l < 4; ++l)
    if (widths[l] < 16 || widths[l] % 16) return ufail(IBM_E_INVAL, "U-Net widths must be multiples of 16");
  auto* n = new ibm_unet();
  std::memcpy(n->w, widths, sizeof(n->w));
  const int* w = n->w;
  auto add = [&](int cin, int cout, bool relu) {
    Conv c{cin, cout, relu, n->nparam, 0, n->npk, n->npkf};
    n->nparam += (size_t)cout * 9 * cin;
    c.b = n->nparam;
    n->nparam += cout;
    n->npk += packed_conv_weights(cin, cout);
    n->npkf += packed_conv_weights(cout, cin);
    n->conv.push_back(c);
  };
  add(16, w[0], true);
  add(w[0], w[0], true);
  for (int l = 1; l < 4; ++l) {
    add(w[l - 1], w[l], true);
    add(w[l], w[l], true);
  }
  add(w[3] + w[2], w[2], true);
  add(w[2], w[2], true);
  add(w[2] + w[1], w[1], true);
  add(w[1], w[1], true);
  add(w[1] + w[0], w[0], true);
  add(w[0], w[0], true);
  add(w[0], 16, false);
  // He-normal initialisation from a seeded generator; biases zero; head x0.1
  std::vector<float> h(n->nparam, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> N01(0.f, 1.f);
  for (size_t ci = 0; ci < n->conv.size(); ++ci) {
    const Conv& c = n->conv[ci];
    float sd = std::sqrt(2.f / (9.f * c.cin)) * (ci == n->conv.size() - 1 ? 0.1f : 1.f);
    for (size_t k = 0; k < (size_t)c.cout * 9 * c.cin; ++k) h[c.w + k] = sd * N01(rng);
  }
  int rc = 0;
  auto A = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess || cudaMemset(*p, 0, bytes) != cudaSuccess) rc = IBM_E_CUDA;
  };
  A((void**)&n->pw, n->nparam * 4);
  A((void**)&n->grad, n->nparam * 4);
  A((void**)&n->m, n->nparam * 4);
  A((void**)&n->v, n->nparam * 4);
  A((void**)&n->wb, n->nparam * 2);
  A((void**)&n->wpk, n->npk * 2);
  A((void**)&n->wpkf, n->npkf * 2);
  std::vector<PackJob> jobs;
  if (!rc) {
    for (const Conv& c : n->conv) {
      jobs.push_back(pack_job(c.cin, c.cout, n->wb + c.w, n->wpk + c.pk, false));
      jobs.push_back(pack_job(c.cout, c.cin, n->wb + c.w, n->wpkf + c.pkf, true));
      n->pack_max = std::max(n->pack_max, (long)std::max(packed_conv_weights(c.cin, c.cout),
                                                          packed_conv_weights(c.cout, c.cin)));
    }
    n->npack = (int)jobs.size();
  }
  A((void**)&n->pack_jobs, jobs.size() * sizeof(PackJob) + 16);
  if (!rc && cudaMemcpy(n->pack_jobs, jobs.data(), jobs.size() * sizeof(PackJob), cudaMemcpyHostToDevice) !=
                 cudaSuccess)
    rc = IBM_E_CUDA;
  A((void**)&n->loss_d, 8);
  if (!rc && cudaMemcpy(n->pw, h.data(), n->nparam * 4, cudaMemcpyHostToDevice) != cudaSuccess) rc = IBM_E_CUDA;
  if (!rc) {
    to_bf16(0, (long)n->nparam, n->pw, n->wb);
    if (cudaDeviceSynchronize() != cudaSuccess) rc = IBM_E_CUDA;
  }
  if (rc) {
    delete n;
    return ufail(IBM_E_CUDA, "U-Net allocation failed");
  }
  *out = n;
  return IBM_OK;
}

void ibm_unet_destroy(ibm_unet* n) { delete n; }

long long ibm_unet_num_params(const ibm_unet* n) { return n ? (long long)n->nparam : 0; }

int ibm_unet_params(ibm_unet* n, float* host, long long count, int set) {
  if (!n || !host || count != (long long)n->nparam) return ufail(IBM_E_INVAL, "parameter count mismatch");
  if (set) {
    UCUDA(cudaMemcpy(n->pw, host, n->nparam * 4, cudaMemcpyHostToDevice));
    to_bf16(0, (long)n->nparam, n->pw, n->wb);
    n->wdirty = true;
    UCUDA(cudaMemset(n->m, 0, n->nparam * 4));
    UCUDA(cudaMemset(n->v, 0, n->nparam * 4));
    n->adam_t = 0;
    UCUDA(cudaDeviceSynchronize());
  } else {
    UCUDA(cudaMemcpy(host, n->pw, n->nparam * 4, cudaMemcpyDeviceToHost));
  }
  return IBM_OK;
}

int ibm_unet_grads(const ibm_unet* n, float* host, long long count) {
  if (!n || !host || count != (long long)n->nparam) return ufail(IBM_E_INVAL, "parameter count mismatch");
  UCUDA(cudaMemcpy(host, n->grad, n->nparam * 4, cudaMemcpyDeviceToHost));
  return IBM_OK;
}

}  // extern "C"

namespace ibm {
// kernels one forward pass launches: input packing, 15 convolutions, 3
// poolings, 3 upsamplings
int unet_forward_launches() { return 1 + 15 + 3 + 3; }
}  // namespace ibm

extern "C" {

int ibm_unet_forward(ibm_unet* n, const float* feat, int H, int W, float* out, void* stream) {
  if (!n || !feat || !out) return ufail(IBM_E_INVAL, "null argument");
  if (H < 8 || W < 8 || H % 8 || W % 8) return ufail(IBM_E_INVAL, "U-Net input sizes must be multiples of 8");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_acts(n, H, W);
  if (rc) return rc;
  if (conv_tc_failed()) return ufail(IBM_E_TIMEOUT, "a U-Net convolution gave up a bounded wait earlier");
  pack_input(s, (long)H * W, 4, 16, feat, n->lv[0].in);
  if (forward(n, s)) return IBM_E_CUDA;
  UCUDA(cudaMemcpy2DAsync(out, sizeof(float), n->outf, 16 * sizeof(float), sizeof(float), (size_t)H * W,
                          cudaMemcpyDeviceToDevice, s));
  UCUDA(cudaGetLastError());
  return IBM_OK;
}

int ibm_unet_train_step(ibm_unet* n, const float* feat, const float* target, int H, int W, float lr, int apply,
                        double* loss, void* stream) {
  if (!n || !feat || !target) return ufail(IBM_E_INVAL, "null argument");
  if (H < 8 || W < 8 || H % 8 || W % 8) return ufail(IBM_E_INVAL, "U-Net input sizes must be multiples of 8");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_acts(n, H, W);
  if (rc) return rc;
  pack_input(s, (long)H * W, 4, 16, feat, n->lv[0].in);
  if (forward(n, s)) return IBM_E_CUDA;
  UCUDA(cudaMemsetAsync(n->grad, 0, n->nparam * 4, s));
  UCUDA(cudaMemsetAsync(n->loss_d, 0, 8, s));
  const long npix = (long)H * W;
  mse(s, npix, n->outf, 16, target, nullptr, 1.f / (float)npix, n->gout, 16, n->loss_d);
  if (backward(n, s)) return IBM_E_CUDA;
  if (apply) {
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)n->adam_t)), c2 = 1.f / (1.f - std::pow(b2, (float)n->adam_t));
    adam(s, (long)n->nparam, n->pw, n->grad, n->m, n->v, n->wb, lr, b1, b2, 1e-8f, c1, c2);
    n->wdirty = true;
  }
  double l = 0.0;
  UCUDA(cudaMemcpyAsync(&l, n->loss_d, 8, cudaMemcpyDeviceToHost, s));
  UCUDA(cudaStreamSynchronize(s));
  if (conv_tc_failed()) return ufail(IBM_E_TIMEOUT, "a U-Net convolution gave up a bounded wait");
  if (loss) *loss = l;
  UCUDA(cudaGetLastError());
  return IBM_OK;
}

}  // extern "C"
