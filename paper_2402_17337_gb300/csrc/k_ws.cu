// Learned warm start of the pressure solve: features for the U-Net, the
// prolongation of its prediction onto the pressure increment, and the
// training targets.
//
// The network works on the grid coarsened 2x in each direction (coarse cell
// (I, J) = fine cells 2I..2I+1 x 2J..2J+1): SOR removes the rough part of an
// error in a few sweeps, so only the smooth part of the increment is worth
// predicting, and the coarse grid doubles the network's reach.  Features of a
// coarse cell (averages over its four fine cells):
//   0  r0 = b - L_p phi^n   (initial residual of the solve)
//   1  b                    (right-hand side)
//   2  fraction of body cells
//   3  p^n                  (pressure)
// each divided by its infinity norm over the grid (scale invariance).  The
// network predicts (phi^{n+1} - phi^n) / (s0 c_T), s0 = ||r0||_inf, c_T a
// constant of the trained model.
#include "ibm_internal.h"

namespace ibm {

namespace {

// block-wide maximum of |v| (IEEE bit patterns of non-negative doubles order
// like the values), one atomic per block
__device__ inline void block_max_abs(double v, unsigned long long* dst) {
  unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, b, o);
    b = w > b ? w : b;
  }
  __shared__ unsigned long long wm[32];
  const int t = threadIdx.x + threadIdx.y * blockDim.x, lane = t & 31, warp = t >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  __syncthreads();  // wm may still be read by a previous call
  if (lane == 0) wm[warp] = b;
  __syncthreads();
  if (warp == 0) {
    b = lane < nw ? wm[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w = __shfl_xor_sync(0xffffffffu, b, o);
      b = w > b ? w : b;
    }
    if (lane == 0 && b) atomicMax(dst, b);
  }
}

__device__ inline double lap_p(const Geo& g, const double* f, int i, int j) {
  const int P = g.pitch;
  size_t c = at(i, j, P);
  double x = f[c];
  double L = g.pE[i] * (f[c + 1] - x);
  L = fma(g.pW[i], f[c - 1] - x, L);
  L = fma(g.pN[j], f[c + P] - x, L);
  L = fma(g.pS[j], f[c - P] - x, L);
  return L;
}

// raw coarse features and their maxima (ws_max[0..3], bit patterns)
__global__ void k_ws_features(Geo g, int Hc, int Wc, const double* __restrict__ b, const double* __restrict__ phi,
                              const double* __restrict__ p, Band B, const uint8_t* __restrict__ fc,
                              float* __restrict__ feat, unsigned long long* __restrict__ ws_max) {
  int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  const bool in = I < Wc && J < Hc;
  double r0 = 0.0, bb = 0.0, body = 0.0, pp = 0.0;
  for (int a = 0; a < 2 && in; ++a)
    for (int c2 = 0; c2 < 2; ++c2) {
      int i = 2 * I + a, j = 2 * J + c2;
      size_t c = at(i, j, g.pitch);
      r0 += b[c] - lap_p(g, phi, i, j);
      bb += b[c];
      pp += p[c];
      int bi = i - B.i0, bj = j - B.j0;
      if (bi >= 0 && bj >= 0 && bi < B.w && bj < B.h && fc[bj * B.w + bi]) body += 1.0;
    }
  if (in) {
    float* f = feat + ((size_t)J * Wc + I) * 4;
    f[0] = (float)(0.25 * r0);
    f[1] = (float)(0.25 * bb);
    f[2] = (float)(0.25 * body);
    f[3] = (float)(0.25 * pp);
  }
  block_max_abs(0.25 * r0, &ws_max[0]);
  block_max_abs(0.25 * bb, &ws_max[1]);
  block_max_abs(0.25 * pp, &ws_max[3]);
}

__device__ inline double bits2d(unsigned long long u) { return __longlong_as_double((long long)u); }

__global__ void k_ws_normalize(long n, float* __restrict__ feat, const unsigned long long* __restrict__ ws_max) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    int ch = (int)(k & 3);
    if (ch == 2) continue;
    double s = bits2d(ws_max[ch]);
    feat[k] = s > 0.0 ? (float)(feat[k] / s) : 0.f;
  }
}

// phi (fine) += s0 * cT * out (coarse), piecewise constant over each coarse cell
__global__ void k_ws_apply(Geo g, int Hc, int Wc, const float* __restrict__ out, double cT,
                           const unsigned long long* __restrict__ ws_max, double* __restrict__ phi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= 2 * Wc || j >= 2 * Hc) return;
  const double s0 = bits2d(ws_max[0]);
  phi[at(i, j, g.pitch)] += s0 * cT * (double)out[(size_t)(j >> 1) * Wc + (i >> 1)];
}

// training target: coarse average of (phi_new - phi_ref) - phi_old, over s0 cT
__global__ void k_ws_target(Geo g, int Hc, int Wc, const double* __restrict__ phi_new,
                            const double* __restrict__ phi_old, const DevScalars* __restrict__ sc, double cT,
                            const unsigned long long* __restrict__ ws_max, float* __restrict__ target) {
  int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= Wc || J >= Hc) return;
  const double ref = sc->phi_ref, s0 = bits2d(ws_max[0]);
  double d = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int c2 = 0; c2 < 2; ++c2) {
      size_t c = at(2 * I + a, 2 * J + c2, g.pitch);
      d += (phi_new[c] - ref) - phi_old[c];
    }
  target[(size_t)J * Wc + I] = s0 > 0.0 ? (float)(0.25 * d / (s0 * cT)) : 0.f;
}

// Linear extrapolation of the pressure increment in time: phi <- 2 phi^n -
// phi^{n-1}, and phi_prev <- phi^n for the next step.
__global__ void k_extrapolate(Geo g, double* __restrict__ phi, double* __restrict__ phi_prev) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const size_t c = at(i, j, g.pitch);
  const double a = phi[c];
  phi[c] = 2.0 * a - phi_prev[c];
  phi_prev[c] = a;
}

// ---- the U-Net as the coarse level of a two-level preconditioner (FCG,
// precision 2).  Channel 0 of the features is the level-1 residual (the
// volume-weighted restriction of the fine residual, colour-split layout)
// over its infinity norm s; channels 1-3 keep the values taken at the start
// of the solve.  The network's output times s c_T is the level-1 correction.
__global__ void k_nnp_features(const MgLevel C, float* __restrict__ feat, unsigned long long* __restrict__ smax) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  float v = 0.f;
  if (I < C.g.nx && J < C.g.ny) {
    v = C.r[rb_at(I, J, C.g.ny, C.g.pk)];
    feat[((size_t)J * C.g.nx + I) * 4] = v;
  }
  block_max_abs((double)v, smax);
}

__global__ void k_nnp_normalize(long npix, float* __restrict__ feat, const unsigned long long* __restrict__ smax) {
  const double s = bits2d(*smax);
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < npix; k += (long)gridDim.x * blockDim.x)
    feat[4 * k] = s > 0.0 ? (float)(feat[4 * k] / s) : 0.f;
}

__global__ void k_nnp_correction(const MgLevel C, const float* __restrict__ out, double cT,
                                 const unsigned long long* __restrict__ smax, float* __restrict__ e) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= C.g.nx || J >= C.g.ny) return;
  const double s = bits2d(*smax);
  e[rb_at(I, J, C.g.ny, C.g.pk)] = (float)(s * cT * (double)out[(size_t)J * C.g.nx + I]);
}

}  // namespace

void launch_nnp_features(cudaStream_t s, const MgLevel& C, float* feat, unsigned long long* smax) {
  cudaMemsetAsync(smax, 0, sizeof(unsigned long long), s);
  dim3 blk(32, 8), grd((C.g.nx + 31) / 32, (C.g.ny + 7) / 8);
  k_nnp_features<<<grd, blk, 0, s>>>(C, feat, smax);
  const long npix = (long)C.g.nx * C.g.ny;
  k_nnp_normalize<<<(unsigned)((npix + 255) / 256 > 1216 ? 1216 : (npix + 255) / 256), 256, 0, s>>>(npix, feat, smax);
}

void launch_nnp_correction(cudaStream_t s, const MgLevel& C, const float* out, double cT,
                           const unsigned long long* smax, float* e) {
  dim3 blk(32, 8), grd((C.g.nx + 31) / 32, (C.g.ny + 7) / 8);
  k_nnp_correction<<<grd, blk, 0, s>>>(C, out, cT, smax, e);
}

void launch_extrapolate(cudaStream_t s, const Geo& g, double* phi, double* phi_prev) {
  dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  k_extrapolate<<<grd, blk, 0, s>>>(g, phi, phi_prev);
}

void launch_ws_features(cudaStream_t s, const Geo& g, int Hc, int Wc, const double* b, const double* phi,
                        const double* p, const Band& band, const uint8_t* fc, float* feat,
                        unsigned long long* ws_max) {
  cudaMemsetAsync(ws_max, 0, 4 * sizeof(unsigned long long), s);
  dim3 blk(32, 8), grd((Wc + 31) / 32, (Hc + 7) / 8);
  k_ws_features<<<grd, blk, 0, s>>>(g, Hc, Wc, b, phi, p, band, fc, feat, ws_max);
  long n = (long)Hc * Wc * 4;
  k_ws_normalize<<<(unsigned)((n + 255) / 256 > 4096 ? 4096 : (n + 255) / 256), 256, 0, s>>>(n, feat, ws_max);
}

void launch_ws_apply(cudaStream_t s, const Geo& g, int Hc, int Wc, const float* out, double cT,
                     const unsigned long long* ws_max, double* phi) {
  dim3 blk(32, 8), grd((2 * Wc + 31) / 32, (2 * Hc + 7) / 8);
  k_ws_apply<<<grd, blk, 0, s>>>(g, Hc, Wc, out, cT, ws_max, phi);
}

void launch_ws_target(cudaStream_t s, const Geo& g, int Hc, int Wc, const double* phi_new, const double* phi_old,
                      const DevScalars* sc, double cT, const unsigned long long* ws_max, float* target) {
  dim3 blk(32, 8), grd((Wc + 31) / 32, (Hc + 7) / 8);
  k_ws_target<<<grd, blk, 0, s>>>(g, Hc, Wc, phi_new, phi_old, sc, cT, ws_max, target);
}

}  // namespace ibm
