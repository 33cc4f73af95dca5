// Red-black Gauss-Seidel SOR kernels ("modified Gauss-Seidel SOR with
// red-black tagging", arXiv 2402.17337 Sec. 2.2 and Sec. 3.1) for the
// pressure Poisson equation and the Crank-Nicolson velocity systems, plus
// their residual infinity norms.
//
// Red cells have (i + j) even.  Within one colour no update reads another
// update of the same colour, so every half-sweep is race-free.
//
// Arithmetic recipe (shared with the CPU oracle so that iteration counts are
// decided identically): 5-point sums and Laplacians are fma chains in the
// order E, W, N, S; the library is built with --fmad=false so that no other
// multiply-add is contracted.  Norms are
// reduced on the IEEE bit pattern of |r|: for non-negative doubles the
// unsigned order is the numeric order, NaN patterns sort above +Inf, and the
// result does not depend on the reduction order.
#include "ibm_internal.h"

namespace ibm {

namespace {

constexpr int TBX = 32, TBY = 8;

__device__ inline void warp_block_max(unsigned long long v, unsigned long long* dst) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  __shared__ unsigned long long wm[32];
  int t = threadIdx.x + threadIdx.y * blockDim.x;
  int lane = t & 31, warp = t >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) wm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? wm[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (lane == 0 && v) atomicMax(dst, v);
  }
}

__device__ inline unsigned long long abs_bits(double r) {
  return (unsigned long long)__double_as_longlong(fabs(r));
}

// ----------------------------------------------------------------- Poisson

// L_p phi = b:  phi_P <- phi_P + omega (GS_P - phi_P),
// GS_P = (sum_nb a_nb phi_nb - b_P) / sum_nb a_nb.
__global__ void k_poisson_half(Geo g, double* __restrict__ phi, const double* __restrict__ b,
                               const double* __restrict__ invd, int colour, double omega) {
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((colour + j) & 1);
  if (j >= g.ny || i >= g.nx) return;
  const int P = g.pitch;
  size_t c = at(i, j, P);
  double s = g.pE[i] * phi[c + 1];
  s = fma(g.pW[i], phi[c - 1], s);
  s = fma(g.pN[j], phi[c + P], s);
  s = fma(g.pS[j], phi[c - P], s);
  double gs = (s - b[c]) * invd[c];
  double x = phi[c];
  phi[c] = fma(omega, gs - x, x);
}

// sum_nb a_nb (x_nb - x_P) in the order E, W, N, S
__device__ inline double lap5(double aE, double aW, double aN, double aS, double xE, double xW, double xN,
                              double xS, double c) {
  double L = aE * (xE - c);
  L = fma(aW, xW - c, L);
  L = fma(aN, xN - c, L);
  L = fma(aS, xS - c, L);
  return L;
}

__global__ void k_poisson_res(Geo g, const double* __restrict__ phi, const double* __restrict__ b,
                              unsigned long long* res_bits) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned long long bits = 0ull;
  if (i < g.nx && j < g.ny) {
    const int P = g.pitch;
    size_t c = at(i, j, P);
    double L = lap5(g.pE[i], g.pW[i], g.pN[j], g.pS[j], phi[c + 1], phi[c - 1], phi[c + P], phi[c - P], phi[c]);
    bits = abs_bits(b[c] - L);
  }
  warp_block_max(bits, res_bits);
}

__global__ void k_poisson_res2(Geo g, const double* __restrict__ pa, const double* __restrict__ pb,
                               const double* __restrict__ b, unsigned long long* bits_a, unsigned long long* bits_b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned long long ba = 0ull, bb = 0ull;
  if (i < g.nx && j < g.ny) {
    const int P = g.pitch;
    size_t c = at(i, j, P);
    const double La = lap5(g.pE[i], g.pW[i], g.pN[j], g.pS[j], pa[c + 1], pa[c - 1], pa[c + P], pa[c - P], pa[c]);
    const double Lb = lap5(g.pE[i], g.pW[i], g.pN[j], g.pS[j], pb[c + 1], pb[c - 1], pb[c + P], pb[c - P], pb[c]);
    ba = abs_bits(b[c] - La);
    bb = abs_bits(b[c] - Lb);
  }
  warp_block_max(ba, bits_a);
  __syncthreads();  // the reduction's shared slots are reused
  warp_block_max(bb, bits_b);
}

__global__ void k_bmax(Geo g, const double* __restrict__ b, unsigned long long* bits_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned long long bits = 0ull;
  if (i < g.nx && j < g.ny) bits = abs_bits(b[at(i, j, g.pitch)]);
  warp_block_max(bits, bits_out);
}

// ---------------------------------------------------- velocity (Helmholtz)

struct HelmCoef {
  const double *E, *W, *N, *S;
  int ilo, ihi, jlo, jhi;
};

__device__ inline HelmCoef helm_coef(const Geo& g, int grid) {
  HelmCoef h;
  if (grid == 0) {
    h.E = g.uE; h.W = g.uW; h.N = g.uN; h.S = g.uS;
    h.ilo = 1; h.ihi = g.nx - 1; h.jlo = 0; h.jhi = g.ny - 1;
  } else {
    h.E = g.vE; h.W = g.vW; h.N = g.vN; h.S = g.vS;
    h.ilo = 0; h.ihi = g.nx - 1; h.jlo = 1; h.jhi = g.ny - 1;
  }
  return h;
}

__device__ inline long opp_offset(int dir, int P) {
  // forcing node whose wall lies in direction dir takes the node on the far side
  return dir == 0 ? 1 : dir == 1 ? -1 : dir == 2 ? (long)P : -(long)P;
}

// (I - beta L) x = R on fluid nodes (SOR); forcing nodes x = Ub + alpha (x_opp - Ub);
// solid nodes keep x = Ub.
__global__ void k_helm_half(Geo g, int grid, double* __restrict__ x, const double* __restrict__ R,
                            const double* __restrict__ invd, Band B, const uint8_t* __restrict__ fl,
                            const double* __restrict__ al, int colour, double omega, double beta, double Ub) {
  HelmCoef h = helm_coef(g, grid);
  int j = blockIdx.y * blockDim.y + threadIdx.y + h.jlo;
  int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((colour + j) & 1);
  if (j > h.jhi || i > h.ihi || i < h.ilo) return;
  const int P = g.pitch;
  size_t c = at(i, j, P);
  int bi = i - B.i0, bj = j - B.j0;
  if (bi >= 0 && bj >= 0 && bi < B.w && bj < B.h) {
    uint8_t f = fl[bj * B.w + bi];
    int kind = f & 3;
    if (kind == K_SOLID) return;
    if (kind == K_FORCE) {
      double a = al[bj * B.w + bi];
      double xo = a != 0.0 ? x[c + opp_offset(f >> 2, P)] : Ub;
      x[c] = fma(a, xo - Ub, Ub);
      return;
    }
  }
  double s = h.E[i] * x[c + 1];
  s = fma(h.W[i], x[c - 1], s);
  s = fma(h.N[j], x[c + P], s);
  s = fma(h.S[j], x[c - P], s);
  double gs = fma(beta, s, R[c]) * invd[c];
  double xp = x[c];
  x[c] = fma(omega, gs - xp, xp);
}

__global__ void k_helm_res(Geo g, int grid, const double* __restrict__ x, const double* __restrict__ R, Band B,
                           const uint8_t* __restrict__ fl, const double* __restrict__ al, double beta, double Ub,
                           unsigned long long* res_bits) {
  HelmCoef h = helm_coef(g, grid);
  int i = blockIdx.x * blockDim.x + threadIdx.x + h.ilo, j = blockIdx.y * blockDim.y + threadIdx.y + h.jlo;
  unsigned long long bits = 0ull;
  if (i <= h.ihi && j <= h.jhi) {
    const int P = g.pitch;
    size_t c = at(i, j, P);
    int bi = i - B.i0, bj = j - B.j0;
    int kind = K_FLUID;
    uint8_t f = 0;
    if (bi >= 0 && bj >= 0 && bi < B.w && bj < B.h) {
      f = fl[bj * B.w + bi];
      kind = f & 3;
    }
    double r;
    double xp = x[c];
    if (kind == K_SOLID) {
      r = Ub - xp;
    } else if (kind == K_FORCE) {
      double a = al[bj * B.w + bi];
      double xo = a != 0.0 ? x[c + opp_offset(f >> 2, P)] : Ub;
      r = fma(a, xo - Ub, Ub) - xp;
    } else {
      double L = lap5(h.E[i], h.W[i], h.N[j], h.S[j], x[c + 1], x[c - 1], x[c + P], x[c - P], xp);
      r = R[c] - fma(-beta, L, xp);
    }
    bits = abs_bits(r);
  }
  warp_block_max(bits, res_bits);
}

// phi -= phi at the gauge cell (value captured beforehand in sc->phi_ref)
__global__ void k_shift(Geo g, double* __restrict__ phi, const DevScalars* __restrict__ sc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i < g.nx && j < g.ny) phi[at(i, j, g.pitch)] -= sc->phi_ref;
}

// x = pseudo-random values in [-1, 1) on the interior cells (an integer
// hash of the cell index; any field with all modes present serves)
__global__ void k_fill_hash(Geo g, double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  unsigned h = (unsigned)i * 0x9E3779B1u ^ ((unsigned)j + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  x[at(i, j, g.pitch)] = (double)(h >> 8) * (1.0 / 8388608.0) - 1.0;
}

inline dim3 grid2(int nx, int ny) { return dim3((nx + TBX - 1) / TBX, (ny + TBY - 1) / TBY); }

}  // namespace

void launch_fill_hash(cudaStream_t s, const Geo& g, double* x) {
  k_fill_hash<<<grid2(g.nx, g.ny), dim3(TBX, TBY), 0, s>>>(g, x);
}

void launch_shift(cudaStream_t s, const Geo& g, double* phi, const DevScalars* sc) {
  k_shift<<<grid2(g.nx, g.ny), dim3(TBX, TBY), 0, s>>>(g, phi, sc);
}

void launch_poisson_half(cudaStream_t s, const Geo& g, double* phi, const double* b, const double* invd,
                         int colour, double omega) {
  k_poisson_half<<<grid2((g.nx + 1) / 2, g.ny), dim3(TBX, TBY), 0, s>>>(g, phi, b, invd, colour, omega);
}

void launch_poisson_res(cudaStream_t s, const Geo& g, const double* phi, const double* b,
                        unsigned long long* res_bits) {
  k_poisson_res<<<grid2(g.nx, g.ny), dim3(TBX, TBY), 0, s>>>(g, phi, b, res_bits);
}

void launch_poisson_res2(cudaStream_t s, const Geo& g, const double* phi_a, const double* phi_b, const double* b,
                         unsigned long long* bits_a, unsigned long long* bits_b) {
  k_poisson_res2<<<grid2(g.nx, g.ny), dim3(TBX, TBY), 0, s>>>(g, phi_a, phi_b, b, bits_a, bits_b);
}

void launch_bmax(cudaStream_t s, const Geo& g, const double* b, unsigned long long* bits) {
  k_bmax<<<grid2(g.nx, g.ny), dim3(TBX, TBY), 0, s>>>(g, b, bits);
}

void launch_helm_half(cudaStream_t s, const Geo& g, int grid, double* x, const double* R, const double* invd,
                      const Band& band, const uint8_t* fl, const double* al, int colour, double omega,
                      double beta, double Ub) {
  int ni = grid == 0 ? g.nx + 1 : g.nx, nj = grid == 0 ? g.ny : g.ny - 1;
  k_helm_half<<<grid2((ni + 1) / 2, nj), dim3(TBX, TBY), 0, s>>>(g, grid, x, R, invd, band, fl, al, colour, omega,
                                                                 beta, Ub);
}

void launch_helm_res(cudaStream_t s, const Geo& g, int grid, const double* x, const double* R, const Band& band,
                     const uint8_t* fl, const double* al, double beta, double Ub, unsigned long long* res_bits) {
  int ni = grid == 0 ? g.nx - 1 : g.nx, nj = grid == 0 ? g.ny : g.ny - 1;
  k_helm_res<<<grid2(ni, nj), dim3(TBX, TBY), 0, s>>>(g, grid, x, R, band, fl, al, beta, Ub, res_bits);
}

// ---- velocity systems in FP32 sweeps inside FP64 defect correction
// (precision >= 1).  The FP64 residual r = R - A x of the system above
// (forcing rows: U_b + alpha (x_opp - U_b) - x; solid rows: U_b - x) is
// stored in FP32, FP32 red-black Gauss-Seidel sweeps solve the correction
// equation A d = r from d = 0, with the homogeneous forms of the side
// conditions (forcing rows d = r + alpha d_opp, solid rows d = r), and the
// FP64 update x += d follows.  Same stopping rule as the FP64 solve.
namespace {

__device__ __forceinline__ void helm_dc_res_body(Geo g, int grid, const double* __restrict__ x, const double* __restrict__ R, Band B,
                              const uint8_t* __restrict__ fl, const double* __restrict__ al, double beta, double Ub,
                              float* __restrict__ r32, unsigned long long* res_bits, int bx, int by) {
  HelmCoef h = helm_coef(g, grid);
  int i = bx * blockDim.x + threadIdx.x + h.ilo, j = by * blockDim.y + threadIdx.y + h.jlo;
  unsigned long long bits = 0ull;
  if (i <= h.ihi && j <= h.jhi) {
    const int P = g.pitch;
    size_t c = at(i, j, P);
    int bi = i - B.i0, bj = j - B.j0;
    int kind = K_FLUID;
    uint8_t f = 0;
    if (bi >= 0 && bj >= 0 && bi < B.w && bj < B.h) {
      f = fl[bj * B.w + bi];
      kind = f & 3;
    }
    double r;
    double xp = x[c];
    if (kind == K_SOLID) {
      r = Ub - xp;
    } else if (kind == K_FORCE) {
      double a = al[bj * B.w + bi];
      double xo = a != 0.0 ? x[c + opp_offset(f >> 2, P)] : Ub;
      r = fma(a, xo - Ub, Ub) - xp;
    } else {
      double L = lap5(h.E[i], h.W[i], h.N[j], h.S[j], x[c + 1], x[c - 1], x[c + P], x[c - P], xp);
      r = R[c] - fma(-beta, L, xp);
    }
    r32[c] = (float)r;
    bits = abs_bits(r);
  }
  warp_block_max(bits, res_bits);
}
__global__ void k_helm_dc_res(Geo g, int grid, const double* __restrict__ x, const double* __restrict__ R, Band B,
                              const uint8_t* __restrict__ fl, const double* __restrict__ al, double beta, double Ub,
                              float* __restrict__ r32, unsigned long long* res_bits) {
  helm_dc_res_body(g, grid, x, R, B, fl, al, beta, Ub, r32, res_bits, blockIdx.x, blockIdx.y);
}

__device__ __forceinline__ void helm32_half_body(Geo g, HelmF32 h32, int grid, float* __restrict__ d, const float* __restrict__ r,
                              const float* __restrict__ invd, Band B, const uint8_t* __restrict__ fl,
                              const double* __restrict__ al, int colour, float omega, float beta, int bx, int by) {
  HelmCoef h = helm_coef(g, grid);
  const float *E = grid == 0 ? h32.uE : h32.vE, *W = grid == 0 ? h32.uW : h32.vW;
  const float *N = grid == 0 ? h32.uN : h32.vN, *S = grid == 0 ? h32.uS : h32.vS;
  int j = by * blockDim.y + threadIdx.y + h.jlo;
  int i = 2 * (bx * blockDim.x + threadIdx.x) + ((colour + j) & 1);
  if (j > h.jhi || i > h.ihi || i < h.ilo) return;
  const int P = g.pitch;
  size_t c = at(i, j, P);
  int bi = i - B.i0, bj = j - B.j0;
  if (bi >= 0 && bj >= 0 && bi < B.w && bj < B.h) {
    uint8_t f = fl[bj * B.w + bi];
    int kind = f & 3;
    if (kind == K_SOLID) {
      d[c] = r[c];
      return;
    }
    if (kind == K_FORCE) {
      float a = (float)al[bj * B.w + bi];
      float dop = a != 0.f ? d[c + opp_offset(f >> 2, P)] : 0.f;
      d[c] = fmaf(a, dop, r[c]);
      return;
    }
  }
  float sum = E[i] * d[c + 1];
  sum = fmaf(W[i], d[c - 1], sum);
  sum = fmaf(N[j], d[c + P], sum);
  sum = fmaf(S[j], d[c - P], sum);
  float gs = fmaf(beta, sum, r[c]) * invd[c];
  float dp = d[c];
  d[c] = fmaf(omega, gs - dp, dp);
}
__global__ void k_helm32_half(Geo g, HelmF32 h32, int grid, float* __restrict__ d, const float* __restrict__ r,
                              const float* __restrict__ invd, Band B, const uint8_t* __restrict__ fl,
                              const double* __restrict__ al, int colour, float omega, float beta) {
  // launched as a programmatic dependent of the previous half-sweep: nothing
  // is read before that launch has completed and its writes are visible
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  helm32_half_body(g, h32, grid, d, r, invd, B, fl, al, colour, omega, beta, blockIdx.x, blockIdx.y);
}

__device__ __forceinline__ void helm_add_body(Geo g, int grid, double* __restrict__ x, const float* __restrict__ d, int bx, int by) {
  HelmCoef h = helm_coef(g, grid);
  int i = bx * blockDim.x + threadIdx.x + h.ilo, j = by * blockDim.y + threadIdx.y + h.jlo;
  if (i > h.ihi || j > h.jhi) return;
  size_t c = at(i, j, g.pitch);
  x[c] += (double)d[c];
}
__global__ void k_helm_add(Geo g, int grid, double* __restrict__ x, const float* __restrict__ d) {
  helm_add_body(g, grid, x, d, blockIdx.x, blockIdx.y);
}

// ---- batched forms over the active cases act[0..na) of a batch (block b
// belongs to active slot k with first[k] <= b < first[k+1]; the grids are
// those of the single-case launches below)
__device__ inline int slot_of(const int* __restrict__ first, int na, int b) {
  int lo = 0, hi = na - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// unknown nodes of grid 0 (u) or 1 (v) along x
__device__ inline int helm_ni(const Geo& g, int grid) { return grid == 0 ? g.nx - 1 : g.nx; }

__global__ void k_helm_dc_res_batch(const StepCase* __restrict__ cs, const int* __restrict__ act,
                                    const int* __restrict__ first, int na, int grid,
                                    unsigned long long* __restrict__ bits) {
  const int k = slot_of(first, na, blockIdx.x);
  const StepCase& s = cs[act[k]];
  const int t = blockIdx.x - first[k], bxn = (helm_ni(s.g, grid) + TBX - 1) / TBX;
  helm_dc_res_body(s.g, grid, grid == 0 ? s.uh : s.vh, grid == 0 ? s.Ru : s.Rv, s.band, grid == 0 ? s.fu : s.fv,
                   grid == 0 ? s.au : s.av, s.beta, grid == 0 ? 0.0 : s.vb, s.hr32, bits + k, t % bxn, t / bxn);
}

// d = 0 over a case's pitched field (64 blocks of 256 threads per case)
__global__ void k_helm_zero_batch(const StepCase* __restrict__ cs, const int* __restrict__ act) {
  const StepCase& s = cs[act[blockIdx.x / 64]];
  for (int e = (blockIdx.x % 64) * 256 + threadIdx.x; e < s.nelem; e += 64 * 256) s.hd32[e] = 0.f;
}

__global__ void k_helm32_half_batch(const StepCase* __restrict__ cs, const int* __restrict__ act,
                                    const int* __restrict__ first, int na, int grid, int colour) {
  const int k = slot_of(first, na, blockIdx.x);
  const StepCase& s = cs[act[k]];
  const int t = blockIdx.x - first[k], bxn = ((helm_ni(s.g, grid) + 1) / 2 + TBX - 1) / TBX;
  helm32_half_body(s.g, s.h32, grid, s.hd32, s.hr32, grid == 0 ? s.hinv_u : s.hinv_v, s.band,
                   grid == 0 ? s.fu : s.fv, grid == 0 ? s.au : s.av, colour, s.omega_h, (float)s.beta, t % bxn,
                   t / bxn);
}

__global__ void k_helm_add_batch(const StepCase* __restrict__ cs, const int* __restrict__ act,
                                 const int* __restrict__ first, int na, int grid) {
  const int k = slot_of(first, na, blockIdx.x);
  const StepCase& s = cs[act[k]];
  const int t = blockIdx.x - first[k], bxn = (helm_ni(s.g, grid) + TBX - 1) / TBX;
  helm_add_body(s.g, grid, grid == 0 ? s.uh : s.vh, s.hd32, t % bxn, t / bxn);
}

}  // namespace

int helm_batch_blocks(const StepCase& c, int grid, int half) {
  const int ni = grid == 0 ? c.g.nx - 1 : c.g.nx, nj = grid == 0 ? c.g.ny : c.g.ny - 1;
  const int cols = half ? (ni + 1) / 2 : ni;
  return ((cols + TBX - 1) / TBX) * ((nj + TBY - 1) / TBY);
}

void launch_helm_dc_res_batch(cudaStream_t s, const StepCase* cs, const int* act, const int* first, int na,
                              int total, int grid, unsigned long long* bits) {
  k_helm_dc_res_batch<<<total, dim3(TBX, TBY), 0, s>>>(cs, act, first, na, grid, bits);
}

void launch_helm_zero_batch(cudaStream_t s, const StepCase* cs, const int* act, int na) {
  k_helm_zero_batch<<<na * 64, 256, 0, s>>>(cs, act);
}

void launch_helm32_half_batch(cudaStream_t s, const StepCase* cs, const int* act, const int* first, int na,
                              int total, int grid, int colour) {
  k_helm32_half_batch<<<total, dim3(TBX, TBY), 0, s>>>(cs, act, first, na, grid, colour);
}

void launch_helm_add_batch(cudaStream_t s, const StepCase* cs, const int* act, const int* first, int na,
                           int total, int grid) {
  k_helm_add_batch<<<total, dim3(TBX, TBY), 0, s>>>(cs, act, first, na, grid);
}

void launch_helm_dc_res(cudaStream_t s, const Geo& g, int grid, const double* x, const double* R, const Band& band,
                        const uint8_t* fl, const double* al, double beta, double Ub, float* r32,
                        unsigned long long* res_bits) {
  int ni = grid == 0 ? g.nx - 1 : g.nx, nj = grid == 0 ? g.ny : g.ny - 1;
  k_helm_dc_res<<<grid2(ni, nj), dim3(TBX, TBY), 0, s>>>(g, grid, x, R, band, fl, al, beta, Ub, r32, res_bits);
}

void launch_helm32_half(cudaStream_t s, const Geo& g, const HelmF32& h32, int grid, float* d, const float* r,
                        const float* invd, const Band& band, const uint8_t* fl, const double* al, int colour,
                        float omega, float beta) {
  int ni = grid == 0 ? g.nx - 1 : g.nx, nj = grid == 0 ? g.ny : g.ny - 1;
  cudaLaunchConfig_t lc{};
  lc.gridDim = grid2((ni + 1) / 2, nj);
  lc.blockDim = dim3(TBX, TBY);
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaLaunchKernelEx(&lc, k_helm32_half, g, h32, grid, d, r, invd, band, fl, al, colour, omega, beta);
}

void launch_helm_add(cudaStream_t s, const Geo& g, int grid, double* x, const float* d) {
  int ni = grid == 0 ? g.nx - 1 : g.nx, nj = grid == 0 ? g.ny : g.ny - 1;
  k_helm_add<<<grid2(ni, nj), dim3(TBX, TBY), 0, s>>>(g, grid, x, d);
}

}  // namespace ibm
