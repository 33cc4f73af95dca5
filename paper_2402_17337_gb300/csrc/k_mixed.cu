// Pressure solve in FP32 sweeps inside FP64 defect correction.
//
// The red-black SOR of the pressure equation (arXiv 2402.17337, Sec. 2.2,
// Sec. 3.1) is split into
//   outer (FP64):  phi <- phi + e,  r = b - L_p phi,  ||r||_inf  (k_dc_residual)
//   inner (FP32):  red-black SOR sweeps on L_p e = r from e = 0   (k_sor32_tile)
// so the residual, the pressure update and the norm stay in FP64 while the
// sweeps, which carry the work, run at the FP32 rate.  Each inner launch
// performs K half-sweeps on a shared-memory tile that carries a halo of K
// cells, so the tile is read and written once for K/2 full sweeps; the halo
// cells are recomputed by the neighbouring tiles (temporal blocking).  The
// inner iterates are exactly those of red-black SOR applied to the
// correction equation.
#include "ibm_internal.h"

namespace ibm {

namespace {

__device__ inline unsigned long long abs_bits(double r) {
  return (unsigned long long)__double_as_longlong(fabs(r));
}

__device__ inline void block_max_bits(unsigned long long v, unsigned long long* dst) {
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

// FP64 update and residual.  With add_e the increment e of the last inner
// solve is added (phi_out = phi_in + e, neighbours included on the fly, so
// phi_out must differ from phi_in); r is stored in FP32 as the next inner
// right-hand side.
__global__ void k_dc_residual(Geo g, const double* __restrict__ phi_in, double* __restrict__ phi_out,
                              const float* __restrict__ e, const double* __restrict__ b, float* __restrict__ r32,
                              int add_e, unsigned long long* __restrict__ res_bits) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned long long bits = 0ull;
  if (i < g.nx && j < g.ny) {
    const int P = g.pitch;
    size_t c = at(i, j, P);
    double fP = phi_in[c], fE = phi_in[c + 1], fW = phi_in[c - 1], fN = phi_in[c + P], fS = phi_in[c - P];
    if (add_e) {
      fP += (double)e[c];
      fE += (double)e[c + 1];
      fW += (double)e[c - 1];
      fN += (double)e[c + P];
      fS += (double)e[c - P];
      phi_out[c] = fP;
    }
    double L = g.pE[i] * (fE - fP);
    L = fma(g.pW[i], fW - fP, L);
    L = fma(g.pN[j], fN - fP, L);
    L = fma(g.pS[j], fS - fP, L);
    double r = b[c] - L;
    r32[c] = (float)r;
    bits = abs_bits(r);
  }
  block_max_bits(bits, res_bits);
}

// K half-sweeps of FP32 red-black SOR on L_p e = r over a TX x TY tile.
// Loaded region: the tile plus a halo of K cells; after half-sweep h the
// values are exact for cells at least h+1 cells inside the loaded region, so
// after K half-sweeps the tile itself is exact.  Cells outside the domain
// are loaded as zero and never updated; boundary cells have zero
// coefficients towards them (homogeneous Neumann).
template <int TX, int TY, int K>
__global__ void __launch_bounds__(256) k_sor32_tile(const Geo32 g, float* __restrict__ e, const float* __restrict__ r,
                                                    const float* __restrict__ invd, float omega, int zero_init) {
  constexpr int H = K, LX = TX + 2 * H, LY = TY + 2 * H;
  extern __shared__ float smem[];
  float* se = smem;                 // LY x LX
  float* sr = se + LX * LY;         // LY x LX
  float* sd = sr + LX * LY;         // LY x LX
  float* cE = sd + LX * LY;         // LX
  float* cW = cE + LX;              // LX
  float* cN = cW + LX;              // LY
  float* cS = cN + LY;              // LY
  const int nx = g.nx, ny = g.ny, P = g.pitch;
  const int gx0 = blockIdx.x * TX - H, gy0 = blockIdx.y * TY - H;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int t = tid; t < LX * LY; t += nth) {
    int lx = t % LX, ly = t / LX, i = gx0 + lx, j = gy0 + ly;
    bool in = i >= 0 && i < nx && j >= 0 && j < ny;
    size_t c = in ? at(i, j, P) : 0;
    se[t] = (in && !zero_init) ? e[c] : 0.f;
    sr[t] = in ? r[c] : 0.f;
    sd[t] = in ? invd[c] : 0.f;
  }
  for (int t = tid; t < LX; t += nth) {
    int i = gx0 + t;
    bool in = i >= 0 && i < nx;
    cE[t] = in ? g.pE[i] : 0.f;
    cW[t] = in ? g.pW[i] : 0.f;
  }
  for (int t = tid; t < LY; t += nth) {
    int j = gy0 + t;
    bool in = j >= 0 && j < ny;
    cN[t] = in ? g.pN[j] : 0.f;
    cS[t] = in ? g.pS[j] : 0.f;
  }
  __syncthreads();
  // parity of the loaded origin: colour of local (lx, ly) = (gx0 + gy0 + lx + ly) & 1
  const int par0 = (gx0 + gy0) & 1;
#pragma unroll 1
  for (int h = 0; h < K; ++h) {
    const int colour = h & 1;  // red first
    const int lo = h + 1, hx = LX - 2 - h, hy = LY - 2 - h;
    const int w2 = (hx - lo + 2) / 2;  // cells of one colour per row (upper bound)
    const int rows = hy - lo + 1;
    for (int t = tid; t < w2 * rows; t += nth) {
      int ly = lo + t / w2;
      int k = t % w2;
      // first lx >= lo with the right colour
      int lx = lo + ((colour + par0 + lo + ly) & 1) + 2 * k;
      if (lx > hx) continue;
      int i = gx0 + lx, j = gy0 + ly;
      if (i < 0 || i >= nx || j < 0 || j >= ny) continue;
      int q = ly * LX + lx;
      float s = cE[lx] * se[q + 1];
      s = fmaf(cW[lx], se[q - 1], s);
      s = fmaf(cN[ly], se[q + LX], s);
      s = fmaf(cS[ly], se[q - LX], s);
      float gs = (s - sr[q]) * sd[q];
      float x = se[q];
      se[q] = fmaf(omega, gs - x, x);
    }
    __syncthreads();
  }
  for (int t = tid; t < TX * TY; t += nth) {
    int lx = H + t % TX, ly = H + t / TX, i = gx0 + lx, j = gy0 + ly;
    if (i < nx && j < ny) e[at(i, j, P)] = se[ly * LX + lx];
  }
}

template <int TX, int TY, int K>
constexpr size_t tile_smem() {
  return sizeof(float) * (3 * (TX + 2 * K) * (TY + 2 * K) + 2 * (TX + 2 * K) + 2 * (TY + 2 * K));
}

constexpr int STX = 64, STY = 32, SK = 8;  // tile and half-sweeps per launch

}  // namespace

int sor32_half_sweeps_per_launch() { return SK; }

void launch_dc_residual(cudaStream_t s, const Geo& g, const double* phi_in, double* phi_out, const float* e,
                        const double* b, float* r32, int add_e, unsigned long long* res_bits) {
  dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  k_dc_residual<<<grd, blk, 0, s>>>(g, phi_in, phi_out, e, b, r32, add_e, res_bits);
}

void launch_sor32(cudaStream_t s, const Geo32& g, float* e, const float* r, const float* invd, float omega,
                  int zero_init) {
  constexpr size_t sm = tile_smem<STX, STY, SK>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sor32_tile<STX, STY, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  dim3 grd((g.nx + STX - 1) / STX, (g.ny + STY - 1) / STY);
  k_sor32_tile<STX, STY, SK><<<grd, 256, sm, s>>>(g, e, r, invd, omega, zero_init);
}

}  // namespace ibm
