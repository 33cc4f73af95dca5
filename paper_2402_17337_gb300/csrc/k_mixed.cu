// Pressure solve in FP32 sweeps inside FP64 defect correction.
//
// The red-black SOR of the pressure equation (arXiv 2402.17337, Sec. 2.2,
// Sec. 3.1) is split into
//   outer (FP64):  phi <- phi + e,  r = b - L_p phi,  ||r||_inf  (k_dc_residual)
//   inner (FP32):  red-black SOR sweeps on L_p e = r from e = 0   (k_sor32_rb)
// so the residual, the pressure update and the norm stay in FP64 while the
// sweeps, which carry the work, run at the FP32 rate.  The inner iterates
// are exactly those of red-black SOR applied to the correction equation.
//
// k_sor32_rb performs K half-sweeps per launch on a tile that carries a halo
// of K cells (temporal blocking): the tile is read and written once for K/2
// full sweeps and the halo is recomputed by the neighbouring tiles.  The
// FP32 arrays are stored split by colour (Geo32), so a half-sweep reads its
// neighbours contiguously; each thread keeps its own cells' correction,
// update coefficients a = omega / d and b = -a r (formed from the
// right-hand side and the reciprocal diagonal) in registers for the whole launch
// and shared memory only carries the values the neighbours read.
#include <type_traits>

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
// phi_out must differ from phi_in); r is stored in FP32, split by colour, as
// the next inner right-hand side.
// phi_out = phi_in + e (the update; one conversion and one FP64 add a cell)
__global__ void k_dc_update(Geo g, int pk, const double* __restrict__ phi_in, double* __restrict__ phi_out,
                            const float* __restrict__ e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const size_t c = at(i, j, g.pitch);
  phi_out[c] = phi_in[c] + (double)e[rb_at(i, j, g.ny, pk)];
}

// r = b - L_p phi in FP64 (stored in FP32, split by colour) and its norm;
// grid-stride over 32 x 8 tiles with a bounded number of blocks
__global__ void k_dc_residual(Geo g, int pk, const double* __restrict__ phi, const double* __restrict__ b,
                              float* __restrict__ r32, unsigned long long* __restrict__ res_bits) {
  unsigned long long bits = 0ull;
  const int nx = g.nx, ny = g.ny, P = g.pitch;
  const int tx = (nx + 31) / 32, nt = tx * ((ny + 7) / 8);
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int i = (t % tx) * 32 + threadIdx.x, j = (t / tx) * 8 + threadIdx.y;
    if (i >= nx || j >= ny) continue;
    const size_t c = at(i, j, P);
    const double fP = phi[c];
    double L = g.pE[i] * (phi[c + 1] - fP);
    L = fma(g.pW[i], phi[c - 1] - fP, L);
    L = fma(g.pN[j], phi[c + P] - fP, L);
    L = fma(g.pS[j], phi[c - P] - fP, L);
    const double r = b[c] - L;
    r32[rb_at(i, j, ny, pk)] = (float)r;
    const unsigned long long rb = abs_bits(r);
    bits = rb > bits ? rb : bits;
  }
  block_max_bits(bits, res_bits);
}

// Batched FP64 update + residual: block b belongs to the case whose block
// range holds it; each case has its own grid, buffers and norm slot.
__global__ void k_dc_residual_batch(const DcCase* __restrict__ cases, int ncases) {
  const int b = blockIdx.x;
  int lo = 0, hi = ncases - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (cases[mid].first <= b) lo = mid; else hi = mid - 1;
  }
  const DcCase& c = cases[lo];
  const Geo& g = c.g;
  const int t = b - c.first, bxn = (g.nx + 31) / 32;
  const int i = (t % bxn) * 32 + threadIdx.x, j = (t / bxn) * 8 + threadIdx.y;
  const int nx = g.nx, ny = g.ny, pk = c.pk;
  unsigned long long bits = 0ull;
  if (i < nx && j < ny) {
    const int P = g.pitch;
    size_t cc = at(i, j, P);
    const double* phi_in = c.phi_in;
    double fP = phi_in[cc], fE = phi_in[cc + 1], fW = phi_in[cc - 1], fN = phi_in[cc + P], fS = phi_in[cc - P];
    if (c.add_e) {
      const float* e = c.e;
      fP += (double)e[rb_at(i, j, ny, pk)];
      if (i < nx - 1) fE += (double)e[rb_at(i + 1, j, ny, pk)];
      if (i > 0) fW += (double)e[rb_at(i - 1, j, ny, pk)];
      if (j < ny - 1) fN += (double)e[rb_at(i, j + 1, ny, pk)];
      if (j > 0) fS += (double)e[rb_at(i, j - 1, ny, pk)];
      c.phi_out[cc] = fP;
    }
    double L = g.pE[i] * (fE - fP);
    L = fma(g.pW[i], fW - fP, L);
    L = fma(g.pN[j], fN - fP, L);
    L = fma(g.pS[j], fS - fP, L);
    double r = c.b[cc] - L;
    c.r32[rb_at(i, j, ny, pk)] = (float)r;
    bits = abs_bits(r);
  }
  block_max_bits(bits, c.res_bits);
}

// One SOR update.  x <- x + omega (gs - x) with the Gauss-Seidel value
// gs = (sum - r) / d is evaluated as x <- a sum + ((1 - omega) x + b), where
// a = omega / d and b = -a r are formed once per cell and launch (sor_ab):
// after the neighbour sum an update costs two FMAs, the first of which does
// not wait for the sum.  The neighbour sum takes the N and S terms first and
// the W/E term of the neighbour across the packed column (a shared-memory
// read) last.  Every tile form below uses exactly these operations in this
// order, so all give identical iterates.
__device__ __forceinline__ void sor_ab(float omega, float rr, float dd, float& a, float& b) {
  a = omega * dd;
  b = -(a * rr);
}
__device__ __forceinline__ float sor_update(float cN, float xN, float cS, float xS, float cSelf, float xSelf,
                                            float cOther, float xOther, float a, float b, float omc, float x) {
  float sum = cN * xN;
  sum = fmaf(cS, xS, sum);
  sum = fmaf(cSelf, xSelf, sum);
  sum = fmaf(cOther, xOther, sum);
  return fmaf(a, sum, fmaf(omc, x, b));
}

// K half-sweeps (red first) of FP32 red-black SOR on L_p e = r, from e_in
// into e_out.  The two buffers must differ: a tile's halo is read from cells
// that neighbouring tiles write, and tiles of later waves would otherwise
// read values that are already K half-sweeps ahead.
//
// Block (32, NY); the loaded region is LY = TY + 2K rows by LK = 64 colour
// columns (k) per colour, i.e. 128 cells in x; the written tile is TY rows
// by TK = LK - 2 HK colour columns, HK = ceil(K/2).  Thread (tx, ty) owns
// colour columns tx and tx + 32 of rows ty, ty + NY, ... for both colours;
// it keeps its cells' values in registers, and shared memory holds the
// values and update coefficients a, b of the whole region.
// Every half-sweep updates all cells that have their four neighbours in the
// region; a value that is wrong because the region is finite moves inwards
// by one cell per half-sweep, so after K half-sweeps the tile, at least K
// cells from every edge, is exact.  Cells outside the domain are never
// updated and hold zero; boundary cells have zero coefficients towards them
// (homogeneous Neumann).
template <int TY, int K, int NY>
struct Sor32Shape {
  static constexpr int LK = 64, HK = (K + 1) / 2, TK = LK - 2 * HK, LY = TY + 2 * K;
  static constexpr int RPT = (LY + NY - 1) / NY;
  static constexpr size_t smem = sizeof(float) * 3 * 2 * LY * LK;
};

template <int TY, int K, int NY>
__device__ __forceinline__ void sor32_tile(const Geo32& g, const float* __restrict__ e_in, float* __restrict__ e_out,
                                           const float* __restrict__ r, const float* __restrict__ invd, float omega,
                                           int zero_init, int bx, int by, float* smem) {
  using S = Sor32Shape<TY, K, NY>;
  constexpr int LK = S::LK, HK = S::HK, TK = S::TK, LY = S::LY, RPT = S::RPT;
  float(*se)[LY][LK] = reinterpret_cast<float(*)[LY][LK]>(smem);                    // [2][LY][LK]
  float(*sb)[LY][LK] = reinterpret_cast<float(*)[LY][LK]>(smem + 2 * LY * LK);      // [2][LY][LK]
  float(*sa)[LY][LK] = reinterpret_cast<float(*)[LY][LK]>(smem + 4 * LY * LK);      // [2][LY][LK]
  const int nx = g.nx, ny = g.ny, pk = g.pk;
  const int k0 = bx * TK - HK, j0 = by * TY - K;
  const int tx = threadIdx.x, ty = threadIdx.y;
  float ev[2][RPT][2];
  const float omc = 1.f - omega;
  float cE[2][2], cW[2][2], cN[RPT], cS[RPT];
  unsigned live = 0u, upd = 0u;  // bit (c, q, m): inside the domain / updated each half-sweep
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    int k = k0 + tx + 32 * m;
    bool ok = k >= 0 && k < pk;
    cE[m][0] = ok ? g.cE0[k] : 0.f;
    cE[m][1] = ok ? g.cE1[k] : 0.f;
    cW[m][0] = ok ? g.cW0[k] : 0.f;
    cW[m][1] = ok ? g.cW1[k] : 0.f;
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ty + NY * q, j = j0 + ly;
    const bool rowok = ly < LY && j >= 0 && j < ny;
    cN[q] = rowok ? g.pN[j] : 0.f;
    cS[q] = rowok ? g.pS[j] : 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m, k = k0 + kk, s = (c + j) & 1, i = 2 * k + s;
        const bool in = rowok && k >= 0 && i < nx;
        const size_t o = (size_t)(c * ny + j) * pk + k;
        const float x = (in && !zero_init) ? e_in[o] : 0.f;
        ev[c][q][m] = x;
        const int bit = (c * RPT + q) * 2 + m, li = 2 * kk + s;
        if (in) live |= 1u << bit;
        if (in && ly >= 1 && ly <= LY - 2 && li >= 1 && li <= 2 * LK - 2) upd |= 1u << bit;
        if (ly < LY) {
          float aa, bb;
          sor_ab(omega, in ? r[o] : 0.f, in ? invd[o] : 0.f, aa, bb);
          se[c][ly][kk] = x;
          sb[c][ly][kk] = bb;
          sa[c][ly][kk] = aa;
        }
      }
  }
  __syncthreads();
  // one half-sweep of colour C (compile-time, so the register arrays are
  // indexed statically)
  auto half = [&](auto colour) {
    constexpr int c = decltype(colour)::value, oc = c ^ 1;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int ly = ty + NY * q;
      const int s = (c + j0 + ly) & 1;  // colour c sits at i = 2k + s in this row
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        if (!(upd >> ((c * RPT + q) * 2 + m) & 1u)) continue;
        const int kk = tx + 32 * m;
        // neighbours of the other colour: N and S, the one in this packed
        // column (W if s, else E) and the one across the next (E if s, else W)
        const float xSelf = se[oc][ly][kk], xOther = se[oc][ly][kk + (s ? 1 : -1)];
        const float xN = se[oc][ly + 1][kk], xS = se[oc][ly - 1][kk];
        const float cself = s ? cW[m][1] : cE[m][0], cother = s ? cE[m][1] : cW[m][0];
        const float nxv = sor_update(cN[q], xN, cS[q], xS, cself, xSelf, cother, xOther, sa[c][ly][kk],
                                     sb[c][ly][kk], omc, ev[c][q][m]);
        ev[c][q][m] = nxv;
        se[c][ly][kk] = nxv;
      }
    }
    __syncthreads();
  };
#pragma unroll 1
  for (int h = 0; h < K; h += 2) {
    half(std::integral_constant<int, 0>{});  // red
    half(std::integral_constant<int, 1>{});  // black
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ty + NY * q;
    if (ly < K || ly >= K + TY) continue;
    const int j = j0 + ly;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m;
        if (kk < HK || kk >= HK + TK) continue;
        if (!(live >> ((c * RPT + q) * 2 + m) & 1u)) continue;
        e_out[(size_t)(c * ny + j) * pk + (k0 + kk)] = ev[c][q][m];
      }
  }
}

// Second form of the tile sweep (same iterates, fewer instructions per
// update).  The region is stored with one zero row and column on each side
// and cells outside the domain carry r = 0 and a zero reciprocal diagonal
// (a = b = 0, so an update multiplies them by 1 - omega),
// so every cell of the region is updated without a test: a cell outside the
// domain stays exactly zero, and a cell on the region's edge takes wrong
// values that, like any value spoiled by the region's finite size, move
// inwards by one cell per half-sweep (the written tile is K cells inside).
// Because NY is even, the colour parity s of a thread's cells is the same in
// all its rows, so coefficient selection and neighbour offsets are fixed per
// thread and colour; of the W and E neighbours one is the thread's own cell
// of the other colour (register) and the other is read from shared memory.
// The arithmetic of an update is the same as in sor32_tile, in the same
// order, so both forms give identical iterates.  With RDREG the update
// coefficients a, b of a thread's cells stay in registers.
template <int TY, int K, int NY, bool RDREG>
struct Sor32ShapeV4 {
  static constexpr int LK = 64, HK = (K + 1) / 2, TK = LK - 2 * HK, LY = TY + 2 * K;
  static constexpr int RPT = LY / NY, PY = LY + 2, PK = LK + 2;
  static constexpr size_t smem = sizeof(float) * (RDREG ? 2 : 6) * PY * PK;
  static_assert(LY % NY == 0, "rows per thread must be whole");
  static_assert(NY % 2 == 0, "an even number of thread rows keeps a thread's colour parity fixed");
};

template <int TY, int K, int NY, bool RDREG>
__device__ __forceinline__ void sor32_tile_v4(const Geo32& g, const float* __restrict__ e_in, float* __restrict__ e_out,
                                              const float* __restrict__ r, const float* __restrict__ invd,
                                              float omega, int zero_init, int bx, int by, float* smem) {
  using S = Sor32ShapeV4<TY, K, NY, RDREG>;
  constexpr int HK = S::HK, TK = S::TK, LY = S::LY, RPT = S::RPT, PY = S::PY, PK = S::PK;
  float(*se)[PY][PK] = reinterpret_cast<float(*)[PY][PK]>(smem);  // [2][PY][PK], cell (ly, kk) at [ly+1][kk+1]
  float(*sb)[PY][PK] = reinterpret_cast<float(*)[PY][PK]>(smem + 2 * PY * PK);
  float(*sa)[PY][PK] = reinterpret_cast<float(*)[PY][PK]>(smem + 4 * PY * PK);
  const int nx = g.nx, ny = g.ny, pk = g.pk;
  const int k0 = bx * TK - HK, j0 = by * TY - K;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int sc[2] = {(j0 + ty) & 1, (1 + j0 + ty) & 1};  // colour c sits at i = 2k + sc[c] in all rows of this thread
  // zero padding of the correction (rows -1 and LY, columns -1 and LK)
  for (int t = ty * 32 + tx; t < 2 * (2 * PK + 2 * LY); t += 32 * NY) {
    const int c = t / (2 * PK + 2 * LY), u = t % (2 * PK + 2 * LY);
    if (u < 2 * PK)
      se[c][u < PK ? 0 : PY - 1][u % PK] = 0.f;
    else
      se[c][1 + (u - 2 * PK) / 2][(u & 1) ? PK - 1 : 0] = 0.f;
  }
  float ev[2][RPT][2];
  const float omc = 1.f - omega;
  float bv[RDREG ? 2 : 1][RDREG ? RPT : 1][2], av[RDREG ? 2 : 1][RDREG ? RPT : 1][2];
  float ce[2][2], cw[2][2], cN[RPT], cS[RPT];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int k = k0 + tx + 32 * m;
    const bool ok = k >= 0 && k < pk;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      ce[c][m] = ok ? (sc[c] ? g.cE1[k] : g.cE0[k]) : 0.f;
      cw[c][m] = ok ? (sc[c] ? g.cW1[k] : g.cW0[k]) : 0.f;
    }
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ty + NY * q, j = j0 + ly;
    const bool rowok = j >= 0 && j < ny;
    cN[q] = rowok ? g.pN[j] : 0.f;
    cS[q] = rowok ? g.pS[j] : 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m, k = k0 + kk, i = 2 * k + sc[c];
        const bool in = rowok && k >= 0 && i < nx;
        const size_t o = (size_t)(c * ny + j) * pk + k;
        const float x = (in && !zero_init) ? e_in[o] : 0.f;
        float aa, bb;  // a and b of the update
        sor_ab(omega, in ? r[o] : 0.f, in ? invd[o] : 0.f, aa, bb);
        ev[c][q][m] = x;
        se[c][ly + 1][kk + 1] = x;
        if constexpr (RDREG) {
          bv[c][q][m] = bb;
          av[c][q][m] = aa;
        } else {
          sb[c][ly + 1][kk + 1] = bb;
          sa[c][ly + 1][kk + 1] = aa;
        }
      }
  }
  __syncthreads();
  auto half = [&](auto colour) {
    constexpr int c = decltype(colour)::value, oc = c ^ 1;
    const int s = sc[c];
    const int off = s ? 2 : 0;  // padded column of the neighbour of the other colour in shared memory: kk+1 -/+ 1
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int ly = ty + NY * q;
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m;
        const float xSelf = ev[oc][q][m];                 // the other colour in this packed column
        const float xOther = se[oc][ly + 1][kk + off];    // the other colour one packed column away
        const float xN = se[oc][ly + 2][kk + 1], xS = se[oc][ly][kk + 1];
        float aa, bb;  // a and b of the update
        if constexpr (RDREG) {
          bb = bv[c][q][m];
          aa = av[c][q][m];
        } else {
          bb = sb[c][ly + 1][kk + 1];
          aa = sa[c][ly + 1][kk + 1];
        }
        const float nxv = sor_update(cN[q], xN, cS[q], xS, s ? cw[c][m] : ce[c][m], xSelf, s ? ce[c][m] : cw[c][m],
                                     xOther, aa, bb, omc, ev[c][q][m]);
        ev[c][q][m] = nxv;
        se[c][ly + 1][kk + 1] = nxv;
      }
    }
    __syncthreads();
  };
#pragma unroll 1
  for (int h = 0; h < K; h += 2) {
    half(std::integral_constant<int, 0>{});
    half(std::integral_constant<int, 1>{});
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ty + NY * q;
    if (ly < K || ly >= K + TY) continue;
    const int j = j0 + ly;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m;
        const int k = k0 + kk;
        if (kk < HK || kk >= HK + TK || j < 0 || j >= ny || k < 0 || 2 * k + ((c + j) & 1) >= nx) continue;
        e_out[(size_t)(c * ny + j) * pk + (k0 + kk)] = ev[c][q][m];
      }
  }
}

// Third form: like the second, but a thread owns RPT consecutive rows (not
// rows NY apart), so the N and S neighbours of its cells of the other
// colour come from its own registers except at the ends of its run; only
// those end rows and the W/E neighbour of the other colour are read from
// shared memory.  The colour parity now alternates along a thread's rows; it
// is fixed per warp and half-sweep (the start row parity), so each half-sweep
// is compiled for both start parities and picked by a warp-uniform branch.
// Same arithmetic in the same order as the other forms: identical iterates.
// waits until the previous grid on the stream has completed and its writes
// are visible (a no-op unless launched as a programmatic dependent)
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// lets the next programmatic dependent launch start once every CTA of this
// grid has released it
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <int TY, int K, int NY, bool RDREG, bool SPLIT = false>
__device__ __forceinline__ void sor32_tile_v6(const Geo32& g, const float* __restrict__ e_in, float* __restrict__ e_out,
                                              const float* __restrict__ r, const float* __restrict__ invd,
                                              float omega, int zero_init, int bx, int by, float* smem) {
  using S = Sor32ShapeV4<TY, K, NY, RDREG>;
  constexpr int HK = S::HK, TK = S::TK, LY = S::LY, RPT = S::RPT, PY = S::PY, PK = S::PK;
  float(*se)[PY][PK] = reinterpret_cast<float(*)[PY][PK]>(smem);  // [2][PY][PK], cell (ly, kk) at [ly+1][kk+1]
  float(*sb)[PY][PK] = reinterpret_cast<float(*)[PY][PK]>(smem + 2 * PY * PK);
  float(*sa)[PY][PK] = reinterpret_cast<float(*)[PY][PK]>(smem + 4 * PY * PK);
  const int nx = g.nx, ny = g.ny, pk = g.pk;
  const int k0 = bx * TK - HK, j0 = by * TY - K;
  const int tx = threadIdx.x, ty = threadIdx.y, ly0 = ty * RPT;
  for (int t = ty * 32 + tx; t < 2 * (2 * PK + 2 * LY); t += 32 * NY) {
    const int c = t / (2 * PK + 2 * LY), u = t % (2 * PK + 2 * LY);
    if (u < 2 * PK)
      se[c][u < PK ? 0 : PY - 1][u % PK] = 0.f;
    else
      se[c][1 + (u - 2 * PK) / 2][(u & 1) ? PK - 1 : 0] = 0.f;
  }
  float ev[2][RPT][2];
  const float omc = 1.f - omega;
  float bv[RDREG ? 2 : 1][RDREG ? RPT : 1][2], av[RDREG ? 2 : 1][RDREG ? RPT : 1][2];
  float cE[2][2], cW[2][2], cN[RPT], cS[RPT];  // cE[m][s]: coefficient of the cell at i = 2k + s
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int k = k0 + tx + 32 * m;
    const bool ok = k >= 0 && k < pk;
    cE[m][0] = ok ? g.cE0[k] : 0.f;
    cE[m][1] = ok ? g.cE1[k] : 0.f;
    cW[m][0] = ok ? g.cW0[k] : 0.f;
    cW[m][1] = ok ? g.cW1[k] : 0.f;
  }
  // Early loads of r and 1/d.  The PTX ISA defines griddepcontrol.wait to
  // block until every prerequisite grid has completed and its memory
  // operations are performed and visible to the waiting grid, and
  // griddepcontrol.launch_dependents to let the dependent grid be scheduled
  // once every CTA of the issuing grid has executed it (or exited).  Every
  // CTA here executes the wait before the release.  So when a launch L2 that
  // follows a sweep launch L1 (zero_init = 0) starts, every CTA of L1 has
  // returned from its wait: the kernel before L1, which wrote r (1/d is
  // written at set-up), has completed and its writes are performed.  L1
  // itself writes only e.  L2 may therefore load r and 1/d before its own
  // wait, while L1 still runs, provided the loads read the device-coherent
  // L2 cache (ld.global.cg) and not this SM's L1, which is not coherent with
  // writes made on other SMs and may still hold lines of an earlier kernel
  // for a grid that starts this early (plain loads here gave wrong
  // iterates).  The first launch of a run (zero_init = 1) follows the kernel
  // that wrote r and waits first.
  if (zero_init) {
    griddep_wait();
    griddep_release();
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ly0 + q, j = j0 + ly;
    const bool rowok = j >= 0 && j < ny;
    cN[q] = rowok ? g.pN[j] : 0.f;
    cS[q] = rowok ? g.pS[j] : 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m, k = k0 + kk, i = 2 * k + ((c + j) & 1);
        const bool in = rowok && k >= 0 && i < nx;
        const size_t o = (size_t)(c * ny + j) * pk + k;
        float aa, bb;  // a and b of the update
        sor_ab(omega, in ? __ldcg(r + o) : 0.f, in ? __ldcg(invd + o) : 0.f, aa, bb);
        if constexpr (RDREG) {
          bv[c][q][m] = bb;
          av[c][q][m] = aa;
        } else {
          sb[c][ly + 1][kk + 1] = bb;
          sa[c][ly + 1][kk + 1] = aa;
        }
      }
  }
  if (!zero_init) {
    griddep_wait();
    griddep_release();
  }
  // e of this thread's cells, addressed from one row pointer per colour
  const float* e_row[2] = {e_in + ((size_t)(j0 + ly0) * pk + (k0 + tx)),
                           e_in + ((size_t)(ny + j0 + ly0) * pk + (k0 + tx))};
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ly0 + q, j = j0 + ly;
    const bool rowok = j >= 0 && j < ny;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m, k = k0 + kk, i = 2 * k + ((c + j) & 1);
        const bool in = rowok && k >= 0 && i < nx;
        const float x = (in && !zero_init) ? __ldcg(e_row[c] + ((size_t)q * pk + 32 * m)) : 0.f;
        ev[c][q][m] = x;
        se[c][ly + 1][kk + 1] = x;
      }
  }
  __syncthreads();
  // one half-sweep of colour C whose first row has parity S0 (all
  // compile-time), over the rows selected by PART: 0 all rows, 1 the rows
  // inside the thread's run, 2 its first and last row
  auto half_rows = [&](auto colour, auto start, auto part) {
    constexpr int c = decltype(colour)::value, oc = c ^ 1, S0 = decltype(start)::value;
    constexpr int PART = decltype(part)::value;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      if constexpr (PART != 0) {
        const bool edge = q == 0 || q == RPT - 1;
        if ((PART == 2) != edge) continue;
      }
      const int s = S0 ^ (q & 1);
      const int ly = ly0 + q;
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m;
        const float xSelf = ev[oc][q][m];
        const float xOther = se[oc][ly + 1][kk + (s ? 2 : 0)];
        const float xN = q < RPT - 1 ? ev[oc][q < RPT - 1 ? q + 1 : q][m] : se[oc][ly + 2][kk + 1];
        const float xS = q > 0 ? ev[oc][q > 0 ? q - 1 : q][m] : se[oc][ly][kk + 1];
        float aa, bb;  // a and b of the update
        if constexpr (RDREG) {
          bb = bv[c][q][m];
          aa = av[c][q][m];
        } else {
          bb = sb[c][ly + 1][kk + 1];
          aa = sa[c][ly + 1][kk + 1];
        }
        const float nxv = sor_update(cN[q], xN, cS[q], xS, s ? cW[m][1] : cE[m][0], xSelf, s ? cE[m][1] : cW[m][0],
                                     xOther, aa, bb, omc, ev[c][q][m]);
        ev[c][q][m] = nxv;
        se[c][ly + 1][kk + 1] = nxv;
      }
    }
  };
  // A half-sweep of a thread row (one warp) reads other threads' cells only
  // in the last row of the thread row above and the first row of the one
  // below; its other rows read the row's own cells (registers, and shared
  // memory written by the same warp).  With SPLIT the barrier between
  // half-sweeps comes after the rows inside each run and before its first
  // and last rows: those read the neighbours' edge rows of the previous
  // half-sweep (written before the barrier) and overwrite cells the
  // neighbours last read before it, and the inside rows of the next
  // half-sweep, which depend on no other warp, can interleave with them.
  // The same updates, each from the same values: identical iterates.
  auto half = [&](auto colour, auto start) {
    if constexpr (SPLIT) {
      half_rows(colour, start, std::integral_constant<int, 1>{});
      __syncthreads();
      half_rows(colour, start, std::integral_constant<int, 2>{});
    } else {
      half_rows(colour, start, std::integral_constant<int, 0>{});
      __syncthreads();
    }
  };
  const int p0 = (j0 + ly0) & 1;  // parity of this thread's first row
#pragma unroll 1
  for (int h = 0; h < K; h += 2) {
    if (p0) {
      half(std::integral_constant<int, 0>{}, std::integral_constant<int, 1>{});
      half(std::integral_constant<int, 1>{}, std::integral_constant<int, 0>{});
    } else {
      half(std::integral_constant<int, 0>{}, std::integral_constant<int, 0>{});
      half(std::integral_constant<int, 1>{}, std::integral_constant<int, 1>{});
    }
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ly0 + q;
    if (ly < K || ly >= K + TY) continue;
    const int j = j0 + ly;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int kk = tx + 32 * m;
        const int k = k0 + kk;
        if (kk < HK || kk >= HK + TK || j < 0 || j >= ny || k < 0 || 2 * k + ((c + j) & 1) >= nx) continue;
        e_out[(size_t)(c * ny + j) * pk + (k0 + kk)] = ev[c][q][m];
      }
  }
}

// Fourth form (9, 10): as sor32_tile_v6 with the coefficients in registers,
// but a thread owns the two adjacent packed columns 2 tx and 2 tx + 1 (not
// tx and tx + 32).  Of a cell's W and E neighbours one is the thread's own
// cell of the other colour in the same packed column and the other lies in
// the next packed column, which is the thread's other column or, once per
// row and half-sweep, the adjacent lane's (a shuffle): no shared memory is
// read or written for W and E.  Shared memory carries only the first and
// last row of each thread's run, which the thread rows above and below read
// as N and S neighbours, stored as pairs.  At the region's left and right
// edges the shuffle returns the lane's own value in place of the missing
// neighbour; like any value spoiled by the region's finite size it moves
// inwards by one cell per half-sweep and stays in the halo, and a cell
// outside the domain (a = b = 0) stays zero whatever it reads.  The update
// is sor_update with the same operands: identical iterates.  Form 10 puts
// the barrier between the rows inside each run and its edge rows (as
// form 8 does).
template <int TY, int K, int NY>
struct Sor32ShapeV9 {
  static constexpr int LK = 64, HK = K / 2, TK = LK - 2 * HK, LY = TY + 2 * K;
  static constexpr int RPT = LY / NY, PY = LY + 2;
  static constexpr size_t smem = sizeof(float) * 2 * PY * LK;
  static_assert(K % 4 == 0, "an even halo keeps a thread's column pair inside or outside the written tile");
  static_assert(LY % NY == 0, "rows per thread must be whole");
  static_assert(LY / NY >= 3, "a run needs a row between its first and last");
};

template <int TY, int K, int NY, bool SPLIT>
__device__ __forceinline__ void sor32_tile_v9(const Geo32& g, const float* __restrict__ e_in, float* __restrict__ e_out,
                                              const float* __restrict__ r, const float* __restrict__ invd,
                                              float omega, int zero_init, int bx, int by, float* smem) {
  using S = Sor32ShapeV9<TY, K, NY>;
  constexpr int LK = S::LK, HK = S::HK, TK = S::TK, RPT = S::RPT, PY = S::PY;
  constexpr unsigned FULL = 0xffffffffu;
  float(*se)[PY][LK] = reinterpret_cast<float(*)[PY][LK]>(smem);  // [2][PY][LK], cell (ly, kk) at [ly + 1][kk]
  const int nx = g.nx, ny = g.ny, pk = g.pk;
  const int k0 = bx * TK - HK, j0 = by * TY - K;  // k0 is even, and so is every thread's first column
  const int tx = threadIdx.x, ty = threadIdx.y, ly0 = ty * RPT, kk0 = 2 * tx;
  for (int t = ty * 32 + tx; t < 2 * 2 * LK; t += 32 * NY) {  // zero rows above and below the region
    const int c = t / (2 * LK), u = t % (2 * LK);
    se[c][u < LK ? 0 : PY - 1][u % LK] = 0.f;
  }
  float ev[2][RPT][2], av[2][RPT][2], bv[2][RPT][2];
  float cE[2][2], cW[2][2], cN[RPT], cS[RPT];  // cE[m][s]: coefficient of the cell at i = 2k + s
  const float omc = 1.f - omega;
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int k = k0 + kk0 + m;
    const bool ok = k >= 0 && k < pk;
    cE[m][0] = ok ? g.cE0[k] : 0.f;
    cE[m][1] = ok ? g.cE1[k] : 0.f;
    cW[m][0] = ok ? g.cW0[k] : 0.f;
    cW[m][1] = ok ? g.cW1[k] : 0.f;
  }
  // early loads of r and 1/d, before the wait, on the argument given in
  // sor32_tile_v6
  if (zero_init) {
    griddep_wait();
    griddep_release();
  }
  const int kp = k0 + kk0;  // first packed column of the pair; rows hold pk (even) entries, so the pair is in one row
  const bool pair_ok = kp >= 0 && kp < pk;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ly0 + q, j = j0 + ly;
    const bool rowok = j >= 0 && j < ny;
    cN[q] = rowok ? g.pN[j] : 0.f;
    cS[q] = rowok ? g.pS[j] : 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float2 rr = make_float2(0.f, 0.f), dd = make_float2(0.f, 0.f);
      if (rowok && pair_ok) {
        const size_t o = (size_t)(c * ny + j) * pk + kp;
        rr = __ldcg(reinterpret_cast<const float2*>(r + o));
        dd = __ldcg(reinterpret_cast<const float2*>(invd + o));
      }
      const int s = (c + j) & 1;
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const bool in = rowok && pair_ok && 2 * (kp + m) + s < nx;
        sor_ab(omega, in ? (m ? rr.y : rr.x) : 0.f, in ? (m ? dd.y : dd.x) : 0.f, av[c][q][m], bv[c][q][m]);
      }
    }
  }
  if (!zero_init) {
    griddep_wait();
    griddep_release();
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ly0 + q, j = j0 + ly;
    const bool rowok = j >= 0 && j < ny;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float2 x = make_float2(0.f, 0.f);
      if (rowok && pair_ok && !zero_init)
        x = __ldcg(reinterpret_cast<const float2*>(e_in + (size_t)(c * ny + j) * pk + kp));
      const int s = (c + j) & 1;
      ev[c][q][0] = (rowok && pair_ok && 2 * kp + s < nx) ? x.x : 0.f;
      ev[c][q][1] = (rowok && pair_ok && 2 * (kp + 1) + s < nx) ? x.y : 0.f;
      if (q == 0 || q == RPT - 1)
        *reinterpret_cast<float2*>(&se[c][ly + 1][kk0]) = make_float2(ev[c][q][0], ev[c][q][1]);
    }
  }
  __syncthreads();
  // one half-sweep of colour C whose first row has parity S0, over the rows
  // selected by PART (0 all, 1 inside the run, 2 its first and last row)
  auto half_rows = [&](auto colour, auto start, auto part) {
    constexpr int c = decltype(colour)::value, oc = c ^ 1, S0 = decltype(start)::value;
    constexpr int PART = decltype(part)::value;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const bool edge = q == 0 || q == RPT - 1;
      if constexpr (PART != 0) {
        if ((PART == 2) != edge) continue;
      }
      const int s = S0 ^ (q & 1);
      const int ly = ly0 + q;
      // the neighbour across the packed column: W (column k - 1) if s = 0,
      // else E (column k + 1)
      float xo[2];
      if (s) {
        xo[0] = ev[oc][q][1];
        xo[1] = __shfl_down_sync(FULL, ev[oc][q][0], 1);
      } else {
        xo[0] = __shfl_up_sync(FULL, ev[oc][q][1], 1);
        xo[1] = ev[oc][q][0];
      }
      float2 nN = make_float2(0.f, 0.f), nS = make_float2(0.f, 0.f);
      if (q == RPT - 1) nN = *reinterpret_cast<const float2*>(&se[oc][ly + 2][kk0]);
      if (q == 0) nS = *reinterpret_cast<const float2*>(&se[oc][ly][kk0]);
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const float xN = q < RPT - 1 ? ev[oc][q < RPT - 1 ? q + 1 : q][m] : (m ? nN.y : nN.x);
        const float xS = q > 0 ? ev[oc][q > 0 ? q - 1 : q][m] : (m ? nS.y : nS.x);
        ev[c][q][m] = sor_update(cN[q], xN, cS[q], xS, s ? cW[m][1] : cE[m][0], ev[oc][q][m],
                                 s ? cE[m][1] : cW[m][0], xo[m], av[c][q][m], bv[c][q][m], omc, ev[c][q][m]);
      }
      if (edge) *reinterpret_cast<float2*>(&se[c][ly + 1][kk0]) = make_float2(ev[c][q][0], ev[c][q][1]);
    }
  };
  auto half = [&](auto colour, auto start) {
    if constexpr (SPLIT) {
      half_rows(colour, start, std::integral_constant<int, 1>{});
      __syncthreads();
      half_rows(colour, start, std::integral_constant<int, 2>{});
    } else {
      half_rows(colour, start, std::integral_constant<int, 0>{});
      __syncthreads();
    }
  };
  const int p0 = (j0 + ly0) & 1;  // parity of this thread's first row
#pragma unroll 1
  for (int h = 0; h < K; h += 2) {
    if (p0) {
      half(std::integral_constant<int, 0>{}, std::integral_constant<int, 1>{});
      half(std::integral_constant<int, 1>{}, std::integral_constant<int, 0>{});
    } else {
      half(std::integral_constant<int, 0>{}, std::integral_constant<int, 0>{});
      half(std::integral_constant<int, 1>{}, std::integral_constant<int, 1>{});
    }
  }
  if (kk0 < HK || kk0 >= HK + TK || !pair_ok) return;  // the pair lies in the halo or outside the rows
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int ly = ly0 + q;
    if (ly < K || ly >= K + TY) continue;
    const int j = j0 + ly;
    if (j < 0 || j >= ny) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int s = (c + j) & 1;
      float* dst = e_out + (size_t)(c * ny + j) * pk + kp;
      if (2 * (kp + 1) + s < nx)
        *reinterpret_cast<float2*>(dst) = make_float2(ev[c][q][0], ev[c][q][1]);
      else if (2 * kp + s < nx)
        dst[0] = ev[c][q][0];
    }
  }
}

// A tile shape: rows per tile, half-sweeps per launch, thread rows, form
// (3: sor32_tile; 4: sor32_tile_v4 with a and b in shared memory; 5: with
// a and b in registers; 6, 7: sor32_tile_v6 likewise; 8: as 7 with the
// barrier between the inside rows of each thread's run and its edge rows;
// 9, 10: sor32_tile_v9, without and with that split)
// and minimum resident CTAs per SM.
template <int TY_, int K_, int NY_, int V_, int MINB_>
struct Cfg {
  static constexpr int TY = TY_, K = K_, NY = NY_, V = V_, MINB = MINB_;
  static constexpr int HK = (K + 1) / 2, TK = 64 - 2 * HK;
  static constexpr size_t smem =
      std::conditional_t<V == 3, Sor32Shape<TY, K, NY>,
                         std::conditional_t<(V >= 9), Sor32ShapeV9<TY, K, NY>,
                                            Sor32ShapeV4<TY, K, NY, V == 5 || V >= 7>>>::smem;
};

template <class C>
__device__ __forceinline__ void tile(const Geo32& g, const float* e_in, float* e_out, const float* r,
                                     const float* invd, float omega, int zero_init, int bx, int by, float* smem) {
  if constexpr (C::V == 3)
    sor32_tile<C::TY, C::K, C::NY>(g, e_in, e_out, r, invd, omega, zero_init, bx, by, smem);
  else if constexpr (C::V == 4 || C::V == 5)
    sor32_tile_v4<C::TY, C::K, C::NY, C::V == 5>(g, e_in, e_out, r, invd, omega, zero_init, bx, by, smem);
  else if constexpr (C::V <= 8)
    sor32_tile_v6<C::TY, C::K, C::NY, C::V >= 7, C::V == 8>(g, e_in, e_out, r, invd, omega, zero_init, bx, by,
                                                              smem);
  else
    sor32_tile_v9<C::TY, C::K, C::NY, C::V == 10>(g, e_in, e_out, r, invd, omega, zero_init, bx, by, smem);
}

template <class C>
__global__ void __launch_bounds__(32 * C::NY, C::MINB)
    k_sor32_rb(const Geo32 g, const float* __restrict__ e_in, float* __restrict__ e_out, const float* __restrict__ r,
               const float* __restrict__ invd, float omega, int zero_init) {
  extern __shared__ float smem[];
  // programmatic dependent launch (a no-op unless the launch asks for it):
  // this launch reads what the previous kernel wrote only after that kernel
  // has completed and its writes are visible, and then lets the next sweep
  // launch start (forms 6 and 7 do both inside, after loading r and 1/d)
  if constexpr (C::V < 6) {
    griddep_wait();
    griddep_release();
  }
  tile<C>(g, e_in, e_out, r, invd, omega, zero_init, blockIdx.x, blockIdx.y, smem);
}

// Batched form: one launch sweeps the tiles of many cases (uneven grids).
// CTA b belongs to the case whose tile range [first, first + count) holds b.
template <class C>
__global__ void __launch_bounds__(32 * C::NY, C::MINB)
    k_sor32_rb_batch(const Sor32Case* __restrict__ cases, int ncases, int zero_init, int q) {
  extern __shared__ float smem[];
  __shared__ Sor32Case c;  // the case's descriptor, read from shared memory where needed
  // programmatic dependent launch (a no-op unless the launch asks for it):
  // the descriptor tables are rewritten between rounds, so every CTA waits
  // for the previous kernel before its first load and then lets the next
  // launch start (forms 6 and 7 wait and release again inside; both return
  // at once the second time)
  griddep_wait();
  griddep_release();
  const int b = blockIdx.x;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {  // last case with first <= b
      int mid = (lo + hi + 1) >> 1;
      if (cases[mid].first <= b) lo = mid; else hi = mid - 1;
    }
    c = cases[lo];
  }
  __syncthreads();
  if (q >= c.pairs) return;  // this case's sweeps of the round are done (uniform over the CTA)
  const int t = b - c.first;
  tile<C>(c.g, c.e_in, c.e_out, c.r, c.invd, c.omega, zero_init, t % c.tiles_x, t / c.tiles_x, smem);
}

// Tile shapes the autotuner chooses from.
struct Sor32Config {
  int TY, K, NY, V;
  void (*launch)(cudaStream_t, const Geo32&, const float*, float*, const float*, const float*, float, int, int);
  void (*launch_batch)(cudaStream_t, const Sor32Case*, int, int, int, int, int);
  cudaError_t (*prepare)();
  void (*tiles)(const Geo32&, int*, int*);
};

// dynamic shared memory limits of both kernels of a shape; set once, outside
// any stream capture
template <class C>
cudaError_t prepare_shape() {
  cudaError_t e = cudaFuncSetAttribute(k_sor32_rb<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_sor32_rb_batch<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
}

template <class C>
void launch_shape(cudaStream_t s, const Geo32& g, const float* e_in, float* e_out, const float* r, const float* invd,
                  float omega, int zero_init, int pdl) {
  static bool attr = false;
  if (!attr) {
    prepare_shape<C>();
    attr = true;
  }
  const int ncol = (g.nx + 1) / 2;
  dim3 grd((ncol + C::TK - 1) / C::TK, (g.ny + C::TY - 1) / C::TY);
  if (!pdl) {
    k_sor32_rb<C><<<grd, dim3(32, C::NY), C::smem, s>>>(g, e_in, e_out, r, invd, omega, zero_init);
    return;
  }
  cudaLaunchConfig_t lc{};
  lc.gridDim = grd;
  lc.blockDim = dim3(32, C::NY);
  lc.dynamicSmemBytes = C::smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaLaunchKernelEx(&lc, k_sor32_rb<C>, g, e_in, e_out, r, invd, omega, zero_init);
}

template <class C>
void launch_shape_batch(cudaStream_t s, const Sor32Case* cases, int ncases, int total_tiles, int zero_init,
                        int pdl, int q) {
  if (total_tiles <= 0) return;
  if (!pdl) {
    k_sor32_rb_batch<C><<<total_tiles, dim3(32, C::NY), C::smem, s>>>(cases, ncases, zero_init, q);
    return;
  }
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3(total_tiles);
  lc.blockDim = dim3(32, C::NY);
  lc.dynamicSmemBytes = C::smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaLaunchKernelEx(&lc, k_sor32_rb_batch<C>, cases, ncases, zero_init, q);
}

template <class C>
void shape_tiles(const Geo32& g, int* tx, int* ty) {
  *tx = ((g.nx + 1) / 2 + C::TK - 1) / C::TK;
  *ty = (g.ny + C::TY - 1) / C::TY;
}

template <class C>
constexpr Sor32Config shape() {
  return {C::TY, C::K, C::NY, C::V, launch_shape<C>, launch_shape_batch<C>, prepare_shape<C>, shape_tiles<C>};
}

const Sor32Config kConfigs[] = {
    shape<Cfg<32, 8, 16, 3, 2>>(),  shape<Cfg<48, 8, 16, 3, 2>>(),  shape<Cfg<16, 8, 8, 3, 2>>(),
    shape<Cfg<32, 4, 8, 3, 2>>(),   shape<Cfg<64, 16, 16, 3, 2>>(), shape<Cfg<32, 12, 16, 3, 2>>(),
    shape<Cfg<32, 8, 16, 4, 2>>(),  shape<Cfg<48, 8, 16, 4, 2>>(),  shape<Cfg<40, 12, 16, 4, 2>>(),
    shape<Cfg<16, 8, 8, 4, 3>>(),   shape<Cfg<24, 4, 8, 4, 3>>(),   shape<Cfg<64, 16, 16, 4, 1>>(),
    shape<Cfg<16, 8, 8, 5, 2>>(),   shape<Cfg<32, 8, 16, 5, 1>>(),  shape<Cfg<24, 4, 8, 5, 2>>(),
    shape<Cfg<32, 8, 8, 6, 3>>(),   shape<Cfg<48, 8, 16, 6, 2>>(),  shape<Cfg<40, 12, 16, 6, 2>>(),
    shape<Cfg<64, 16, 16, 6, 1>>(), shape<Cfg<24, 4, 8, 6, 3>>(),   shape<Cfg<32, 8, 8, 7, 2>>(),
    shape<Cfg<48, 8, 16, 7, 1>>(),  shape<Cfg<24, 4, 8, 7, 2>>(),   shape<Cfg<48, 8, 8, 6, 2>>(),
    shape<Cfg<48, 8, 8, 7, 1>>(),   shape<Cfg<40, 12, 8, 6, 2>>(),  shape<Cfg<80, 16, 16, 6, 1>>(),
    shape<Cfg<96, 16, 16, 6, 1>>(), shape<Cfg<64, 16, 16, 7, 1>>(), shape<Cfg<80, 16, 16, 7, 1>>(),
    shape<Cfg<64, 16, 16, 8, 1>>(), shape<Cfg<80, 16, 16, 8, 1>>(), shape<Cfg<80, 16, 16, 9, 1>>(),
    shape<Cfg<80, 16, 16, 10, 1>>(), shape<Cfg<64, 16, 16, 10, 1>>(), shape<Cfg<48, 8, 16, 10, 1>>(),
    shape<Cfg<32, 8, 8, 10, 2>>(),
};
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

}  // namespace

int sor32_num_configs() { return kNumConfigs; }
int sor32_find_shape(int ty, int k, int form) {
  for (int i = 0; i < kNumConfigs; ++i)
    if (kConfigs[i].TY == ty && kConfigs[i].K == k && kConfigs[i].V == form) return i;
  return -1;
}
int sor32_half_sweeps(int cfg) { return kConfigs[cfg].K; }
void sor32_describe(int cfg, int* ty, int* k, int* ny, int* form) {
  *ty = kConfigs[cfg].TY;
  *k = kConfigs[cfg].K;
  *ny = kConfigs[cfg].NY;
  *form = kConfigs[cfg].V;
}

void launch_dc_residual(cudaStream_t s, const Geo& g, int pk, const double* phi_in, double* phi_out, const float* e,
                        const double* b, float* r32, int add_e, unsigned long long* res_bits) {
  const int nt = ((g.nx + 31) / 32) * ((g.ny + 7) / 8);
  if (add_e) k_dc_update<<<dim3((g.nx + 31) / 32, (g.ny + 7) / 8), dim3(32, 8), 0, s>>>(g, pk, phi_in, phi_out, e);
  k_dc_residual<<<nt < 1216 ? nt : 1216, dim3(32, 8), 0, s>>>(g, pk, add_e ? phi_out : phi_in, b, r32, res_bits);
}

void launch_sor32(cudaStream_t s, int cfg, const Geo32& g, const float* e_in, float* e_out, const float* r,
                  const float* invd, float omega, int zero_init, int pdl) {
  kConfigs[cfg].launch(s, g, e_in, e_out, r, invd, omega, zero_init, pdl);
}

void sor32_tiles(int cfg, const Geo32& g, int* tiles_x, int* tiles_y) { kConfigs[cfg].tiles(g, tiles_x, tiles_y); }

cudaError_t sor32_batch_prepare(int cfg) { return kConfigs[cfg].prepare(); }

void launch_sor32_batch(cudaStream_t s, int cfg, const Sor32Case* cases_dev, int ncases, int total_tiles,
                        int zero_init, int pdl, int q) {
  kConfigs[cfg].launch_batch(s, cases_dev, ncases, total_tiles, zero_init, pdl, q);
}

void launch_dc_residual_batch(cudaStream_t s, const DcCase* cases_dev, int ncases, int total_blocks) {
  if (total_blocks <= 0) return;
  k_dc_residual_batch<<<total_blocks, dim3(32, 8), 0, s>>>(cases_dev, ncases);
}

}  // namespace ibm
