// Step kernels of the immersed-boundary fractional step (arXiv 2402.17337,
// Sec. 2.2): outflow boundary values, fluid/solid classification and forcing
// data, explicit momentum predictor (Adams-Bashforth convection,
// Crank-Nicolson diffusion), divergence right-hand side with the mass source
// q (Eq. 4), surface forces, and the projection with the divergence check.
//
// All fields are FP64 in the shared pitched layout (ibm_internal.h).  The
// arithmetic follows the recipe shared with the CPU oracle: reciprocals of
// the grid spacings, fma chains for the 5-point Laplacian, plain expressions
// elsewhere (no contraction: the library is built with --fmad=false), and the
// outflow-flux and body-source sums accumulated in a fixed two-level index
// order.
#include "ibm_internal.h"

namespace ibm {

namespace {

constexpr int TBX = 32, TBY = 8;

__device__ inline int band_index(const Band& B, int i, int j) {
  int bi = i - B.i0, bj = j - B.j0;
  if (bi < 0 || bj < 0 || bi >= B.w || bj >= B.h) return -1;
  return bj * B.w + bi;
}

// Integer decisions (solid or not, which wall direction) are taken with
// explicitly rounded operations so that no multiply-add is contracted.
__device__ inline bool inside_ellipse(double x, double y, double xb, double yb, double a, double b) {
  double xi = __ddiv_rn(__dsub_rn(x, xb), a);
  double eta = __ddiv_rn(__dsub_rn(y, yb), b);
  return __dadd_rn(__dmul_rn(xi, xi), __dmul_rn(eta, eta)) <= 1.0;
}

// deterministic block reduction of up to 4 doubles (blockDim.x = 256)
template <int N>
__device__ inline void block_sum(double (&v)[N], double* out) {
  __shared__ double sm[N][256];
  for (int k = 0; k < N; ++k) sm[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < N; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < N; ++k) out[k] = sm[k][0];
}

__device__ inline void block_max_bits(unsigned long long v, unsigned long long* dst) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  __shared__ unsigned long long wm[32];
  int lane = (threadIdx.x + threadIdx.y * blockDim.x) & 31;
  int warp = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
  int nw = (blockDim.x * blockDim.y + 31) >> 5;
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

// --------------------------------------------------------- boundary values

// Inflow u = u_in; convective outflow du/dt + u_in du/dx = 0 by explicit Euler,
// then a uniform shift so that the outflow flux equals the inflow flux.
__device__ __forceinline__ void outflow_bc_body(Geo g, const double* __restrict__ u, double* __restrict__ uh, double u_in,
                             double dt, int bx, int by) {
  const int nx = g.nx, ny = g.ny, P = g.pitch;
  // convective update, one row per thread
  for (int j = threadIdx.x; j < ny; j += blockDim.x) {
    double ub = u[at(nx, j, P)], um = u[at(nx - 1, j, P)];
    uh[at(0, j, P)] = u_in;
    uh[at(nx, j, P)] = ub - dt * u_in * (ub - um) * g.idx[nx - 1];
  }
  __syncthreads();
  // fluxes: each thread sums one chunk of 32 rows in row order, then thread 0
  // sums the chunk sums in order (the shift feeds back into the flow, so the
  // order of the additions is fixed)
  __shared__ double part[3][256];
  __shared__ double corr;
  const int nchunk = (ny + 31) / 32;
  for (int ch = threadIdx.x; ch < nchunk; ch += blockDim.x) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int j = 32 * ch; j < 32 * ch + 32 && j < ny; ++j) {
      a += u_in * g.dy[j];
      b += uh[at(nx, j, P)] * g.dy[j];
      c += g.dy[j];
    }
    part[0][ch] = a;
    part[1][ch] = b;
    part[2][ch] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double qin = 0.0, qout = 0.0, ly = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) {
      qin += part[0][ch];
      qout += part[1][ch];
      ly += part[2][ch];
    }
    corr = (qin - qout) / ly;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ny; j += blockDim.x) uh[at(nx, j, P)] += corr;
}
__global__ void k_outflow_bc(Geo g, const double* __restrict__ u, double* __restrict__ uh, double u_in,
                             double dt) {
  outflow_bc_body(g, u, uh, u_in, dt, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------- classification

__device__ __forceinline__ void classify_solid_body(Geo g, Band B, double xb, double yb, double a, double b,
                                 uint8_t* __restrict__ fu, uint8_t* __restrict__ fv, uint8_t* __restrict__ fc,
                                 double* __restrict__ au, double* __restrict__ av, int bx, int by) {
  int bi = bx * blockDim.x + threadIdx.x, bj = by * blockDim.y + threadIdx.y;
  if (bi >= B.w || bj >= B.h) return;
  int i = B.i0 + bi, j = B.j0 + bj, k = bj * B.w + bi;
  const int nx = g.nx, ny = g.ny;
  bool su = i >= 1 && i <= nx - 1 && j >= 0 && j <= ny - 1 && inside_ellipse(g.xf[i], g.yc[j], xb, yb, a, b);
  bool sv = i >= 0 && i <= nx - 1 && j >= 1 && j <= ny - 1 && inside_ellipse(g.xc[i], g.yf[j], xb, yb, a, b);
  bool sc = i >= 0 && i <= nx - 1 && j >= 0 && j <= ny - 1 && inside_ellipse(g.xc[i], g.yc[j], xb, yb, a, b);
  fu[k] = su ? K_SOLID : K_FLUID;
  fv[k] = sv ? K_SOLID : K_FLUID;
  fc[k] = sc ? 1 : 0;
  au[k] = 0.0;
  av[k] = 0.0;
}
__global__ void k_classify_solid(Geo g, Band B, double xb, double yb, double a, double b,
                                 uint8_t* __restrict__ fu, uint8_t* __restrict__ fv, uint8_t* __restrict__ fc,
                                 double* __restrict__ au, double* __restrict__ av) {
  classify_solid_body(g, B, xb, yb, a, b, fu, fv, fc, au, av, blockIdx.x, blockIdx.y);
}

__device__ inline bool band_solid(const uint8_t* f, const Band& B, int i, int j) {
  int k = band_index(B, i, j);
  return k >= 0 && (f[k] & 3) == K_SOLID;
}

__device__ inline bool band_has_solid_nb(const uint8_t* f, const Band& B, int i, int j) {
  return band_solid(f, B, i - 1, j) || band_solid(f, B, i + 1, j) || band_solid(f, B, i, j - 1) ||
         band_solid(f, B, i, j + 1);
}

// Forcing nodes: fluid nodes with a solid 4-neighbour on their own grid.  The
// wall crossing is found analytically along each grid line towards a solid
// neighbour; the nearest one (ties: -x, +x, -y, +y) sets the direction, and
// the node takes u_F = U_b + alpha (u_opp - U_b), alpha = d / (d + D), with
// u_opp the node on the far side at distance D.  alpha = 0 (u_F = U_b) when
// that node is solid, a forcing node, or not an unknown of the grid.
__device__ __forceinline__ void classify_forcing_body(Geo g, Band B, int grid, double xb, double yb, double a, double b,
                                   uint8_t* __restrict__ fl, double* __restrict__ al, int bx, int by) {
  int bi = bx * blockDim.x + threadIdx.x, bj = by * blockDim.y + threadIdx.y;
  if (bi >= B.w || bj >= B.h) return;
  int i = B.i0 + bi, j = B.j0 + bj, k = bj * B.w + bi;
  const int nx = g.nx, ny = g.ny;
  int ilo = grid == 0 ? 1 : 0, ihi = nx - 1;
  int jlo = grid == 0 ? 0 : 1, jhi = ny - 1;
  if (i < ilo || i > ihi || j < jlo || j > jhi) return;
  if ((fl[k] & 3) == K_SOLID || !band_has_solid_nb(fl, B, i, j)) return;
  const double* gx = grid == 0 ? g.xf : g.xc;
  const double* gy = grid == 0 ? g.yc : g.yf;
  double x = gx[i], y = gy[j];
  double best = 1.0 / 0.0;
  int bd = -1;
  const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
  for (int d = 0; d < 4; ++d) {
    int ni = i + di[d], nj = j + dj[d];
    if (!band_solid(fl, B, ni, nj)) continue;
    double dist, span;
    if (d < 2) {
      double eta = __ddiv_rn(__dsub_rn(y, yb), b);
      double s = __dmul_rn(a, __dsqrt_rn(fmax(0.0, __dsub_rn(1.0, __dmul_rn(eta, eta)))));
      if (d == 0) {
        dist = __dsub_rn(x, __dadd_rn(xb, s));
        span = __dsub_rn(x, gx[i - 1]);
      } else {
        dist = __dsub_rn(__dsub_rn(xb, s), x);
        span = __dsub_rn(gx[i + 1], x);
      }
    } else {
      double xi = __ddiv_rn(__dsub_rn(x, xb), a);
      double s = __dmul_rn(b, __dsqrt_rn(fmax(0.0, __dsub_rn(1.0, __dmul_rn(xi, xi)))));
      if (d == 2) {
        dist = __dsub_rn(y, __dadd_rn(yb, s));
        span = __dsub_rn(y, gy[j - 1]);
      } else {
        dist = __dsub_rn(__dsub_rn(yb, s), y);
        span = __dsub_rn(gy[j + 1], y);
      }
    }
    dist = dist < 0.0 ? 0.0 : dist;
    dist = dist > span ? span : dist;
    if (dist < best) {
      best = dist;
      bd = d;
    }
  }
  int oi = i - di[bd], oj = j - dj[bd];
  bool ok = oi >= ilo && oi <= ihi && oj >= jlo && oj <= jhi;
  if (ok) ok = !band_solid(fl, B, oi, oj) && !band_has_solid_nb(fl, B, oi, oj);
  double alpha = 0.0;
  if (ok) {
    double D = bd < 2 ? fabs(__dsub_rn(gx[oi], x)) : fabs(__dsub_rn(gy[oj], y));
    alpha = __ddiv_rn(best, __dadd_rn(best, D));
  }
  // the kind bits of this node change from fluid to forcing; other threads
  // only ever test for "solid", which this write cannot change
  fl[k] = (uint8_t)(K_FORCE | (bd << 2));
  al[k] = alpha;
}
__global__ void k_classify_forcing(Geo g, Band B, int grid, double xb, double yb, double a, double b,
                                   uint8_t* __restrict__ fl, double* __restrict__ al) {
  classify_forcing_body(g, B, grid, xb, yb, a, b, fl, al, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------- explicit predictor

// sum_nb a_nb (x_nb - x_P) in the order E, W, N, S
__device__ inline double lap5(double aE, double aW, double aN, double aS, double xE, double xW, double xN,
                              double xS, double c) {
  double L = aE * (xE - c);
  L = fma(aW, xW - c, L);
  L = fma(aN, xN - c, L);
  L = fma(aS, xS - c, L);
  return L;
}

// u node (i = 1..nx-1, j = 0..ny-1): control volume [xc_{i-1}, xc_i] x [yf_j, yf_{j+1}]
__device__ __forceinline__ void predict_u_body(Geo g, const double* __restrict__ u, const double* __restrict__ v,
                            const double* __restrict__ p, double* __restrict__ Hu,
                            const double* __restrict__ Huo, double* __restrict__ Ru, double* __restrict__ uh,
                            Band B, const uint8_t* __restrict__ fu, double dt, double beta, int first, int bx, int by) {
  int i = bx * blockDim.x + threadIdx.x + 1, j = by * blockDim.y + threadIdx.y;
  if (i > g.nx - 1 || j > g.ny - 1) return;
  const int P = g.pitch;
  size_t c = at(i, j, P);
  double uP = u[c], uE = u[c + 1], uW = u[c - 1], uN = u[c + P], uS = u[c - P];
  // v at the north and south corners of the control volume (v row j+1 and j)
  size_t cv = c;  // v(i, j) shares the index of u(i, j)
  double wx = g.wx[i];
  double vn = (1.0 - wx) * v[cv + P - 1] + wx * v[cv + P];
  double vs = (1.0 - wx) * v[cv - 1] + wx * v[cv];
  double un = (1.0 - g.wy[j + 1]) * uP + g.wy[j + 1] * uN;
  double us = (1.0 - g.wy[j]) * uS + g.wy[j] * uP;
  double ue = 0.5 * (uP + uE), uw = 0.5 * (uW + uP);
  double H = (ue * ue - uw * uw) * g.idxc[i] + (vn * un - vs * us) * g.idy[j];
  double Ho = first ? H : Huo[c];
  double gp = (p[c] - p[c - 1]) * g.idxc[i];
  double L = lap5(g.uE[i], g.uW[i], g.uN[j], g.uS[j], uE, uW, uN, uS, uP);
  Hu[c] = H;
  Ru[c] = uP + dt * (-1.5 * H + 0.5 * Ho - gp) + beta * L;
  int k = band_index(B, i, j);
  uh[c] = (k >= 0 && (fu[k] & 3) == K_SOLID) ? 0.0 : uP;
}
__global__ void k_predict_u(Geo g, const double* __restrict__ u, const double* __restrict__ v,
                            const double* __restrict__ p, double* __restrict__ Hu,
                            const double* __restrict__ Huo, double* __restrict__ Ru, double* __restrict__ uh,
                            Band B, const uint8_t* __restrict__ fu, double dt, double beta, int first) {
  predict_u_body(g, u, v, p, Hu, Huo, Ru, uh, B, fu, dt, beta, first, blockIdx.x, blockIdx.y);
}

// v node (i = 0..nx-1, j = 1..ny-1): control volume [xf_i, xf_{i+1}] x [yc_{j-1}, yc_j]
__device__ __forceinline__ void predict_v_body(Geo g, const double* __restrict__ u, const double* __restrict__ v,
                            const double* __restrict__ p, double* __restrict__ Hv,
                            const double* __restrict__ Hvo, double* __restrict__ Rv, double* __restrict__ vh,
                            Band B, const uint8_t* __restrict__ fv, double dt, double beta, double vb,
                            int first, int bx, int by) {
  int i = bx * blockDim.x + threadIdx.x, j = by * blockDim.y + threadIdx.y + 1;
  if (i > g.nx - 1 || j > g.ny - 1) return;
  const int P = g.pitch;
  size_t c = at(i, j, P);
  double vP = v[c], vN = v[c + P], vS = v[c - P], vE = v[c + 1], vW = v[c - 1];
  double wy = g.wy[j];
  // u at the east and west corners (u columns i+1 and i, rows j-1 and j)
  double ue = (1.0 - wy) * u[c + 1 - P] + wy * u[c + 1];
  double uw = (1.0 - wy) * u[c - P] + wy * u[c];
  double ve = (1.0 - g.wx[i + 1]) * vP + g.wx[i + 1] * vE;
  double vw = (1.0 - g.wx[i]) * vW + g.wx[i] * vP;
  double vn = 0.5 * (vP + vN), vs = 0.5 * (vS + vP);
  double H = (ue * ve - uw * vw) * g.idx[i] + (vn * vn - vs * vs) * g.idyc[j];
  double Ho = first ? H : Hvo[c];
  double gp = (p[c] - p[c - P]) * g.idyc[j];
  double L = lap5(g.vE[i], g.vW[i], g.vN[j], g.vS[j], vE, vW, vN, vS, vP);
  Hv[c] = H;
  Rv[c] = vP + dt * (-1.5 * H + 0.5 * Ho - gp) + beta * L;
  int k = band_index(B, i, j);
  vh[c] = (k >= 0 && (fv[k] & 3) == K_SOLID) ? vb : vP;
}
__global__ void k_predict_v(Geo g, const double* __restrict__ u, const double* __restrict__ v,
                            const double* __restrict__ p, double* __restrict__ Hv,
                            const double* __restrict__ Hvo, double* __restrict__ Rv, double* __restrict__ vh,
                            Band B, const uint8_t* __restrict__ fv, double dt, double beta, double vb,
                            int first) {
  predict_v_body(g, u, v, p, Hv, Hvo, Rv, vh, B, fv, dt, beta, vb, first, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------- right-hand side and q

__device__ __forceinline__ void rhs_body(Geo g, const double* __restrict__ uh, const double* __restrict__ vh, double* __restrict__ b,
                      double idt, int bx, int by) {
  int i = bx * blockDim.x + threadIdx.x, j = by * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int P = g.pitch;
  size_t c = at(i, j, P);
  double D = (uh[c + 1] - uh[c]) * g.idx[i] + (vh[c + P] - vh[c]) * g.idy[j];
  b[c] = D * idt;
}
__global__ void k_rhs(Geo g, const double* __restrict__ uh, const double* __restrict__ vh, double* __restrict__ b,
                      double idt) {
  rhs_body(g, uh, vh, b, idt, blockIdx.x, blockIdx.y);
}

__device__ inline double cell_div(const Geo& g, const double* uh, const double* vh, int i, int j) {
  size_t c = at(i, j, g.pitch);
  return (uh[c + 1] - uh[c]) * g.idx[i] + (vh[c + g.pitch] - vh[c]) * g.idy[j];
}

// sum of D V and of V over body cells: one thread per band row sums along
// the row in order, then one thread sums the row sums in order (the mean
// feeds back into the flow, so the order of the additions is fixed)
__device__ __forceinline__ void body_sums_body(Geo g, Band B, const uint8_t* __restrict__ fc, const double* __restrict__ uh,
                            const double* __restrict__ vh, double* __restrict__ rowsum, DevScalars* sc, int bx, int by) {
  for (int bj = threadIdx.x; bj < B.h; bj += blockDim.x) {
    double a = 0.0, b = 0.0;
    const int j = B.j0 + bj;
    for (int bi = 0; bi < B.w; ++bi) {
      if (!fc[bj * B.w + bi]) continue;
      int i = B.i0 + bi;
      double V = g.dx[i] * g.dy[j];
      a += cell_div(g, uh, vh, i, j) * V;
      b += V;
    }
    rowsum[2 * bj] = a;
    rowsum[2 * bj + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sdv = 0.0, sv = 0.0;
  for (int bj = 0; bj < B.h; ++bj) {
    sdv += rowsum[2 * bj];
    sv += rowsum[2 * bj + 1];
  }
  sc->body_sum[0] = sdv;
  sc->body_sum[1] = sv;
  sc->cbar = sv > 0.0 ? sdv / sv : 0.0;
}

// The same sums over many SMs: one warp per band row, whose lanes evaluate 32
// consecutive cells at a time while every lane adds the body cells' values
// in increasing i (broadcast by shuffles), the order of the sequential loop
// above, so the row sums are the same bit for bit; k_body_total then adds
// the rows in order.
__global__ void k_body_rows(Geo g, Band B, const uint8_t* __restrict__ fc, const double* __restrict__ uh,
                            const double* __restrict__ vh, double* __restrict__ rowsum) {
  const int bj = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (bj >= B.h) return;  // the whole warp
  const int j = B.j0 + bj;
  double a = 0.0, b = 0.0;
  for (int c0 = 0; c0 < B.w; c0 += 32) {
    const int bi = c0 + lane;
    double dv = 0.0, v = 0.0;
    const bool on = bi < B.w && fc[bj * B.w + bi];
    if (on) {
      const int i = B.i0 + bi;
      v = g.dx[i] * g.dy[j];
      dv = cell_div(g, uh, vh, i, j) * v;
    }
    for (unsigned m = __ballot_sync(0xffffffffu, on); m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      a += __shfl_sync(0xffffffffu, dv, src);
      b += __shfl_sync(0xffffffffu, v, src);
    }
  }
  if (lane == 0) {
    rowsum[2 * bj] = a;
    rowsum[2 * bj + 1] = b;
  }
}
__global__ void k_body_total(Band B, const double* __restrict__ rowsum, DevScalars* sc) {
  double sdv = 0.0, sv = 0.0;
#pragma unroll 8
  for (int bj = 0; bj < B.h; ++bj) {
    sdv += rowsum[2 * bj];
    sv += rowsum[2 * bj + 1];
  }
  sc->body_sum[0] = sdv;
  sc->body_sum[1] = sv;
  sc->cbar = sv > 0.0 ? sdv / sv : 0.0;
}

// On body cells (centre inside the body) continuity is replaced by div u = q,
// q = D(uhat) - cbar, cbar the mean over those cells (zero net source).
__device__ __forceinline__ void body_fix_body(Geo g, Band B, const uint8_t* __restrict__ fc, const double* __restrict__ uh,
                           const double* __restrict__ vh, double* __restrict__ b, double* __restrict__ qband,
                           double idt, const DevScalars* __restrict__ sc, int bx, int by) {
  int bi = bx * blockDim.x + threadIdx.x, bj = by * blockDim.y + threadIdx.y;
  if (bi >= B.w || bj >= B.h) return;
  int k = bj * B.w + bi;
  if (!fc[k]) {
    qband[k] = 0.0;
    return;
  }
  int i = B.i0 + bi, j = B.j0 + bj;
  double D = cell_div(g, uh, vh, i, j);
  double q = D - sc->cbar;
  qband[k] = q;
  b[at(i, j, g.pitch)] = (D - q) * idt;
}
__global__ void k_body_fix(Geo g, Band B, const uint8_t* __restrict__ fc, const double* __restrict__ uh,
                           const double* __restrict__ vh, double* __restrict__ b, double* __restrict__ qband,
                           double idt, const DevScalars* __restrict__ sc) {
  body_fix_body(g, B, fc, uh, vh, b, qband, idt, sc, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------ forces

// f = ((I - beta L) uhat - R) / dt on solid and forcing nodes;
// F = -sum f dV + d/dt sum_solid uhat dV;  C_d = 2 F_x / c, C_l = 2 F_y / c.
__device__ __forceinline__ void force_partials_body(Geo g, Band B, const uint8_t* __restrict__ fu, const uint8_t* __restrict__ fv,
                                 const double* __restrict__ uh, const double* __restrict__ vh,
                                 const double* __restrict__ Ru, const double* __restrict__ Rv, double beta,
                                 double idt, double* __restrict__ partials, int bx, int by, int nblk) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // fx dV, fy dV, Sx, Sy
  const int P = g.pitch;
  for (int k = bx * blockDim.x + threadIdx.x; k < B.w * B.h; k += nblk * blockDim.x) {
    int i = B.i0 + k % B.w, j = B.j0 + k / B.w;
    size_t c = at(i, j, P);
    int ku = fu[k] & 3;
    if (ku != K_FLUID) {
      double x = uh[c];
      double L = g.uE[i] * (uh[c + 1] - x) + g.uW[i] * (uh[c - 1] - x) + g.uN[j] * (uh[c + P] - x) +
                 g.uS[j] * (uh[c - P] - x);
      double dV = g.dxc[i] * g.dy[j];
      acc[0] += ((x - beta * L) - Ru[c]) * idt * dV;
      if (ku == K_SOLID) acc[2] += x * dV;
    }
    int kv = fv[k] & 3;
    if (kv != K_FLUID) {
      double x = vh[c];
      double L = g.vE[i] * (vh[c + 1] - x) + g.vW[i] * (vh[c - 1] - x) + g.vN[j] * (vh[c + P] - x) +
                 g.vS[j] * (vh[c - P] - x);
      double dV = g.dx[i] * g.dyc[j];
      acc[1] += ((x - beta * L) - Rv[c]) * idt * dV;
      if (kv == K_SOLID) acc[3] += x * dV;
    }
  }
  double out[4];
  block_sum<4>(acc, out);
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) partials[4 * bx + q] = out[q];
}
__global__ void k_force_partials(Geo g, Band B, const uint8_t* __restrict__ fu, const uint8_t* __restrict__ fv,
                                 const double* __restrict__ uh, const double* __restrict__ vh,
                                 const double* __restrict__ Ru, const double* __restrict__ Rv, double beta,
                                 double idt, double* __restrict__ partials) {
  force_partials_body(g, B, fu, fv, uh, vh, Ru, Rv, beta, idt, partials, blockIdx.x, blockIdx.y, gridDim.x);
}

__device__ __forceinline__ void force_final_body(const double* __restrict__ partials, int nblk, double idt, double chord,
                              DevScalars* sc, double* cl_hist, double* cd_hist, int n, int bx, int by) {
  if (threadIdx.x != 0) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < nblk; ++k)
    for (int q = 0; q < 4; ++q) s[q] += partials[4 * k + q];
  double Fx = -s[0] + (s[2] - sc->S_prev[0]) * idt;
  double Fy = -s[1] + (s[3] - sc->S_prev[1]) * idt;
  sc->S_prev[0] = s[2];
  sc->S_prev[1] = s[3];
  sc->force[0] = Fx;
  sc->force[1] = Fy;
  cd_hist[n] = 2.0 * Fx / chord;
  cl_hist[n] = 2.0 * Fy / chord;
}
__global__ void k_force_final(const double* __restrict__ partials, int nblk, double idt, double chord,
                              DevScalars* sc, double* cl_hist, double* cd_hist, int n) {
  force_final_body(partials, nblk, idt, chord, sc, cl_hist, cd_hist, n, blockIdx.x, blockIdx.y);
}

__global__ void k_body_momentum0(Geo g, Band B, const uint8_t* __restrict__ fv, double vb,
                                 double* __restrict__ partials) {
  double acc[1] = {0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < B.w * B.h; k += gridDim.x * blockDim.x) {
    if ((fv[k] & 3) != K_SOLID) continue;
    int i = B.i0 + k % B.w, j = B.j0 + k / B.w;
    acc[0] += vb * (g.dx[i] * g.dyc[j]);
  }
  double out[1];
  block_sum<1>(acc, out);
  if (threadIdx.x == 0) partials[blockIdx.x] = out[0];
}

__global__ void k_body_momentum0_final(const double* __restrict__ partials, int nblk, DevScalars* sc) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < nblk; ++k) s += partials[k];
  sc->S_prev[0] = 0.0;
  sc->S_prev[1] = s;
}

// -------------------------------------------------------------- projection

__device__ __forceinline__ void phi_ref_body(Geo g, const double* __restrict__ phi, DevScalars* sc, int bx, int by) {
  if (threadIdx.x == 0 && bx == 0) sc->phi_ref = phi[at(g.nx - 1, 0, g.pitch)];
}
__global__ void k_phi_ref(Geo g, const double* __restrict__ phi, DevScalars* sc) {
  phi_ref_body(g, phi, sc, blockIdx.x, blockIdx.y);
}

// u = uhat - dt G phi on interior faces (boundary faces keep uhat), p += phi,
// the stored increment is shifted so that the gauge cell (nx-1, 0) is zero,
// and max |div u| is taken over cells whose centre is in the fluid.
__device__ __forceinline__ void project_body(Geo g, const double* __restrict__ uh, const double* __restrict__ vh,
                          const double* __restrict__ phi, double* __restrict__ u, double* __restrict__ v,
                          double* __restrict__ p, double* __restrict__ phi_store, Band B,
                          const uint8_t* __restrict__ fc, double dt, DevScalars* sc, int bx, int by) {
  int i = bx * blockDim.x + threadIdx.x, j = by * blockDim.y + threadIdx.y;
  const int nx = g.nx, ny = g.ny, P = g.pitch;
  unsigned long long bits = 0ull;
  if (i < nx && j < ny) {
    size_t c = at(i, j, P);
    // the increment in its gauge (cell (nx-1, 0) zero) before it is used
    const double ref = sc->phi_ref;
    double fP = phi[c] - ref;
    double uw = i == 0 ? uh[c] : uh[c] - dt * ((fP - (phi[c - 1] - ref)) * g.idxc[i]);
    double ue = i == nx - 1 ? uh[c + 1] : uh[c + 1] - dt * (((phi[c + 1] - ref) - fP) * g.idxc[i + 1]);
    double vs = j == 0 ? vh[c] : vh[c] - dt * ((fP - (phi[c - P] - ref)) * g.idyc[j]);
    double vn = j == ny - 1 ? vh[c + P] : vh[c + P] - dt * (((phi[c + P] - ref) - fP) * g.idyc[j + 1]);
    u[c] = uw;
    v[c] = vs;
    if (i == nx - 1) u[c + 1] = ue;
    if (j == ny - 1) v[c + P] = vn;
    p[c] += fP;
    phi_store[c] = fP;
    int k = band_index(B, i, j);
    if (!(k >= 0 && fc[k])) {
      double d = (ue - uw) * g.idx[i] + (vn - vs) * g.idy[j];
      bits = (unsigned long long)__double_as_longlong(fabs(d));
    }
  }
  block_max_bits(bits, &sc->div_bits);
}
__global__ void k_project(Geo g, const double* __restrict__ uh, const double* __restrict__ vh,
                          const double* __restrict__ phi, double* __restrict__ u, double* __restrict__ v,
                          double* __restrict__ p, double* __restrict__ phi_store, Band B,
                          const uint8_t* __restrict__ fc, double dt, DevScalars* sc) {
  project_body(g, uh, vh, phi, u, v, p, phi_store, B, fc, dt, sc, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------- batched forms
// One launch covers the blocks of every case of a batch: block b belongs to
// the case whose range [first[c], first[c+1]) holds it, and runs the same
// body as the single-case kernel with that case's arguments and its block
// coordinates within the case's own grid (32 x 8 threads, as above).

// the last case c with first[c] <= b
__device__ inline int case_of(const int* __restrict__ first, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ inline int blocks_in_x(int n) { return (n + TBX - 1) / TBX; }

// pass 0: solid nodes and body cells; 1, 2: forcing nodes of the u and v grids
__global__ void k_classify_batch(const StepCase* __restrict__ cs, const int* __restrict__ first, int n, int pass) {
  const int c = case_of(first, n, blockIdx.x);
  const StepCase& s = cs[c];
  if (!s.has_body) return;
  const int t = blockIdx.x - first[c], bxn = blocks_in_x(s.band.w);
  if (pass == 0)
    classify_solid_body(s.g, s.band, s.xb, s.yb, s.ea, s.eb, s.fu, s.fv, s.fc, s.au, s.av, t % bxn, t / bxn);
  else
    classify_forcing_body(s.g, s.band, pass - 1, s.xb, s.yb, s.ea, s.eb, pass == 1 ? s.fu : s.fv,
                          pass == 1 ? s.au : s.av, t % bxn, t / bxn);
}

// one block per case
__global__ void k_outflow_bc_batch(const StepCase* __restrict__ cs) {
  const StepCase& s = cs[blockIdx.x];
  if (s.g.bc == 0) outflow_bc_body(s.g, s.u, s.uh, s.u_in, s.dt, 0, 0);
}

__global__ void k_predict_u_batch(const StepCase* __restrict__ cs, const int* __restrict__ first, int n) {
  const int c = case_of(first, n, blockIdx.x);
  const StepCase& s = cs[c];
  const int t = blockIdx.x - first[c], bxn = blocks_in_x(s.g.nx - 1);
  predict_u_body(s.g, s.u, s.v, s.p, s.Hu, s.Huo, s.Ru, s.uh, s.band, s.fu, s.dt, s.beta, s.first_step, t % bxn,
                 t / bxn);
}

__global__ void k_predict_v_batch(const StepCase* __restrict__ cs, const int* __restrict__ first, int n) {
  const int c = case_of(first, n, blockIdx.x);
  const StepCase& s = cs[c];
  const int t = blockIdx.x - first[c], bxn = blocks_in_x(s.g.nx);
  predict_v_body(s.g, s.u, s.v, s.p, s.Hv, s.Hvo, s.Rv, s.vh, s.band, s.fv, s.dt, s.beta, s.vb, s.first_step,
                 t % bxn, t / bxn);
}

__global__ void k_rhs_batch(const StepCase* __restrict__ cs, const int* __restrict__ first, int n) {
  const int c = case_of(first, n, blockIdx.x);
  const StepCase& s = cs[c];
  const int t = blockIdx.x - first[c], bxn = blocks_in_x(s.g.nx);
  rhs_body(s.g, s.uh, s.vh, s.b, 1.0 / s.dt, t % bxn, t / bxn);
}

// one block of 1024 threads per case
__global__ void k_body_sums_batch(const StepCase* __restrict__ cs) {
  const StepCase& s = cs[blockIdx.x];
  if (s.has_body) body_sums_body(s.g, s.band, s.fc, s.uh, s.vh, s.rowsum, s.sc, 0, 0);
}

__global__ void k_body_fix_batch(const StepCase* __restrict__ cs, const int* __restrict__ first, int n) {
  const int c = case_of(first, n, blockIdx.x);
  const StepCase& s = cs[c];
  if (!s.has_body) return;
  const int t = blockIdx.x - first[c], bxn = blocks_in_x(s.band.w);
  body_fix_body(s.g, s.band, s.fc, s.uh, s.vh, s.b, s.qband, 1.0 / s.dt, s.sc, t % bxn, t / bxn);
}

// RED_BLOCKS blocks of 256 threads per case
__global__ void k_force_partials_batch(const StepCase* __restrict__ cs) {
  const StepCase& s = cs[blockIdx.x / RED_BLOCKS];
  if (s.has_body)
    force_partials_body(s.g, s.band, s.fu, s.fv, s.uh, s.vh, s.Ru, s.Rv, s.beta, 1.0 / s.dt, s.partials,
                        blockIdx.x % RED_BLOCKS, 0, RED_BLOCKS);
}

// one block of 32 threads per case; a case without a body has no force
__global__ void k_force_final_batch(const StepCase* __restrict__ cs) {
  const StepCase& s = cs[blockIdx.x];
  if (s.has_body) {
    force_final_body(s.partials, RED_BLOCKS, 1.0 / s.dt, s.chord, s.sc, s.cl_hist, s.cd_hist, s.n, 0, 0);
  } else if (threadIdx.x == 0) {
    s.cl_hist[s.n] = 0.0;
    s.cd_hist[s.n] = 0.0;
  }
}

// one block of 32 threads per case: the gauge value, and the divergence
// maximum cleared before the projection accumulates it
__global__ void k_phi_ref_batch(const StepCase* __restrict__ cs) {
  const StepCase& s = cs[blockIdx.x];
  phi_ref_body(s.g, s.phi, s.sc, 0, 0);
  if (threadIdx.x == 0) s.sc->div_bits = 0ull;
}

__global__ void k_project_batch(const StepCase* __restrict__ cs, const int* __restrict__ first, int n) {
  const int c = case_of(first, n, blockIdx.x);
  const StepCase& s = cs[c];
  const int t = blockIdx.x - first[c], bxn = blocks_in_x(s.g.nx);
  project_body(s.g, s.uh, s.vh, s.phi, s.u, s.v, s.p, s.phi_store, s.band, s.fc, s.dt, s.sc, t % bxn, t / bxn);
}

// the scalars each case's step reads back, gathered for one copy to the host
__global__ void k_gather_batch(const StepCase* __restrict__ cs, StepReadback* __restrict__ out) {
  const StepCase& s = cs[blockIdx.x];
  if (threadIdx.x != 0) return;
  out[blockIdx.x].sc = *s.sc;
  out[blockIdx.x].cl = s.cl_hist[s.n];
  out[blockIdx.x].cd = s.cd_hist[s.n];
}

inline dim3 grid2(int nx, int ny) { return dim3((nx + TBX - 1) / TBX, (ny + TBY - 1) / TBY); }

}  // namespace

// ---------------------------------------------------------------- launchers

void launch_outflow_bc(cudaStream_t s, const Geo& g, const double* u, double* uh, double*, double u_in,
                       double dt) {
  k_outflow_bc<<<1, 256, 0, s>>>(g, u, uh, u_in, dt);
}

void launch_classify(cudaStream_t s, const Geo& g, const Band& band, double xb, double yb, double a, double b,
                     uint8_t* fu, uint8_t* fv, uint8_t* fc, double* au, double* av) {
  dim3 blk(TBX, TBY), grd = grid2(band.w, band.h);
  k_classify_solid<<<grd, blk, 0, s>>>(g, band, xb, yb, a, b, fu, fv, fc, au, av);
  k_classify_forcing<<<grd, blk, 0, s>>>(g, band, 0, xb, yb, a, b, fu, au);
  k_classify_forcing<<<grd, blk, 0, s>>>(g, band, 1, xb, yb, a, b, fv, av);
}

void launch_predict(cudaStream_t s, const Geo& g, const double* u, const double* v, const double* p, double* Hu,
                    double* Hv, const double* Huo, const double* Hvo, double* Ru, double* Rv, double* uh,
                    double* vh, const Band& band, const uint8_t* fu, const uint8_t* fv, double dt, double beta,
                    double vb, int first) {
  dim3 blk(TBX, TBY);
  k_predict_u<<<grid2(g.nx - 1, g.ny), blk, 0, s>>>(g, u, v, p, Hu, Huo, Ru, uh, band, fu, dt, beta, first);
  k_predict_v<<<grid2(g.nx, g.ny - 1), blk, 0, s>>>(g, u, v, p, Hv, Hvo, Rv, vh, band, fv, dt, beta, vb, first);
}

void launch_rhs(cudaStream_t s, const Geo& g, const double* uh, const double* vh, double* b, double dt) {
  k_rhs<<<grid2(g.nx, g.ny), dim3(TBX, TBY), 0, s>>>(g, uh, vh, b, 1.0 / dt);
}

void launch_body_source(cudaStream_t s, const Geo& g, const Band& band, const uint8_t* fc, const double* uh,
                        const double* vh, double* b, double* qband, double dt, double* rowsum,
                        DevScalars* sc) {
  k_body_rows<<<(band.h + 7) / 8, 256, 0, s>>>(g, band, fc, uh, vh, rowsum);
  k_body_total<<<1, 1, 0, s>>>(band, rowsum, sc);
  k_body_fix<<<grid2(band.w, band.h), dim3(TBX, TBY), 0, s>>>(g, band, fc, uh, vh, b, qband, 1.0 / dt, sc);
}

void launch_forces(cudaStream_t s, const Geo& g, const Band& band, const uint8_t* fu, const uint8_t* fv,
                   const double* uh, const double* vh, const double* Ru, const double* Rv, double beta, double dt,
                   double chord, double* partials, DevScalars* sc, double* cl_hist, double* cd_hist, int n) {
  k_force_partials<<<RED_BLOCKS, 256, 0, s>>>(g, band, fu, fv, uh, vh, Ru, Rv, beta, 1.0 / dt, partials);
  k_force_final<<<1, 32, 0, s>>>(partials, RED_BLOCKS, 1.0 / dt, chord, sc, cl_hist, cd_hist, n);
}

void launch_init_body_momentum(cudaStream_t s, const Geo& g, const Band& band, const uint8_t* fv, double vb,
                               double* partials, DevScalars* sc) {
  k_body_momentum0<<<RED_BLOCKS, 256, 0, s>>>(g, band, fv, vb, partials);
  k_body_momentum0_final<<<1, 32, 0, s>>>(partials, RED_BLOCKS, sc);
}

void launch_phi_ref(cudaStream_t s, const Geo& g, const double* phi, DevScalars* sc) {
  k_phi_ref<<<1, 32, 0, s>>>(g, phi, sc);
}

void launch_project(cudaStream_t s, const Geo& g, const double* uh, const double* vh, const double* phi, double* u,
                    double* v, double* p, double* phi_store, const Band& band, const uint8_t* fc, double dt,
                    DevScalars* sc) {
  k_project<<<grid2(g.nx, g.ny), dim3(TBX, TBY), 0, s>>>(g, uh, vh, phi, u, v, p, phi_store, band, fc, dt, sc);
}

}  // namespace ibm

namespace ibm {

int batch_blocks(const StepCase& c, int kind) {
  auto g2 = [](int nx, int ny) { return ((nx + 31) / 32) * ((ny + 7) / 8); };
  switch (kind) {
    case BK_BAND: return g2(c.band.w, c.band.h);
    case BK_PREDICT_U: return g2(c.g.nx - 1, c.g.ny);
    case BK_PREDICT_V: return g2(c.g.nx, c.g.ny - 1);
    default: return g2(c.g.nx, c.g.ny);
  }
}

void launch_classify_batch(cudaStream_t s, const StepCase* cs, const int* first, int n, int total) {
  for (int pass = 0; pass < 3; ++pass) k_classify_batch<<<total, dim3(TBX, TBY), 0, s>>>(cs, first, n, pass);
}

void launch_outflow_bc_batch(cudaStream_t s, const StepCase* cs, int n) {
  k_outflow_bc_batch<<<n, 256, 0, s>>>(cs);
}

void launch_predict_batch(cudaStream_t s, const StepCase* cs, const int* first_u, int total_u, const int* first_v,
                          int total_v, int n) {
  k_predict_u_batch<<<total_u, dim3(TBX, TBY), 0, s>>>(cs, first_u, n);
  k_predict_v_batch<<<total_v, dim3(TBX, TBY), 0, s>>>(cs, first_v, n);
}

void launch_rhs_batch(cudaStream_t s, const StepCase* cs, const int* first_cells, int total_cells,
                      const int* first_band, int total_band, int n) {
  k_rhs_batch<<<total_cells, dim3(TBX, TBY), 0, s>>>(cs, first_cells, n);
  k_body_sums_batch<<<n, 1024, 0, s>>>(cs);
  k_body_fix_batch<<<total_band, dim3(TBX, TBY), 0, s>>>(cs, first_band, n);
}

void launch_forces_batch(cudaStream_t s, const StepCase* cs, int n) {
  k_force_partials_batch<<<n * RED_BLOCKS, 256, 0, s>>>(cs);
  k_force_final_batch<<<n, 32, 0, s>>>(cs);
}

void launch_project_batch(cudaStream_t s, const StepCase* cs, const int* first_cells, int total_cells, int n,
                          StepReadback* out) {
  k_phi_ref_batch<<<n, 32, 0, s>>>(cs);
  k_project_batch<<<total_cells, dim3(TBX, TBY), 0, s>>>(cs, first_cells, n);
  k_gather_batch<<<n, 32, 0, s>>>(cs, out);
}

}  // namespace ibm
