// Geometric multigrid for the pressure correction equation L_p e = r
// (FP32, inside the FP64 defect correction).
//
// The paper solves the pressure equation by red-black SOR (Sec. 2.2); this
// is a variant that reaches the same FP64 residual tolerance in fewer
// sweeps.  The hierarchy coarsens the stretched grid (Sec. 2.3) by merging
// pairs of cells (level l+1 has the faces x_f[0], x_f[2], ... of level l),
// and every level carries the same five-point operator per unit volume,
// rediscretised from its own faces:
//   (L e)_ij = pE_i (e_E - e) + pW_i (e_W - e) + pN_j (e_N - e) + pS_j (e_S - e).
// Transfers:
//   restriction  r_c(I,J) = sum over children of (dx_i / dX_I)(dy_j / dY_J) res_f(i,j)
//                (the volume-weighted average of the fine residual);
//   prolongation e_f(i,j) += bilinear interpolation of e_c between the
//                centre of the parent cell and the centres of the neighbours
//                on the fine cell's side, in the stretched coordinates (zero
//                slope at the domain boundary).
// Interpolation of order 2 and restriction of order 1 add up to more than
// the order of the operator, as cell-centred multigrid needs for V-cycles
// whose convergence does not degrade with the number of levels; piecewise
// constant interpolation (1 + 1) lost convergence on deep hierarchies.
// Smoothing is red-black Gauss-Seidel by the FP32 tile kernel of k_mixed.cu;
// the coarsest level (a few dozen cells) is solved by red-black SOR inside
// one CTA.  All arrays use the colour-split layout rb_at of the FP32 sweeps.
#include "ibm_internal.h"

namespace ibm {

namespace {

__device__ inline float level_res(const MgLevel& L, const float* __restrict__ e, int i, int j) {
  const int nx = L.g.nx, ny = L.g.ny, pk = L.g.pk;
  const float x = e[rb_at(i, j, ny, pk)];
  const float xE = i < nx - 1 ? e[rb_at(i + 1, j, ny, pk)] : x;
  const float xW = i > 0 ? e[rb_at(i - 1, j, ny, pk)] : x;
  const float xN = j < ny - 1 ? e[rb_at(i, j + 1, ny, pk)] : x;
  const float xS = j > 0 ? e[rb_at(i, j - 1, ny, pk)] : x;
  float Le = L.pE[i] * (xE - x);
  Le = fmaf(L.pW[i], xW - x, Le);
  Le = fmaf(L.g.pN[j], xN - x, Le);
  Le = fmaf(L.g.pS[j], xS - x, Le);
  return L.r[rb_at(i, j, ny, pk)] - Le;
}

// one thread per coarse cell: residual of its (up to four) children, restricted
__global__ void k_mg_restrict(const MgLevel F, const float* __restrict__ ef, MgLevel C) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= C.g.nx || J >= C.g.ny) return;
  float acc = 0.f;
  for (int b = 0; b < 2; ++b) {
    const int j = 2 * J + b;
    if (j >= F.g.ny) break;
    float row = 0.f;
    for (int a = 0; a < 2; ++a) {
      const int i = 2 * I + a;
      if (i >= F.g.nx) break;
      row = fmaf(F.wx[i], level_res(F, ef, i, j), row);
    }
    acc = fmaf(F.wy[j], row, acc);
  }
  C.r[rb_at(I, J, C.g.ny, C.g.pk)] = acc;
}

// one thread per fine cell: parent I = i/2 and neighbour I + ox_i (ox_i in
// {-1, 0, +1}, 0 at the boundary) with weight ax_i on the neighbour, the same
// in y
__global__ void k_mg_prolong(const MgLevel C, const float* __restrict__ ec, MgLevel F, float* __restrict__ ef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= F.g.nx || j >= F.g.ny) return;
  const int I = i >> 1, J = j >> 1, I2 = I + F.ox[i], J2 = J + F.oy[j];
  const float ax = F.ax[i], ay = F.ay[j];
  const int ny = C.g.ny, pk = C.g.pk;
  const float e00 = ec[rb_at(I, J, ny, pk)], e10 = ec[rb_at(I2, J, ny, pk)];
  const float e01 = ec[rb_at(I, J2, ny, pk)], e11 = ec[rb_at(I2, J2, ny, pk)];
  const float lo = fmaf(ax, e10 - e00, e00), hi = fmaf(ax, e11 - e01, e01);
  ef[rb_at(i, j, F.g.ny, F.g.pk)] += fmaf(ay, hi - lo, lo);
}

// coarsest level: red-black SOR from e = 0 in shared memory, one CTA
constexpr int kCoarseMax = 1024;  // cells the coarsest level may hold

__global__ void __launch_bounds__(1024) k_mg_coarse(MgLevel L, float* __restrict__ e_out, float omega, int sweeps) {
  __shared__ float se[kCoarseMax], sr[kCoarseMax], sd[kCoarseMax];
  const int nx = L.g.nx, ny = L.g.ny, n = nx * ny;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % nx, j = t / nx;
    const size_t o = rb_at(i, j, ny, L.g.pk);
    se[t] = 0.f;
    sr[t] = L.r[o];
    sd[t] = L.invd[o];
  }
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 2; ++c) {
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int i = t % nx, j = t / nx;
        if (((i + j) & 1) != c) continue;
        const float xE = i < nx - 1 ? se[t + 1] : 0.f, xW = i > 0 ? se[t - 1] : 0.f;
        const float xN = j < ny - 1 ? se[t + nx] : 0.f, xS = j > 0 ? se[t - nx] : 0.f;
        float sum = L.pE[i] * xE;
        sum = fmaf(L.pW[i], xW, sum);
        sum = fmaf(L.g.pN[j], xN, sum);
        sum = fmaf(L.g.pS[j], xS, sum);
        const float gs = (sum - sr[t]) * sd[t];
        se[t] = fmaf(omega, gs - se[t], se[t]);
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % nx, j = t / nx;
    e_out[rb_at(i, j, ny, L.g.pk)] = se[t];
  }
}

inline dim3 grid_for(int nx, int ny) { return dim3((nx + 31) / 32, (ny + 7) / 8); }

// ---- flexible conjugate gradients, FCG(1), preconditioned by the V-cycle,
// on level 0 in the volume-weighted inner product <a, b> = sum V_ij a_ij b_ij
// (L is self-adjoint in it).  Scalars stay on the device: sc[0] = <p, Lp>,
// sc[1] = <p, r>, sc[2] = <z, q>.

__device__ inline void block_sum_add(double v, double* dst) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double ws[32];
  const int t = threadIdx.x + threadIdx.y * blockDim.x, lane = t & 31, warp = t >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? ws[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(dst, v);
  }
}

// sc[2] = <z, q>
__global__ void k_fcg_dot(const MgLevel L, const float* __restrict__ dxv, const float* __restrict__ dyv,
                          const float* __restrict__ z, const float* __restrict__ q, double* __restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  double v = 0.0;
  if (i < L.g.nx && j < L.g.ny) {
    const size_t o = rb_at(i, j, L.g.ny, L.g.pk);
    v = (double)(dxv[i] * dyv[j]) * (double)z[o] * (double)q[o];
  }
  block_sum_add(v, &sc[2]);
}

// p = z (first) or p = z + beta p, beta = -<z, q> / <p, Lp> of the previous direction
__global__ void k_fcg_dir(const MgLevel L, const float* __restrict__ z, float* __restrict__ p,
                          const double* __restrict__ sc, int first) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.g.nx || j >= L.g.ny) return;
  const size_t o = rb_at(i, j, L.g.ny, L.g.pk);
  if (first) {
    p[o] = z[o];
  } else {
    const float beta = sc[0] != 0.0 ? (float)(-sc[2] / sc[0]) : 0.f;
    p[o] = fmaf(beta, p[o], z[o]);
  }
}

// q = L p, sc[0] += <p, q>, sc[1] += <p, r>
__global__ void k_fcg_apply(const MgLevel L, const float* __restrict__ dxv, const float* __restrict__ dyv,
                            const float* __restrict__ p, const float* __restrict__ r, float* __restrict__ q,
                            double* __restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  double vpq = 0.0, vpr = 0.0;
  const int nx = L.g.nx, ny = L.g.ny, pk = L.g.pk;
  if (i < nx && j < ny) {
    const size_t o = rb_at(i, j, ny, pk);
    const float x = p[o];
    const float xE = i < nx - 1 ? p[rb_at(i + 1, j, ny, pk)] : x;
    const float xW = i > 0 ? p[rb_at(i - 1, j, ny, pk)] : x;
    const float xN = j < ny - 1 ? p[rb_at(i, j + 1, ny, pk)] : x;
    const float xS = j > 0 ? p[rb_at(i, j - 1, ny, pk)] : x;
    float Lp = L.pE[i] * (xE - x);
    Lp = fmaf(L.pW[i], xW - x, Lp);
    Lp = fmaf(L.g.pN[j], xN - x, Lp);
    Lp = fmaf(L.g.pS[j], xS - x, Lp);
    q[o] = Lp;
    const double V = (double)(dxv[i] * dyv[j]);
    vpq = V * (double)x * (double)Lp;
    vpr = V * (double)x * (double)r[o];
  }
  block_sum_add(vpq, &sc[0]);
  block_sum_add(vpr, &sc[1]);
}

// alpha = <p, r> / <p, Lp>; x += alpha p; r -= alpha q
__global__ void k_fcg_update(const MgLevel L, const float* __restrict__ p, const float* __restrict__ q,
                             float* __restrict__ x, float* __restrict__ r, const double* __restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.g.nx || j >= L.g.ny) return;
  const size_t o = rb_at(i, j, L.g.ny, L.g.pk);
  const float alpha = sc[0] != 0.0 ? (float)(sc[1] / sc[0]) : 0.f;
  x[o] = fmaf(alpha, p[o], x[o]);
  r[o] = fmaf(-alpha, q[o], r[o]);
}

}  // namespace

void launch_fcg_dot(cudaStream_t s, const MgLevel& L, const float* dxv, const float* dyv, const float* z,
                    const float* q, double* sc) {
  k_fcg_dot<<<grid_for(L.g.nx, L.g.ny), dim3(32, 8), 0, s>>>(L, dxv, dyv, z, q, sc);
}
void launch_fcg_dir(cudaStream_t s, const MgLevel& L, const float* z, float* p, const double* sc, int first) {
  k_fcg_dir<<<grid_for(L.g.nx, L.g.ny), dim3(32, 8), 0, s>>>(L, z, p, sc, first);
}
void launch_fcg_apply(cudaStream_t s, const MgLevel& L, const float* dxv, const float* dyv, const float* p,
                      const float* r, float* q, double* sc) {
  k_fcg_apply<<<grid_for(L.g.nx, L.g.ny), dim3(32, 8), 0, s>>>(L, dxv, dyv, p, r, q, sc);
}
void launch_fcg_update(cudaStream_t s, const MgLevel& L, const float* p, const float* q, float* x, float* r,
                       const double* sc) {
  k_fcg_update<<<grid_for(L.g.nx, L.g.ny), dim3(32, 8), 0, s>>>(L, p, q, x, r, sc);
}

int mg_coarse_max() { return kCoarseMax; }

void launch_mg_restrict(cudaStream_t s, const MgLevel& F, const float* ef, const MgLevel& C) {
  k_mg_restrict<<<grid_for(C.g.nx, C.g.ny), dim3(32, 8), 0, s>>>(F, ef, C);
}

void launch_mg_prolong(cudaStream_t s, const MgLevel& C, const float* ec, const MgLevel& F, float* ef) {
  k_mg_prolong<<<grid_for(F.g.nx, F.g.ny), dim3(32, 8), 0, s>>>(C, ec, F, ef);
}

void launch_mg_coarse(cudaStream_t s, const MgLevel& L, float* e_out, float omega, int sweeps) {
  k_mg_coarse<<<1, 1024, 0, s>>>(L, e_out, omega, sweeps);
}

}  // namespace ibm
