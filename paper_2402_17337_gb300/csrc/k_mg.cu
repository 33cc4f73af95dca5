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

// ---- the small levels of the hierarchy in one CTA: the V-cycle below a
// level whose cells (with all coarser levels) fit in shared memory runs in a
// single launch instead of four launches per level, each of which would be
// mostly launch latency.  Same operations as the per-level kernels: two
// red-black Gauss-Seidel sweeps before and after, residual and restriction,
// bilinear prolongation, SOR on the coarsest level; corrections from zero.
__device__ inline float tail_sum(const MgLevel& L, const float* e, int i, int j) {
  const int nx = L.g.nx, ny = L.g.ny, t = j * nx + i;
  const float xE = i < nx - 1 ? e[t + 1] : 0.f, xW = i > 0 ? e[t - 1] : 0.f;
  const float xN = j < ny - 1 ? e[t + nx] : 0.f, xS = j > 0 ? e[t - nx] : 0.f;
  float sum = L.pE[i] * xE;
  sum = fmaf(L.pW[i], xW, sum);
  sum = fmaf(L.g.pN[j], xN, sum);
  sum = fmaf(L.g.pS[j], xS, sum);
  return sum;
}

__device__ inline void tail_relax(const MgLevel& L, float* e, const float* r, float omega, int sweeps) {
  const int nx = L.g.nx, n = nx * L.g.ny;
  for (int s = 0; s < sweeps; ++s)
    for (int c = 0; c < 2; ++c) {
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int i = t % nx, j = t / nx;
        if (((i + j) & 1) != c) continue;
        const float gs = (tail_sum(L, e, i, j) - r[t]) * L.invd[rb_at(i, j, L.g.ny, L.g.pk)];
        e[t] = fmaf(omega, gs - e[t], e[t]);
      }
      __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_mg_tail(const MgTail T, float* __restrict__ e_top) {
  extern __shared__ float tail_smem[];
  float* se = tail_smem;               // corrections of all tail levels
  float* sr = tail_smem + kTailCells;  // right-hand sides
  const MgLevel& top = T.lv[0];
  for (int t = threadIdx.x; t < top.g.nx * top.g.ny; t += blockDim.x) {
    const int i = t % top.g.nx, j = t / top.g.nx;
    sr[t] = top.r[rb_at(i, j, top.g.ny, top.g.pk)];
  }
  for (int l = 0; l < T.n; ++l) {
    const MgLevel& A = T.lv[l];
    float *e = se + T.off[l], *r = sr + T.off[l];
    const int n = A.g.nx * A.g.ny;
    for (int t = threadIdx.x; t < n; t += blockDim.x) e[t] = 0.f;
    __syncthreads();
    if (l == T.n - 1) {
      tail_relax(A, e, r, T.omega_c, T.sweeps_c);
      break;
    }
    tail_relax(A, e, r, 1.0f, 2);
    const MgLevel& C = T.lv[l + 1];
    float* rc = sr + T.off[l + 1];
    for (int t = threadIdx.x; t < C.g.nx * C.g.ny; t += blockDim.x) {
      const int I = t % C.g.nx, J = t / C.g.nx;
      float acc = 0.f;
      for (int b = 0; b < 2; ++b) {
        const int j = 2 * J + b;
        if (j >= A.g.ny) break;
        float row = 0.f;
        for (int a = 0; a < 2; ++a) {
          const int i = 2 * I + a;
          if (i >= A.g.nx) break;
          const int u = j * A.g.nx + i;
          const float x = e[u];
          const float xE = i < A.g.nx - 1 ? e[u + 1] : x, xW = i > 0 ? e[u - 1] : x;
          const float xN = j < A.g.ny - 1 ? e[u + A.g.nx] : x, xS = j > 0 ? e[u - A.g.nx] : x;
          float Le = A.pE[i] * (xE - x);
          Le = fmaf(A.pW[i], xW - x, Le);
          Le = fmaf(A.g.pN[j], xN - x, Le);
          Le = fmaf(A.g.pS[j], xS - x, Le);
          row = fmaf(A.wx[i], r[u] - Le, row);
        }
        acc = fmaf(A.wy[j], row, acc);
      }
      rc[t] = acc;
    }
    __syncthreads();
  }
  for (int l = T.n - 2; l >= 0; --l) {
    const MgLevel& A = T.lv[l];
    const MgLevel& C = T.lv[l + 1];
    float *e = se + T.off[l], *r = sr + T.off[l];
    const float* ec = se + T.off[l + 1];
    for (int t = threadIdx.x; t < A.g.nx * A.g.ny; t += blockDim.x) {
      const int i = t % A.g.nx, j = t / A.g.nx;
      const int I = i >> 1, J = j >> 1, I2 = I + A.ox[i], J2 = J + A.oy[j];
      const float ax = A.ax[i], ay = A.ay[j];
      const float e00 = ec[J * C.g.nx + I], e10 = ec[J * C.g.nx + I2];
      const float e01 = ec[J2 * C.g.nx + I], e11 = ec[J2 * C.g.nx + I2];
      const float lo = fmaf(ax, e10 - e00, e00), hi = fmaf(ax, e11 - e01, e01);
      e[t] += fmaf(ay, hi - lo, lo);
    }
    __syncthreads();
    tail_relax(A, e, r, 1.0f, 2);
  }
  for (int t = threadIdx.x; t < top.g.nx * top.g.ny; t += blockDim.x) {
    const int i = t % top.g.nx, j = t / top.g.nx;
    e_top[rb_at(i, j, top.g.ny, top.g.pk)] = se[t];
  }
}

constexpr int kFcgSlots = 128;

// ---- flexible conjugate gradients, FCG(1), preconditioned by the V-cycle,
// on level 0 in the volume-weighted inner product <a, b> = sum V_ij a_ij b_ij
// (L is self-adjoint in it).  Scalars stay on the device in FcgScalars:
// each inner product is accumulated in kFcgSlots FP64 slots (block b adds
// into slot b mod kFcgSlots, so the atomics do not pile onto one address);
// the last block of a reduction kernel (found by a counter after a memory
// fence) sums the slots, derives alpha or beta, and clears the slots and
// the counter for the next use.  Products and warp sums are FP32, block and
// slot sums FP64.
struct FcgScalars {
  double slot[3][kFcgSlots];  // <p, Lp>, <p, r>, <z, q>
  double pq;                  // <p, Lp> of the current direction
  float alpha, beta;
  unsigned int count;
};

// adds the block's sum of v into slots; returns true in the block that
// finished last (all other blocks' additions are then visible)
__device__ inline bool block_sum_add(float v, double* slots, unsigned int* count, bool last_check) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double ws[32];
  __shared__ bool last;
  const int t = threadIdx.x + threadIdx.y * blockDim.x, lane = t & 31, warp = t >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  __syncthreads();  // ws may still be read by a previous call
  if (lane == 0) ws[warp] = (double)v;
  __syncthreads();
  if (t == 0) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += ws[w];
    atomicAdd(&slots[(blockIdx.x + gridDim.x * blockIdx.y) % kFcgSlots], a);
    if (last_check) {
      __threadfence();
      last = atomicAdd(count, 1u) == gridDim.x * gridDim.y - 1;
    }
  }
  __syncthreads();
  return last_check && last;
}

// sum of one scalar's slots (warp 0 of the calling block), slots cleared
__device__ inline double take_slots(double* slots) {
  __shared__ double out;
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
  if (t < 32) {
    double a = 0.0;
    for (int k = t; k < kFcgSlots; k += 32) {
      a += *(volatile double*)&slots[k];
      slots[k] = 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (t == 0) out = a;
  }
  __syncthreads();
  return out;
}

// The two reduction kernels run a grid-stride loop over 32 x 8 tiles with at
// most kReduceBlocks blocks, so the slot and counter atomics stay few.
constexpr int kReduceBlocks = 1216;  // 8 CTAs of 8 warps per SM: full occupancy to hide load latency

// <z, q>; the last block sets beta = -<z, q> / <p, Lp> of the previous direction
__global__ void k_fcg_dot(const MgLevel L, const float* __restrict__ dxv, const float* __restrict__ dyv,
                          const float* __restrict__ z, const float* __restrict__ q, FcgScalars* __restrict__ sc) {
  const int tx = (L.g.nx + 31) / 32, nt = tx * ((L.g.ny + 7) / 8);
  float v = 0.f;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int i = (t % tx) * 32 + threadIdx.x, j = (t / tx) * 8 + threadIdx.y;
    if (i < L.g.nx && j < L.g.ny) {
      const size_t o = rb_at(i, j, L.g.ny, L.g.pk);
      v = fmaf(dxv[i] * dyv[j] * z[o], q[o], v);
    }
  }
  if (block_sum_add(v, sc->slot[2], &sc->count, true)) {
    const double zq = take_slots(sc->slot[2]);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      sc->beta = sc->pq != 0.0 ? (float)(-zq / sc->pq) : 0.f;
      sc->count = 0u;
    }
  }
}

// p = z (first) or p = z + beta p
__global__ void k_fcg_dir(const MgLevel L, const float* __restrict__ z, float* __restrict__ p,
                          const FcgScalars* __restrict__ sc, int first) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.g.nx || j >= L.g.ny) return;
  const size_t o = rb_at(i, j, L.g.ny, L.g.pk);
  p[o] = first ? z[o] : fmaf(sc->beta, p[o], z[o]);
}

// q = L p, <p, q>, <p, r>; the last block sets alpha = <p, r> / <p, q>
__global__ void k_fcg_apply(const MgLevel L, const float* __restrict__ dxv, const float* __restrict__ dyv,
                            const float* __restrict__ p, const float* __restrict__ r, float* __restrict__ q,
                            FcgScalars* __restrict__ sc) {
  float vpq = 0.f, vpr = 0.f;
  const int nx = L.g.nx, ny = L.g.ny, pk = L.g.pk;
  const int tx = (nx + 31) / 32, nt = tx * ((ny + 7) / 8);
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int i = (t % tx) * 32 + threadIdx.x, j = (t / tx) * 8 + threadIdx.y;
    if (i >= nx || j >= ny) continue;
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
    const float Vx = dxv[i] * dyv[j] * x;
    vpq = fmaf(Vx, Lp, vpq);
    vpr = fmaf(Vx, r[o], vpr);
  }
  block_sum_add(vpq, sc->slot[0], &sc->count, false);
  if (block_sum_add(vpr, sc->slot[1], &sc->count, true)) {
    const double pq = take_slots(sc->slot[0]);
    const double pr = take_slots(sc->slot[1]);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      sc->pq = pq;
      sc->alpha = pq != 0.0 ? (float)(pr / pq) : 0.f;
      sc->count = 0u;
    }
  }
}

// x += alpha p; r -= alpha q
__global__ void k_fcg_update(const MgLevel L, const float* __restrict__ p, const float* __restrict__ q,
                             float* __restrict__ x, float* __restrict__ r, const FcgScalars* __restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.g.nx || j >= L.g.ny) return;
  const size_t o = rb_at(i, j, L.g.ny, L.g.pk);
  const float alpha = sc->alpha;
  x[o] = fmaf(alpha, p[o], x[o]);
  r[o] = fmaf(-alpha, q[o], r[o]);
}

}  // namespace

size_t fcg_scalars_bytes() { return sizeof(FcgScalars); }

inline int reduce_blocks(const MgLevel& L) {
  const int nt = ((L.g.nx + 31) / 32) * ((L.g.ny + 7) / 8);
  return nt < kReduceBlocks ? nt : kReduceBlocks;
}

void launch_fcg_dot(cudaStream_t s, const MgLevel& L, const float* dxv, const float* dyv, const float* z,
                    const float* q, void* sc) {
  k_fcg_dot<<<reduce_blocks(L), dim3(32, 8), 0, s>>>(L, dxv, dyv, z, q, (FcgScalars*)sc);
}
void launch_fcg_dir(cudaStream_t s, const MgLevel& L, const float* z, float* p, const void* sc, int first) {
  k_fcg_dir<<<grid_for(L.g.nx, L.g.ny), dim3(32, 8), 0, s>>>(L, z, p, (const FcgScalars*)sc, first);
}
void launch_fcg_apply(cudaStream_t s, const MgLevel& L, const float* dxv, const float* dyv, const float* p,
                      const float* r, float* q, void* sc) {
  k_fcg_apply<<<reduce_blocks(L), dim3(32, 8), 0, s>>>(L, dxv, dyv, p, r, q, (FcgScalars*)sc);
}
void launch_fcg_update(cudaStream_t s, const MgLevel& L, const float* p, const float* q, float* x, float* r,
                       const void* sc) {
  k_fcg_update<<<grid_for(L.g.nx, L.g.ny), dim3(32, 8), 0, s>>>(L, p, q, x, r, (const FcgScalars*)sc);
}

int mg_coarse_max() { return kCoarseMax; }

cudaError_t prepare_mg_tail() {
  return cudaFuncSetAttribute(k_mg_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(2 * kTailCells * sizeof(float)));
}

void launch_mg_tail(cudaStream_t s, const MgTail& T, float* e_top) {
  k_mg_tail<<<1, 1024, 2 * kTailCells * sizeof(float), s>>>(T, e_top);
}

void launch_mg_restrict(cudaStream_t s, const MgLevel& F, const float* ef, const MgLevel& C) {
  k_mg_restrict<<<grid_for(C.g.nx, C.g.ny), dim3(32, 8), 0, s>>>(F, ef, C);
}

void launch_mg_prolong(cudaStream_t s, const MgLevel& C, const float* ec, const MgLevel& F, float* ef) {
  k_mg_prolong<<<grid_for(F.g.nx, F.g.ny), dim3(32, 8), 0, s>>>(C, ec, F, ef);
}

void launch_mg_coarse(cudaStream_t s, const MgLevel& L, float* e_out, float omega, int sweeps) {
  const int n = L.g.nx * L.g.ny, threads = n >= 1024 ? 1024 : (n + 31) / 32 * 32;  // few warps: cheap barriers
  k_mg_coarse<<<1, threads, 0, s>>>(L, e_out, omega, sweeps);
}

}  // namespace ibm
