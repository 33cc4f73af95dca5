// Pressure solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host application whose device
// memory is owned by its own allocator or a pool sized up front, a framework
// that forbids allocation on its hot path, or a real-time loop that cannot
// take the device-wide synchronisation an allocation may cause.  This
// variant of the red-black SOR pressure solve therefore keeps its scratch
// (the 1-D coefficient arrays and the residual-norm accumulator) in one
// file-scope __device__ array of fixed size, so the caller only passes its
// own input and output buffers.  Every GPU that loads the library holds this
// array (256 KB) until the process exits.
//
// The iterates are those of ibm_poisson_solve on an FP64 (precision 0)
// context of the same grid: same sweep order, same fma chains, same
// reciprocal diagonal (1/(aE+aW+aN+aS), computed here on the device with the
// same IEEE operations).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/ibm.h"
#include "ibm_internal.h"

namespace {

constexpr int NOALLOC_MAX_N = 8192;  // largest nx and ny
constexpr int COEF = 4 * NOALLOC_MAX_N;

// [0, COEF): pE, pW (x), pN, pS (y); then the norm accumulator and the gauge value
static __device__ __align__(256) double g_noalloc_scratch[COEF + 8];

constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mutex;

// device address of the scratch array for the current device (looked up
// once per device, with that device current)
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return IBM_E_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return IBM_E_CUDA;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return IBM_OK;
}

struct NoAllocGrid {
  int nx, ny;
  const double *pE, *pW, *pN, *pS;
};

__device__ inline unsigned long long abs_bits(double r) {
  return (unsigned long long)__double_as_longlong(fabs(r));
}

// Red-black half-sweep on the caller's compact layout (phi[j*nx + i]);
// neighbours outside the grid read as zero and carry zero coefficients.
__global__ void k_na_half(NoAllocGrid g, double* __restrict__ phi, const double* __restrict__ b, int colour,
                          double omega) {
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((colour + j) & 1);
  if (j >= g.ny || i >= g.nx) return;
  const int nx = g.nx;
  size_t c = (size_t)j * nx + i;
  double xE = i < nx - 1 ? phi[c + 1] : 0.0;
  double xW = i > 0 ? phi[c - 1] : 0.0;
  double xN = j < g.ny - 1 ? phi[c + nx] : 0.0;
  double xS = j > 0 ? phi[c - nx] : 0.0;
  double s = g.pE[i] * xE;
  s = fma(g.pW[i], xW, s);
  s = fma(g.pN[j], xN, s);
  s = fma(g.pS[j], xS, s);
  double invd = 1.0 / (g.pE[i] + g.pW[i] + g.pN[j] + g.pS[j]);
  double gs = (s - b[c]) * invd;
  double x = phi[c];
  phi[c] = fma(omega, gs - x, x);
}

__global__ void k_na_res(NoAllocGrid g, const double* __restrict__ phi, const double* __restrict__ b,
                         unsigned long long* __restrict__ bits_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned long long bits = 0ull;
  if (i < g.nx && j < g.ny) {
    const int nx = g.nx;
    size_t c = (size_t)j * nx + i;
    double x = phi[c];
    double xE = i < nx - 1 ? phi[c + 1] : 0.0;
    double xW = i > 0 ? phi[c - 1] : 0.0;
    double xN = j < g.ny - 1 ? phi[c + nx] : 0.0;
    double xS = j > 0 ? phi[c - nx] : 0.0;
    double L = g.pE[i] * (xE - x);
    L = fma(g.pW[i], xW - x, L);
    L = fma(g.pN[j], xN - x, L);
    L = fma(g.pS[j], xS - x, L);
    bits = abs_bits(b[c] - L);
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = w > bits ? w : bits;
  }
  if (((threadIdx.x + threadIdx.y * blockDim.x) & 31) == 0 && bits) atomicMax(bits_out, bits);
}

__global__ void k_na_ref(const double* __restrict__ phi, int nx, double* __restrict__ ref) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *ref = phi[nx - 1];  // cell (nx-1, 0)
}

__global__ void k_na_shift(double* __restrict__ phi, size_t n, const double* __restrict__ ref) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n) phi[k] -= *ref;
}

// 1-D coefficients of the pressure Laplacian from face coordinates, with the
// same operations (and rounding) as the context's grid set-up.
void axis_coefficients(const double* f, int n, double* aPlus, double* aMinus) {
  // centre spacing between cells m-1 and m
  auto dc = [f](int m) { return 0.5 * (f[m] + f[m + 1]) - 0.5 * (f[m - 1] + f[m]); };
  for (int m = 0; m < n; ++m) {
    double d = f[m + 1] - f[m];
    aPlus[m] = m < n - 1 ? 1.0 / (d * dc(m + 1)) : 0.0;
    aMinus[m] = m > 0 ? 1.0 / (d * dc(m)) : 0.0;
  }
}

// host staging of the coefficients (guarded by g_scratch_mutex; the copy
// from pageable memory has consumed the buffer when cudaMemcpyAsync returns)
double g_coef[COEF];

// sets the thread's error message for a failed CUDA call and returns IBM_E_CUDA
int cuda_fail(const char* what, cudaError_t e) {
  char msg[200];
  snprintf(msg, sizeof msg, "ibm_poisson_solve_noalloc: %s failed: %s", what, cudaGetErrorString(e));
  ibm::set_last_error(msg);
  return IBM_E_CUDA;
}

// index of the first face that does not exceed its predecessor, or -1
int first_non_increasing(const double* f, int n) {
  for (int m = 0; m < n; ++m)
    if (!(f[m + 1] > f[m])) return m + 1;
  return -1;
}

}  // namespace

extern "C" int ibm_poisson_solve_noalloc(int nx, int ny, const double* xf, const double* yf, const double* b_dev,
                                         double* phi_dev, double omega, double tol, int check_every, int max_sweeps,
                                         void* stream, int* sweeps, double* res) {
  char msg[200];
  if (nx > NOALLOC_MAX_N || ny > NOALLOC_MAX_N) {
    snprintf(msg, sizeof msg, "ibm_poisson_solve_noalloc: nx=%d, ny=%d exceed the static scratch limit of %d per axis",
             nx, ny, NOALLOC_MAX_N);
    ibm::set_last_error(msg);
    return IBM_E_INVAL;
  }
  if (nx < 2 || ny < 2 || !xf || !yf || !b_dev || !phi_dev || !(tol > 0.0) || !(omega > 0.0 && omega < 2.0)) {
    ibm::set_last_error("ibm_poisson_solve_noalloc: invalid argument");
    return IBM_E_INVAL;
  }
  for (int a = 0; a < 2; ++a) {
    const int bad = first_non_increasing(a ? yf : xf, a ? ny : nx);
    if (bad >= 0) {
      snprintf(msg, sizeof msg, "ibm_poisson_solve_noalloc: %s[%d] does not exceed %s[%d] (faces must increase)",
               a ? "yf" : "xf", bad, a ? "yf" : "xf", bad - 1);
      ibm::set_last_error(msg);
      return IBM_E_INVAL;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) {
    ibm::set_last_error("ibm_poisson_solve_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return rc;
  }
  {
    // only the segments this grid uses: nx values of pE and pW, ny of pN and pS
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    axis_coefficients(xf, nx, g_coef, g_coef + NOALLOC_MAX_N);
    axis_coefficients(yf, ny, g_coef + 2 * NOALLOC_MAX_N, g_coef + 3 * NOALLOC_MAX_N);
    for (int seg = 0; seg < 4; ++seg) {
      const size_t off = (size_t)seg * NOALLOC_MAX_N, len = seg < 2 ? nx : ny;
      const cudaError_t e =
          cudaMemcpyAsync(scratch + off, g_coef + off, sizeof(double) * len, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync of the coefficients", e);
    }
  }
  NoAllocGrid g{nx, ny, scratch, scratch + NOALLOC_MAX_N, scratch + 2 * NOALLOC_MAX_N, scratch + 3 * NOALLOC_MAX_N};
  unsigned long long* norm = (unsigned long long*)(scratch + COEF);
  double* ref = scratch + COEF + 1;
  const int m = check_every > 0 ? check_every : 8;
  const int maxs = max_sweeps > 0 ? max_sweeps : 1000000;
  dim3 blk(32, 8), grd_res((nx + 31) / 32, (ny + 7) / 8), grd_half(((nx + 1) / 2 + 31) / 32, (ny + 7) / 8);
  for (int it = 0;; ++it) {
    if (it % m == 0) {
      unsigned long long bits = 0;
      cudaError_t e = cudaMemsetAsync(norm, 0, sizeof(unsigned long long), s);
      if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync of the norm", e);
      k_na_res<<<grd_res, blk, 0, s>>>(g, phi_dev, b_dev, norm);
      e = cudaMemcpyAsync(&bits, norm, sizeof bits, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync of the norm", e);
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail("the residual check (cudaStreamSynchronize)", e);
      double r;
      std::memcpy(&r, &bits, sizeof r);
      if (sweeps) *sweeps = it;
      if (res) *res = r;
      if (!std::isfinite(r)) {
        ibm::set_last_error("ibm_poisson_solve_noalloc: residual is not finite");
        return IBM_E_DIVERGED;
      }
      if (r <= tol) break;
    }
    if (it >= maxs) {
      ibm::set_last_error("ibm_poisson_solve_noalloc: max_sweeps reached before the tolerance");
      return IBM_E_NOCONV;
    }
    k_na_half<<<grd_half, blk, 0, s>>>(g, phi_dev, b_dev, 0, omega);
    k_na_half<<<grd_half, blk, 0, s>>>(g, phi_dev, b_dev, 1, omega);
  }
  const size_t n = (size_t)nx * ny;
  k_na_ref<<<1, 32, 0, s>>>(phi_dev, nx, ref);
  k_na_shift<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(phi_dev, n, ref);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("a kernel launch", e);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail("the final cudaStreamSynchronize", e);
  return IBM_OK;
}
