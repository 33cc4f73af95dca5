// Host side of libibm: the C ABI declared in include/ibm.h, grid
// construction (Sec. 2.3), device memory of a context and the fractional-step
// driver (Sec. 2.2).
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ibm.h"
#include "ibm_internal.h"

using namespace ibm;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return fail(IBM_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------ grid (Sec. 2.3)

// hmin * (r + r^2 + ... + r^n), accumulated from the first term up
double progression_length(double hmin, double r, int n) {
  double term = 1.0, total = 0.0;
  for (int m = 0; m < n; ++m) {
    term *= r;
    total += term;
  }
  return hmin * total;
}

// Growth ratio r >= 1 of n cells hmin*r^m (m = 1..n) that fill length L:
// bracket [1, 2^k], then halve the bracket until it no longer shrinks.
bool growth_ratio(double hmin, int n, double L, double* r) {
  if (n == 0) {
    *r = 1.0;
    return true;
  }
  double lo = 1.0, hi = 2.0;
  if (progression_length(hmin, lo, n) > L) return false;
  while (progression_length(hmin, hi, n) < L) {
    hi *= 2.0;
    if (hi > 1e6) return false;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    (progression_length(hmin, mid, n) < L ? lo : hi) = mid;
  }
  *r = 0.5 * (lo + hi);
  return true;
}

// Face coordinates of one axis: uniform when hmin <= 0; otherwise a block of
// round((b1-b0)/hmin) cells of size hmin from b0, flanked by geometric
// progressions filling [a0, b0] and [block end, a1], the remaining cells
// shared in proportion to the two lengths.
bool build_axis(double a0, double a1, double b0, double b1, int n, double hmin, std::vector<double>& f) {
  f.assign(n + 1, 0.0);
  if (n < 1 || !(a1 > a0)) return false;
  if (hmin <= 0.0) {
    const double h = (a1 - a0) / n;
    for (int i = 0; i < n; ++i) f[i] = a0 + i * h;
    f[n] = a1;
    return true;
  }
  if (!(b0 >= a0 && b1 <= a1 && b1 > b0)) return false;
  const int nb = (int)std::lround((b1 - b0) / hmin);
  if (nb < 1 || nb > n) return false;
  const double bend = b0 + nb * hmin;
  if (bend > a1) return false;
  const double left = b0 - a0, right = a1 - bend;
  const int spare = n - nb;
  const int nl = (left + right > 0.0) ? (int)std::lround(spare * (left / (left + right))) : 0;
  const int nr = spare - nl;
  if ((nl == 0) != (left == 0.0) || (nr == 0) != (right == 0.0)) return false;
  double rl, rr;
  if (!growth_ratio(hmin, nl, left, &rl) || !growth_ratio(hmin, nr, right, &rr)) return false;
  for (int m = 0; m <= nb; ++m) f[nl + m] = b0 + m * hmin;
  for (int m = 1; m <= nl; ++m) f[nl - m] = b0 - progression_length(hmin, rl, m);
  for (int m = 1; m <= nr; ++m) f[nl + nb + m] = bend + progression_length(hmin, rr, m);
  f[0] = a0;
  f[n] = a1;
  return true;
}

}  // namespace

struct ibm_ctx {
  ibm_grid_params P;
  int nx = 0, ny = 0, pitch = 0, rows = 0;
  size_t nelem = 0;  // elements of one pitched field
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<double> xf, yf;
  std::vector<void*> allocs;
  Geo geo{};
  // fields (FP64, pitched)
  double *u = nullptr, *v = nullptr, *p = nullptr, *phi = nullptr, *phi2 = nullptr, *b = nullptr;
  double *uh = nullptr, *vh = nullptr, *Ru = nullptr, *Rv = nullptr;
  double *Hu = nullptr, *Hv = nullptr, *Huo = nullptr, *Hvo = nullptr;
  double *invd_p = nullptr, *invd_u = nullptr, *invd_v = nullptr;
  // mixed precision (FP32 correction, residual and reciprocal diagonal)
  Geo32 geo32{};
  float *e32 = nullptr, *e32b = nullptr, *r32 = nullptr, *invd32 = nullptr;  // e32/e32b: ping-pong
  // velocity systems in FP32 sweeps (precision >= 1): coefficients, reciprocal
  // diagonals (pitched, u and v), correction and residual (pitched)
  HelmF32 h32{};
  float *hinv_u = nullptr, *hinv_v = nullptr, *hd32 = nullptr, *hr32 = nullptr;
  int m_inner = 32;  // inner sweeps between FP64 checks (adapted)
  int sor_cfg = -1;          // tile shape of the FP32 sweeps, -1: not tuned yet
  double sor_us = 0.0;       // its measured time per full sweep
  // geometric multigrid on the correction equation (precision 2)
  std::vector<MgLevel> mg;
  int mg_shape = -1;                                 // tile shape of the smoother
  int mg_cycles = 2;                                 // V-cycles between FP64 checks (adapted)
  int mg_coarse_sweeps = 0;
  float mg_coarse_omega = 1.f;
  int mg_tail = -1;  // first level run by the one-CTA tail kernel (-1: none)
  cudaGraphExec_t mg_graph[2] = {nullptr, nullptr};  // one FCG iteration: first / later
  bool mg_graph_failed = false;
  float *fcg_x = nullptr, *fcg_p = nullptr, *fcg_q = nullptr;  // level-0 FCG vectors
  void* fcg_sc = nullptr;                                     // device scalars of the FCG iteration
  const float *mg_dxv = nullptr, *mg_dyv = nullptr;           // level-0 cell widths (inner products)
  // preconditioner of the FCG iteration: 0 the V-cycle, 1 a two-level cycle
  // whose coarse level (level 1) is corrected by a U-Net
  int pc_kind = 0;
  int pc_pre = 1;  // pre-smoothing launches (0 or 1) of the two-level cycle
  ibm_unet* pc_net = nullptr;
  double pc_cT = 1.0;
  float *pc_feat = nullptr, *pc_out = nullptr;
  unsigned long long* pc_max = nullptr;
  // body and band
  bool has_body = false;
  double chord = 1, tc = 0.12, h = 0, k = 0, xb = 0, yb0 = 0;
  Band band{0, 0, 1, 1};
  uint8_t *fu = nullptr, *fv = nullptr, *fc = nullptr;
  double *au = nullptr, *av = nullptr, *qband = nullptr, *rowsum = nullptr;
  double* partials = nullptr;
  DevScalars* sc = nullptr;
  DevScalars* sc_host = nullptr;  // pinned mirror
  // history
  double *cl_d = nullptr, *cd_d = nullptr;
  int hist_cap = 0;
  int n = 0;
  ibm_step_stats last{};
  // warm start: 0 previous increment, 1 learned (U-Net), 2 previous increment + sample capture
  int ws_mode = 0;
  int ws_base = 0;             // base guess: 0 previous increment, 1 linear extrapolation in time
  double* phi_prev = nullptr;  // increment of the previous step (ws_base 1)
  ibm_unet* ws_net = nullptr;
  double ws_cT = 1.0;
  int Hc = 0, Wc = 0;
  float *ws_feat = nullptr, *ws_out = nullptr, *ws_target = nullptr;
  double* phi_old = nullptr;
  unsigned long long* ws_max = nullptr;
  bool has_sample = false;
  // profiling
  ibm_profile prof{};
  bool profiling = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  ~ibm_ctx() {
    for (cudaGraphExec_t g : mg_graph)
      if (g) cudaGraphExecDestroy(g);
    for (void* a : allocs) cudaFree(a);
    if (sc_host) cudaFreeHost(sc_host);
    if (cl_d) cudaFree(cl_d);
    if (cd_d) cudaFree(cd_d);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  template <class T>
  int alloc(T** ptr, size_t count) {
    void* q = nullptr;
    CUDA_TRY(cudaMalloc(&q, sizeof(T) * (count ? count : 1)));
    CUDA_TRY(cudaMemset(q, 0, sizeof(T) * (count ? count : 1)));
    allocs.push_back(q);
    *ptr = (T*)q;
    return IBM_OK;
  }
  template <class T>
  int upload(const T** ptr, const std::vector<T>& h) {
    T* d = nullptr;
    int rc = alloc(&d, h.size());
    if (rc) return rc;
    CUDA_TRY(cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    *ptr = d;
    return IBM_OK;
  }
};

namespace {

// Five-point coefficients per unit volume on the cells between the faces xf,
// yf (homogeneous Neumann: no coupling across the domain boundary); the same
// formulas as the fine grid's.
void laplace_coefs(const std::vector<double>& xf, std::vector<double>& pE, std::vector<double>& pW) {
  const int n = (int)xf.size() - 1;
  std::vector<double> dx(n), xc(n);
  for (int i = 0; i < n; ++i) {
    dx[i] = xf[i + 1] - xf[i];
    xc[i] = 0.5 * (xf[i] + xf[i + 1]);
  }
  pE.assign(n, 0.0);
  pW.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    if (i < n - 1) pE[i] = 1.0 / (dx[i] * (xc[i + 1] - xc[i]));
    if (i > 0) pW[i] = 1.0 / (dx[i] * (xc[i] - xc[i - 1]));
  }
}

std::vector<double> coarse_faces(const std::vector<double>& xf) {
  const int n = (int)xf.size() - 1, nc = (n + 1) / 2;
  std::vector<double> out(nc + 1);
  for (int I = 0; I <= nc; ++I) out[I] = xf[2 * I < n ? 2 * I : n];
  return out;
}

int build_mg(ibm_ctx* c);

int setup_geometry(ibm_ctx* c) {
  const int nx = c->nx, ny = c->ny;
  const auto& xf = c->xf;
  const auto& yf = c->yf;
  std::vector<double> xc(nx), yc(ny), dx(nx), dy(ny), idx(nx), idy(ny);
  for (int i = 0; i < nx; ++i) {
    dx[i] = xf[i + 1] - xf[i];
    xc[i] = 0.5 * (xf[i] + xf[i + 1]);
    idx[i] = 1.0 / dx[i];
  }
  for (int j = 0; j < ny; ++j) {
    dy[j] = yf[j + 1] - yf[j];
    yc[j] = 0.5 * (yf[j] + yf[j + 1]);
    idy[j] = 1.0 / dy[j];
  }
  // centre spacings and face interpolation weights; the end entries encode
  // the boundary conditions (see the predictor kernels)
  std::vector<double> dxc(nx + 1, 0.0), dyc(ny + 1, 0.0), idxc(nx + 1, 0.0), idyc(ny + 1, 0.0);
  std::vector<double> wx(nx + 1, 0.5), wy(ny + 1, 0.5);
  for (int i = 1; i < nx; ++i) {
    dxc[i] = xc[i] - xc[i - 1];
    idxc[i] = 1.0 / dxc[i];
    wx[i] = (xf[i] - xc[i - 1]) / dxc[i];
  }
  for (int j = 1; j < ny; ++j) {
    dyc[j] = yc[j] - yc[j - 1];
    idyc[j] = 1.0 / dyc[j];
    wy[j] = (yf[j] - yc[j - 1]) / dyc[j];
  }
  // v at x0 for the convective flux: inflow v = 0 (weight 0 on the zero
  // ghost) or free slip (weight 1 on v itself); at x1 zero gradient.
  wx[0] = c->P.bc == 0 ? 0.0 : 1.0;
  wx[nx] = 0.0;
  // Laplacian coefficients
  std::vector<double> pE(nx), pW(nx), pN(ny), pS(ny);
  for (int i = 0; i < nx; ++i) {
    pE[i] = i < nx - 1 ? 1.0 / (dx[i] * dxc[i + 1]) : 0.0;
    pW[i] = i > 0 ? 1.0 / (dx[i] * dxc[i]) : 0.0;
  }
  for (int j = 0; j < ny; ++j) {
    pN[j] = j < ny - 1 ? 1.0 / (dy[j] * dyc[j + 1]) : 0.0;
    pS[j] = j > 0 ? 1.0 / (dy[j] * dyc[j]) : 0.0;
  }
  std::vector<double> uE(nx + 1, 0.0), uW(nx + 1, 0.0), uN(ny), uS(ny);
  for (int i = 1; i < nx; ++i) {
    uE[i] = 1.0 / (dx[i] * dxc[i]);
    uW[i] = 1.0 / (dx[i - 1] * dxc[i]);
  }
  for (int j = 0; j < ny; ++j) {
    uN[j] = j < ny - 1 ? 1.0 / (dyc[j + 1] * dy[j]) : 0.0;  // free slip: no flux through the wall
    uS[j] = j > 0 ? 1.0 / (dyc[j] * dy[j]) : 0.0;
  }
  std::vector<double> vE(nx), vW(nx), vN(ny + 1, 0.0), vS(ny + 1, 0.0);
  for (int i = 0; i < nx; ++i) {
    vE[i] = i < nx - 1 ? 1.0 / (dxc[i + 1] * dx[i]) : 0.0;
    // inflow: v = 0 on x0, half a cell from the node (ghost value 0 at the
    // mirrored point, doubled coefficient); free slip: no flux
    vW[i] = i > 0 ? 1.0 / (dxc[i] * dx[i]) : (c->P.bc == 0 ? 2.0 / (dx[0] * dx[0]) : 0.0);
  }
  for (int j = 1; j < ny; ++j) {
    vN[j] = 1.0 / (dy[j] * dyc[j]);
    vS[j] = 1.0 / (dy[j - 1] * dyc[j]);
  }
  Geo& g = c->geo;
  g.nx = nx;
  g.ny = ny;
  g.pitch = c->pitch;
  g.bc = c->P.bc;
  int rc = 0;
  rc |= c->upload(&g.xf, xf);
  rc |= c->upload(&g.yf, yf);
  rc |= c->upload(&g.xc, xc);
  rc |= c->upload(&g.yc, yc);
  rc |= c->upload(&g.dx, dx);
  rc |= c->upload(&g.dy, dy);
  rc |= c->upload(&g.idx, idx);
  rc |= c->upload(&g.idy, idy);
  rc |= c->upload(&g.dxc, dxc);
  rc |= c->upload(&g.dyc, dyc);
  rc |= c->upload(&g.idxc, idxc);
  rc |= c->upload(&g.idyc, idyc);
  rc |= c->upload(&g.wx, wx);
  rc |= c->upload(&g.wy, wy);
  rc |= c->upload(&g.pE, pE);
  rc |= c->upload(&g.pW, pW);
  rc |= c->upload(&g.pN, pN);
  rc |= c->upload(&g.pS, pS);
  rc |= c->upload(&g.uE, uE);
  rc |= c->upload(&g.uW, uW);
  rc |= c->upload(&g.uN, uN);
  rc |= c->upload(&g.uS, uS);
  rc |= c->upload(&g.vE, vE);
  rc |= c->upload(&g.vW, vW);
  rc |= c->upload(&g.vN, vN);
  rc |= c->upload(&g.vS, vS);
  if (rc) return IBM_E_CUDA;
  // reciprocal diagonals of the SOR updates (pitched tables)
  const double beta = c->P.dt / (2.0 * c->P.Re);
  std::vector<double> ip(c->nelem, 0.0), iu(c->nelem, 0.0), iv(c->nelem, 0.0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double d = pE[i] + pW[i] + pN[j] + pS[j];
      ip[at(i, j, c->pitch)] = 1.0 / d;
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i) iu[at(i, j, c->pitch)] = 1.0 / (1.0 + beta * (uE[i] + uW[i] + uN[j] + uS[j]));
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) iv[at(i, j, c->pitch)] = 1.0 / (1.0 + beta * (vE[i] + vW[i] + vN[j] + vS[j]));
  const double *a, *bb, *cc;
  rc |= c->upload(&a, ip);
  rc |= c->upload(&bb, iu);
  rc |= c->upload(&cc, iv);
  if (rc) return IBM_E_CUDA;
  c->invd_p = const_cast<double*>(a);
  c->invd_u = const_cast<double*>(bb);
  c->invd_v = const_cast<double*>(cc);
  if (c->P.precision >= 1) {
    // colour-split FP32 data of the inner sweeps (Geo32)
    Geo32& g32 = c->geo32;
    const int pk = ((nx + 1) / 2 + 31) / 32 * 32;
    g32.nx = nx;
    g32.ny = ny;
    g32.pk = pk;
    std::vector<float> ce0(pk, 0.f), ce1(pk, 0.f), cw0(pk, 0.f), cw1(pk, 0.f), pn(ny), ps(ny);
    for (int k = 0; k < pk; ++k) {
      if (2 * k < nx) ce0[k] = (float)pE[2 * k], cw0[k] = (float)pW[2 * k];
      if (2 * k + 1 < nx) ce1[k] = (float)pE[2 * k + 1], cw1[k] = (float)pW[2 * k + 1];
    }
    for (int j = 0; j < ny; ++j) pn[j] = (float)pN[j], ps[j] = (float)pS[j];
    rc |= c->upload(&g32.cE0, ce0);
    rc |= c->upload(&g32.cE1, ce1);
    rc |= c->upload(&g32.cW0, cw0);
    rc |= c->upload(&g32.cW1, cw1);
    rc |= c->upload(&g32.pN, pn);
    rc |= c->upload(&g32.pS, ps);
    const size_t n32 = (size_t)2 * ny * pk;
    std::vector<float> ip32(n32, 0.0f);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        float d = (float)pE[i] + (float)pW[i] + (float)pN[j] + (float)pS[j];
        ip32[rb_at(i, j, ny, pk)] = 1.0f / d;
      }
    const float* d32;
    rc |= c->upload(&d32, ip32);
    rc |= c->alloc(&c->e32, n32);
    rc |= c->alloc(&c->e32b, n32);
    rc |= c->alloc(&c->r32, n32);
    if (rc) return IBM_E_CUDA;
    c->invd32 = const_cast<float*>(d32);
    // velocity systems
    auto f32 = [](const std::vector<double>& a) {
      std::vector<float> o(a.size());
      for (size_t k = 0; k < a.size(); ++k) o[k] = (float)a[k];
      return o;
    };
    rc |= c->upload(&c->h32.uE, f32(uE));
    rc |= c->upload(&c->h32.uW, f32(uW));
    rc |= c->upload(&c->h32.uN, f32(uN));
    rc |= c->upload(&c->h32.uS, f32(uS));
    rc |= c->upload(&c->h32.vE, f32(vE));
    rc |= c->upload(&c->h32.vW, f32(vW));
    rc |= c->upload(&c->h32.vN, f32(vN));
    rc |= c->upload(&c->h32.vS, f32(vS));
    std::vector<float> iu32(c->nelem, 0.f), iv32(c->nelem, 0.f);
    const float b32 = (float)beta;
    for (int j = 0; j < ny; ++j)
      for (int i = 1; i < nx; ++i)
        iu32[at(i, j, c->pitch)] =
            1.0f / (1.0f + b32 * ((float)uE[i] + (float)uW[i] + (float)uN[j] + (float)uS[j]));
    for (int j = 1; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        iv32[at(i, j, c->pitch)] =
            1.0f / (1.0f + b32 * ((float)vE[i] + (float)vW[i] + (float)vN[j] + (float)vS[j]));
    const float *hu, *hv;
    rc |= c->upload(&hu, iu32);
    rc |= c->upload(&hv, iv32);
    rc |= c->alloc(&c->hd32, c->nelem);
    rc |= c->alloc(&c->hr32, c->nelem);
    if (rc) return IBM_E_CUDA;
    c->hinv_u = const_cast<float*>(hu);
    c->hinv_v = const_cast<float*>(hv);
  }
  if (c->P.precision == 2) return build_mg(c);
  return IBM_OK;
}

int ensure_history(ibm_ctx* c, int need) {
  if (need <= c->hist_cap) return IBM_OK;
  int cap = c->hist_cap ? c->hist_cap : 1024;
  while (cap < need) cap *= 2;
  double *ncl = nullptr, *ncd = nullptr;
  CUDA_TRY(cudaMalloc(&ncl, sizeof(double) * cap));
  CUDA_TRY(cudaMalloc(&ncd, sizeof(double) * cap));
  if (c->hist_cap) {
    CUDA_TRY(cudaMemcpyAsync(ncl, c->cl_d, sizeof(double) * c->hist_cap, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(ncd, c->cd_d, sizeof(double) * c->hist_cap, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    cudaFree(c->cl_d);
    cudaFree(c->cd_d);
  }
  c->cl_d = ncl;
  c->cd_d = ncd;
  c->hist_cap = cap;
  return IBM_OK;
}

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}

int read_norm(ibm_ctx* c, const unsigned long long* dev_bits, double* out);

// Level hierarchy of the multigrid: level 0 is the fine grid (its FP32
// arrays are those of the inner sweeps); each coarser level merges pairs of
// cells in both directions until at most 64 cells remain.
int build_mg(ibm_ctx* c) {
  c->mg_shape = sor32_find_shape(24, 4, 4);
  if (c->mg_shape < 0) return fail(IBM_E_CUDA, "multigrid smoother shape missing");
  CUDA_TRY(sor32_batch_prepare(c->mg_shape));
  CUDA_TRY(prepare_mg_tail());
  std::vector<double> xf = c->xf, yf = c->yf;
  int rc = 0;
  for (int l = 0;; ++l) {
    const int nx = (int)xf.size() - 1, ny = (int)yf.size() - 1;
    std::vector<double> pE, pW, pN, pS;
    laplace_coefs(xf, pE, pW);
    laplace_coefs(yf, pN, pS);
    MgLevel L{};
    L.cur = 0;
    std::vector<float> pe(nx), pw(nx);
    for (int i = 0; i < nx; ++i) pe[i] = (float)pE[i], pw[i] = (float)pW[i];
    rc |= c->upload(&L.pE, pe);
    rc |= c->upload(&L.pW, pw);
    if (l == 0) {
      L.g = c->geo32;
      L.e[0] = c->e32;
      L.e[1] = c->e32b;
      L.r = c->r32;
      L.invd = c->invd32;
    } else {
      Geo32& g = L.g;
      const int pk = ((nx + 1) / 2 + 31) / 32 * 32;
      g.nx = nx;
      g.ny = ny;
      g.pk = pk;
      std::vector<float> ce0(pk, 0.f), ce1(pk, 0.f), cw0(pk, 0.f), cw1(pk, 0.f), pn(ny), ps(ny);
      for (int k = 0; k < pk; ++k) {
        if (2 * k < nx) ce0[k] = (float)pE[2 * k], cw0[k] = (float)pW[2 * k];
        if (2 * k + 1 < nx) ce1[k] = (float)pE[2 * k + 1], cw1[k] = (float)pW[2 * k + 1];
      }
      for (int j = 0; j < ny; ++j) pn[j] = (float)pN[j], ps[j] = (float)pS[j];
      rc |= c->upload(&g.cE0, ce0);
      rc |= c->upload(&g.cE1, ce1);
      rc |= c->upload(&g.cW0, cw0);
      rc |= c->upload(&g.cW1, cw1);
      rc |= c->upload(&g.pN, pn);
      rc |= c->upload(&g.pS, ps);
      const size_t n32 = (size_t)2 * ny * pk;
      std::vector<float> ip(n32, 0.f);
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const float d = (float)pE[i] + (float)pW[i] + (float)pN[j] + (float)pS[j];
          ip[rb_at(i, j, ny, pk)] = d > 0.f ? 1.0f / d : 0.f;
        }
      rc |= c->upload(&L.invd, ip);
      rc |= c->alloc(&L.e[0], n32);
      rc |= c->alloc(&L.e[1], n32);
      rc |= c->alloc(&L.r, n32);
    }
    const bool last = (long)nx * ny <= 64 || (nx <= 2 && ny <= 2) || l == 15;
    if (!last) {
      // restriction weights: a cell's share of its parent's width
      std::vector<double> xfc = coarse_faces(xf), yfc = coarse_faces(yf);
      std::vector<float> wx(nx), wy(ny);
      for (int i = 0; i < nx; ++i) wx[i] = (float)((xf[i + 1] - xf[i]) / (xfc[i / 2 + 1] - xfc[i / 2]));
      for (int j = 0; j < ny; ++j) wy[j] = (float)((yf[j + 1] - yf[j]) / (yfc[j / 2 + 1] - yfc[j / 2]));
      rc |= c->upload(&L.wx, wx);
      rc |= c->upload(&L.wy, wy);
      // bilinear prolongation: each fine centre between its parent's centre
      // and the centre of the parent's neighbour on its side
      auto interp = [](const std::vector<double>& f, const std::vector<double>& fc, std::vector<int>& o,
                       std::vector<float>& a) {
        const int n = (int)f.size() - 1, ncoarse = (int)fc.size() - 1;
        o.assign(n, 0);
        a.assign(n, 0.f);
        for (int i = 0; i < n; ++i) {
          const int I = i / 2;
          const double x = 0.5 * (f[i] + f[i + 1]), X = 0.5 * (fc[I] + fc[I + 1]);
          const int side = x < X ? -1 : (x > X ? 1 : 0);
          const int I2 = I + side;
          if (side == 0 || I2 < 0 || I2 >= ncoarse) continue;  // at the boundary: zero slope
          const double X2 = 0.5 * (fc[I2] + fc[I2 + 1]);
          o[i] = side;
          a[i] = (float)((x - X) / (X2 - X));
        }
      };
      std::vector<int> ox, oy;
      std::vector<float> ax, ay;
      interp(xf, xfc, ox, ax);
      interp(yf, yfc, oy, ay);
      rc |= c->upload(&L.ox, ox);
      rc |= c->upload(&L.oy, oy);
      rc |= c->upload(&L.ax, ax);
      rc |= c->upload(&L.ay, ay);
      xf.swap(xfc);
      yf.swap(yfc);
    }
    if (rc) return IBM_E_CUDA;
    c->mg.push_back(L);
    if (last) {
      if ((long)nx * ny > mg_coarse_max()) return fail(IBM_E_INVAL, "multigrid: coarsest level too large");
      const int m = nx > ny ? nx : ny;
      c->mg_coarse_omega = (float)(2.0 / (1.0 + std::sin(M_PI / (m + 1))));
      c->mg_coarse_sweeps = 2 * (nx + ny) + 8;
      break;
    }
  }
  // the tail: the coarsest levels whose cells together fit in one CTA's
  // shared memory (level 0 stays with the FCG vectors)
  {
    long cells = 0;
    int lt = -1;
    for (int l = (int)c->mg.size() - 1; l >= 1 && (int)c->mg.size() - l <= kTailLevels; --l) {
      cells += (long)c->mg[l].g.nx * c->mg[l].g.ny;
      if (cells > kTailCells) break;
      lt = l;
    }
    c->mg_tail = ((int)c->mg.size() - lt >= 2 && lt >= 1) ? lt : -1;
  }
  const size_t n32 = (size_t)2 * c->ny * c->geo32.pk;
  std::vector<float> dxv(c->nx), dyv(c->ny);
  for (int i = 0; i < c->nx; ++i) dxv[i] = (float)(c->xf[i + 1] - c->xf[i]);
  for (int j = 0; j < c->ny; ++j) dyv[j] = (float)(c->yf[j + 1] - c->yf[j]);
  rc |= c->upload(&c->mg_dxv, dxv);
  rc |= c->upload(&c->mg_dyv, dyv);
  rc |= c->alloc(&c->fcg_x, n32);
  rc |= c->alloc(&c->fcg_p, n32);
  rc |= c->alloc(&c->fcg_q, n32);
  {
    unsigned char* scb = nullptr;
    rc |= c->alloc(&scb, fcg_scalars_bytes());  // zeroed: empty slots, counter 0
    c->fcg_sc = scb;
  }
  return rc ? IBM_E_CUDA : IBM_OK;
}

// One V(2,2)-cycle on the correction equation of level 0: smoothing by two
// red-black Gauss-Seidel sweeps (one tile launch of four half-sweeps) before
// and after the coarse-grid correction.  Each level's correction ends in the
// buffer it started in, so the launch sequence is the same every cycle.
void mg_vcycle(ibm_ctx* c, int zero_first) {
  const int n = (int)c->mg.size();
  const int bottom = c->mg_tail >= 1 ? c->mg_tail : n - 1;  // first level not handled level by level
  for (int l = 0; l < bottom; ++l) {
    MgLevel& A = c->mg[l];
    launch_sor32(c->stream, c->mg_shape, A.g, A.e[A.cur], A.e[A.cur ^ 1], A.r, A.invd, 1.0f, l > 0 || zero_first);
    A.cur ^= 1;
    launch_mg_restrict(c->stream, A, A.e[A.cur], c->mg[l + 1]);
  }
  if (c->mg_tail >= 1) {
    MgTail T{};
    T.n = n - bottom;
    int off = 0;
    for (int k = 0; k < T.n; ++k) {
      T.lv[k] = c->mg[bottom + k];
      T.off[k] = off;
      off += T.lv[k].g.nx * T.lv[k].g.ny;
    }
    T.omega_c = c->mg_coarse_omega;
    T.sweeps_c = c->mg_coarse_sweeps;
    MgLevel& B = c->mg[bottom];
    launch_mg_tail(c->stream, T, B.e[B.cur]);
  } else {
    MgLevel& Z = c->mg[n - 1];
    launch_mg_coarse(c->stream, Z, Z.e[Z.cur], c->mg_coarse_omega, c->mg_coarse_sweeps);
  }
  for (int l = bottom - 1; l >= 0; --l) {
    MgLevel& A = c->mg[l];
    const MgLevel& B = c->mg[l + 1];
    launch_mg_prolong(c->stream, B, B.e[B.cur], A, A.e[A.cur]);
    launch_sor32(c->stream, c->mg_shape, A.g, A.e[A.cur], A.e[A.cur ^ 1], A.r, A.invd, 1.0f, 0);
    A.cur ^= 1;
  }
  c->prof.launches += 4 * bottom + 1;
}

// Two-level cycle with the U-Net as the coarse level (the preconditioner
// the network provides): optional pre-smoothing by two red-black
// Gauss-Seidel sweeps from zero, the residual restricted to level 1 (the
// grid the network works on), the network's correction of level 1 from that
// residual (channel 0) and the values of b, body fraction and p taken at the
// start of the solve (channels 1-3), bilinear prolongation, two
// post-smoothing sweeps.  The network replaces the whole coarse hierarchy of
// the V-cycle; FCG tolerates a preconditioner that is neither linear nor
// symmetric.
void nn_cycle(ibm_ctx* c) {
  MgLevel& A = c->mg[0];
  MgLevel& B = c->mg[1];
  if (c->pc_pre) {
    launch_sor32(c->stream, c->mg_shape, A.g, A.e[A.cur], A.e[A.cur ^ 1], A.r, A.invd, 1.0f, 1);
    A.cur ^= 1;
  } else {
    cudaMemsetAsync(A.e[A.cur], 0, (size_t)2 * A.g.ny * A.g.pk * sizeof(float), c->stream);
  }
  launch_mg_restrict(c->stream, A, A.e[A.cur], B);
  launch_nnp_features(c->stream, B, c->pc_feat, c->pc_max);
  ibm_unet_forward(c->pc_net, c->pc_feat, B.g.ny, B.g.nx, c->pc_out, c->stream);
  launch_nnp_correction(c->stream, B, c->pc_out, c->pc_cT, c->pc_max, B.e[B.cur]);
  launch_mg_prolong(c->stream, B, B.e[B.cur], A, A.e[A.cur]);
  launch_sor32(c->stream, c->mg_shape, A.g, A.e[A.cur], A.e[A.cur ^ 1], A.r, A.invd, 1.0f, 0);
  A.cur ^= 1;
  c->prof.launches += c->pc_pre + 6 + unet_forward_launches();
}

// One iteration of flexible conjugate gradients, FCG(1), on level 0's
// correction equation L x = r (r is level 0's right-hand side, updated in
// place), preconditioned by one V-cycle: z = V(r); p = z + beta p with
// beta = -<z, q>/<p, Lp> (p = z first); q = L p; alpha = <p, r>/<p, Lp>;
// x += alpha p; r -= alpha q.  The Krylov recurrence removes the few error
// components the V-cycle reduces slowly (cells of large aspect ratio where
// the stretched directions cross).
void fcg_iter(ibm_ctx* c, int first) {
  MgLevel& L0 = c->mg[0];
  if (c->pc_kind == 1)
    nn_cycle(c);
  else
    mg_vcycle(c, 1);
  const float* z = L0.e[L0.cur];
  if (!first) launch_fcg_dot(c->stream, L0, c->mg_dxv, c->mg_dyv, z, c->fcg_q, c->fcg_sc);
  launch_fcg_dir(c->stream, L0, z, c->fcg_p, c->fcg_sc, first);
  launch_fcg_apply(c->stream, L0, c->mg_dxv, c->mg_dyv, c->fcg_p, L0.r, c->fcg_q, c->fcg_sc);
  launch_fcg_update(c->stream, L0, c->fcg_p, c->fcg_q, c->fcg_x, L0.r, c->fcg_sc);
  c->prof.launches += first ? 3 : 4;
}

int fcg_launches(const ibm_ctx* c) {
  if (c->pc_kind == 1) return c->pc_pre + 6 + unet_forward_launches() + 4;
  const int bottom = c->mg_tail >= 1 ? c->mg_tail : (int)c->mg.size() - 1;
  return 4 * bottom + 1 + 4;
}

// CUDA graphs of one FCG iteration (first and later); direct launches if the
// stream cannot be captured.
void mg_capture(ibm_ctx* c) {
  // the two-level cycle runs as direct launches: its graph would hold
  // pointers into the network's buffers, which another use of the same
  // network at other sizes reallocates
  if (c->mg_graph[0] || c->mg_graph_failed || c->pc_kind == 1) return;
  for (int z = 0; z < 2; ++z) {
    cudaGraph_t g = nullptr;
    const long long launches = c->prof.launches;
    bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      fcg_iter(c, z == 0);
      ok = cudaStreamEndCapture(c->stream, &g) == cudaSuccess;
    }
    c->prof.launches = launches;
    if (ok) ok = cudaGraphInstantiate(&c->mg_graph[z], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      cudaGetLastError();
      for (cudaGraphExec_t& e : c->mg_graph)
        if (e) cudaGraphExecDestroy(e), e = nullptr;
      c->mg_graph_failed = true;
      return;
    }
  }
}

int fcg_iters(ibm_ctx* c, int m) {
  CUDA_TRY(cudaMemsetAsync(c->fcg_x, 0, (size_t)2 * c->ny * c->geo32.pk * sizeof(float), c->stream));
  for (int k = 0; k < m; ++k) {
    if (c->mg_graph[0] && c->pc_kind == 0) {
      CUDA_TRY(cudaGraphLaunch(c->mg_graph[k == 0 ? 0 : 1], c->stream));
      c->prof.launches += fcg_launches(c) - (k == 0 ? 1 : 0);
    } else {
      fcg_iter(c, k == 0);
    }
  }
  CUDA_TRY(cudaGetLastError());
  return IBM_OK;
}

// Defect correction with FP32 multigrid-preconditioned FCG as the inner
// solver: FP64 update, residual and norm as in solve_poisson_mixed; the
// number of FCG iterations (one V-cycle each) per check adapts to the
// observed reduction per iteration, aiming at the tolerance or at a
// reduction of 1e-4 (about the resolution of an FP32 correction).  *cycles
// receives the V-cycles performed.
int solve_poisson_mg(ibm_ctx* c, double tol, int maxc, int* cycles, double* res) {
  const Geo& g = c->geo;
  mg_capture(c);
  MgLevel& L0 = c->mg[0];
  if (c->pc_kind == 1) {  // channels 1-3 of the network's features, fixed during the solve
    launch_ws_features(c->stream, g, c->Hc, c->Wc, c->b, c->phi, c->p, c->band, c->fc, c->pc_feat, c->pc_max);
    c->prof.launches += 2;
  }
  double* cur = c->phi;
  double* alt = c->phi2;
  int s = 0, add = 0, m = 0;
  double prev = 0.0;
  bool timing = false;
  for (;;) {
    if (timing) CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->sc->res_bits, 0, 8, c->stream));
    launch_dc_residual(c->stream, g, c->geo32.pk, cur, alt, c->fcg_x, c->b, L0.r, add, &c->sc->res_bits);
    c->prof.launches += 1;
    if (add) std::swap(cur, alt);
    double r;
    int rc = read_norm(c, &c->sc->res_bits, &r);
    if (rc) return rc;
    if (timing) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      c->prof.sweep_ms += ms;
      timing = false;
    }
    *cycles = s;
    *res = r;
    c->phi = cur;
    c->phi2 = alt;
    if (!std::isfinite(r)) return fail(IBM_E_DIVERGED, "pressure residual is not finite after %d V-cycles", s);
    if (r <= tol) return IBM_OK;
    if (s >= maxc) return fail(IBM_E_NOCONV, "pressure solve: %d V-cycles, residual %.3e > %.3e", s, r, tol);
    if (m > 0 && prev > r && r > 0.0) {
      const double rate = std::log(r / prev) / m;  // per cycle, < 0
      double target = std::log(tol / r);
      if (target < std::log(1e-4)) target = std::log(1e-4);
      const int want = (int)std::ceil(target / rate);
      // a V-cycle reduces the residual by about 0.5 or better, so 64 cycles
      // always reach 1e-4; the two-level cycle without a coarse hierarchy
      // needs longer Krylov runs
      const int run_max = c->pc_kind == 1 ? 512 : 64;
      c->mg_cycles = want < 1 ? 1 : (want > run_max ? run_max : want);
    }
    m = c->mg_cycles;
    if (s + m > maxc) m = maxc - s;
    if (c->profiling) {
      CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
      timing = true;
      c->prof.sweep_launches += (long long)m * fcg_launches(c);
      c->prof.sweep_cells += (long long)m * c->nx * c->ny;
    }
    rc = fcg_iters(c, m);
    if (rc) return rc;
    prev = r;
    s += m;
    add = 1;
  }
}

// Reads one norm accumulator back (waits for the stream).
int read_norm(ibm_ctx* c, const unsigned long long* dev_bits, double* out) {
  CUDA_TRY(cudaMemcpyAsync(&c->sc_host->res_bits, dev_bits, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  *out = bits_to_double(c->sc_host->res_bits);
  return IBM_OK;
}

// Red-black SOR for the pressure: residual checked before the first sweep
// and every m sweeps.
int solve_poisson(ibm_ctx* c, double tol, double rtol, int m, int maxs, int* sweeps, double* res) {
  const Geo& g = c->geo;
  double thr = tol;
  if (rtol > 0.0) {
    CUDA_TRY(cudaMemsetAsync(&c->sc->bmax_bits, 0, 8, c->stream));
    launch_bmax(c->stream, g, c->b, &c->sc->bmax_bits);
    double bmax;
    int rc = read_norm(c, &c->sc->bmax_bits, &bmax);
    if (rc) return rc;
    thr = std::fmax(tol, rtol * bmax);
  }
  if (m < 1) m = 1;
  const double omega = c->P.omega_p;
  int pending = 0;  // sweep launches inside the open event bracket
  for (int s = 0;; ++s) {
    if (s % m == 0) {
      if (pending) CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
      CUDA_TRY(cudaMemsetAsync(&c->sc->res_bits, 0, 8, c->stream));
      launch_poisson_res(c->stream, g, c->phi, c->b, &c->sc->res_bits);
      c->prof.launches += 1;
      double r;
      int rc = read_norm(c, &c->sc->res_bits, &r);
      if (rc) return rc;
      if (pending) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        c->prof.sweep_ms += ms;
        c->prof.sweep_launches += pending;
        c->prof.sweep_cells += (long long)pending * c->nx * c->ny;
        pending = 0;
      }
      *sweeps = s;
      *res = r;
      if (!std::isfinite(r)) return fail(IBM_E_DIVERGED, "pressure residual is not finite after %d sweeps", s);
      if (r <= thr) return IBM_OK;
      if (s < maxs && c->profiling) {
        CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        pending = 0;
      }
    }
    if (s >= maxs) return fail(IBM_E_NOCONV, "pressure solve: %d sweeps, residual %.3e > %.3e", s, *res, thr);
    launch_poisson_half(c->stream, g, c->phi, c->b, c->invd_p, 0, omega);
    launch_poisson_half(c->stream, g, c->phi, c->b, c->invd_p, 1, omega);
    c->prof.launches += 2;
    if (c->profiling) pending += 2;
  }
}

// Autotuner of the FP32 sweep kernel: times every tile shape on this
// context's grid and arrays (CUDA events, a few launches each) and keeps the
// fastest per full sweep.  Runs before the first mixed solve; the arrays'
// contents are rewritten by the solve (each inner solve starts from e = 0
// and the residual kernel rewrites r).
int tune_sor32(ibm_ctx* c) {
  cudaEvent_t a = nullptr, b = nullptr;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  const float omega = (float)c->P.omega_p;
  double best = 1e300;
  int best_cfg = 0;
  for (int cfg = 0; cfg < sor32_num_configs(); ++cfg) {
    const int reps = 8;
    for (int w = 0; w < 2; ++w) {
      launch_sor32(c->stream, cfg, c->geo32, c->e32, c->e32b, c->r32, c->invd32, omega, 1, 1);
      std::swap(c->e32, c->e32b);
    }
    CUDA_TRY(cudaEventRecord(a, c->stream));
    for (int l = 0; l < reps; ++l) {
      launch_sor32(c->stream, cfg, c->geo32, c->e32, c->e32b, c->r32, c->invd32, omega, l == 0 ? 1 : 0, 1);
      std::swap(c->e32, c->e32b);
    }
    CUDA_TRY(cudaEventRecord(b, c->stream));
    CUDA_TRY(cudaEventSynchronize(b));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    const double us_sweep = 1e3 * ms / (reps * (sor32_half_sweeps(cfg) / 2));
    c->prof.launches += reps + 2;
    if (us_sweep < best) {
      best = us_sweep;
      best_cfg = cfg;
    }
  }
  CUDA_TRY(cudaGetLastError());
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->sor_cfg = best_cfg;
  c->sor_us = best;
  return IBM_OK;
}

// Relaxation factor of the pressure SOR from its observed convergence
// (adaptive SOR): for a consistently ordered matrix (red-black ordering of
// the five-point operator is one) and omega below the optimum, the SOR
// spectral radius rho and the Jacobi spectral radius mu satisfy Young's
// relation (rho + omega - 1)^2 = rho omega^2 mu^2, and the optimum is
// omega_opt = 2 / (1 + sqrt(1 - mu^2)).  At or above the optimum rho equals
// omega - 1 and says nothing about mu: omega is returned unchanged.
double omega_from_rate(double omega, double rho) {
  if (!(rho > 0.0) || !(rho < 1.0) || !(omega > 0.0) || !(omega < 2.0)) return omega;
  if (rho <= omega - 1.0) return omega;
  double mu = (rho + omega - 1.0) / (std::sqrt(rho) * omega);
  if (!(mu < 1.0)) return omega;
  return 2.0 / (1.0 + std::sqrt((1.0 - mu) * (1.0 + mu)));
}

// Asymptotic convergence factor per sweep of FP64 red-black SOR on the
// homogeneous pressure system (b = 0) from a pseudo-random start.  The
// residual's infinity norm is read every 64 sweeps until it has fallen by
// 1e-10 (well above the rounding floor) or S sweeps have run; the factor is
// taken over the second half of the sweeps run.
int sor_rate(ibm_ctx* c, double* x, const double* zero, double omega, int S, double* rho) {
  const Geo& g = c->geo;
  const int C = 64;
  CUDA_TRY(cudaMemsetAsync(x, 0, c->nelem * sizeof(double), c->stream));
  launch_fill_hash(c->stream, g, x);
  std::vector<double> r;
  for (int s = 0;; s += C) {
    double v = 0.0;
    CUDA_TRY(cudaMemsetAsync(&c->sc->res_bits, 0, 8, c->stream));
    launch_poisson_res(c->stream, g, x, zero, &c->sc->res_bits);
    int rc = read_norm(c, &c->sc->res_bits, &v);
    if (rc) return rc;
    r.push_back(v);
    c->prof.launches += 1;
    if (!(v > 1e-10 * r[0]) || s + C > S) break;
    for (int k = 0; k < C; ++k) {
      launch_poisson_half(c->stream, g, x, zero, c->invd_p, 0, omega);
      launch_poisson_half(c->stream, g, x, zero, c->invd_p, 1, omega);
    }
    c->prof.launches += 2 * C;
  }
  CUDA_TRY(cudaGetLastError());
  const int b = (int)r.size() - 1, a = b / 2;
  *rho = (b > a && r[a] > 0.0 && r[b] > 0.0) ? std::pow(r[b] / r[a], 1.0 / (C * (b - a))) : 0.0;
  return IBM_OK;
}

int tune_omega(ibm_ctx* c, int S, double* out) {
  if (S <= 0) {
    S = 8 * (c->nx > c->ny ? c->nx : c->ny);
    S = S < 2048 ? 2048 : (S > 32768 ? 32768 : S);
  }
  double *x = nullptr, *zero = nullptr;
  CUDA_TRY(cudaMalloc((void**)&x, c->nelem * sizeof(double)));
  if (cudaMalloc((void**)&zero, c->nelem * sizeof(double)) != cudaSuccess) {
    cudaFree(x);
    return fail(IBM_E_CUDA, "tune_omega: allocation failed");
  }
  int rc = cudaMemsetAsync(zero, 0, c->nelem * sizeof(double), c->stream) == cudaSuccess ? IBM_OK : IBM_E_CUDA;
  const double w0 = c->P.omega_p;
  double rho0 = 0.0, rho1 = 0.0, w1 = w0;
  if (!rc) rc = sor_rate(c, x, zero, w0, S, &rho0);
  if (!rc) w1 = omega_from_rate(w0, rho0);
  if (!rc && w1 != w0) rc = sor_rate(c, x, zero, w1, S, &rho1);
  cudaStreamSynchronize(c->stream);
  cudaFree(x);
  cudaFree(zero);
  if (rc) return rc;
  if (w1 != w0 && rho1 > 0.0 && rho1 < rho0) c->P.omega_p = w1;
  *out = c->P.omega_p;
  return IBM_OK;
}

// FP32 sweeps between two FP64 checks: a share of the predicted remaining
// count, capped below the reduction one FP32 correction resolves (measured on
// 2048x1024: 0.9 and 4096 took 12 % more sweeps per step than 0.7 and 1024)
constexpr double kInnerFrac = 0.7;
constexpr int kInnerMax = 1024;

// Defect correction: FP64 residual and update around FP32 red-black SOR
// sweeps on the correction equation.  The number of inner sweeps between two
// FP64 checks adapts to the observed convergence rate.
int solve_poisson_mixed(ibm_ctx* c, double tol, int maxs, int* sweeps, double* res) {
  const Geo& g = c->geo;
  if (c->sor_cfg < 0) {
    int rc = tune_sor32(c);
    if (rc) return rc;
  }
  const int cfg = c->sor_cfg;
  const int K2 = sor32_half_sweeps(cfg) / 2;  // full sweeps per launch
  double* cur = c->phi;
  double* alt = c->phi2;
  int s = 0, add = 0, inner = 0;
  double prev = 0.0;
  int pending = 0;
  const float omega = (float)c->P.omega_p;
  for (;;) {
    if (pending) CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->sc->res_bits, 0, 8, c->stream));
    launch_dc_residual(c->stream, g, c->geo32.pk, cur, alt, c->e32, c->b, c->r32, add, &c->sc->res_bits);
    c->prof.launches += 1;
    if (add) std::swap(cur, alt);
    double r;
    int rc = read_norm(c, &c->sc->res_bits, &r);
    if (rc) return rc;
    if (pending) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      c->prof.sweep_ms += ms;
      c->prof.sweep_launches += pending;
      c->prof.sweep_cells += (long long)pending * c->nx * c->ny;
      pending = 0;
    }
    *sweeps = s;
    *res = r;
    c->phi = cur;
    c->phi2 = alt;
    if (!std::isfinite(r)) return fail(IBM_E_DIVERGED, "pressure residual is not finite after %d sweeps", s);
    if (r <= tol) return IBM_OK;
    if (s >= maxs) return fail(IBM_E_NOCONV, "pressure solve: %d sweeps, residual %.3e > %.3e", s, r, tol);
    // inner sweeps until the next check: kInnerFrac of the predicted
    // remaining count, 16 .. kInnerMax sweeps, whole launches
    if (inner > 0 && prev > r && r > 0.0) {
      double rate = std::log(r / prev) / inner;  // per sweep, < 0
      double need = std::log(tol / r) / rate;
      int m = (int)(kInnerFrac * need);
      c->m_inner = m < 16 ? 16 : (m > kInnerMax ? kInnerMax : m);
    }
    inner = (c->m_inner + K2 - 1) / K2 * K2;
    if (s + inner > maxs) inner = ((maxs - s) + K2 - 1) / K2 * K2;
    if (c->profiling) CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    for (int l = 0; l < inner / K2; ++l) {
      // read e32, write e32b, swap: the final correction ends in e32
      launch_sor32(c->stream, cfg, c->geo32, c->e32, c->e32b, c->r32, c->invd32, omega, l == 0 ? 1 : 0, 1);
      std::swap(c->e32, c->e32b);
      c->prof.launches += 1;
      if (c->profiling) pending += 1;
    }
    prev = r;
    s += inner;
    add = 1;
  }
}

// Velocity system in FP32 sweeps inside FP64 defect correction: FP64
// residual (stored in FP32) and norm, 4 FP32 red-black sweeps on the
// correction equation from zero (the Gauss-Seidel contraction of these
// systems, (I - beta L) with beta / h^2 small, reaches the resolution of an
// FP32 correction in a few sweeps), FP64 update; *sweeps counts FP32 sweeps.
int solve_helm_mixed(ibm_ctx* c, int grid, double beta, double Ub, int* sweeps, double* res) {
  const Geo& g = c->geo;
  double* x = grid == 0 ? c->uh : c->vh;
  const double* R = grid == 0 ? c->Ru : c->Rv;
  const float* invd = grid == 0 ? c->hinv_u : c->hinv_v;
  const uint8_t* fl = grid == 0 ? c->fu : c->fv;
  const double* al = grid == 0 ? c->au : c->av;
  const int m = 4;
  for (int s = 0;; s += m) {
    CUDA_TRY(cudaMemsetAsync(&c->sc->res_bits, 0, 8, c->stream));
    launch_helm_dc_res(c->stream, g, grid, x, R, c->band, fl, al, beta, Ub, c->hr32, &c->sc->res_bits);
    c->prof.launches += 1;
    double r;
    int rc = read_norm(c, &c->sc->res_bits, &r);
    if (rc) return rc;
    *sweeps = s;
    *res = r;
    if (!std::isfinite(r)) return fail(IBM_E_DIVERGED, "velocity residual is not finite");
    if (r <= c->P.helm_tol) return IBM_OK;
    if (s >= c->P.max_sweeps) return fail(IBM_E_NOCONV, "velocity solve (grid %d) did not converge", grid);
    CUDA_TRY(cudaMemsetAsync(c->hd32, 0, c->nelem * sizeof(float), c->stream));
    for (int k = 0; k < m; ++k) {
      launch_helm32_half(c->stream, g, c->h32, grid, c->hd32, c->hr32, invd, c->band, fl, al, 0,
                         (float)c->P.omega_h, (float)beta);
      launch_helm32_half(c->stream, g, c->h32, grid, c->hd32, c->hr32, invd, c->band, fl, al, 1,
                         (float)c->P.omega_h, (float)beta);
    }
    launch_helm_add(c->stream, g, grid, x, c->hd32);
    c->prof.launches += 2 * m + 1;
  }
}

int solve_helm(ibm_ctx* c, int grid, double beta, double Ub, int* sweeps, double* res) {
  if (c->P.precision >= 1) return solve_helm_mixed(c, grid, beta, Ub, sweeps, res);
  const Geo& g = c->geo;
  double* x = grid == 0 ? c->uh : c->vh;
  const double* R = grid == 0 ? c->Ru : c->Rv;
  const double* invd = grid == 0 ? c->invd_u : c->invd_v;
  const uint8_t* fl = grid == 0 ? c->fu : c->fv;
  const double* al = grid == 0 ? c->au : c->av;
  int m = c->P.check_every_h;
  for (int s = 0;; ++s) {
    if (s % m == 0) {
      CUDA_TRY(cudaMemsetAsync(&c->sc->res_bits, 0, 8, c->stream));
      launch_helm_res(c->stream, g, grid, x, R, c->band, fl, al, beta, Ub, &c->sc->res_bits);
      c->prof.launches += 1;
      double r;
      int rc = read_norm(c, &c->sc->res_bits, &r);
      if (rc) return rc;
      *sweeps = s;
      *res = r;
      if (!std::isfinite(r)) return fail(IBM_E_DIVERGED, "velocity residual is not finite");
      if (r <= c->P.helm_tol) return IBM_OK;
    }
    if (s >= c->P.max_sweeps) return fail(IBM_E_NOCONV, "velocity solve (grid %d) did not converge", grid);
    launch_helm_half(c->stream, g, grid, x, R, invd, c->band, fl, al, 0, c->P.omega_h, beta, Ub);
    launch_helm_half(c->stream, g, grid, x, R, invd, c->band, fl, al, 1, c->P.omega_h, beta, Ub);
    c->prof.launches += 2;
  }
}

// Part of a step before the pressure solve (a1-a7); *thr receives the
// pressure tolerance of the step.
int step_pre(ibm_ctx* c, ibm_step_stats* st, double* thr) {
  const Geo& g = c->geo;
  const ibm_grid_params& P = c->P;
  const double dt = P.dt, beta = dt / (2.0 * P.Re);
  const double t1 = (c->n + 1) * dt;
  double yb = c->yb0, vb = 0.0;
  *st = ibm_step_stats{};
  int rc = ensure_history(c, c->n + 1);
  if (rc) return rc;
  // a1: kinematics at t^{n+1} (Eqs. 1-2)
  if (c->has_body) {
    NvtxRange r("a1-a3 kinematics and classification");
    yb = c->yb0 + c->h * std::sin(c->k * t1);
    vb = c->k * c->h * std::cos(c->k * t1);
    // a2/a3: classification and forcing data
    launch_classify(c->stream, g, c->band, c->xb, yb, 0.5 * c->chord, 0.5 * c->tc * c->chord, c->fu, c->fv,
                    c->fc, c->au, c->av);
    c->prof.launches += 3;
  }
  // boundary values of the intermediate velocity at t^{n+1}
  if (P.bc == 0) {
    launch_outflow_bc(c->stream, g, c->u, c->uh, c->vh, P.u_in, dt);
    c->prof.launches += 1;
  }
  // a4: explicit predictor and initial guess
  NvtxRange r4("a4 explicit predictor");
  launch_predict(c->stream, g, c->u, c->v, c->p, c->Hu, c->Hv, c->Huo, c->Hvo, c->Ru, c->Rv, c->uh, c->vh,
                 c->band, c->fu, c->fv, dt, beta, vb, c->n == 0 ? 1 : 0);
  c->prof.launches += 2;
  // a5: implicit velocity solves
  {
    NvtxRange r("a5 velocity solves");
    rc = solve_helm(c, 0, beta, 0.0, &st->sweeps_u, &st->res_u);
    if (rc) return rc;
    rc = solve_helm(c, 1, beta, vb, &st->sweeps_v, &st->res_v);
    if (rc) return rc;
  }
  // a6: right-hand side with the mass source on body cells
  NvtxRange r6("a6 right-hand side and mass source");
  launch_rhs(c->stream, g, c->uh, c->vh, c->b, dt);
  c->prof.launches += 1;
  if (c->has_body) {
    launch_body_source(c->stream, g, c->band, c->fc, c->uh, c->vh, c->b, c->qband, dt, c->rowsum, c->sc);
    c->prof.launches += 3;  // row sums, their total, the mass source
  }
  // a7: warm start.  The solve starts from the previous increment, or from
  // its linear extrapolation in time; the learned form adds the U-Net's
  // prediction of the remaining change.
  NvtxRange r7("a7 warm start");
  if (c->ws_base == 1) {
    launch_extrapolate(c->stream, g, c->phi, c->phi_prev);
    c->prof.launches += 1;
  }
  if (c->ws_mode) {
    launch_ws_features(c->stream, g, c->Hc, c->Wc, c->b, c->phi, c->p, c->band, c->fc, c->ws_feat, c->ws_max);
    c->prof.launches += 2;
    if (c->ws_mode == 2)
      CUDA_TRY(cudaMemcpyAsync(c->phi_old, c->phi, c->nelem * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (c->ws_mode == 1) {
      // the plain guess is kept; the learned one replaces it only if it
      // starts the solve with less than half the residual (the plain
      // iteration is the fallback and decides when the solve ends; a merely
      // smaller maximum residual did not mean fewer sweeps)
      rc = ibm_unet_forward(c->ws_net, c->ws_feat, c->Hc, c->Wc, c->ws_out, c->stream);
      if (rc) return rc;
      CUDA_TRY(cudaMemcpyAsync(c->phi_old, c->phi, c->nelem * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      launch_ws_apply(c->stream, g, c->Hc, c->Wc, c->ws_out, c->ws_cT, c->ws_max, c->phi);
      // both residual norms in one pass and one wait
      CUDA_TRY(cudaMemsetAsync(&c->sc->res_bits, 0, 8, c->stream));
      CUDA_TRY(cudaMemsetAsync(&c->sc->res2_bits, 0, 8, c->stream));
      launch_poisson_res2(c->stream, g, c->phi, c->phi_old, c->b, &c->sc->res_bits, &c->sc->res2_bits);
      CUDA_TRY(cudaMemcpyAsync(&c->sc_host->res2_bits, &c->sc->res2_bits, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, c->stream));
      double r_learned = 0.0, r_plain = 0.0;
      rc = read_norm(c, &c->sc->res_bits, &r_learned);  // waits for the stream
      if (rc) return rc;
      r_plain = bits_to_double(c->sc_host->res2_bits);
      c->prof.launches += unet_forward_launches() + 2;
      c->prof.ws_applied += 1;
      if (r_learned < 0.5 * r_plain)
        c->prof.ws_kept += 1;
      else
        std::swap(c->phi, c->phi_old);
    }
  }
  *thr = P.poisson_tol;
  if (P.poisson_rtol > 0.0) {
    CUDA_TRY(cudaMemsetAsync(&c->sc->bmax_bits, 0, 8, c->stream));
    launch_bmax(c->stream, g, c->b, &c->sc->bmax_bits);
    double bmax;
    rc = read_norm(c, &c->sc->bmax_bits, &bmax);
    if (rc) return rc;
    *thr = std::fmax(*thr, P.poisson_rtol * bmax);
  }
  return IBM_OK;
}

// Part of a step after the pressure solve (a9-a11): samples, forces,
// projection, divergence, statistics.
int step_post(ibm_ctx* c, ibm_step_stats* st) {
  const Geo& g = c->geo;
  const ibm_grid_params& P = c->P;
  const double dt = P.dt, beta = dt / (2.0 * P.Re);
  NvtxRange r("a9-a11 forces, projection and divergence");
  if (c->ws_mode == 2) {
    launch_phi_ref(c->stream, g, c->phi, c->sc);
    launch_ws_target(c->stream, g, c->Hc, c->Wc, c->phi, c->phi_old, c->sc, c->ws_cT, c->ws_max, c->ws_target);
    c->prof.launches += 2;
    c->has_sample = true;
  }
  // a10: forces (before the projection overwrites nothing they need)
  if (c->has_body) {
    launch_forces(c->stream, g, c->band, c->fu, c->fv, c->uh, c->vh, c->Ru, c->Rv, beta, dt, c->chord, c->partials,
                  c->sc, c->cl_d, c->cd_d, c->n);
    c->prof.launches += 2;
  } else {
    CUDA_TRY(cudaMemsetAsync(c->cl_d + c->n, 0, sizeof(double), c->stream));
    CUDA_TRY(cudaMemsetAsync(c->cd_d + c->n, 0, sizeof(double), c->stream));
  }
  // a9 + a11: projection, pressure update, divergence check
  launch_phi_ref(c->stream, g, c->phi, c->sc);
  CUDA_TRY(cudaMemsetAsync(&c->sc->div_bits, 0, 8, c->stream));
  launch_project(c->stream, g, c->uh, c->vh, c->phi, c->u, c->v, c->p, c->phi2, c->band, c->fc, dt, c->sc);
  c->prof.launches += 2;
  CUDA_TRY(cudaGetLastError());
  // read the scalars of the step
  CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
  double clcd[2] = {0.0, 0.0};
  CUDA_TRY(cudaMemcpyAsync(&clcd[0], c->cl_d + c->n, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(&clcd[1], c->cd_d + c->n, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  std::swap(c->phi, c->phi2);
  std::swap(c->Hu, c->Huo);
  std::swap(c->Hv, c->Hvo);
  c->n += 1;
  c->prof.steps += 1;
  c->prof.poisson_sweeps += st->sweeps_p;
  c->prof.helm_sweeps += st->sweeps_u + st->sweeps_v;
  st->n = c->n;
  st->t = c->n * dt;
  st->div_max = bits_to_double(c->sc_host->div_bits);
  st->cl = clcd[0];
  st->cd = clcd[1];
  c->last = *st;
  return IBM_OK;
}

int one_step(ibm_ctx* c) {
  NvtxRange step("ibm_step");
  ibm_step_stats st;
  double thr;
  int rc = step_pre(c, &st, &thr);
  if (rc) return rc;
  {
    NvtxRange r("a8 pressure solve");
    if (c->P.precision == 2)
      rc = solve_poisson_mg(c, thr, c->P.max_sweeps, &st.sweeps_p, &st.res_p);
    else if (c->P.precision == 1)
      rc = solve_poisson_mixed(c, thr, c->P.max_sweeps, &st.sweeps_p, &st.res_p);
    else
      rc = solve_poisson(c, c->P.poisson_tol, c->P.poisson_rtol, c->P.check_every_p, c->P.max_sweeps,
                         &st.sweeps_p, &st.res_p);
  }
  if (rc) return rc;
  return step_post(c, &st);
}


}  // namespace

// ------------------------------------------------------------------ batch
// Many cases advance together.  Per case, the parts of a step before and
// after the pressure solve run as for a single context (on the batch's
// stream); the pressure solves of all cases run as one defect-correction
// loop in which every FP32 sweep launch and every FP64 residual launch
// covers the tiles of all cases that have not converged yet.  Cases leave
// the launches as they converge.  Inner sweeps run in pairs of launches
// (e32 -> e32b -> e32), so each case's correction always ends in e32; the
// pairs are replayed from CUDA graphs captured per active set.
struct ibm_batch {
  std::vector<ibm_ctx*> cs;
  cudaStream_t stream = nullptr;
  int cfg = -1;
  double sor_us = 0.0;
  bool use_graphs = true;
  bool budgets = true;  // each case its own sweeps per round (direct launches); off: shared rounds
  bool profiling = false;
  Sor32Case *h_sor = nullptr, *d_sor = nullptr;  // tables A (e32 -> e32b) at [0, n), B (e32b -> e32) at [n, 2n)
  DcCase *h_dc = nullptr, *d_dc = nullptr;
  unsigned long long *h_bits = nullptr, *d_bits = nullptr;
  // whole-step batching: the case table, the first block of every case per
  // launch kind, the active-case tables of the velocity solves (one region
  // for the residual launch, one for the sweep launches) and the scalars
  // read back at the end of a step
  StepCase *h_cases = nullptr, *d_cases = nullptr;
  int *h_first = nullptr, *d_first = nullptr;  // [BK_NUM][n]
  int total[BK_NUM] = {0, 0, 0, 0};
  bool first_ready = false;
  int *h_hres = nullptr, *d_hres = nullptr;    // [2][n]: active cases, first blocks
  int *h_hswp = nullptr, *d_hswp = nullptr;    // [3][n]: active cases, first blocks of half-sweeps, of updates
  StepReadback *h_rb = nullptr, *d_rb = nullptr;
  std::vector<cudaEvent_t> ev;
  cudaEvent_t ev_b = nullptr, t0 = nullptr, t1 = nullptr;
  struct Graphs {
    cudaGraphExec_t first = nullptr, pair = nullptr, many = nullptr;
  };
  std::map<std::pair<int, int>, Graphs> graphs;
  ibm_profile prof{};

  void drop_graphs() {
    for (auto& kv : graphs) {
      if (kv.second.first) cudaGraphExecDestroy(kv.second.first);
      if (kv.second.pair) cudaGraphExecDestroy(kv.second.pair);
      if (kv.second.many) cudaGraphExecDestroy(kv.second.many);
    }
    graphs.clear();
  }
  ~ibm_batch() {
    drop_graphs();
    if (h_sor) cudaFreeHost(h_sor);
    if (h_dc) cudaFreeHost(h_dc);
    if (h_bits) cudaFreeHost(h_bits);
    if (d_sor) cudaFree(d_sor);
    if (d_dc) cudaFree(d_dc);
    if (d_bits) cudaFree(d_bits);
    for (void* q : {(void*)h_cases, (void*)h_first, (void*)h_hres, (void*)h_hswp, (void*)h_rb})
      if (q) cudaFreeHost(q);
    for (void* q : {(void*)d_cases, (void*)d_first, (void*)d_hres, (void*)d_hswp, (void*)d_rb})
      if (q) cudaFree(q);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (ev_b) cudaEventDestroy(ev_b);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

constexpr int kPairsPerGraph = 8;

// Sweep tables of the cases act[0..na) for tile shape cfg; *tiles receives
// the CTAs of one launch; pairs (may be NULL: no limit) the launch pairs of
// the round per active case.  Copied to the device on the batch's stream.
int batch_sor_tables(ibm_batch* B, int cfg, const std::vector<int>& act, int* tiles,
                     const std::vector<int>* pairs = nullptr) {
  const int n = (int)B->cs.size(), na = (int)act.size();
  int first = 0;
  for (int k = 0; k < na; ++k) {
    ibm_ctx* c = B->cs[act[k]];
    int tx = 0, ty = 0;
    sor32_tiles(cfg, c->geo32, &tx, &ty);
    const float om = (float)c->P.omega_p;
    const int np = pairs ? (*pairs)[k] : INT_MAX;
    B->h_sor[k] = Sor32Case{c->geo32, c->e32, c->e32b, c->r32, c->invd32, om, first, tx, np};
    B->h_sor[n + k] = Sor32Case{c->geo32, c->e32b, c->e32, c->r32, c->invd32, om, first, tx, np};
    first += tx * ty;
  }
  *tiles = first;
  CUDA_TRY(cudaMemcpyAsync(B->d_sor, B->h_sor, 2 * n * sizeof(Sor32Case), cudaMemcpyHostToDevice, B->stream));
  return IBM_OK;
}

void batch_launch_pair(ibm_batch* B, int na, int tiles, int zero_first, int pdl) {
  const int n = (int)B->cs.size();
  launch_sor32_batch(B->stream, B->cfg, B->d_sor, na, tiles, zero_first, pdl);
  launch_sor32_batch(B->stream, B->cfg, B->d_sor + n, na, tiles, 0, pdl);
}

int batch_capture(ibm_batch* B, int na, int tiles, int pairs, int zero_first, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
  for (int q = 0; q < pairs; ++q) batch_launch_pair(B, na, tiles, q == 0 ? zero_first : 0, 0);
  CUDA_TRY(cudaStreamEndCapture(B->stream, &g));
  cudaError_t e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(IBM_E_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
  return IBM_OK;
}

// `pairs` launch pairs over the active set (tables already on the device),
// the first one starting from e = 0.
int batch_sweeps(ibm_batch* B, int na, int tiles, int pairs) {
  B->prof.launches += 2 * pairs;
  if (!B->use_graphs) {  // direct launches, as programmatic dependents
    for (int q = 0; q < pairs; ++q) batch_launch_pair(B, na, tiles, q == 0, 1);
    CUDA_TRY(cudaGetLastError());
    return IBM_OK;
  }
  auto key = std::make_pair(na, tiles);
  auto it = B->graphs.find(key);
  if (it == B->graphs.end()) {
    if (B->graphs.size() >= 512) B->drop_graphs();
    ibm_batch::Graphs G;
    int rc = batch_capture(B, na, tiles, 1, 1, &G.first);
    if (!rc) rc = batch_capture(B, na, tiles, 1, 0, &G.pair);
    if (!rc) rc = batch_capture(B, na, tiles, kPairsPerGraph, 0, &G.many);
    if (rc) {
      if (G.first) cudaGraphExecDestroy(G.first);
      if (G.pair) cudaGraphExecDestroy(G.pair);
      return rc;
    }
    it = B->graphs.emplace(key, G).first;
  }
  const ibm_batch::Graphs& G = it->second;
  CUDA_TRY(cudaGraphLaunch(G.first, B->stream));
  int rem = pairs - 1;
  for (; rem >= kPairsPerGraph; rem -= kPairsPerGraph) CUDA_TRY(cudaGraphLaunch(G.many, B->stream));
  for (; rem > 0; --rem) CUDA_TRY(cudaGraphLaunch(G.pair, B->stream));
  return IBM_OK;
}

// Common tile shape of the batch: every shape timed over all cases.
int batch_tune(ibm_batch* B) {
  const int n = (int)B->cs.size();
  std::vector<int> all(n);
  for (int i = 0; i < n; ++i) all[i] = i;
  double best = 1e300;
  int best_cfg = 0;
  const bool graphs = B->use_graphs;
  B->use_graphs = false;
  for (int cfg = 0; cfg < sor32_num_configs(); ++cfg) {
    CUDA_TRY(sor32_batch_prepare(cfg));
    B->cfg = cfg;
    int tiles = 0;
    int rc = batch_sor_tables(B, cfg, all, &tiles);
    if (!rc) rc = batch_sweeps(B, n, tiles, 1);
    CUDA_TRY(cudaEventRecord(B->t0, B->stream));
    const int pairs = 3;
    if (!rc) rc = batch_sweeps(B, n, tiles, pairs);
    if (rc) {
      B->use_graphs = graphs;
      return rc;
    }
    CUDA_TRY(cudaEventRecord(B->t1, B->stream));
    CUDA_TRY(cudaEventSynchronize(B->t1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, B->t0, B->t1));
    const double us = 1e3 * ms / (2 * pairs * (sor32_half_sweeps(cfg) / 2));
    if (us < best) {
      best = us;
      best_cfg = cfg;
    }
  }
  B->use_graphs = graphs;
  B->cfg = best_cfg;
  B->sor_us = best;
  B->drop_graphs();
  return IBM_OK;
}

// Pressure solves of all cases (defect correction, as solve_poisson_mixed,
// with one check of every active case per round).  thr: tolerance per case.
int batch_solve(ibm_batch* B, const std::vector<double>& thr, std::vector<ibm_step_stats>& st) {
  const int n = (int)B->cs.size();
  if (B->cfg < 0) {
    int rc = batch_tune(B);
    if (rc) return rc;
  }
  const int pair_sweeps = sor32_half_sweeps(B->cfg);  // full sweeps of one launch pair
  struct State {
    double *cur, *alt;
    int s = 0, add = 0, inner = 0;
    double prev = 0.0;
  };
  std::vector<State> S(n);
  std::vector<int> act(n), next;
  for (int i = 0; i < n; ++i) {
    S[i].cur = B->cs[i]->phi;
    S[i].alt = B->cs[i]->phi2;
    act[i] = i;
  }
  std::vector<int> want(n, 0);
  bool timing = false;
  while (!act.empty()) {
    // FP64 update + residual of every active case
    const int na = (int)act.size();
    int first = 0;
    for (int k = 0; k < na; ++k) {
      const int i = act[k];
      ibm_ctx* c = B->cs[i];
      B->h_dc[k] = DcCase{c->geo, c->geo32.pk, S[i].add, first, S[i].cur, S[i].alt, c->e32, c->b, c->r32,
                          B->d_bits + k};
      first += ((c->nx + 31) / 32) * ((c->ny + 7) / 8);
    }
    if (timing) CUDA_TRY(cudaEventRecord(B->t1, B->stream));
    CUDA_TRY(cudaMemcpyAsync(B->d_dc, B->h_dc, na * sizeof(DcCase), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemsetAsync(B->d_bits, 0, na * sizeof(unsigned long long), B->stream));
    launch_dc_residual_batch(B->stream, B->d_dc, na, first);
    B->prof.launches += 1;
    CUDA_TRY(cudaMemcpyAsync(B->h_bits, B->d_bits, na * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    CUDA_TRY(cudaGetLastError());
    if (timing) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, B->t0, B->t1));
      B->prof.sweep_ms += ms;
      timing = false;
    }
    next.clear();
    int round = 1 << 30;
    for (int k = 0; k < na; ++k) {
      const int i = act[k];
      ibm_ctx* c = B->cs[i];
      State& q = S[i];
      if (q.add) std::swap(q.cur, q.alt);
      const double r = bits_to_double(B->h_bits[k]);
      st[i].sweeps_p = q.s;
      st[i].res_p = r;
      c->phi = q.cur;
      c->phi2 = q.alt;
      if (!std::isfinite(r))
        return fail(IBM_E_DIVERGED, "batch case %d: pressure residual is not finite after %d sweeps", i, q.s);
      if (r <= thr[i]) continue;
      if (q.s >= c->P.max_sweeps)
        return fail(IBM_E_NOCONV, "batch case %d: pressure solve: %d sweeps, residual %.3e > %.3e", i, q.s, r,
                    thr[i]);
      if (q.inner > 0 && q.prev > r && r > 0.0) {
        const double rate = std::log(r / q.prev) / q.inner;
        const int m = (int)(kInnerFrac * std::log(thr[i] / r) / rate);
        c->m_inner = m < 16 ? 16 : (m > kInnerMax ? kInnerMax : m);
      }
      int w = (c->m_inner + pair_sweeps - 1) / pair_sweeps * pair_sweeps;
      const int left = (c->P.max_sweeps - q.s + pair_sweeps - 1) / pair_sweeps * pair_sweeps;
      want[i] = w < left ? w : left;
      round = std::min(round, want[i]);
      q.prev = r;
      next.push_back(i);
    }
    act.swap(next);
    if (act.empty()) break;
    // FP32 sweeps of every active case: with budgets each case takes the
    // sweeps it asked for (its CTAs skip the launch pairs beyond them) and
    // the round lasts as long as the largest request; otherwise every case
    // takes the shortest request
    std::vector<int> pairs(act.size());
    int round_pairs = 0;
    for (size_t k = 0; k < act.size(); ++k) {
      pairs[k] = (B->budgets ? want[act[k]] : round) / pair_sweeps;
      round_pairs = std::max(round_pairs, pairs[k]);
    }
    int tiles = 0;
    int rc = batch_sor_tables(B, B->cfg, act, &tiles, B->budgets ? &pairs : nullptr);
    if (rc) return rc;
    if (B->profiling) {
      CUDA_TRY(cudaEventRecord(B->t0, B->stream));
      timing = true;
      long long cells = 0;
      for (size_t k = 0; k < act.size(); ++k) cells += (long long)B->cs[act[k]]->nx * B->cs[act[k]]->ny * pairs[k];
      B->prof.sweep_launches += 2 * round_pairs;
      B->prof.sweep_cells += cells * 2;
    }
    if (B->budgets) {
      // direct launches (programmatic dependents): the pair index varies per launch
      B->prof.launches += 2 * round_pairs;
      for (int q = 0; q < round_pairs; ++q) {
        launch_sor32_batch(B->stream, B->cfg, B->d_sor, (int)act.size(), tiles, q == 0, 1, q);
        launch_sor32_batch(B->stream, B->cfg, B->d_sor + n, (int)act.size(), tiles, 0, 1, q);
      }
      CUDA_TRY(cudaGetLastError());
    } else {
      rc = batch_sweeps(B, (int)act.size(), tiles, round_pairs);
      if (rc) return rc;
    }
    for (size_t k = 0; k < act.size(); ++k) {
      const int i = act[k];
      S[i].s += pairs[k] * pair_sweeps;
      S[i].add = 1;
      S[i].inner = pairs[k] * pair_sweeps;
    }
  }
  for (int i = 0; i < n; ++i) B->prof.poisson_sweeps += st[i].sweeps_p;
  return IBM_OK;
}

// ---- whole-step batching
// The case table entry of context c for the step it is about to take (a1:
// the body's position and velocity at t^{n+1}, Eqs. 1-2).
StepCase step_case(const ibm_ctx* c) {
  StepCase s{};
  const ibm_grid_params& P = c->P;
  s.g = c->geo;
  s.band = c->band;
  s.h32 = c->h32;
  s.u = c->u; s.v = c->v; s.p = c->p; s.Hu = c->Hu; s.Hv = c->Hv; s.Huo = c->Huo; s.Hvo = c->Hvo;
  s.Ru = c->Ru; s.Rv = c->Rv; s.uh = c->uh; s.vh = c->vh; s.b = c->b; s.phi = c->phi; s.phi_store = c->phi2;
  s.au = c->au; s.av = c->av; s.qband = c->qband; s.rowsum = c->rowsum; s.partials = c->partials;
  s.cl_hist = c->cl_d; s.cd_hist = c->cd_d;
  s.fu = c->fu; s.fv = c->fv; s.fc = c->fc;
  s.hd32 = c->hd32; s.hr32 = c->hr32; s.hinv_u = c->hinv_u; s.hinv_v = c->hinv_v;
  s.sc = c->sc;
  s.dt = P.dt;
  s.beta = P.dt / (2.0 * P.Re);
  const double t1 = (c->n + 1) * P.dt;
  s.yb = c->yb0;
  s.vb = 0.0;
  if (c->has_body) {
    s.yb = c->yb0 + c->h * std::sin(c->k * t1);
    s.vb = c->k * c->h * std::cos(c->k * t1);
  }
  s.xb = c->xb;
  s.ea = 0.5 * c->chord;
  s.eb = 0.5 * c->tc * c->chord;
  s.u_in = P.u_in;
  s.chord = c->chord;
  s.omega_h = (float)P.omega_h;
  s.first_step = c->n == 0 ? 1 : 0;
  s.n = c->n;
  s.has_body = c->has_body ? 1 : 0;
  s.nelem = (int)c->nelem;
  return s;
}

// The velocity system of `grid` for every case: the defect-correction rounds
// of solve_helm_mixed (an FP64 residual check, then 4 FP32 red-black sweeps
// from d = 0 and x += d), with one residual launch and one host check for
// all cases per round and shared sweep launches; cases leave as they
// converge, each after exactly the sweeps it would take alone.
int batch_helm(ibm_batch* B, int grid, std::vector<ibm_step_stats>& st) {
  const int n = (int)B->cs.size(), m = 4;
  std::vector<int> act(n), next;
  for (int i = 0; i < n; ++i) act[i] = i;
  for (int s = 0;; s += m) {
    int na = (int)act.size(), tot = 0;
    for (int k = 0; k < na; ++k) {
      B->h_hres[k] = act[k];
      B->h_hres[n + k] = tot;
      tot += helm_batch_blocks(B->h_cases[act[k]], grid, 0);
    }
    CUDA_TRY(cudaMemcpyAsync(B->d_hres, B->h_hres, 2 * n * sizeof(int), cudaMemcpyHostToDevice, B->stream));
    CUDA_TRY(cudaMemsetAsync(B->d_bits, 0, na * sizeof(unsigned long long), B->stream));
    launch_helm_dc_res_batch(B->stream, B->d_cases, B->d_hres, B->d_hres + n, na, tot, grid, B->d_bits);
    CUDA_TRY(cudaMemcpyAsync(B->h_bits, B->d_bits, na * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    CUDA_TRY(cudaGetLastError());
    B->prof.launches += 1;
    next.clear();
    for (int k = 0; k < na; ++k) {
      const int i = act[k];
      const double r = bits_to_double(B->h_bits[k]);
      (grid == 0 ? st[i].sweeps_u : st[i].sweeps_v) = s;
      (grid == 0 ? st[i].res_u : st[i].res_v) = r;
      if (!std::isfinite(r)) return fail(IBM_E_DIVERGED, "batch case %d: velocity residual is not finite", i);
      if (r <= B->cs[i]->P.helm_tol) continue;
      if (s >= B->cs[i]->P.max_sweeps)
        return fail(IBM_E_NOCONV, "batch case %d: velocity solve (grid %d) did not converge", i, grid);
      next.push_back(i);
    }
    act.swap(next);
    if (act.empty()) return IBM_OK;
    na = (int)act.size();
    int th = 0, tf = 0;
    for (int k = 0; k < na; ++k) {
      B->h_hswp[k] = act[k];
      B->h_hswp[n + k] = th;
      B->h_hswp[2 * n + k] = tf;
      th += helm_batch_blocks(B->h_cases[act[k]], grid, 1);
      tf += helm_batch_blocks(B->h_cases[act[k]], grid, 0);
    }
    CUDA_TRY(cudaMemcpyAsync(B->d_hswp, B->h_hswp, 3 * n * sizeof(int), cudaMemcpyHostToDevice, B->stream));
    launch_helm_zero_batch(B->stream, B->d_cases, B->d_hswp, na);
    for (int k = 0; k < m; ++k) {
      launch_helm32_half_batch(B->stream, B->d_cases, B->d_hswp, B->d_hswp + n, na, th, grid, 0);
      launch_helm32_half_batch(B->stream, B->d_cases, B->d_hswp, B->d_hswp + n, na, th, grid, 1);
    }
    launch_helm_add_batch(B->stream, B->d_cases, B->d_hswp, B->d_hswp + 2 * n, na, tf, grid);
    B->prof.launches += 2 * m + 2;
  }
}

// One step of every case with each part of the step (a1-a11) as shared
// launches: the number of launches per step does not grow with the number
// of cases, and the host waits once per defect-correction round of the
// velocity and pressure solves and once at the end.  Per case the
// arithmetic is that of one_step on precision 1, so every case takes the
// step it would take alone.
int batch_one_step_fused(ibm_batch* B) {
  const int n = (int)B->cs.size();
  std::vector<ibm_step_stats> st(n);
  std::vector<double> thr(n);
  for (int i = 0; i < n; ++i) {
    int rc = ensure_history(B->cs[i], B->cs[i]->n + 1);
    if (rc) return rc;
    B->h_cases[i] = step_case(B->cs[i]);
    thr[i] = B->cs[i]->P.poisson_tol;
  }
  if (!B->first_ready) {
    for (int k = 0; k < BK_NUM; ++k) {
      int tot = 0;
      for (int i = 0; i < n; ++i) {
        B->h_first[k * n + i] = tot;
        tot += batch_blocks(B->h_cases[i], k);
      }
      B->total[k] = tot;
    }
    CUDA_TRY(cudaMemcpyAsync(B->d_first, B->h_first, BK_NUM * n * sizeof(int), cudaMemcpyHostToDevice, B->stream));
    B->first_ready = true;
  }
  CUDA_TRY(cudaMemcpyAsync(B->d_cases, B->h_cases, n * sizeof(StepCase), cudaMemcpyHostToDevice, B->stream));
  const int* first = B->d_first;
  {
    NvtxRange r("a1-a4 classification, boundary values, predictor (batch)");
    launch_classify_batch(B->stream, B->d_cases, first + BK_BAND * n, n, B->total[BK_BAND]);
    launch_outflow_bc_batch(B->stream, B->d_cases, n);
    launch_predict_batch(B->stream, B->d_cases, first + BK_PREDICT_U * n, B->total[BK_PREDICT_U],
                         first + BK_PREDICT_V * n, B->total[BK_PREDICT_V], n);
    B->prof.launches += 6;
  }
  int rc;
  {
    NvtxRange r("a5 velocity solves (batch)");
    rc = batch_helm(B, 0, st);
    if (!rc) rc = batch_helm(B, 1, st);
  }
  if (rc) return rc;
  {
    NvtxRange r("a6 right-hand side and mass source (batch)");
    launch_rhs_batch(B->stream, B->d_cases, first + BK_CELLS * n, B->total[BK_CELLS], first + BK_BAND * n,
                     B->total[BK_BAND], n);
    B->prof.launches += 3;
  }
  {
    NvtxRange r("a8 pressure solves of the batch");
    rc = batch_solve(B, thr, st);
  }
  if (rc) return rc;
  // the solve leaves each case's increment in phi (its buffers may have swapped)
  for (int i = 0; i < n; ++i) {
    B->h_cases[i].phi = B->cs[i]->phi;
    B->h_cases[i].phi_store = B->cs[i]->phi2;
  }
  {
    NvtxRange r("a9-a11 forces, projection and divergence (batch)");
    CUDA_TRY(cudaMemcpyAsync(B->d_cases, B->h_cases, n * sizeof(StepCase), cudaMemcpyHostToDevice, B->stream));
    launch_forces_batch(B->stream, B->d_cases, n);
    launch_project_batch(B->stream, B->d_cases, first + BK_CELLS * n, B->total[BK_CELLS], n, B->d_rb);
    CUDA_TRY(cudaMemcpyAsync(B->h_rb, B->d_rb, n * sizeof(StepReadback), cudaMemcpyDeviceToHost, B->stream));
    CUDA_TRY(cudaStreamSynchronize(B->stream));
    CUDA_TRY(cudaGetLastError());
    B->prof.launches += 5;
  }
  for (int i = 0; i < n; ++i) {
    ibm_ctx* c = B->cs[i];
    *c->sc_host = B->h_rb[i].sc;
    std::swap(c->phi, c->phi2);
    std::swap(c->Hu, c->Huo);
    std::swap(c->Hv, c->Hvo);
    c->n += 1;
    c->prof.steps += 1;
    c->prof.poisson_sweeps += st[i].sweeps_p;
    c->prof.helm_sweeps += st[i].sweeps_u + st[i].sweeps_v;
    st[i].n = c->n;
    st[i].t = c->n * c->P.dt;
    st[i].div_max = bits_to_double(c->sc_host->div_bits);
    st[i].cl = B->h_rb[i].cl;
    st[i].cd = B->h_rb[i].cd;
    c->last = st[i];
  }
  B->prof.steps += 1;
  return IBM_OK;
}

int batch_one_step(ibm_batch* B) {
  const int n = (int)B->cs.size();
  // cases with a learned or extrapolated warm start, samples or a relative
  // pressure tolerance take the parts before and after the pressure solve
  // case by case
  bool fused = true;
  for (ibm_ctx* c : B->cs)
    if (c->ws_mode != 0 || c->ws_base != 0 || c->P.poisson_rtol > 0.0) fused = false;
  if (fused) return batch_one_step_fused(B);
  std::vector<ibm_step_stats> st(n);
  std::vector<double> thr(n);
  for (int i = 0; i < n; ++i) {
    int rc = step_pre(B->cs[i], &st[i], &thr[i]);
    if (rc) return rc;
  }
  int rc;
  {
    NvtxRange r("a8 pressure solves of the batch");
    rc = batch_solve(B, thr, st);
  }
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    rc = step_post(B->cs[i], &st[i]);
    if (rc) return rc;
  }
  B->prof.steps += 1;
  return IBM_OK;
}

}  // namespace

namespace {

struct FieldDesc {
  double* ptr;
  int w, h;
};

FieldDesc field_desc(const ibm_ctx* c, int which) {
  const int nx = c->nx, ny = c->ny;
  switch (which) {
    case IBM_U: return {c->u, nx + 1, ny};
    case IBM_V: return {c->v, nx, ny + 1};
    case IBM_P: return {c->p, nx, ny};
    case IBM_PHI: return {c->phi, nx, ny};
    case IBM_B: return {c->b, nx, ny};
    case IBM_UHAT: return {c->uh, nx + 1, ny};
    case IBM_VHAT: return {c->vh, nx, ny + 1};
    case IBM_RU: return {c->Ru, nx + 1, ny};
    case IBM_RV: return {c->Rv, nx, ny + 1};
    case IBM_HU: return {c->Huo, nx + 1, ny};  // swapped after the step: Huo holds H^n
    case IBM_HV: return {c->Hvo, nx, ny + 1};
    default: return {nullptr, 0, 0};
  }
}

}  // namespace

namespace ibm {
// records the message returned by ibm_last_error() on this thread
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace ibm

extern "C" {

const char* ibm_last_error(void) { return g_err.c_str(); }

int ibm_create_grid(const ibm_grid_params* params, ibm_ctx** out) {
  if (!params || !out) return fail(IBM_E_INVAL, "null argument");
  *out = nullptr;
  ibm_grid_params P = *params;
  if (P.nx < 4 || P.ny < 4) return fail(IBM_E_INVAL, "nx, ny must be >= 4");
  if (P.ny > 8192) return fail(IBM_E_INVAL, "ny must be <= 8192 (outflow flux reduction)");
  if (!(P.Re > 0.0) || !(P.dt > 0.0)) return fail(IBM_E_INVAL, "Re and dt must be positive");
  if (P.bc != 0 && P.bc != 1) return fail(IBM_E_INVAL, "bc must be 0 or 1");
  if (P.precision < 0 || P.precision > 2) return fail(IBM_E_INVAL, "precision must be 0, 1 or 2");
  if (P.omega_p <= 0.0) P.omega_p = 2.0 / (1.0 + std::sin(M_PI / (P.nx > P.ny ? P.nx : P.ny)));
  if (P.omega_h <= 0.0) P.omega_h = 1.0;
  if (!(P.omega_p < 2.0) || !(P.omega_h < 2.0)) return fail(IBM_E_INVAL, "omega must lie in (0, 2)");
  if (P.check_every_p <= 0) P.check_every_p = 8;
  if (P.check_every_h <= 0) P.check_every_h = 2;
  if (P.max_sweeps <= 0) P.max_sweeps = 1000000;
  if (P.helm_tol <= 0.0) P.helm_tol = 1e-12;
  if (P.poisson_tol <= 0.0 && P.poisson_rtol <= 0.0) return fail(IBM_E_INVAL, "a Poisson tolerance is required");
  auto* c = new ibm_ctx();
  c->P = P;
  c->nx = P.nx;
  c->ny = P.ny;
  if (!build_axis(P.x0, P.x1, P.ubox[0], P.ubox[1], P.nx, P.hmin, c->xf) ||
      !build_axis(P.y0, P.y1, P.ubox[2], P.ubox[3], P.ny, P.hmin, c->yf)) {
    delete c;
    return fail(IBM_E_INVAL, "cannot build the grid (check domain, uniform box and hmin)");
  }
  c->pitch = ((P.nx + 2 + XOFF) + 31) / 32 * 32;
  c->rows = P.ny + 3;
  c->nelem = (size_t)c->pitch * c->rows;
  if (P.cuda_stream) {
    c->stream = (cudaStream_t)P.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return fail(IBM_E_CUDA, "cannot create a stream");
    }
    c->own_stream = true;
  }
  int rc = 0;
  double** fields[] = {&c->u, &c->v, &c->p, &c->phi, &c->phi2, &c->b, &c->uh, &c->vh,
                       &c->Ru, &c->Rv, &c->Hu, &c->Hv, &c->Huo, &c->Hvo};
  for (double** f : fields) rc |= c->alloc(f, c->nelem);
  rc |= c->alloc(&c->sc, 1);
  rc |= c->alloc(&c->partials, 4 * RED_BLOCKS);
  if (!rc) rc = setup_geometry(c);
  if (!rc && cudaMallocHost((void**)&c->sc_host, sizeof(DevScalars)) != cudaSuccess) rc = IBM_E_CUDA;
  if (!rc) rc = ensure_history(c, 1024);
  // band arrays exist (1 x 1) even without a body
  if (!rc) {
    rc |= c->alloc(&c->fu, 1);
    rc |= c->alloc(&c->fv, 1);
    rc |= c->alloc(&c->fc, 1);
    rc |= c->alloc(&c->au, 1);
    rc |= c->alloc(&c->av, 1);
    rc |= c->alloc(&c->qband, 1);
    c->band = Band{-100, -100, 1, 1};
  }
  if (!rc && P.bc == 0) {
    std::vector<double> col(P.ny, P.u_in);
    if (cudaMemcpy2D(c->u + at(0, 0, c->pitch), c->pitch * sizeof(double), col.data(), sizeof(double),
                     sizeof(double), P.ny, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = IBM_E_CUDA;
  }
  if (rc) {
    std::string keep = g_err;
    delete c;
    g_err = keep.empty() ? "allocation failed" : keep;
    return rc < 0 ? rc : IBM_E_CUDA;
  }
  *out = c;
  return IBM_OK;
}

int ibm_set_body(ibm_ctx* c, double chord, double tc, double h, double k, double xc, double yc) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (c->n != 0) return fail(IBM_E_INVAL, "the body must be set before the first step");
  if (!(chord > 0.0) || !(tc > 0.0)) return fail(IBM_E_INVAL, "chord and thickness ratio must be positive");
  const double a = 0.5 * chord, bsemi = 0.5 * tc * chord;
  const double xlo = xc - a, xhi = xc + a, ylo = yc - std::fabs(h) - bsemi, yhi = yc + std::fabs(h) + bsemi;
  const int nx = c->nx, ny = c->ny;
  // band: every node index whose coordinate can lie inside the body, plus 4
  int i0 = 0, i1 = nx, j0 = 0, j1 = ny;
  while (i0 < nx && c->xf[i0 + 1] < xlo) ++i0;
  while (i1 > 0 && c->xf[i1 - 1] > xhi) --i1;
  while (j0 < ny && c->yf[j0 + 1] < ylo) ++j0;
  while (j1 > 0 && c->yf[j1 - 1] > yhi) --j1;
  i0 -= 4;
  j0 -= 4;
  i1 += 4;
  j1 += 4;
  if (i0 < 2 || j0 < 2 || i1 > nx - 2 || j1 > ny - 2)
    return fail(IBM_E_INVAL, "the body's swept region reaches the domain boundary");
  Band B{i0, j0, i1 - i0 + 1, j1 - j0 + 1};
  size_t nb = (size_t)B.w * B.h;
  int rc = 0;
  rc |= c->alloc(&c->fu, nb);
  rc |= c->alloc(&c->fv, nb);
  rc |= c->alloc(&c->fc, nb);
  rc |= c->alloc(&c->au, nb);
  rc |= c->alloc(&c->av, nb);
  rc |= c->alloc(&c->qband, nb);
  rc |= c->alloc(&c->rowsum, 2 * (size_t)B.h);
  if (rc) return IBM_E_CUDA;
  c->band = B;
  c->has_body = true;
  c->chord = chord;
  c->tc = tc;
  c->h = h;
  c->k = k;
  c->xb = xc;
  c->yb0 = yc;
  // momentum carried inside the body at t = 0 (first internal-mass term)
  launch_classify(c->stream, c->geo, B, xc, yc, a, bsemi, c->fu, c->fv, c->fc, c->au, c->av);
  launch_init_body_momentum(c->stream, c->geo, B, c->fv, k * h, c->partials, c->sc);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

int ibm_step(ibm_ctx* c, int nsteps, ibm_step_stats* last) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (nsteps < 0) return fail(IBM_E_INVAL, "nsteps < 0");
  for (int s = 0; s < nsteps; ++s) {
    int rc = one_step(c);
    if (rc) return rc;
  }
  if (last) *last = c->last;
  return IBM_OK;
}

int ibm_forces(const ibm_ctx* c, double* cl, double* cd, int cap, int* n_out) {
  if (!c || !n_out) return fail(IBM_E_INVAL, "null argument");
  int n = c->n < cap ? c->n : cap;
  if (n > 0 && cl) CUDA_TRY(cudaMemcpyAsync(cl, c->cl_d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  if (n > 0 && cd) CUDA_TRY(cudaMemcpyAsync(cd, c->cd_d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  *n_out = c->n;
  return IBM_OK;
}

int ibm_get_field(const ibm_ctx* c, int which, double* host, size_t n) {
  if (!c || !host) return fail(IBM_E_INVAL, "null argument");
  if (which == IBM_Q) {
    if (n != (size_t)c->nx * c->ny) return fail(IBM_E_INVAL, "size mismatch");
    std::memset(host, 0, n * sizeof(double));
    if (!c->has_body) return IBM_OK;
    const Band& B = c->band;
    std::vector<double> q((size_t)B.w * B.h);
    CUDA_TRY(cudaMemcpyAsync(q.data(), c->qband, q.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int bj = 0; bj < B.h; ++bj)
      for (int bi = 0; bi < B.w; ++bi) {
        int i = B.i0 + bi, j = B.j0 + bj;
        if (i >= 0 && i < c->nx && j >= 0 && j < c->ny) host[(size_t)j * c->nx + i] = q[(size_t)bj * B.w + bi];
      }
    return IBM_OK;
  }
  FieldDesc f = field_desc(c, which);
  if (!f.ptr) return fail(IBM_E_INVAL, "unknown field %d", which);
  if (n != (size_t)f.w * f.h) return fail(IBM_E_INVAL, "size mismatch: %zu vs %d", n, f.w * f.h);
  CUDA_TRY(cudaMemcpy2DAsync(host, f.w * sizeof(double), f.ptr + at(0, 0, c->pitch), c->pitch * sizeof(double),
                             f.w * sizeof(double), f.h, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

int ibm_set_field(ibm_ctx* c, int which, const double* host, size_t n) {
  if (!c || !host) return fail(IBM_E_INVAL, "null argument");
  if (which < IBM_U || which > IBM_PHI) return fail(IBM_E_INVAL, "only u, v, p, phi can be set");
  FieldDesc f = field_desc(c, which);
  if (n != (size_t)f.w * f.h) return fail(IBM_E_INVAL, "size mismatch");
  CUDA_TRY(cudaMemcpy2DAsync(f.ptr + at(0, 0, c->pitch), c->pitch * sizeof(double), host, f.w * sizeof(double),
                             f.w * sizeof(double), f.h, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

int ibm_get_flags(const ibm_ctx* c, int grid, unsigned char* kind, unsigned char* dir, double* alpha, size_t n) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  const int nx = c->nx, ny = c->ny;
  int w = grid == 0 ? nx + 1 : nx, h = grid == 1 ? ny + 1 : ny;
  if (grid < 0 || grid > 2) return fail(IBM_E_INVAL, "grid must be 0, 1 or 2");
  if (n != (size_t)w * h) return fail(IBM_E_INVAL, "size mismatch");
  if (kind) std::memset(kind, 0, n);
  if (dir) std::memset(dir, 0, n);
  if (alpha) std::memset(alpha, 0, n * sizeof(double));
  if (!c->has_body) return IBM_OK;
  const Band& B = c->band;
  size_t nb = (size_t)B.w * B.h;
  std::vector<uint8_t> f(nb);
  std::vector<double> a(nb);
  const uint8_t* fsrc = grid == 0 ? c->fu : grid == 1 ? c->fv : c->fc;
  CUDA_TRY(cudaMemcpyAsync(f.data(), fsrc, nb, cudaMemcpyDeviceToHost, c->stream));
  if (grid < 2) CUDA_TRY(cudaMemcpyAsync(a.data(), grid == 0 ? c->au : c->av, nb * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int bj = 0; bj < B.h; ++bj)
    for (int bi = 0; bi < B.w; ++bi) {
      int i = B.i0 + bi, j = B.j0 + bj;
      if (i < 0 || i >= w || j < 0 || j >= h) continue;
      size_t o = (size_t)j * w + i, k = (size_t)bj * B.w + bi;
      if (kind) kind[o] = grid == 2 ? f[k] : (f[k] & 3);
      if (dir && grid < 2) dir[o] = (f[k] & 3) == K_FORCE ? (f[k] >> 2) : 0;
      if (alpha && grid < 2) alpha[o] = a[k];
    }
  return IBM_OK;
}

int ibm_get_grid(const ibm_ctx* c, double* xf, double* yf) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (xf) std::memcpy(xf, c->xf.data(), sizeof(double) * (c->nx + 1));
  if (yf) std::memcpy(yf, c->yf.data(), sizeof(double) * (c->ny + 1));
  return IBM_OK;
}

int ibm_poisson_solve(ibm_ctx* c, const double* b_dev, double* phi_dev, double tol, int check_every, int max_sweeps,
                      int* sweeps, double* res) {
  if (!c || !b_dev || !phi_dev) return fail(IBM_E_INVAL, "null argument");
  if (!(tol > 0.0)) return fail(IBM_E_INVAL, "tol must be positive");
  const size_t rowb = c->nx * sizeof(double), pb = c->pitch * sizeof(double);
  CUDA_TRY(cudaMemcpy2DAsync(c->b + at(0, 0, c->pitch), pb, b_dev, rowb, rowb, c->ny, cudaMemcpyDeviceToDevice,
                             c->stream));
  CUDA_TRY(cudaMemcpy2DAsync(c->phi + at(0, 0, c->pitch), pb, phi_dev, rowb, rowb, c->ny, cudaMemcpyDeviceToDevice,
                             c->stream));
  int s = 0;
  double r = 0.0;
  const int maxs = max_sweeps > 0 ? max_sweeps : c->P.max_sweeps;
  if (c->P.precision == 1 && check_every > 0) c->m_inner = check_every;  // first run of FP32 sweeps
  int rc = c->P.precision == 2   ? solve_poisson_mg(c, tol, maxs, &s, &r)
           : c->P.precision == 1 ? solve_poisson_mixed(c, tol, maxs, &s, &r)
                                 : solve_poisson(c, tol, 0.0, check_every, maxs, &s, &r);
  if (sweeps) *sweeps = s;
  if (res) *res = r;
  if (rc && rc != IBM_E_NOCONV) return rc;
  if (!rc) {
    launch_phi_ref(c->stream, c->geo, c->phi, c->sc);
    launch_shift(c->stream, c->geo, c->phi, c->sc);
  }
  CUDA_TRY(cudaMemcpy2DAsync(phi_dev, rowb, c->phi + at(0, 0, c->pitch), pb, rowb, c->ny, cudaMemcpyDeviceToDevice,
                             c->stream));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return rc;
}

int ibm_set_profiling(ibm_ctx* c, int on) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if ((on || c->P.precision == 1) && !c->ev0) {
    CUDA_TRY(cudaEventCreate(&c->ev0));
    CUDA_TRY(cudaEventCreate(&c->ev1));
  }
  c->profiling = on != 0;
  c->prof = ibm_profile{};
  return IBM_OK;
}

int ibm_get_profile(const ibm_ctx* c, ibm_profile* out) {
  if (!c || !out) return fail(IBM_E_INVAL, "null argument");
  *out = c->prof;
  out->sor_shape[0] = out->sor_shape[1] = out->sor_shape[2] = 0;
  out->sor_us_per_sweep = c->sor_us;
  out->sor_index = c->sor_cfg;
  if (c->sor_cfg >= 0)
    sor32_describe(c->sor_cfg, &out->sor_shape[0], &out->sor_shape[1], &out->sor_shape[2], &out->sor_form);
  return IBM_OK;
}

int ibm_set_warmstart(ibm_ctx* c, int mode, ibm_unet* net, double target_scale) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (mode < 0 || mode > 2) return fail(IBM_E_INVAL, "warm-start mode must be 0, 1 or 2");
  if (mode == 1 && !net) return fail(IBM_E_INVAL, "the learned warm start needs a network");
  if (mode != 0 && (c->nx % 16 || c->ny % 16))
    return fail(IBM_E_INVAL, "the learned warm start needs nx and ny divisible by 16");
  if (mode != 0 && !(target_scale > 0.0)) return fail(IBM_E_INVAL, "target_scale must be positive");
  if (mode != 0 && !c->ws_feat) {
    c->Hc = c->ny / 2;
    c->Wc = c->nx / 2;
    const size_t nc = (size_t)c->Hc * c->Wc;
    int rc = 0;
    rc |= c->alloc(&c->ws_feat, 4 * nc);
    rc |= c->alloc(&c->ws_out, nc);
    rc |= c->alloc(&c->ws_target, nc);
    rc |= c->alloc(&c->phi_old, c->nelem);
    rc |= c->alloc(&c->ws_max, 4);
    if (rc) return IBM_E_CUDA;
  }
  c->ws_mode = mode;
  c->ws_net = net;
  c->ws_cT = mode ? target_scale : 1.0;
  c->has_sample = false;
  return IBM_OK;
}

namespace {

// Checkpoint layout: this header, then the pitched FP64 arrays u, v, p, phi
// (the last pressure increment, the next solve's start), H^n of u and v
// (AB2 history), the C_l and C_d histories (n values each) and, when the
// warm start extrapolates in time, the increment of the step before.
struct StateHeader {
  char magic[8];
  int32_t version, nx, ny, pitch;
  int64_t nelem;
  int32_t n, has_body, m_inner, mg_cycles, has_phi_prev, precision;
  int32_t sor_cfg, reserved;  // FP32 sweep shape (its sweeps per launch round the inner runs)
  double body[6];  // chord, thickness ratio, h, k, x and y of the centre
  double dt, Re;
  double S_prev[2];  // momentum inside the body at step n (added-mass term of the force)
};
constexpr char kStateMagic[8] = {'I', 'B', 'M', 'S', 'T', 'A', 'T', 'E'};

size_t state_bytes(const ibm_ctx* c) {
  const size_t fields = 6 + (c->phi_prev ? 1 : 0);
  return sizeof(StateHeader) + fields * c->nelem * sizeof(double) + 2 * (size_t)c->n * sizeof(double);
}

}  // namespace

int ibm_state_bytes(const ibm_ctx* c, size_t* bytes) {
  if (!c || !bytes) return fail(IBM_E_INVAL, "null argument");
  *bytes = state_bytes(c);
  return IBM_OK;
}

int ibm_save_state(const ibm_ctx* c, void* host, size_t bytes) {
  if (!c || !host) return fail(IBM_E_INVAL, "null argument");
  if (bytes < state_bytes(c)) return fail(IBM_E_INVAL, "state buffer too small: %zu < %zu", bytes, state_bytes(c));
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, 8);
  h.version = 1;
  h.nx = c->nx;
  h.ny = c->ny;
  h.pitch = c->pitch;
  h.nelem = (int64_t)c->nelem;
  h.n = c->n;
  h.has_body = c->has_body ? 1 : 0;
  h.m_inner = c->m_inner;
  h.mg_cycles = c->mg_cycles;
  h.has_phi_prev = c->phi_prev ? 1 : 0;
  h.precision = c->P.precision;
  h.sor_cfg = c->sor_cfg;
  const double body[6] = {c->chord, c->tc, c->h, c->k, c->xb, c->yb0};
  std::memcpy(h.body, body, sizeof body);
  h.dt = c->P.dt;
  h.Re = c->P.Re;
  CUDA_TRY(cudaMemcpyAsync(&c->sc_host->S_prev, &c->sc->S_prev, sizeof(h.S_prev), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  std::memcpy(h.S_prev, c->sc_host->S_prev, sizeof(h.S_prev));
  unsigned char* out = static_cast<unsigned char*>(host);
  std::memcpy(out, &h, sizeof h);
  out += sizeof h;
  const double* fields[7] = {c->u, c->v, c->p, c->phi, c->Huo, c->Hvo, c->phi_prev};
  const size_t fb = c->nelem * sizeof(double);
  for (int f = 0; f < 6 + h.has_phi_prev; ++f, out += fb)
    CUDA_TRY(cudaMemcpyAsync(out, fields[f], fb, cudaMemcpyDeviceToHost, c->stream));
  if (c->n > 0) {
    CUDA_TRY(cudaMemcpyAsync(out, c->cl_d, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    out += (size_t)c->n * sizeof(double);
    CUDA_TRY(cudaMemcpyAsync(out, c->cd_d, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

int ibm_load_state(ibm_ctx* c, const void* host, size_t bytes) {
  if (!c || !host) return fail(IBM_E_INVAL, "null argument");
  if (bytes < sizeof(StateHeader)) return fail(IBM_E_INVAL, "state buffer too small for its header");
  StateHeader h;
  std::memcpy(&h, host, sizeof h);
  if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1) return fail(IBM_E_INVAL, "not a state of this format");
  if (h.nx != c->nx || h.ny != c->ny || h.pitch != c->pitch || h.nelem != (int64_t)c->nelem)
    return fail(IBM_E_INVAL, "state of a %dx%d grid, context %dx%d", h.nx, h.ny, c->nx, c->ny);
  if (h.dt != c->P.dt || h.Re != c->P.Re) return fail(IBM_E_INVAL, "state taken with another dt or Re");
  if (h.n < 0) return fail(IBM_E_INVAL, "bad step count in the state");
  const double body[6] = {c->chord, c->tc, c->h, c->k, c->xb, c->yb0};
  if (h.has_body != (c->has_body ? 1 : 0) || (h.has_body && std::memcmp(h.body, body, sizeof body) != 0))
    return fail(IBM_E_INVAL, "the context's body differs from the state's (set the same body first)");
  if ((c->phi_prev != nullptr) && !h.has_phi_prev)
    return fail(IBM_E_INVAL, "the context extrapolates the warm start in time but the state has no history for it");
  const size_t fb = c->nelem * sizeof(double);
  const size_t need = sizeof h + (6 + (size_t)h.has_phi_prev) * fb + 2 * (size_t)h.n * sizeof(double);
  if (bytes < need) return fail(IBM_E_INVAL, "state buffer too small: %zu < %zu", bytes, need);
  int rc = ensure_history(c, h.n > 0 ? h.n : 1);
  if (rc) return rc;
  const unsigned char* in = static_cast<const unsigned char*>(host) + sizeof h;
  double* fields[6] = {c->u, c->v, c->p, c->phi, c->Huo, c->Hvo};
  for (int f = 0; f < 6; ++f, in += fb) CUDA_TRY(cudaMemcpyAsync(fields[f], in, fb, cudaMemcpyHostToDevice, c->stream));
  if (h.has_phi_prev) {
    if (c->phi_prev) CUDA_TRY(cudaMemcpyAsync(c->phi_prev, in, fb, cudaMemcpyHostToDevice, c->stream));
    in += fb;
  }
  if (h.n > 0) {
    CUDA_TRY(cudaMemcpyAsync(c->cl_d, in, (size_t)h.n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    in += (size_t)h.n * sizeof(double);
    CUDA_TRY(cudaMemcpyAsync(c->cd_d, in, (size_t)h.n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  std::memcpy(c->sc_host->S_prev, h.S_prev, sizeof(h.S_prev));
  CUDA_TRY(cudaMemcpyAsync(&c->sc->S_prev, c->sc_host->S_prev, sizeof(h.S_prev), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (h.sor_cfg >= sor32_num_configs()) return fail(IBM_E_INVAL, "unknown sweep shape in the state");
  c->n = h.n;
  c->m_inner = h.m_inner;
  c->mg_cycles = h.mg_cycles;
  if (h.sor_cfg >= 0) c->sor_cfg = h.sor_cfg;
  c->has_sample = false;
  return IBM_OK;
}

int ibm_set_preconditioner(ibm_ctx* c, int kind, ibm_unet* net, double target_scale, int pre_smooth) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (c->P.precision != 2) return fail(IBM_E_INVAL, "the preconditioner applies to precision 2 (FCG) only");
  if (kind < 0 || kind > 1) return fail(IBM_E_INVAL, "preconditioner kind must be 0 or 1");
  if (kind == 1) {
    if (!net) return fail(IBM_E_INVAL, "the two-level preconditioner needs a network");
    if (c->nx % 16 || c->ny % 16) return fail(IBM_E_INVAL, "the two-level preconditioner needs nx and ny divisible by 16");
    if (!(target_scale > 0.0)) return fail(IBM_E_INVAL, "target_scale must be positive");
    if (pre_smooth < 0 || pre_smooth > 1) return fail(IBM_E_INVAL, "pre_smooth must be 0 or 1");
    if (c->mg.size() < 2 || c->mg[1].g.nx != c->nx / 2 || c->mg[1].g.ny != c->ny / 2)
      return fail(IBM_E_INVAL, "level 1 of the hierarchy is not the 2x coarsened grid");
    if (!c->pc_feat) {
      c->Hc = c->ny / 2;
      c->Wc = c->nx / 2;
      const size_t nc = (size_t)c->Hc * c->Wc;
      int rc = 0;
      rc |= c->alloc(&c->pc_feat, 4 * nc);
      rc |= c->alloc(&c->pc_out, nc);
      rc |= c->alloc(&c->pc_max, 4);
      if (rc) return IBM_E_CUDA;
    }
  }
  c->pc_kind = kind;
  c->pc_net = kind ? net : nullptr;
  c->pc_cT = kind ? target_scale : 1.0;
  c->pc_pre = kind ? pre_smooth : 1;
  return IBM_OK;
}

int ibm_set_warmstart_base(ibm_ctx* c, int base) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (base != 0 && base != 1) return fail(IBM_E_INVAL, "warm-start base must be 0 or 1");
  if (base == 1 && !c->phi_prev) {
    int rc = c->alloc(&c->phi_prev, c->nelem);
    if (rc) return rc;
  }
  if (base == 1 && c->ws_base == 0)  // no history yet: the first extrapolation is the previous increment
    CUDA_TRY(cudaMemcpyAsync(c->phi_prev, c->phi, c->nelem * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  c->ws_base = base;
  return IBM_OK;
}

int ibm_get_sample(const ibm_ctx* c, float* feat, float* target, int* Hc, int* Wc) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (Hc) *Hc = c->Hc;
  if (Wc) *Wc = c->Wc;
  if (!feat && !target) return IBM_OK;
  if (!c->has_sample) return fail(IBM_E_INVAL, "no sample: capture (mode 2) and step first");
  const size_t nc = (size_t)c->Hc * c->Wc;
  if (feat) CUDA_TRY(cudaMemcpyAsync(feat, c->ws_feat, 4 * nc * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (target) CUDA_TRY(cudaMemcpyAsync(target, c->ws_target, nc * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return IBM_OK;
}

int ibm_sor_num_shapes(void) { return sor32_num_configs(); }

int ibm_set_sor_shape(ibm_ctx* c, int index) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (index < -1 || index >= sor32_num_configs())
    return fail(IBM_E_INVAL, "sweep shape %d out of range (-1 .. %d)", index, sor32_num_configs() - 1);
  if (index >= 0) {
    cudaError_t e = sor32_batch_prepare(index);
    if (e != cudaSuccess) return fail(IBM_E_CUDA, "sweep shape %d: %s", index, cudaGetErrorString(e));
  }
  c->sor_cfg = index;
  c->sor_us = 0.0;
  return IBM_OK;
}

int ibm_tune(ibm_ctx* c) {
  if (!c) return fail(IBM_E_INVAL, "null context");
  if (c->P.precision != 1) return IBM_OK;  // only the FP32 sweeps have shapes to choose
  int rc = tune_sor32(c);
  if (!rc) CUDA_TRY(cudaStreamSynchronize(c->stream));
  return rc;
}

void ibm_destroy(ibm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  delete c;
}

int ibm_batch_create(ibm_ctx* const* cases, int n, ibm_batch** out) {
  if (!cases || !out || n < 1) return fail(IBM_E_INVAL, "null argument or empty batch");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!cases[i]) return fail(IBM_E_INVAL, "batch case %d is null", i);
    if (cases[i]->P.precision != 1) return fail(IBM_E_INVAL, "batch case %d: precision must be 1", i);
    for (int k = 0; k < i; ++k)
      if (cases[k] == cases[i]) return fail(IBM_E_INVAL, "batch cases %d and %d are the same context", k, i);
  }
  auto* B = new ibm_batch();
  B->cs.assign(cases, cases + n);
  bool ok = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&B->h_sor, 2 * n * sizeof(Sor32Case)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&B->h_dc, n * sizeof(DcCase)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&B->h_bits, n * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&B->d_sor, 2 * n * sizeof(Sor32Case)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&B->d_dc, n * sizeof(DcCase)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&B->d_bits, n * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&B->h_cases, n * sizeof(StepCase)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&B->d_cases, n * sizeof(StepCase)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&B->h_first, BK_NUM * n * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&B->d_first, BK_NUM * n * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&B->h_hres, 2 * n * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&B->d_hres, 2 * n * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&B->h_hswp, 3 * n * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&B->d_hswp, 3 * n * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&B->h_rb, n * sizeof(StepReadback)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&B->d_rb, n * sizeof(StepReadback)) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&B->ev_b, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreate(&B->t0) == cudaSuccess && cudaEventCreate(&B->t1) == cudaSuccess;
  B->ev.resize(n, nullptr);
  for (int i = 0; ok && i < n; ++i) ok = cudaEventCreateWithFlags(&B->ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    delete B;
    return fail(IBM_E_CUDA, "batch allocation failed");
  }
  *out = B;
  return IBM_OK;
}

int ibm_batch_step(ibm_batch* B, int nsteps, ibm_step_stats* last) {
  if (!B || nsteps < 0) return fail(IBM_E_INVAL, "invalid argument");
  const int n = (int)B->cs.size();
  // all work of the batch runs on its stream, after what the cases' own
  // streams hold, and the cases' streams wait for it afterwards
  std::vector<cudaStream_t> own(n);
  for (int i = 0; i < n; ++i) {
    own[i] = B->cs[i]->stream;
    CUDA_TRY(cudaEventRecord(B->ev[i], own[i]));
    CUDA_TRY(cudaStreamWaitEvent(B->stream, B->ev[i], 0));
    B->cs[i]->stream = B->stream;
  }
  int rc = IBM_OK;
  for (int s = 0; s < nsteps && rc == IBM_OK; ++s) rc = batch_one_step(B);
  for (int i = 0; i < n; ++i) B->cs[i]->stream = own[i];
  cudaEventRecord(B->ev_b, B->stream);
  for (int i = 0; i < n; ++i) cudaStreamWaitEvent(own[i], B->ev_b, 0);
  if (rc) return rc;
  if (last)
    for (int i = 0; i < n; ++i) last[i] = B->cs[i]->last;
  return IBM_OK;
}

double ibm_omega_from_rate(double omega, double rho) { return omega_from_rate(omega, rho); }

int ibm_tune_omega(ibm_ctx* c, int sweeps, double* omega) {
  if (!c || !omega) return fail(IBM_E_INVAL, "null argument");
  return tune_omega(c, sweeps, omega);
}

int ibm_batch_set_sor_shape(ibm_batch* B, int index) {
  if (!B) return fail(IBM_E_INVAL, "null batch");
  if (index < -1 || index >= sor32_num_configs())
    return fail(IBM_E_INVAL, "sweep shape %d out of range (-1 .. %d)", index, sor32_num_configs() - 1);
  if (index >= 0) CUDA_TRY(sor32_batch_prepare(index));
  B->cfg = index;
  B->sor_us = 0.0;
  B->drop_graphs();
  return IBM_OK;
}

void* ibm_batch_stream(const ibm_batch* B) { return B ? (void*)B->stream : nullptr; }

int ibm_batch_set_graphs(ibm_batch* B, int on) {
  if (!B) return fail(IBM_E_INVAL, "null batch");
  B->use_graphs = on != 0;
  return IBM_OK;
}

int ibm_batch_set_budgets(ibm_batch* B, int on) {
  if (!B) return fail(IBM_E_INVAL, "null batch");
  B->budgets = on != 0;
  return IBM_OK;
}

int ibm_batch_set_profiling(ibm_batch* B, int on) {
  if (!B) return fail(IBM_E_INVAL, "null batch");
  B->profiling = on != 0;
  B->prof = ibm_profile{};
  for (ibm_ctx* c : B->cs) c->prof = ibm_profile{};
  return IBM_OK;
}

int ibm_batch_get_profile(const ibm_batch* B, ibm_profile* out) {
  if (!B || !out) return fail(IBM_E_INVAL, "null argument");
  *out = B->prof;
  out->sor_index = B->cfg;
  if (B->cfg >= 0) sor32_describe(B->cfg, &out->sor_shape[0], &out->sor_shape[1], &out->sor_shape[2], &out->sor_form);
  out->sor_us_per_sweep = B->sor_us;
  for (ibm_ctx* c : B->cs) {
    out->launches += c->prof.launches;
    out->helm_sweeps += c->prof.helm_sweeps;
  }
  return IBM_OK;
}

void ibm_batch_destroy(ibm_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  delete B;
}

}  // extern "C"
