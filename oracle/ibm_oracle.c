/*
 * Plain FP64 CPU oracle of the discrete-forcing immersed-boundary fractional
 * step (Sundar, Majumdar, Shah & Sarkar, arXiv 2402.17337).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the scheme that the GPU path is checked against.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (paper sections in brackets):
 *   - plunge kinematics y = h sin(k t), ydot = k h cos(k t)      [Sec. 2.1, Eqs. 1-2]
 *   - incompressible N-S with momentum forcing f and mass source q
 *     on a staggered Cartesian grid                               [Sec. 2.2, Eqs. 3-4]
 *   - fluid/solid classification at the start of every step      [Sec. 2.2]
 *   - semi-implicit fractional step: Adams-Bashforth convection,
 *     Crank-Nicolson diffusion, pressure and velocity correction
 *     solved by red-black Gauss-Seidel SOR                          [Sec. 2.2, Sec. 3.1]
 *   - stretched grid: uniform in the body region, geometric
 *     progression outward                                          [Sec. 2.3]
 *   - lift/drag histories                                          [Sec. 4.1]
 * The paper delegates the scheme's details to other papers; the readings used
 * here (boundary conditions, interpolation rule, mass source, pinned gauge,
 * force formula) are stated beside the code that implements them.
 *
 * Conventions: non-dimensional (chord = U_inf = rho = 1 in the paper's
 * setting).  Canonical layouts, x fastest:
 *   u   (nx+1) x ny   u[j*(nx+1)+i], face x_f[i], centre y_c[j]
 *   v   nx x (ny+1)   v[j*nx+i],     centre x_c[i], face y_f[j]
 *   p   nx x ny       p[j*nx+i]
 * Build with -ffp-contract=off so every product and sum is rounded alone.
 *
 * Arithmetic recipe.  Where floating point decides an integer (the SOR
 * iteration count, a node's kind) the GPU path must take the same decision,
 * so both follow one recipe: divisions by grid spacings are multiplications
 * by reciprocals computed once, the 5-point operators are fused
 * multiply-add chains in the order E, W, N, S (fma() below), and the two
 * sums that feed back into the flow are accumulated in a fixed two-level
 * index order (outflow flux: rows within chunks of 32, then the chunks;
 * body-cell source: along each row, then the rows).  Everything else is a
 * plain expression.
 *
 * Textbook form.  Compiled with -DORACLE_PLAIN the same file computes every
 * operator in its textbook form instead: flux differences divided by the
 * spacings, every product and sum rounded on its own (no fused
 * multiply-add), SOR updates written as (1 - omega) x + omega GS with the
 * Gauss-Seidel value divided by the diagonal, and the feedback sums in one
 * pass in index order.  The two forms are the same mathematics; the tests
 * compare them operator by operator and over whole steps, so a slip shared
 * by the recipe's two implementations (oracle and GPU) cannot hide in the
 * recipe itself.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_E_INVAL -1
#define OR_E_NOCONV -3
#define OR_E_DIVERGED -4

/* flags on the u and v grids */
#define FL_FLUID 0
#define FL_SOLID 1
#define FL_FORCE 2

typedef struct {
  double x0, x1, y0, y1; /* domain */
  int nx, ny;            /* cells */
  double hmin;           /* <=0: uniform grid */
  double ubox[4];        /* uniform box bx0,bx1,by0,by1 (stretched only) */
  int bc;                /* 0 inflow/convective outflow/free-slip walls; 1 free-slip box */
  double u_in;           /* inflow velocity (bc 0) */
  double Re, dt;
  double ptol, prtol;    /* Poisson: stop at ||r|| <= max(ptol, prtol*||b||) */
  double htol;           /* velocity systems: absolute tolerance */
  int check_p, check_h;  /* residual checked every m full sweeps */
  int max_sweeps;
  double omega_p, omega_h;
} or_params;

typedef struct {
  int n;          /* steps done */
  double t;
  int sweeps_u, sweeps_v, sweeps_p;
  double res_u, res_v, res_p;
  double div_max;  /* max |D u| over fluid (uncut) cells after the step */
  double cl, cd;
  double sum_q;    /* sum of q*V over cut cells (zero by construction) */
} or_stats;

typedef struct {
  or_params P;
  int nx, ny;
  /* grid */
  double *xf, *yf, *dx, *dy, *xc, *yc;
  double *dxc, *dyc; /* dxc[i] = xc[i]-xc[i-1], i=1..nx-1 (index 0, nx unused) */
  double *wx, *wy;   /* face interpolation weights, i=1..nx-1 */
  double *idx, *idy, *idxc, *idyc;      /* reciprocals of dx, dy, dxc, dyc */
  /* 5-point coefficients a_nb of sum_nb a_nb (x_nb - x_P); zero through walls */
  double *pE, *pW, *pN, *pS, *uE, *uW, *uN, *uS, *vE, *vW, *vN, *vS;
  double *ipd, *iud, *ivd;              /* reciprocal SOR diagonals per node */
  /* fields */
  double *u, *v, *p, *phi;
  double *uh, *vh, *Ru, *Rv, *Hu, *Hv, *Huo, *Hvo;
  double *D, *q, *b;
  /* classification */
  unsigned char *fu, *fv;  /* flags */
  unsigned char *du, *dv;  /* direction of the opposite node for forcing nodes */
  double *au, *av;         /* interpolation weight alpha */
  unsigned char *cut;      /* per cell: 1 when the cell centre lies inside the body */
  /* body */
  int has_body;
  double chord, tc, h, k, xb, yb0;
  double S_prev[2];
  /* history */
  int n;
  double *cl, *cd;
  int cap;
  or_stats last;
  int threads;
} or_sim;

/* ------------------------------------------------------------------ grid */

/* Sum_{m=1..ns} r^m, accumulated in order. */
static double geo_sum(double r, int ns) {
  double s = 0.0, pw = 1.0;
  for (int m = 1; m <= ns; ++m) {
    pw = pw * r;
    s = s + pw;
  }
  return s;
}

/* Ratio r >= 1 with hmin * sum_{m=1..ns} r^m = L, by bisection (Sec. 2.3:
 * geometric progression outward from the uniform region). */
static int solve_ratio(double hmin, int ns, double L, double* r_out) {
  if (ns == 0) {
    *r_out = 1.0;
    return 0;
  }
  double lo = 1.0, hi = 2.0;
  if (hmin * geo_sum(lo, ns) > L) return -1; /* the side cannot be stretched outward */
  while (hmin * geo_sum(hi, ns) < L) {
    hi = hi * 2.0;
    if (hi > 1e6) return -1;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (hmin * geo_sum(mid, ns) < L)
      lo = mid;
    else
      hi = mid;
  }
  *r_out = 0.5 * (lo + hi);
  return 0;
}

/* Face coordinates of one axis (n+1 values).  hmin<=0: uniform.  Otherwise a
 * uniform block of spacing hmin starting at b0 (round((b1-b0)/hmin) cells),
 * and on each side a geometric progression hmin*r^m, m=1..ns, summing to
 * the side length; the remaining cells are split between the two sides in
 * proportion to their lengths (rounded). */
int or_build_axis(double a0, double a1, double b0, double b1, int n, double hmin, double* f) {
  if (n < 1 || !(a1 > a0)) return OR_E_INVAL;
  if (hmin <= 0.0) {
    double hh = (a1 - a0) / n;
    for (int i = 0; i < n; ++i) f[i] = a0 + i * hh;
    f[n] = a1;
    return OR_OK;
  }
  if (!(b0 >= a0 && b1 <= a1 && b1 > b0)) return OR_E_INVAL;
  int nb = (int)lround((b1 - b0) / hmin);
  if (nb < 1 || nb > n) return OR_E_INVAL;
  double be = b0 + nb * hmin;
  if (be > a1) return OR_E_INVAL;
  double Ll = b0 - a0, Lr = a1 - be;
  int nrest = n - nb;
  int nl = (Ll + Lr > 0.0) ? (int)lround(nrest * (Ll / (Ll + Lr))) : 0;
  int nr = nrest - nl;
  if ((nl == 0) != (Ll == 0.0) || (nr == 0) != (Lr == 0.0)) return OR_E_INVAL;
  double rl, rr;
  if (solve_ratio(hmin, nl, Ll, &rl) || solve_ratio(hmin, nr, Lr, &rr)) return OR_E_INVAL;
  for (int m = 0; m <= nb; ++m) f[nl + m] = b0 + m * hmin;
  for (int m = 1; m <= nl; ++m) f[nl - m] = b0 - hmin * geo_sum(rl, m);
  for (int m = 1; m <= nr; ++m) f[nl + nb + m] = be + hmin * geo_sum(rr, m);
  f[0] = a0;
  f[n] = a1;
  return OR_OK;
}

static void* xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

/* ------------------------------------------------------------------ sim */

or_sim* or_create(const or_params* P) {
  if (P->nx < 2 || P->ny < 2) return NULL;
  or_sim* S = (or_sim*)xcalloc(1, sizeof(or_sim));
  S->P = *P;
  int nx = S->nx = P->nx, ny = S->ny = P->ny;
  S->threads = 1;
  S->xf = xcalloc(nx + 1, 8); S->yf = xcalloc(ny + 1, 8);
  if (or_build_axis(P->x0, P->x1, P->ubox[0], P->ubox[1], nx, P->hmin, S->xf) ||
      or_build_axis(P->y0, P->y1, P->ubox[2], P->ubox[3], ny, P->hmin, S->yf)) {
    free(S->xf); free(S->yf); free(S);
    return NULL;
  }
  S->dx = xcalloc(nx, 8); S->dy = xcalloc(ny, 8);
  S->xc = xcalloc(nx, 8); S->yc = xcalloc(ny, 8);
  S->dxc = xcalloc(nx + 1, 8); S->dyc = xcalloc(ny + 1, 8);
  S->wx = xcalloc(nx + 1, 8); S->wy = xcalloc(ny + 1, 8);
  for (int i = 0; i < nx; ++i) {
    S->dx[i] = S->xf[i + 1] - S->xf[i];
    S->xc[i] = 0.5 * (S->xf[i] + S->xf[i + 1]);
  }
  for (int j = 0; j < ny; ++j) {
    S->dy[j] = S->yf[j + 1] - S->yf[j];
    S->yc[j] = 0.5 * (S->yf[j] + S->yf[j + 1]);
  }
  for (int i = 1; i < nx; ++i) {
    S->dxc[i] = S->xc[i] - S->xc[i - 1];
    S->wx[i] = (S->xf[i] - S->xc[i - 1]) / S->dxc[i];
  }
  for (int j = 1; j < ny; ++j) {
    S->dyc[j] = S->yc[j] - S->yc[j - 1];
    S->wy[j] = (S->yf[j] - S->yc[j - 1]) / S->dyc[j];
  }
  S->idx = xcalloc(nx, 8); S->idy = xcalloc(ny, 8);
  S->idxc = xcalloc(nx + 1, 8); S->idyc = xcalloc(ny + 1, 8);
  for (int i = 0; i < nx; ++i) S->idx[i] = 1.0 / S->dx[i];
  for (int j = 0; j < ny; ++j) S->idy[j] = 1.0 / S->dy[j];
  for (int i = 1; i < nx; ++i) S->idxc[i] = 1.0 / S->dxc[i];
  for (int j = 1; j < ny; ++j) S->idyc[j] = 1.0 / S->dyc[j];
  /* pressure grid: homogeneous Neumann (no flux through the boundary) */
  S->pE = xcalloc(nx, 8); S->pW = xcalloc(nx, 8); S->pN = xcalloc(ny, 8); S->pS = xcalloc(ny, 8);
  for (int i = 0; i < nx; ++i) {
    S->pE[i] = i < nx - 1 ? 1.0 / (S->dx[i] * S->dxc[i + 1]) : 0.0;
    S->pW[i] = i > 0 ? 1.0 / (S->dx[i] * S->dxc[i]) : 0.0;
  }
  for (int j = 0; j < ny; ++j) {
    S->pN[j] = j < ny - 1 ? 1.0 / (S->dy[j] * S->dyc[j + 1]) : 0.0;
    S->pS[j] = j > 0 ? 1.0 / (S->dy[j] * S->dyc[j]) : 0.0;
  }
  /* u grid (CV [xc_{i-1},xc_i] x [yf_j,yf_{j+1}]): faces i=0, nx carry
   * Dirichlet values; free-slip walls y0, y1 pass no flux */
  S->uE = xcalloc(nx + 1, 8); S->uW = xcalloc(nx + 1, 8); S->uN = xcalloc(ny, 8); S->uS = xcalloc(ny, 8);
  for (int i = 1; i < nx; ++i) {
    S->uE[i] = 1.0 / (S->dx[i] * S->dxc[i]);
    S->uW[i] = 1.0 / (S->dx[i - 1] * S->dxc[i]);
  }
  for (int j = 0; j < ny; ++j) {
    S->uN[j] = j < ny - 1 ? 1.0 / (S->dyc[j + 1] * S->dy[j]) : 0.0;
    S->uS[j] = j > 0 ? 1.0 / (S->dyc[j] * S->dy[j]) : 0.0;
  }
  /* v grid (CV [xf_i,xf_{i+1}] x [yc_{j-1},yc_j]): rows j=0, ny carry v = 0.
   * At x0 the inflow (bc 0) holds v = 0 on the boundary, half a cell from
   * the node: flux 2 (0 - v)/dx, i.e. twice the coefficient with a zero
   * neighbour; free slip (bc 1) passes no flux.  At x1 zero flux. */
  S->vE = xcalloc(nx, 8); S->vW = xcalloc(nx, 8); S->vN = xcalloc(ny + 1, 8); S->vS = xcalloc(ny + 1, 8);
  for (int i = 0; i < nx; ++i) {
    S->vE[i] = i < nx - 1 ? 1.0 / (S->dxc[i + 1] * S->dx[i]) : 0.0;
    S->vW[i] = i > 0 ? 1.0 / (S->dxc[i] * S->dx[i]) : (P->bc == 0 ? 2.0 / (S->dx[0] * S->dx[0]) : 0.0);
  }
  for (int j = 1; j < ny; ++j) {
    S->vN[j] = 1.0 / (S->dy[j] * S->dyc[j]);
    S->vS[j] = 1.0 / (S->dy[j - 1] * S->dyc[j]);
  }
  {
    double beta = P->dt / (2.0 * P->Re);
    S->ipd = xcalloc((size_t)nx * ny, 8);
    S->iud = xcalloc((size_t)(nx + 1) * ny, 8);
    S->ivd = xcalloc((size_t)nx * (ny + 1), 8);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) S->ipd[(size_t)j * nx + i] = 1.0 / (S->pE[i] + S->pW[i] + S->pN[j] + S->pS[j]);
    for (int j = 0; j < ny; ++j)
      for (int i = 1; i < nx; ++i)
        S->iud[(size_t)j * (nx + 1) + i] = 1.0 / (1.0 + beta * (S->uE[i] + S->uW[i] + S->uN[j] + S->uS[j]));
    for (int j = 1; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        S->ivd[(size_t)j * nx + i] = 1.0 / (1.0 + beta * (S->vE[i] + S->vW[i] + S->vN[j] + S->vS[j]));
  }
  size_t nu = (size_t)(nx + 1) * ny, nv = (size_t)nx * (ny + 1), np = (size_t)nx * ny;
  S->u = xcalloc(nu, 8); S->uh = xcalloc(nu, 8); S->Ru = xcalloc(nu, 8);
  S->Hu = xcalloc(nu, 8); S->Huo = xcalloc(nu, 8);
  S->v = xcalloc(nv, 8); S->vh = xcalloc(nv, 8); S->Rv = xcalloc(nv, 8);
  S->Hv = xcalloc(nv, 8); S->Hvo = xcalloc(nv, 8);
  S->p = xcalloc(np, 8); S->phi = xcalloc(np, 8); S->D = xcalloc(np, 8);
  S->q = xcalloc(np, 8); S->b = xcalloc(np, 8);
  S->fu = xcalloc(nu, 1); S->fv = xcalloc(nv, 1);
  S->du = xcalloc(nu, 1); S->dv = xcalloc(nv, 1);
  S->au = xcalloc(nu, 8); S->av = xcalloc(nv, 8);
  S->cut = xcalloc(np, 1);
  /* initial state: zero interior flow; inflow face at u_in (bc 0) */
  if (P->bc == 0)
    for (int j = 0; j < ny; ++j) S->u[j * (nx + 1)] = P->u_in;
  S->cap = 0;
  return S;
}

void or_destroy(or_sim* S) {
  if (!S) return;
  void* ptrs[] = {S->xf, S->yf, S->dx, S->dy, S->xc, S->yc, S->dxc, S->dyc, S->wx, S->wy,
                  S->u, S->uh, S->Ru, S->Hu, S->Huo, S->v, S->vh, S->Rv, S->Hv, S->Hvo,
                  S->p, S->phi, S->D, S->q, S->b, S->fu, S->fv, S->du, S->dv, S->au, S->av,
                  S->cut, S->cl, S->cd, S->idx, S->idy, S->idxc, S->idyc, S->pE, S->pW, S->pN, S->pS,
                  S->uE, S->uW, S->uN, S->uS, S->vE, S->vW, S->vN, S->vS, S->ipd, S->iud, S->ivd};
  for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
  free(S);
}

void or_set_threads(or_sim* S, int t) { S->threads = t > 0 ? t : 1; }

int or_get_grid(const or_sim* S, double* xf, double* yf) {
  memcpy(xf, S->xf, sizeof(double) * (S->nx + 1));
  memcpy(yf, S->yf, sizeof(double) * (S->ny + 1));
  return OR_OK;
}

#define UI(i, j) ((size_t)(j) * (nx + 1) + (i))
#define VI(i, j) ((size_t)(j) * nx + (i))
#define PI_(i, j) ((size_t)(j) * nx + (i))

/* The two arithmetic forms (see the file header).  MULADD(a, b, c) is
 * a*b + c, fused in the recipe and rounded twice in the textbook form;
 * OVER(x, d, id) is x/d, computed as x times the stored reciprocal id = 1/d
 * in the recipe. */
#ifdef ORACLE_PLAIN
#define MULADD(a, b, c) ((a) * (b) + (c))
#define OVER(x, d, id) ((x) / (d))
#else
#define MULADD(a, b, c) fma((a), (b), (c))
#define OVER(x, d, id) ((x) * (id))
#endif

/* ------------------------------------------------- discrete operators (Sec. 2.2) */

#ifndef ORACLE_PLAIN
/* 5-point finite-volume Laplacian sum_nb a_nb (x_nb - x_P) as an fma chain
 * in the order E, W, N, S; a missing neighbour (outside the node range)
 * enters with value 0 and, except at an inflow face, a zero coefficient. */
static double lap5(double aE, double aW, double aN, double aS, double xE, double xW, double xN, double xS,
                   double c) {
  double L = aE * (xE - c);
  L = fma(aW, xW - c, L);
  L = fma(aN, xN - c, L);
  L = fma(aS, xS - c, L);
  return L;
}

/* Laplacian on the u grid at unknown nodes i = 1..nx-1, j = 0..ny-1 */
static double lap_u_at(const or_sim* S, const double* u, int i, int j) {
  int nx = S->nx, ny = S->ny;
  double c = u[UI(i, j)];
  double xN = j < ny - 1 ? u[UI(i, j + 1)] : 0.0;
  double xS = j > 0 ? u[UI(i, j - 1)] : 0.0;
  return lap5(S->uE[i], S->uW[i], S->uN[j], S->uS[j], u[UI(i + 1, j)], u[UI(i - 1, j)], xN, xS, c);
}

/* Laplacian on the v grid at unknown nodes i = 0..nx-1, j = 1..ny-1 */
static double lap_v_at(const or_sim* S, const double* v, int i, int j) {
  int nx = S->nx;
  double c = v[VI(i, j)];
  double xE = i < nx - 1 ? v[VI(i + 1, j)] : 0.0;
  double xW = i > 0 ? v[VI(i - 1, j)] : 0.0;
  return lap5(S->vE[i], S->vW[i], S->vN[j], S->vS[j], xE, xW, v[VI(i, j + 1)], v[VI(i, j - 1)], c);
}

/* Pressure Laplacian L_p = D G with homogeneous Neumann boundaries. */
static double lap_p_at(const or_sim* S, const double* f, int i, int j) {
  int nx = S->nx, ny = S->ny;
  double c = f[PI_(i, j)];
  double xE = i < nx - 1 ? f[PI_(i + 1, j)] : 0.0;
  double xW = i > 0 ? f[PI_(i - 1, j)] : 0.0;
  double xN = j < ny - 1 ? f[PI_(i, j + 1)] : 0.0;
  double xS = j > 0 ? f[PI_(i, j - 1)] : 0.0;
  return lap5(S->pE[i], S->pW[i], S->pN[j], S->pS[j], xE, xW, xN, xS, c);
}
#else
/* Textbook flux form of the same three Laplacians: the face gradients
 * (neighbour difference over the distance between the nodes) differenced
 * across the control volume and divided by its width. */

/* u grid: control volume [xc[i-1], xc[i]] x [yf[j], yf[j+1]]; free-slip walls
 * pass no flux through y0 and y1; the faces i = 0 and i = nx hold Dirichlet
 * values.  Unknown nodes i = 1..nx-1. */
static double lap_u_at(const or_sim* S, const double* u, int i, int j) {
  int nx = S->nx, ny = S->ny;
  double c = u[UI(i, j)];
  double fe = (u[UI(i + 1, j)] - c) / S->dx[i];
  double fw = (c - u[UI(i - 1, j)]) / S->dx[i - 1];
  double fn = (j < ny - 1) ? (u[UI(i, j + 1)] - c) / S->dyc[j + 1] : 0.0;
  double fs = (j > 0) ? (c - u[UI(i, j - 1)]) / S->dyc[j] : 0.0;
  return (fe - fw) / S->dxc[i] + (fn - fs) / S->dy[j];
}

/* v grid: control volume [xf[i], xf[i+1]] x [yc[j-1], yc[j]]; the walls y0,
 * y1 hold v = 0.  At x0 the inflow (bc 0) holds v = 0 on the boundary, half a
 * cell from the node; the free-slip box (bc 1) passes no flux.  At x1 no
 * flux. */
static double lap_v_at(const or_sim* S, const double* v, int i, int j) {
  int nx = S->nx;
  double c = v[VI(i, j)];
  double fe = (i < nx - 1) ? (v[VI(i + 1, j)] - c) / S->dxc[i + 1] : 0.0;
  double fw;
  if (i > 0)
    fw = (c - v[VI(i - 1, j)]) / S->dxc[i];
  else
    fw = (S->P.bc == 0) ? (c - 0.0) / (0.5 * S->dx[0]) : 0.0;
  double fn = (v[VI(i, j + 1)] - c) / S->dy[j];
  double fs = (c - v[VI(i, j - 1)]) / S->dy[j - 1];
  return (fe - fw) / S->dx[i] + (fn - fs) / S->dyc[j];
}

/* Pressure Laplacian L_p = D G with homogeneous Neumann boundaries. */
static double lap_p_at(const or_sim* S, const double* f, int i, int j) {
  int nx = S->nx, ny = S->ny;
  double c = f[PI_(i, j)];
  double fe = (i < nx - 1) ? (f[PI_(i + 1, j)] - c) / S->dxc[i + 1] : 0.0;
  double fw = (i > 0) ? (c - f[PI_(i - 1, j)]) / S->dxc[i] : 0.0;
  double fn = (j < ny - 1) ? (f[PI_(i, j + 1)] - c) / S->dyc[j + 1] : 0.0;
  double fs = (j > 0) ? (c - f[PI_(i, j - 1)]) / S->dyc[j] : 0.0;
  return (fe - fw) / S->dx[i] + (fn - fs) / S->dy[j];
}
#endif

/* Convective flux divergence H = div(u u), second-order central finite volume,
 * linear interpolation in the coordinate to the corners (Sec. 2.2). */
static double conv_u_at(const or_sim* S, const double* u, const double* v, int i, int j) {
  int nx = S->nx, ny = S->ny;
  double ue = 0.5 * (u[UI(i, j)] + u[UI(i + 1, j)]);
  double uw = 0.5 * (u[UI(i - 1, j)] + u[UI(i, j)]);
  double fn = 0.0, fs = 0.0;
  double w = S->wx[i];
  if (j < ny - 1) {
    double vn = (1.0 - w) * v[VI(i - 1, j + 1)] + w * v[VI(i, j + 1)];
    double un = (1.0 - S->wy[j + 1]) * u[UI(i, j)] + S->wy[j + 1] * u[UI(i, j + 1)];
    fn = vn * un;
  }
  if (j > 0) {
    double vs = (1.0 - w) * v[VI(i - 1, j)] + w * v[VI(i, j)];
    double us = (1.0 - S->wy[j]) * u[UI(i, j - 1)] + S->wy[j] * u[UI(i, j)];
    fs = vs * us;
  }
  return OVER(ue * ue - uw * uw, S->dxc[i], S->idxc[i]) + OVER(fn - fs, S->dy[j], S->idy[j]);
}
static double conv_v_at(const or_sim* S, const double* u, const double* v, int i, int j) {
  int nx = S->nx;
  double vn = 0.5 * (v[VI(i, j)] + v[VI(i, j + 1)]);
  double vs = 0.5 * (v[VI(i, j - 1)] + v[VI(i, j)]);
  double w = S->wy[j];
  double ue = (1.0 - w) * u[UI(i + 1, j - 1)] + w * u[UI(i + 1, j)];
  double ve = (i < nx - 1) ? (1.0 - S->wx[i + 1]) * v[VI(i, j)] + S->wx[i + 1] * v[VI(i + 1, j)]
                           : v[VI(i, j)];
  double uw = (1.0 - w) * u[UI(i, j - 1)] + w * u[UI(i, j)];
  double vw;
  if (i > 0)
    vw = (1.0 - S->wx[i]) * v[VI(i - 1, j)] + S->wx[i] * v[VI(i, j)];
  else
    vw = (S->P.bc == 0) ? 0.0 : v[VI(i, j)];
  return OVER(ue * ve - uw * vw, S->dx[i], S->idx[i]) + OVER(vn * vn - vs * vs, S->dyc[j], S->idyc[j]);
}

/* exported operator wrappers (canonical layouts; entries that are not
 * unknowns are left at zero) */
void or_lap_p(const or_sim* S, const double* f, double* out) {
  int nx = S->nx, ny = S->ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) out[PI_(i, j)] = lap_p_at(S, f, i, j);
}
void or_lap_u(const or_sim* S, const double* u, double* out) {
  int nx = S->nx, ny = S->ny;
  memset(out, 0, sizeof(double) * (nx + 1) * ny);
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i) out[UI(i, j)] = lap_u_at(S, u, i, j);
}
void or_lap_v(const or_sim* S, const double* v, double* out) {
  int nx = S->nx, ny = S->ny;
  memset(out, 0, sizeof(double) * nx * (ny + 1));
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) out[VI(i, j)] = lap_v_at(S, v, i, j);
}
void or_conv(const or_sim* S, const double* u, const double* v, double* Hu, double* Hv) {
  int nx = S->nx, ny = S->ny;
  memset(Hu, 0, sizeof(double) * (nx + 1) * ny);
  memset(Hv, 0, sizeof(double) * nx * (ny + 1));
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i) Hu[UI(i, j)] = conv_u_at(S, u, v, i, j);
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) Hv[VI(i, j)] = conv_v_at(S, u, v, i, j);
}
/* gradient of a cell field on the interior faces; boundary faces get 0 */
void or_grad(const or_sim* S, const double* f, double* gu, double* gv) {
  int nx = S->nx, ny = S->ny;
  memset(gu, 0, sizeof(double) * (nx + 1) * ny);
  memset(gv, 0, sizeof(double) * nx * (ny + 1));
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i) gu[UI(i, j)] = OVER(f[PI_(i, j)] - f[PI_(i - 1, j)], S->dxc[i], S->idxc[i]);
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) gv[VI(i, j)] = OVER(f[PI_(i, j)] - f[PI_(i, j - 1)], S->dyc[j], S->idyc[j]);
}
/* divergence of a face field, per cell */
void or_div(const or_sim* S, const double* u, const double* v, double* out) {
  int nx = S->nx, ny = S->ny;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      out[PI_(i, j)] = OVER(u[UI(i + 1, j)] - u[UI(i, j)], S->dx[i], S->idx[i]) +
                       OVER(v[VI(i, j + 1)] - v[VI(i, j)], S->dy[j], S->idy[j]);
}

/* ------------------------------------------ classification (Sec. 2.2, "flagging") */

/* Ellipse level function: solid iff ((x-xb)/a)^2 + ((y-yb)/b)^2 <= 1. */
static int inside(double x, double y, double xb, double yb, double a, double bb) {
  double xi = (x - xb) / a, eta = (y - yb) / bb;
  return xi * xi + eta * eta <= 1.0;
}

/* One grid (u: gx=xf, gy=yc, indices i 1..nx-1, j 0..ny-1; v: gx=xc, gy=yf,
 * i 0..nx-1, j 1..ny-1).  A forcing node is a fluid node with at least one
 * solid 4-neighbour on its own grid.  Among the directions towards a solid
 * neighbour, the one with the shortest distance d to the analytic wall is
 * taken (order -x,+x,-y,+y breaks ties); the node value is interpolated
 * linearly between the wall (body velocity) and the node on the opposite
 * side at distance D:  u_F = U_b + (u_opp - U_b) * d/(d+D).  When the
 * opposite node is solid, a forcing node or outside the unknowns, u_F = U_b
 * (alpha = 0). */
static void classify_grid(int ni, int nj, int ilo, int ihi, int jlo, int jhi, const double* gx,
                          const double* gy, double xb, double yb, double a, double bb,
                          unsigned char* fl, unsigned char* dir, double* al) {
  /* pass 1: solid */
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      size_t id = (size_t)j * ni + i;
      fl[id] = FL_FLUID;
      dir[id] = 0;
      al[id] = 0.0;
      if (i < ilo || i > ihi || j < jlo || j > jhi) continue;
      if (inside(gx[i], gy[j], xb, yb, a, bb)) fl[id] = FL_SOLID;
    }
#define ISSOL(ii, jj) ((ii) >= ilo && (ii) <= ihi && (jj) >= jlo && (jj) <= jhi && fl[(size_t)(jj) * ni + (ii)] == FL_SOLID)
#define HASSOLNB(ii, jj) (ISSOL((ii) - 1, jj) || ISSOL((ii) + 1, jj) || ISSOL(ii, (jj) - 1) || ISSOL(ii, (jj) + 1))
  /* pass 2: forcing nodes and their interpolation data */
  for (int j = jlo; j <= jhi; ++j)
    for (int i = ilo; i <= ihi; ++i) {
      size_t id = (size_t)j * ni + i;
      if (fl[id] == FL_SOLID || !HASSOLNB(i, j)) continue;
      fl[id] = FL_FORCE;
      double x = gx[i], y = gy[j];
      double best = INFINITY;
      int bd = -1;
      int nb_i[4] = {i - 1, i + 1, i, i};
      int nb_j[4] = {j, j, j - 1, j + 1};
      for (int d = 0; d < 4; ++d) {
        if (!ISSOL(nb_i[d], nb_j[d])) continue;
        double dist, span;
        if (d < 2) {
          double eta = (y - yb) / bb;
          double s = a * sqrt(fmax(0.0, 1.0 - eta * eta));
          if (d == 0) {
            dist = x - (xb + s);
            span = x - gx[i - 1];
          } else {
            dist = (xb - s) - x;
            span = gx[i + 1] - x;
          }
        } else {
          double xi = (x - xb) / a;
          double s = bb * sqrt(fmax(0.0, 1.0 - xi * xi));
          if (d == 2) {
            dist = y - (yb + s);
            span = y - gy[j - 1];
          } else {
            dist = (yb - s) - y;
            span = gy[j + 1] - y;
          }
        }
        if (dist < 0.0) dist = 0.0;
        if (dist > span) dist = span;
        if (dist < best) {
          best = dist;
          bd = d;
        }
      }
      /* opposite node */
      int oi = i, oj = j;
      double D;
      if (bd == 0) { oi = i + 1; }
      else if (bd == 1) { oi = i - 1; }
      else if (bd == 2) { oj = j + 1; }
      else { oj = j - 1; }
      dir[id] = (unsigned char)bd;
      int ok = oi >= ilo && oi <= ihi && oj >= jlo && oj <= jhi;
      if (ok) {
        size_t oid = (size_t)oj * ni + oi;
        if (fl[oid] == FL_SOLID || HASSOLNB(oi, oj)) ok = 0;
      }
      if (!ok) {
        al[id] = 0.0;
        continue;
      }
      D = (bd < 2) ? fabs(gx[oi] - x) : fabs(gy[oj] - y);
      al[id] = best / (best + D);
    }
#undef ISSOL
#undef HASSOLNB
}

static void classify(or_sim* S, double yb) {
  int nx = S->nx, ny = S->ny;
  double a = 0.5 * S->chord, bb = 0.5 * S->tc * S->chord;
  classify_grid(nx + 1, ny, 1, nx - 1, 0, ny - 1, S->xf, S->yc, S->xb, yb, a, bb, S->fu, S->du, S->au);
  classify_grid(nx, ny + 1, 0, nx - 1, 1, ny - 1, S->xc, S->yf, S->xb, yb, a, bb, S->fv, S->dv, S->av);
  /* body cells: cell centre inside the body (carry the mass source q) */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) S->cut[PI_(i, j)] = (unsigned char)inside(S->xc[i], S->yc[j], S->xb, yb, a, bb);
}

/* exported: classify at time t (uses the body set by or_set_body) */
int or_classify(or_sim* S, double t) {
  if (!S->has_body) return OR_E_INVAL;
  classify(S, S->yb0 + S->h * sin(S->k * t));
  return OR_OK;
}

int or_get_flags(const or_sim* S, int grid, unsigned char* flags, unsigned char* dir, double* alpha) {
  size_t n = grid == 0 ? (size_t)(S->nx + 1) * S->ny : (grid == 1 ? (size_t)S->nx * (S->ny + 1) : (size_t)S->nx * S->ny);
  if (grid == 2) {
    memcpy(flags, S->cut, n);
    return OR_OK;
  }
  memcpy(flags, grid == 0 ? S->fu : S->fv, n);
  if (dir) memcpy(dir, grid == 0 ? S->du : S->dv, n);
  if (alpha) memcpy(alpha, grid == 0 ? S->au : S->av, n * 8);
  return OR_OK;
}

/* --------------------------------------------- Helmholtz (Crank-Nicolson) solve */

/* node value and neighbours on grid 0 (u) or 1 (v); a neighbour outside the
 * grid's node range reads as 0 */
static void helm_nb(const or_sim* S, int grid, const double* x, int i, int j, double* xE, double* xW, double* xN,
                    double* xS) {
  int nx = S->nx, ny = S->ny;
  if (grid == 0) {
    *xE = x[UI(i + 1, j)];
    *xW = x[UI(i - 1, j)];
    *xN = j < ny - 1 ? x[UI(i, j + 1)] : 0.0;
    *xS = j > 0 ? x[UI(i, j - 1)] : 0.0;
  } else {
    *xE = i < nx - 1 ? x[VI(i + 1, j)] : 0.0;
    *xW = i > 0 ? x[VI(i - 1, j)] : 0.0;
    *xN = x[VI(i, j + 1)];
    *xS = x[VI(i, j - 1)];
  }
}

/* forcing-node value U_b + alpha (x_opp - U_b) from the current opposite node */
static double forcing_value(const or_sim* S, int grid, const double* x, int i, int j, double Ub) {
  int nx = S->nx;
  size_t id = grid == 0 ? UI(i, j) : VI(i, j);
  double al = grid == 0 ? S->au[id] : S->av[id];
  int d = grid == 0 ? S->du[id] : S->dv[id];
  double xo = Ub;
  if (al != 0.0) {
    int oi = i + (d == 0) - (d == 1), oj = j + (d == 2) - (d == 3);
    xo = x[grid == 0 ? UI(oi, oj) : VI(oi, oj)];
  }
  return MULADD(al, xo - Ub, Ub);
}

/* Row residual of (I - beta L) x = R on fluid rows, of the interpolation
 * condition on forcing rows, and of x = U_b on solid rows. */
static double helm_row_res(const or_sim* S, int grid, const double* x, const double* R, int i, int j,
                           double beta, double Ub) {
  int nx = S->nx;
  size_t id = grid == 0 ? UI(i, j) : VI(i, j);
  unsigned char fl = grid == 0 ? S->fu[id] : S->fv[id];
  if (fl == FL_SOLID) return Ub - x[id];
  if (fl == FL_FORCE) return forcing_value(S, grid, x, i, j, Ub) - x[id];
  double L = grid == 0 ? lap_u_at(S, x, i, j) : lap_v_at(S, x, i, j);
  return R[id] - MULADD(-beta, L, x[id]);
}

static double helm_res_inf(const or_sim* S, int grid, const double* x, const double* R, double beta,
                           double Ub, int* bad) {
  int nx = S->nx, ny = S->ny;
  int i0 = grid == 0 ? 1 : 0, i1 = nx - 1;
  int j0 = grid == 0 ? 0 : 1, j1 = ny - 1;
  double m = 0.0;
  int nan = 0;
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i) {
      double r = helm_row_res(S, grid, x, R, i, j, beta, Ub);
      if (r != r || isinf(r)) nan = 1;
      if (fabs(r) > m) m = fabs(r);
    }
  *bad = nan;
  return m;
}

/* Red-black Gauss-Seidel SOR for one grid's implicit velocity system
 * (Sec. 2.2: "modified" Gauss-Seidel SOR with red-black tagging).  Red =
 * (i+j) even, updated first.  Fluid rows: Gauss-Seidel value
 * (R + beta sum a_nb x_nb) / (1 + beta sum a_nb), over-relaxed by omega;
 * forcing rows are assigned from the current opposite node; solid rows stay
 * at U_b.  The residual is checked before the first sweep and every m. */
static int helm_solve(or_sim* S, int grid, double* x, const double* R, double beta, double Ub,
                      int* sweeps, double* res) {
  int nx = S->nx, ny = S->ny;
  int i0 = grid == 0 ? 1 : 0, i1 = nx - 1;
  int j0 = grid == 0 ? 0 : 1, j1 = ny - 1;
  double om = S->P.omega_h;
  int m = S->P.check_h > 0 ? S->P.check_h : 1;
  const double *cE = grid == 0 ? S->uE : S->vE, *cW = grid == 0 ? S->uW : S->vW;
  const double *cN = grid == 0 ? S->uN : S->vN, *cS = grid == 0 ? S->uS : S->vS;
  const double* inv = grid == 0 ? S->iud : S->ivd;
  int s = 0;
  for (;;) {
    if (s % m == 0) {
      int bad;
      double r = helm_res_inf(S, grid, x, R, beta, Ub, &bad);
      *res = r;
      *sweeps = s;
      if (bad) return OR_E_DIVERGED;
      if (r <= S->P.htol) return OR_OK;
    }
    if (s >= S->P.max_sweeps) return OR_E_NOCONV;
    for (int col = 0; col < 2; ++col) {
      for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) {
          if (((i + j) & 1) != col) continue;
          size_t id = grid == 0 ? UI(i, j) : VI(i, j);
          unsigned char fl = grid == 0 ? S->fu[id] : S->fv[id];
          if (fl == FL_SOLID) continue;
          if (fl == FL_FORCE) {
            x[id] = forcing_value(S, grid, x, i, j, Ub);
            continue;
          }
          double xE, xW, xN, xS;
          helm_nb(S, grid, x, i, j, &xE, &xW, &xN, &xS);
#ifndef ORACLE_PLAIN
          double sum = cE[i] * xE;
          sum = fma(cW[i], xW, sum);
          sum = fma(cN[j], xN, sum);
          sum = fma(cS[j], xS, sum);
          double gs = fma(beta, sum, R[id]) * inv[id];
          x[id] = fma(om, gs - x[id], x[id]);
#else
          /* (1 + beta sum a_nb) x_P = R + beta sum a_nb x_nb */
          double offsum = 0.0;
          offsum += cE[i] * xE;
          offsum += cW[i] * xW;
          offsum += cN[j] * xN;
          offsum += cS[j] * xS;
          double diag = cE[i] + cW[i] + cN[j] + cS[j];
          double gs = (R[id] + beta * offsum) / (1.0 + beta * diag);
          x[id] = (1.0 - om) * x[id] + om * gs;
          (void)inv;
#endif
        }
    }
    ++s;
  }
}

/* ----------------------------------------------------- pressure Poisson solve */

static double poisson_res_inf(const or_sim* S, const double* phi, const double* b, int* bad) {
  int nx = S->nx, ny = S->ny;
  double m = 0.0;
  int nan = 0;
#pragma omp parallel for reduction(max : m) reduction(| : nan) num_threads(S->threads)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double r = b[PI_(i, j)] - lap_p_at(S, phi, i, j);
      if (r != r || isinf(r)) nan |= 1;
      if (fabs(r) > m) m = fabs(r);
    }
  *bad = nan;
  return m;
}

/* Red-black SOR for L_p phi = b (Sec. 2.2, Sec. 3.1).  The Neumann problem
 * is singular; its right-hand side is compatible (zero net source), so SOR
 * is run on the singular system itself (pinning one cell would leave it
 * nearly singular and SOR would crawl).  On convergence the gauge is fixed by
 * shifting phi so that the cell (nx-1, 0) is zero; a constant shift leaves
 * L_p phi and the velocity correction unchanged.  The residual infinity norm
 * is checked before the first sweep and every m full sweeps; the solve stops
 * when it is at most max(tol, rtol * ||b||_inf).  Update of a cell:
 * GS = (sum_nb a_nb phi_nb - b) / sum_nb a_nb, phi <- phi + omega (GS - phi). */
int or_poisson(or_sim* S, const double* b, double* phi, double omega, double tol, double rtol, int m,
               int maxs, int* sweeps, double* res) {
  int nx = S->nx, ny = S->ny;
  if (m < 1) m = 1;
  int s = 0;
  const size_t ref = PI_(nx - 1, 0);
  double bmax = 0.0;
  for (size_t id = 0; id < (size_t)nx * ny; ++id)
    if (fabs(b[id]) > bmax) bmax = fabs(b[id]);
  double thr = rtol * bmax > tol ? rtol * bmax : tol;
  for (;;) {
    if (s % m == 0) {
      int bad;
      double r = poisson_res_inf(S, phi, b, &bad);
      *res = r;
      *sweeps = s;
      if (bad) return OR_E_DIVERGED;
      if (r <= thr) {
        double c = phi[ref];
        for (size_t id = 0; id < (size_t)nx * ny; ++id) phi[id] -= c;
        return OR_OK;
      }
    }
    if (s >= maxs) return OR_E_NOCONV;
    for (int col = 0; col < 2; ++col) {
#pragma omp parallel for num_threads(S->threads)
      for (int j = 0; j < ny; ++j)
        for (int i = (j + col) & 1; i < nx; i += 2) {
          size_t id = PI_(i, j);
          double xE = i < nx - 1 ? phi[PI_(i + 1, j)] : 0.0;
          double xW = i > 0 ? phi[PI_(i - 1, j)] : 0.0;
          double xN = j < ny - 1 ? phi[PI_(i, j + 1)] : 0.0;
          double xS = j > 0 ? phi[PI_(i, j - 1)] : 0.0;
#ifndef ORACLE_PLAIN
          double sum = S->pE[i] * xE;
          sum = fma(S->pW[i], xW, sum);
          sum = fma(S->pN[j], xN, sum);
          sum = fma(S->pS[j], xS, sum);
          double gs = (sum - b[id]) * S->ipd[id];
          phi[id] = fma(omega, gs - phi[id], phi[id]);
#else
          double sum = 0.0;
          sum += S->pE[i] * xE;
          sum += S->pW[i] * xW;
          sum += S->pN[j] * xN;
          sum += S->pS[j] * xS;
          double gs = (sum - b[id]) / (S->pE[i] + S->pW[i] + S->pN[j] + S->pS[j]);
          phi[id] = (1.0 - omega) * phi[id] + omega * gs;
#endif
        }
    }
    ++s;
  }
}

/* ------------------------------------------------------------------ body */

int or_set_body(or_sim* S, double chord, double tc, double h, double k, double xc, double yc) {
  if (!(chord > 0.0) || !(tc > 0.0)) return OR_E_INVAL;
  S->has_body = 1;
  S->chord = chord;
  S->tc = tc;
  S->h = h;
  S->k = k;
  S->xb = xc;
  S->yb0 = yc;
  /* momentum of the fluid carried inside the body at t = 0 (internal-mass
   * term of the force, Sec. 4.1 histories) */
  classify(S, yc);
  int nx = S->nx, ny = S->ny;
  double vb = k * h;
  double sy = 0.0;
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (S->fv[VI(i, j)] == FL_SOLID) sy += vb * (S->dx[i] * S->dyc[j]);
  S->S_prev[0] = 0.0;
  S->S_prev[1] = sy;
  return OR_OK;
}

/* ------------------------------------------------------------------ step */

static int one_step(or_sim* S) {
  int nx = S->nx, ny = S->ny;
  const or_params* P = &S->P;
  double dt = P->dt, beta = dt / (2.0 * P->Re), idt = 1.0 / dt;
  double t1 = (S->n + 1) * dt;
  double yb = S->yb0, vb = 0.0;
  or_stats st;
  memset(&st, 0, sizeof(st));
  /* a1: kinematics at t^{n+1} (Eqs. 1-2) */
  if (S->has_body) {
    yb = S->yb0 + S->h * sin(S->k * t1);
    vb = S->k * S->h * cos(S->k * t1);
    /* a2/a3: classification, forcing nodes and interpolation data */
    classify(S, yb);
  } else {
    memset(S->fu, 0, (size_t)(nx + 1) * ny);
    memset(S->fv, 0, (size_t)nx * (ny + 1));
    memset(S->cut, 0, (size_t)nx * ny);
  }
  /* a4: explicit part.  H^n; AB2 with H^{-1} = H^0 on the first step. */
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i) S->Hu[UI(i, j)] = conv_u_at(S, S->u, S->v, i, j);
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) S->Hv[VI(i, j)] = conv_v_at(S, S->u, S->v, i, j);
  if (S->n == 0) {
    memcpy(S->Huo, S->Hu, sizeof(double) * (nx + 1) * ny);
    memcpy(S->Hvo, S->Hv, sizeof(double) * nx * (ny + 1));
  }
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i) {
      size_t id = UI(i, j);
      double gp = OVER(S->p[PI_(i, j)] - S->p[PI_(i - 1, j)], S->dxc[i], S->idxc[i]);
      S->Ru[id] = S->u[id] + dt * (-1.5 * S->Hu[id] + 0.5 * S->Huo[id] - gp) + beta * lap_u_at(S, S->u, i, j);
    }
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t id = VI(i, j);
      double gp = OVER(S->p[PI_(i, j)] - S->p[PI_(i, j - 1)], S->dyc[j], S->idyc[j]);
      S->Rv[id] = S->v[id] + dt * (-1.5 * S->Hv[id] + 0.5 * S->Hvo[id] - gp) + beta * lap_v_at(S, S->v, i, j);
    }
  /* boundary values of the intermediate velocity at t^{n+1} */
  memcpy(S->uh, S->u, sizeof(double) * (nx + 1) * ny);
  memcpy(S->vh, S->v, sizeof(double) * nx * (ny + 1));
  for (int i = 0; i < nx; ++i) {
    S->vh[VI(i, 0)] = 0.0;
    S->vh[VI(i, ny)] = 0.0;
  }
  if (P->bc == 0) {
    /* inflow u = u_in; convective outflow du/dt + U du/dx = 0 (U = u_in,
     * explicit Euler), then a uniform shift so that outflow flux = inflow flux */
    double qin = 0.0, qout = 0.0, ly = 0.0;
    for (int j = 0; j < ny; ++j) {
      S->uh[UI(0, j)] = P->u_in;
      double ub = S->u[UI(nx, j)];
      S->uh[UI(nx, j)] = ub - OVER(dt * P->u_in * (ub - S->u[UI(nx - 1, j)]), S->dx[nx - 1], S->idx[nx - 1]);
    }
#ifndef ORACLE_PLAIN
    /* fluxes: in row order within chunks of 32 rows, then the chunk sums in order */
    for (int j0 = 0; j0 < ny; j0 += 32) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int j = j0; j < j0 + 32 && j < ny; ++j) {
        a += S->uh[UI(0, j)] * S->dy[j];
        b += S->uh[UI(nx, j)] * S->dy[j];
        c += S->dy[j];
      }
      qin += a;
      qout += b;
      ly += c;
    }
#else
    for (int j = 0; j < ny; ++j) {
      qin += S->uh[UI(0, j)] * S->dy[j];
      qout += S->uh[UI(nx, j)] * S->dy[j];
      ly += S->dy[j];
    }
#endif
    double corr = (qin - qout) / ly;
    for (int j = 0; j < ny; ++j) S->uh[UI(nx, j)] += corr;
  } else {
    for (int j = 0; j < ny; ++j) {
      S->uh[UI(0, j)] = 0.0;
      S->uh[UI(nx, j)] = 0.0;
    }
  }
  /* initial guess: u^n, body velocity on solid nodes */
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i)
      if (S->fu[UI(i, j)] == FL_SOLID) S->uh[UI(i, j)] = 0.0;
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (S->fv[VI(i, j)] == FL_SOLID) S->vh[VI(i, j)] = vb;
  /* a5: implicit velocity solves */
  int rc = helm_solve(S, 0, S->uh, S->Ru, beta, 0.0, &st.sweeps_u, &st.res_u);
  if (!rc) rc = helm_solve(S, 1, S->vh, S->Rv, beta, vb, &st.sweeps_v, &st.res_v);
  if (rc) {
    S->last = st;
    return rc;
  }
  /* a6: divergence of the intermediate velocity and the mass source (Eq. 4).
   * Inside the body the continuity equation is replaced by div u = q: q is
   * the divergence of the forced velocity on every cell whose centre lies in
   * the body, less the mean c over those cells, so that the net source is
   * zero (a rigid body neither creates nor removes fluid) and the Neumann
   * problem stays compatible.  Cells whose centre is in the fluid keep q = 0,
   * so the faces a moving body pushes through still drive the pressure.
   * b = (D(uhat) - q)/dt. */
  or_div(S, S->uh, S->vh, S->D);
  double sdv = 0.0, sv = 0.0;
#ifndef ORACLE_PLAIN
  /* sums over body cells: along each row in order, then the row sums in order */
  for (int j = 0; j < ny; ++j) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nx; ++i)
      if (S->cut[PI_(i, j)]) {
        double V = S->dx[i] * S->dy[j];
        a += S->D[PI_(i, j)] * V;
        b += V;
      }
    sdv += a;
    sv += b;
  }
#else
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (S->cut[PI_(i, j)]) {
        double V = S->dx[i] * S->dy[j];
        sdv += S->D[PI_(i, j)] * V;
        sv += V;
      }
#endif
  double cbar = sv > 0.0 ? sdv / sv : 0.0;
  double sq = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t id = PI_(i, j);
      S->q[id] = S->cut[id] ? S->D[id] - cbar : 0.0;
      S->b[id] = (S->D[id] - S->q[id]) * idt;
      if (S->cut[id]) sq += S->q[id] * (S->dx[i] * S->dy[j]);
    }
  st.sum_q = sq;
  /* a7/a8: Poisson solve warm-started from the previous increment */
  rc = or_poisson(S, S->b, S->phi, P->omega_p, P->ptol, P->prtol, P->check_p, P->max_sweeps, &st.sweeps_p, &st.res_p);
  if (rc) {
    S->last = st;
    return rc;
  }
  /* a10: forces.  f = ((I - beta L) uhat - R)/dt on solid and forcing nodes;
   * F = -sum f dV + d/dt sum_{solid} uhat dV ; C = 2F/chord. */
  if (S->has_body) {
    double fx = 0.0, fy = 0.0, sx = 0.0, sy = 0.0;
    for (int j = 0; j < ny; ++j)
      for (int i = 1; i < nx; ++i) {
        size_t id = UI(i, j);
        if (S->fu[id] == FL_FLUID) continue;
        double dV = S->dxc[i] * S->dy[j];
        double f = ((S->uh[id] - beta * lap_u_at(S, S->uh, i, j)) - S->Ru[id]) * idt;
        fx += f * dV;
        if (S->fu[id] == FL_SOLID) sx += S->uh[id] * dV;
      }
    for (int j = 1; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t id = VI(i, j);
        if (S->fv[id] == FL_FLUID) continue;
        double dV = S->dx[i] * S->dyc[j];
        double f = ((S->vh[id] - beta * lap_v_at(S, S->vh, i, j)) - S->Rv[id]) * idt;
        fy += f * dV;
        if (S->fv[id] == FL_SOLID) sy += S->vh[id] * dV;
      }
    double Fx = -fx + (sx - S->S_prev[0]) * idt;
    double Fy = -fy + (sy - S->S_prev[1]) * idt;
    S->S_prev[0] = sx;
    S->S_prev[1] = sy;
    st.cd = 2.0 * Fx / S->chord;
    st.cl = 2.0 * Fy / S->chord;
  }
  /* a9: projection u = uhat - dt G phi on interior faces, p += phi */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      size_t id = UI(i, j);
      if (i == 0 || i == nx)
        S->u[id] = S->uh[id];
      else
        S->u[id] = S->uh[id] - dt * OVER(S->phi[PI_(i, j)] - S->phi[PI_(i - 1, j)], S->dxc[i], S->idxc[i]);
    }
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t id = VI(i, j);
      if (j == 0 || j == ny)
        S->v[id] = S->vh[id];
      else
        S->v[id] = S->vh[id] - dt * OVER(S->phi[PI_(i, j)] - S->phi[PI_(i, j - 1)], S->dyc[j], S->idyc[j]);
    }
  for (size_t id = 0; id < (size_t)nx * ny; ++id) S->p[id] += S->phi[id];
  /* H^n becomes H^{n-1} */
  memcpy(S->Huo, S->Hu, sizeof(double) * (nx + 1) * ny);
  memcpy(S->Hvo, S->Hv, sizeof(double) * nx * (ny + 1));
  /* a11: divergence over uncut cells */
  double dm = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (S->cut[PI_(i, j)]) continue;
      double d = OVER(S->u[UI(i + 1, j)] - S->u[UI(i, j)], S->dx[i], S->idx[i]) +
                 OVER(S->v[VI(i, j + 1)] - S->v[VI(i, j)], S->dy[j], S->idy[j]);
      if (fabs(d) > dm) dm = fabs(d);
    }
  st.div_max = dm;
  S->n += 1;
  st.n = S->n;
  st.t = S->n * dt;
  S->last = st;
  /* history */
  if (S->n > S->cap) {
    int nc = S->cap ? 2 * S->cap : 256;
    S->cl = realloc(S->cl, sizeof(double) * nc);
    S->cd = realloc(S->cd, sizeof(double) * nc);
    S->cap = nc;
  }
  S->cl[S->n - 1] = st.cl;
  S->cd[S->n - 1] = st.cd;
  return OR_OK;
}

int or_step(or_sim* S, int nsteps, or_stats* last) {
  for (int s = 0; s < nsteps; ++s) {
    int rc = one_step(S);
    if (rc) {
      if (last) *last = S->last;
      return rc;
    }
  }
  if (last) *last = S->last;
  return OR_OK;
}

int or_forces(const or_sim* S, double* cl, double* cd, int cap, int* n_out) {
  int n = S->n < cap ? S->n : cap;
  if (cl) memcpy(cl, S->cl, sizeof(double) * n);
  if (cd) memcpy(cd, S->cd, sizeof(double) * n);
  *n_out = S->n;
  return OR_OK;
}

/* field access.  which: 0 u, 1 v, 2 p, 3 phi, 4 b, 5 uhat, 6 vhat, 7 Ru, 8 Rv,
 * 9 Hu, 10 Hv, 11 q, 12 D(uhat) */
static double* field_ptr(const or_sim* S, int which, size_t* n) {
  size_t nu = (size_t)(S->nx + 1) * S->ny, nv = (size_t)S->nx * (S->ny + 1), np = (size_t)S->nx * S->ny;
  switch (which) {
    case 0: *n = nu; return S->u;
    case 1: *n = nv; return S->v;
    case 2: *n = np; return S->p;
    case 3: *n = np; return S->phi;
    case 4: *n = np; return S->b;
    case 5: *n = nu; return S->uh;
    case 6: *n = nv; return S->vh;
    case 7: *n = nu; return S->Ru;
    case 8: *n = nv; return S->Rv;
    case 9: *n = nu; return S->Hu;
    case 10: *n = nv; return S->Hv;
    case 11: *n = np; return S->q;
    case 12: *n = np; return S->D;
    default: *n = 0; return NULL;
  }
}

int or_get(const or_sim* S, int which, double* out) {
  size_t n;
  double* p = field_ptr(S, which, &n);
  if (!p) return OR_E_INVAL;
  memcpy(out, p, n * sizeof(double));
  return OR_OK;
}

/* set u (0), v (1), p (2) or phi (3); the step counter is left alone */
int or_set(or_sim* S, int which, const double* in) {
  if (which < 0 || which > 3) return OR_E_INVAL;
  size_t n;
  double* p = field_ptr(S, which, &n);
  memcpy(p, in, n * sizeof(double));
  return OR_OK;
}

int or_get_stats(const or_sim* S, or_stats* st) {
  *st = S->last;
  return OR_OK;
}

/* exported: one implicit velocity solve on grid 0 (u) or 1 (v) with the
 * current classification; x holds the initial guess and boundary values */
int or_helm_solve(or_sim* S, int grid, double* x, const double* R, double beta, double Ub, int* sweeps,
                  double* res) {
  return helm_solve(S, grid, x, R, beta, Ub, sweeps, res);
}

/* exported: clear the classification (no body anywhere) */
void or_clear_flags(or_sim* S) {
  memset(S->fu, 0, (size_t)(S->nx + 1) * S->ny);
  memset(S->fv, 0, (size_t)S->nx * (S->ny + 1));
  memset(S->cut, 0, (size_t)S->nx * S->ny);
}
