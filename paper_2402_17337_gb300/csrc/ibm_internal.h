// Internal declarations shared by the CUDA translation units of libibm.
// Not part of the public C ABI (include/ibm.h).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

namespace ibm {

// Named NVTX range over a scope (host side: it spans the enqueueing of the
// phase's kernels and any host waits inside it; a profiler attached to the
// process shows the phases of a step, nothing is recorded otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Every staggered field (u, v, p-type) uses one storage geometry: rows
// j = -1 .. ny+1 and columns i = -XOFF .. pitch-XOFF-1, element (i, j) at
// (j + 1) * pitch + i + XOFF.  Ghost entries stay zero; boundary conditions
// live in the 1-D coefficient and weight arrays, so stencils never branch.
constexpr int XOFF = 4;

__host__ __device__ inline size_t at(int i, int j, int pitch) {
  return (size_t)(j + 1) * pitch + (size_t)(i + XOFF);
}

// node kinds in the band flag arrays (bits 0-1); bits 2-3 hold the direction
// of the solid neighbour chosen for a forcing node (0 -x, 1 +x, 2 -y, 3 +y)
enum : uint8_t { K_FLUID = 0, K_SOLID = 1, K_FORCE = 2 };

// Device pointers to the 1-D grid data (all FP64).
struct Geo {
  int nx, ny, pitch, bc;
  const double *xf, *yf, *xc, *yc;     // coordinates (nx+1, ny+1, nx, ny)
  const double *dx, *dy, *idx, *idy;   // cell widths and inverses
  const double *dxc, *dyc;             // centre spacings, index 1..n-1 (n+1 entries)
  const double *idxc, *idyc;           // their inverses (0 where undefined)
  const double *wx, *wy;               // face interpolation weights (n+1 entries)
  // Laplacian coefficients, sum_nb a_nb (x_nb - x_P); zero through walls
  const double *pE, *pW, *pN, *pS;     // pressure grid (nx, nx, ny, ny)
  const double *uE, *uW, *uN, *uS;     // u grid (nx+1, nx+1, ny, ny)
  const double *vE, *vW, *vN, *vS;     // v grid (nx, nx, ny+1, ny+1)
};

// FP32 data of the mixed-precision inner sweeps.  The correction e, its
// right-hand side r and the reciprocal diagonal are stored split by colour:
// cell (i, j) of colour c = (i + j) & 1 lives at [(c ny + j) pk + (i >> 1)],
// so the cells of one colour in a row are contiguous and the neighbours of
// a cell of the other colour are contiguous too.
struct Geo32 {
  int nx, ny, pk;
  const float *cE0, *cE1, *cW0, *cW1;  // pE, pW at i = 2k + s for s = 0, 1 (pk entries)
  const float *pN, *pS;                // ny entries
};

__host__ __device__ inline size_t rb_at(int i, int j, int ny, int pk) {
  return (size_t)(((i + j) & 1) * ny + j) * pk + (size_t)(i >> 1);
}

// Index rectangle that contains every node the body can touch over its
// whole plunge, with a margin; used for all three grids.
struct Band {
  int i0, j0, w, h;
};

// Small device-side scalars of one context (the context's scratch).
struct DevScalars {
  unsigned long long res_bits;   // infinity norm accumulator (bit pattern of |r|)
  unsigned long long div_bits;   // max |div u| over fluid cells
  unsigned long long bmax_bits;  // ||b||_inf
  double body_sum[2];            // sum D V, sum V over body cells
  double cbar;                   // mean divergence over body cells
  double phi_ref;                // phi at the gauge cell
  double S_prev[2];              // momentum inside the body at the previous step
  double force[2];               // Fx, Fy of the last step
  double sum_q;
  unsigned long long res2_bits;  // a second infinity norm accumulator (two residuals in one pass)
};

constexpr int RED_BLOCKS = 64;   // fixed partial-reduction width (deterministic sums)

// ---------------------------------------------------------------- launchers
// (all asynchronous on the given stream)

void launch_outflow_bc(cudaStream_t s, const Geo& g, const double* u, double* uh, double* vh,
                       double u_in, double dt);
void launch_classify(cudaStream_t s, const Geo& g, const Band& band, double xb, double yb, double a,
                     double b, uint8_t* fu, uint8_t* fv, uint8_t* fc, double* au, double* av);
void launch_predict(cudaStream_t s, const Geo& g, const double* u, const double* v, const double* p,
                    double* Hu, double* Hv, const double* Huo, const double* Hvo, double* Ru, double* Rv,
                    double* uh, double* vh, const Band& band, const uint8_t* fu, const uint8_t* fv,
                    double dt, double beta, double vb, int first);
void launch_rhs(cudaStream_t s, const Geo& g, const double* uh, const double* vh, double* b, double dt);
void launch_body_source(cudaStream_t s, const Geo& g, const Band& band, const uint8_t* fc, const double* uh,
                        const double* vh, double* b, double* qband, double dt, double* rowsum,
                        DevScalars* sc);  // rowsum: 2 * band.h doubles
void launch_forces(cudaStream_t s, const Geo& g, const Band& band, const uint8_t* fu, const uint8_t* fv,
                   const double* uh, const double* vh, const double* Ru, const double* Rv, double beta,
                   double dt, double chord, double* partials, DevScalars* sc, double* cl_hist,
                   double* cd_hist, int n);
void launch_phi_ref(cudaStream_t s, const Geo& g, const double* phi, DevScalars* sc);
void launch_project(cudaStream_t s, const Geo& g, const double* uh, const double* vh, const double* phi,
                    double* u, double* v, double* p, double* phi_store, const Band& band, const uint8_t* fc,
                    double dt, DevScalars* sc);
void launch_init_body_momentum(cudaStream_t s, const Geo& g, const Band& band, const uint8_t* fv, double vb,
                               double* partials, DevScalars* sc);

// SOR kernels (FP64 plain path)
void launch_poisson_half(cudaStream_t s, const Geo& g, double* phi, const double* b, const double* invd,
                         int colour, double omega);
void launch_poisson_res(cudaStream_t s, const Geo& g, const double* phi, const double* b,
                        unsigned long long* res_bits);
// ||b - L_p phi_a||_inf and ||b - L_p phi_b||_inf in one pass, each summed as
// by launch_poisson_res
void launch_poisson_res2(cudaStream_t s, const Geo& g, const double* phi_a, const double* phi_b, const double* b,
                         unsigned long long* bits_a, unsigned long long* bits_b);
void launch_shift(cudaStream_t s, const Geo& g, double* phi, const DevScalars* sc);
void launch_bmax(cudaStream_t s, const Geo& g, const double* b, unsigned long long* bits);
void launch_fill_hash(cudaStream_t s, const Geo& g, double* x);
void launch_helm_half(cudaStream_t s, const Geo& g, int grid, double* x, const double* R, const double* invd,
                      const Band& band, const uint8_t* fl, const double* al, int colour, double omega,
                      double beta, double Ub);
// velocity systems in FP32 sweeps inside FP64 defect correction (k_sor.cu)
struct HelmF32 {
  const float *uE, *uW, *uN, *uS, *vE, *vW, *vN, *vS;  // FP32 copies of Geo's velocity coefficients
};
void launch_helm_dc_res(cudaStream_t s, const Geo& g, int grid, const double* x, const double* R, const Band& band,
                        const uint8_t* fl, const double* al, double beta, double Ub, float* r32,
                        unsigned long long* res_bits);
void launch_helm32_half(cudaStream_t s, const Geo& g, const HelmF32& h32, int grid, float* d, const float* r,
                        const float* invd, const Band& band, const uint8_t* fl, const double* al, int colour,
                        float omega, float beta);
void launch_helm_add(cudaStream_t s, const Geo& g, int grid, double* x, const float* d);
void launch_helm_res(cudaStream_t s, const Geo& g, int grid, const double* x, const double* R,
                     const Band& band, const uint8_t* fl, const double* al, double beta, double Ub,
                     unsigned long long* res_bits);

// ---- whole-step batching: one launch covers the blocks of every case
// All that the step kernels of one case read or write in one step (device
// pointers and this step's scalars); a batch keeps a table of them on the
// device.  blocks[k] lists, per kernel kind k, the first block of each case
// in a launch of that kind (cases in table order).
struct StepCase {
  Geo g;
  Band band;
  HelmF32 h32;
  double *u, *v, *p, *Hu, *Hv, *Huo, *Hvo, *Ru, *Rv, *uh, *vh, *b, *phi, *phi_store;
  double *au, *av, *qband, *rowsum, *partials, *cl_hist, *cd_hist;
  uint8_t *fu, *fv, *fc;
  float *hd32, *hr32;
  const float *hinv_u, *hinv_v;
  DevScalars* sc;
  double dt, beta, vb, yb, xb, ea, eb, u_in, chord;
  float omega_h;
  int first_step, n, has_body, nelem;
};
// kinds of batched launches with case-dependent block counts
enum BatchKind { BK_BAND = 0, BK_PREDICT_U, BK_PREDICT_V, BK_CELLS, BK_NUM };
// blocks of one case in a launch of kind k (32 x 8 threads per block)
int batch_blocks(const StepCase& c, int kind);
// host copies of the scalars a step reads back, gathered per case
struct StepReadback {
  DevScalars sc;
  double cl, cd;
};
void launch_classify_batch(cudaStream_t s, const StepCase* cs, const int* first, int n, int total);
void launch_outflow_bc_batch(cudaStream_t s, const StepCase* cs, int n);
void launch_predict_batch(cudaStream_t s, const StepCase* cs, const int* first_u, int total_u, const int* first_v,
                          int total_v, int n);
void launch_rhs_batch(cudaStream_t s, const StepCase* cs, const int* first_cells, int total_cells,
                      const int* first_band, int total_band, int n);
void launch_forces_batch(cudaStream_t s, const StepCase* cs, int n);
void launch_project_batch(cudaStream_t s, const StepCase* cs, const int* first_cells, int total_cells, int n,
                          StepReadback* out);
// velocity systems of the active cases act[0..na): FP64 residual (norm of
// case act[k] into bits[k]), d = 0, FP32 half-sweeps, update x += d
int helm_batch_blocks(const StepCase& c, int grid, int half);
void launch_helm_dc_res_batch(cudaStream_t s, const StepCase* cs, const int* act, const int* first, int na,
                              int total, int grid, unsigned long long* bits);
void launch_helm_zero_batch(cudaStream_t s, const StepCase* cs, const int* act, int na);
void launch_helm32_half_batch(cudaStream_t s, const StepCase* cs, const int* act, const int* first, int na,
                              int total, int grid, int colour);
void launch_helm_add_batch(cudaStream_t s, const StepCase* cs, const int* act, const int* first, int na,
                           int total, int grid);

// batched mixed-precision solve: one launch over the tiles of many cases
struct Sor32Case {
  Geo32 g;
  const float* e_in;
  float* e_out;
  const float* r;
  const float* invd;
  float omega;
  int first, tiles_x;  // first CTA of this case, tiles per row
  int pairs;           // launch pairs of this round for this case (a launch with pair index >= pairs skips it)
};
struct DcCase {
  Geo g;
  int pk, add_e, first;  // first block of this case (blocks of 32 x 8 cells)
  const double* phi_in;
  double* phi_out;
  const float* e;
  const double* b;
  float* r32;
  unsigned long long* res_bits;
};
void sor32_tiles(int cfg, const Geo32& g, int* tiles_x, int* tiles_y);
cudaError_t sor32_batch_prepare(int cfg);
// pdl: launch as a programmatic dependent of the previous kernel on the
// stream (direct launches; the kernel waits for it before its first load)
// q: index of the launch pair within the round (cases with pairs <= q skip it)
void launch_sor32_batch(cudaStream_t s, int cfg, const Sor32Case* cases_dev, int ncases, int total_tiles,
                        int zero_init, int pdl = 0, int q = 0);
void launch_dc_residual_batch(cudaStream_t s, const DcCase* cases_dev, int ncases, int total_blocks);

// geometric multigrid on the FP32 correction equation (k_mg.cu)
struct MgLevel {
  Geo32 g;              // split-colour coefficients of this level (smoothing by the tile kernel)
  const float *pE, *pW;  // the same coefficients by column (nx entries), rows in g.pN, g.pS
  const float *wx, *wy;  // restriction weights of this level's cells into the next coarser level
  const int *ox, *oy;    // prolongation from the next coarser level: neighbour of the parent (-1, 0, +1)
  const float *ax, *ay;  //   and the neighbour's interpolation weight, per column / row
  float* e[2];           // correction (ping-pong of the tile kernel)
  float* r;              // right-hand side
  const float* invd;     // reciprocal diagonal
  int cur;               // buffer holding the current correction
};
int mg_coarse_max();
constexpr int kTailLevels = 8, kTailCells = 5632;  // 44 KB of shared memory: a larger level costs one CTA more than its launches
struct MgTail {             // the small levels, run by one CTA (k_mg_tail)
  MgLevel lv[kTailLevels];  // lv[0] = first tail level, its r from global memory
  int off[kTailLevels];     // offsets of each level's cells in shared memory
  int n;                    // number of tail levels (the last is solved by SOR)
  float omega_c;
  int sweeps_c;
};
cudaError_t prepare_mg_tail();  // dynamic shared memory limit, once, outside graph capture
void launch_mg_tail(cudaStream_t s, const MgTail& T, float* e_top);
size_t fcg_scalars_bytes();  // device scalars of the FCG iteration (zero-initialised)
void launch_mg_restrict(cudaStream_t s, const MgLevel& F, const float* ef, const MgLevel& C);
void launch_mg_prolong(cudaStream_t s, const MgLevel& C, const float* ec, const MgLevel& F, float* ef);
void launch_mg_coarse(cudaStream_t s, const MgLevel& L, float* e_out, float omega, int sweeps);
int sor32_find_shape(int rows_per_tile, int half_sweeps, int form);
void launch_fcg_dot(cudaStream_t s, const MgLevel& L, const float* dxv, const float* dyv, const float* z,
                    const float* q, void* sc);
void launch_fcg_dir(cudaStream_t s, const MgLevel& L, const float* z, float* p, const void* sc, int first);
void launch_fcg_apply(cudaStream_t s, const MgLevel& L, const float* dxv, const float* dyv, const float* p,
                      const float* r, float* q, void* sc);
void launch_fcg_update(cudaStream_t s, const MgLevel& L, const float* p, const float* q, float* x, float* r,
                       const void* sc);

// learned warm start (k_ws.cu): coarse features, prediction, targets; base guess
void launch_extrapolate(cudaStream_t s, const Geo& g, double* phi, double* phi_prev);
void launch_ws_features(cudaStream_t s, const Geo& g, int Hc, int Wc, const double* b, const double* phi,
                        const double* p, const Band& band, const uint8_t* fc, float* feat,
                        unsigned long long* ws_max);
void launch_ws_apply(cudaStream_t s, const Geo& g, int Hc, int Wc, const float* out, double cT,
                     const unsigned long long* ws_max, double* phi);
void launch_ws_target(cudaStream_t s, const Geo& g, int Hc, int Wc, const double* phi_new, const double* phi_old,
                      const DevScalars* sc, double cT, const unsigned long long* ws_max, float* target);
// kernels launched by one ibm_unet_forward
int unet_forward_launches();
// U-Net coarse level of the two-level preconditioner: channel 0 of feat from
// level C's residual (max into *smax), and C's correction from the output
void launch_nnp_features(cudaStream_t s, const MgLevel& C, float* feat, unsigned long long* smax);
void launch_nnp_correction(cudaStream_t s, const MgLevel& C, const float* out, double cT,
                           const unsigned long long* smax, float* e);

// message for ibm_last_error() on the calling thread
void set_last_error(const char* msg);

// mixed precision: FP64 update + residual, FP32 temporally blocked sweeps
int sor32_num_configs();
int sor32_half_sweeps(int cfg);  // half-sweeps per launch of tile shape cfg (even)
void sor32_describe(int cfg, int* rows_per_tile, int* half_sweeps, int* thread_rows, int* form);
void launch_dc_residual(cudaStream_t s, const Geo& g, int pk, const double* phi_in, double* phi_out,
                        const float* e, const double* b, float* r32, int add_e, unsigned long long* res_bits);
// pdl: launch as a programmatic dependent of the previous kernel on the
// stream (consecutive sweep launches outside graph capture).  With
// zero_init = 0 the previous kernel must be a sweep launch of the same run:
// forms 6 and 7 then read r and 1/d before waiting for it.
void launch_sor32(cudaStream_t s, int cfg, const Geo32& g, const float* e_in, float* e_out, const float* r,
                  const float* invd, float omega, int zero_init, int pdl = 0);

}  // namespace ibm
