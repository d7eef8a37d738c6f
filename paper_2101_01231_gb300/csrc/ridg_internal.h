// Internal declarations shared by the RIDG library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/ridg.h"
#include "nl3.h"
#include "tables.h"

namespace ridg {

constexpr int kMaxNB = 12;  // largest supported M + 1 (1D; 2D up to 5, 3D up to 4)

// Per-launch constants of the correction (1D tables and CFL numbers), passed by value.
struct CorrParams {
  double ep[kMaxNB], em[kMaxNB];       // phi_b(+1), phi_b(-1)
  float eph[kMaxNB], epl[kMaxNB];      // phi_b(+1) as a double-float pair
  double D[kMaxNB * kMaxNB];           // int phi_a' phi_b
  double nu[3], nup[3], num[3];        // a_d dt / h_d and its positive / negative parts
  // the same constants as double-float pairs (hi, lo), for the FP32 correction kernels
  float Dh[kMaxNB * kMaxNB], Dl[kMaxNB * kMaxNB];
  float nuh[3], nul[3], nph[3], npl[3], nmh[3], nml[3];
  // nu_d D[a][a-1] as double-float pairs: the one volume-term coefficient of mode a along d
  // for degrees up to 2 (D[a][b] != 0 only for a > b, a + b odd)
  float vdh[3][kMaxNB], vdl[3][kMaxNB];
  // the upwind trace coefficients along d as double-float pairs: nu_d phi_b(+1) for nu_d > 0
  // (the left cell's trace), nu_d phi_b(-1) for nu_d < 0 (the right cell's), 0 for nu_d = 0
  float tch[3][kMaxNB], tcl[3][kMaxNB];
};

struct Grid {
  int dim;
  int n[3];
  long long ncell;
  RegionBox box;  // linear flux: the region cells the prediction reads (tables.h)
};

// ---- FP64 linear path (k_linear.cu) ----
// W[e * wstride + c0 + c] = sum_k P[c][k] X_e[k] for c < nout (rows of P, K = g.box.n theta_S:
// X_e stacks the Q of the box's cells around e, x fastest)
cudaError_t launch_predict_fp64(const Grid& g, int nb, const double* Q, const double* P, int nout,
                                double* W, int wstride, cudaStream_t s);
// Q[e] += correction from the time means Wbar (stride wstride) of e and its face neighbours
// Small 1D meshes: a whole run of nsteps FP64 steps (prediction of the time means with the
// operator's first theta_S rows, then the correction) in one single-CTA launch.
constexpr long long kRun1dMaxCells = 4096;
bool run1d_fits(const Grid& g, int nb);
cudaError_t launch_run1d_fp64(const Grid& g, int nb, double* Q, const double* P, int nsteps,
                              const CorrParams& cp, cudaStream_t s);
cudaError_t launch_correct_linear(const Grid& g, int nb, double* Q, const double* Wbar,
                                  int wstride, const CorrParams& cp, cudaStream_t s);

// ---- mixed BF16 tensor-core prediction (k_mixed.cu) ----
struct MixedOp {
  int nout = 0, npad = 0, K = 0, Kpad = 0, slices = 0, bits = 0, gmax = 0;
  void* b_slices = nullptr;     // device, core-matrix layout bf16 digits of the operator rows
  double* row_scale = nullptr;  // device, 2^(g_c - 16) per row
  float* row_mul = nullptr;     // device, 2^(g_c - gmax) per row
};
// Device-side state of the mixed path: the ghost-padded BF16 digit planes of the current
// state, the TMA descriptor over them, and the exponent / maximum bookkeeping.
struct MixedState {
  void* planes = nullptr;                 // [digit x mode group][y + 2][x + 2][8] bf16
  alignas(64) unsigned char map[128];     // CUtensorMap over the planes (fused step)
  alignas(64) unsigned char map_pred[128];  // the same for the full prediction
  int* exps = nullptr;                    // [0] exponent of the planes, [1] of the outputs,
                                          // [2] 1 if the digits are FP16 (else BF16)
  unsigned long long* maxbits = nullptr;  // [0] max |Q| of the current state, [1] accumulator
  int* status = nullptr;                  // shared status word
  bool valid = false;                     // planes describe the current state
};
bool mixed_supported(int dim, int nb, int nout);
// Digits of the operator rows P (nout x K): K = box.n theta_S columns, the upwind box's
// cells x fastest.
// Digits as BF16 bit patterns, or FP16 if f16 (exact either way).
int mixed_build(int dim, int nb, const std::vector<double>& P, int nout, int slices,
                const RegionBox& box, std::vector<unsigned short>& digits,
                std::vector<double>& rscale, std::vector<float>& rowmul, MixedOp& op, bool f16);
size_t mixed_plane_bytes(const Grid& g, int nb, int slices);
int mixed_make_map(const Grid& g, int nb, int slices, int nout, void* planes, void* map_out);
// Y[e * ys_e + c * ys_c] = (G X_e)[c]: FP64 (fused == false) or, for the fused step
// operator, double-float pairs output-major with the exponent in exps[1]
cudaError_t launch_mixed_gemm(const Grid& g, int nb, const MixedOp& op, MixedState& ms, void* Y,
                              long long ys_e, long long ys_c, bool fused, cudaStream_t s);
// max |Q| and the digit planes of Q (after the state changed outside the mixed step)
cudaError_t launch_mixed_refresh(const Grid& g, int nb, int slices, const double* Q,
                                 MixedState& ms, cudaStream_t s);
// the correction from the fused outputs, plus the new state's planes and maximum
cudaError_t launch_mixed_correct(const Grid& g, int nb, int slices, double* Q, const void* Y,
                                 int gmax, const CorrParams& cp, int sgnx, int sgny,
                                 MixedState& ms, cudaStream_t s);

// ---- mixed BF16 tensor-core prediction in 3D (k_mixed3.cu) ----
bool mixed3_supported(int nb, int slices);
// The fused step operator C P-bar of the 3D step (rows: the volume term, theta_S, then the
// upwind face traces, NB^2 lines per direction): its row count, and whether its digits fit
// the GEMM (two TMEM stages of slices x padded rows <= 256 columns)
int mixed3_fused_nout(int nb);
bool mixed3_fused_fits(int nb, int slices);
size_t mixed3_plane_bytes(const Grid& g, int nb, int slices);
int mixed3_make_map(const Grid& g, int nb, int slices, void* planes, void* map_out);
// Y[c * cells + e] = (G X_e)[c] as double-float pairs from the digit planes in ms (value
// (hi + lo) 2^(exps[1] + gmax - 16)); G = op's rows (P-bar, the fused step operator, or a
// block of P's rows for ridg_predict), at most 64
// (slots: depth of the plane-operand ring, 0 = as many as fit; the autotuner's choice.
// step: the launch is the step's prediction -- it rotates the running maximum and records
// the outputs' exponent in exps[1]; ridg_predict's launches leave both alone, their
// outputs carry the planes' exponent exps[0])
cudaError_t launch_mixed3_gemm(const Grid& g, int nb, const MixedOp& op, MixedState& ms, void* Y,
                               int slots, cudaStream_t s, bool step);
// W[e * wstride + c0 + c] = the double-float outputs Y[c * cells + e] of a prediction launch
// (c < nout), as FP64 with the planes' exponent (through a shared-memory tile)
cudaError_t launch_mixed3_to_w(const Grid& g, int nout, int c0, int wstride, const void* Y,
                               int gmax, const MixedState& ms, double* W, cudaStream_t s);
// ridg_predict's block: W[e * wstride + c0 + c] = (G X_e)[c] in FP64 (c < op.nout), written by
// the GEMM's epilogue (the planes' exponent; the step's bookkeeping left alone)
cudaError_t launch_mixed3_predict(const Grid& g, int nb, const MixedOp& op, MixedState& ms,
                                  double* W, int wstride, int c0, int slots, cudaStream_t s);
// the ring depth a slot cap gives for this configuration (0: it does not fit)
int mixed3_gemm_slots(int nb, int slices, int npad, const RegionBox& box, int cap);
// the correction from those outputs, plus the new state's digit planes and maximum: fused =
// the outputs of the fused step operator (volume term and face traces), else the time means
// (face values from each cell's own and upstream neighbours' time means)
// (block: 64, 128 or 256 threads, the autotuner's choice)
cudaError_t launch_mixed3_correct(const Grid& g, int nb, int slices, double* Q, const void* Y,
                                  int gmax, const CorrParams& cp, MixedState& ms, int block,
                                  bool fused, cudaStream_t s);
// max |Q| and the 3D digit planes of Q
cudaError_t launch_mixed3_refresh(const Grid& g, int nb, int slices, const double* Q,
                                  MixedState& ms, cudaStream_t s);

// ---- nonlinear flux, 2D: Newton prediction (k_newton*.cu) and correction (k_nonlinear.cu) ----
// Device copies of the host-built tables (nl_tables.h), all inside one allocation.
struct NlDev {
  const double *Mt, *em;                // time term, psi_a(-1)
  const double *V1, *V1T, *dV1, *ep1, *em1;  // 1D residual rule (nl_tables.h)
  const double *PsiV, *dPsiV, *wV;      // residual volume rule
  const double *PsiF, *wF;              // residual face rule
  const double *PhiV, *dPhiV, *PhiF;    // spatial basis at the same points (correction)
  const double *PsiAtP, *PsiAtFP, *P1;  // projection rule of eq. Jacproj
  const double* PhiEq;                  // spatial basis on a 6 x 6 equispaced grid (wave speed)
  const int *bptr[2], *bp[2];           // volume triple-product lists per direction
  const double* bval[2];
  const int *gptr[8], *gp[8];           // face lists, index dd * 4 + side_k * 2 + side_l
  const double* gval[8];
  // merged assembly lists (nl_tables.h) with packed entries: {int offset; int pad; double c}
  // for FP64 assembly, {int offset; float c} for FP32 assembly
  const int* dptr;
  const void *dent_d, *dent_f;
  const int* optr[4];
  const void *oent_d[4], *oent_f[4];
  // FP32 copies of the projection tables and the time term (FP32 assembly)
  const float *Mt_f, *PsiAtP_f, *PsiAtFP_f, *P1_f;
  // FP32 1D triple products [a][b][p] (int phi_a phi_b phi_p; with phi_a') and the traces
  // phi_b(+1), phi_b(-1): the factors of the sum-factorised FP32 assembly
  const float *T0_f, *T1_f, *ep1_f, *em1_f;
};
// Block elimination plan for the 3 x 3 region: blocks are eliminated corners first, then the
// edge cells, then the centre; each pivot's later neighbours and the fill they create.
struct NlPlan {
  int order[9];
  int nn[9];
  int nbr[9][3];
  int slot[81];        // storage slot of block (i, j), -1 if it stays zero
  int first[9][3][3];  // 1: this update creates the block (write, do not accumulate)
  int pos[9];          // elimination step of each region cell (order[pos[r]] == r)
  int nslots;
};
NlPlan build_elim_plan();
struct NlDevTables {
  NlDev tb{};
  void* mem = nullptr;
  size_t bytes = 0;
};
// Build the tables for degree nb - 1 and copy them into `mem` (device, `bytes` long; call
// with mem == nullptr first to get the size).
int nl_tables_upload(int nb, NlDevTables& out, void* mem, size_t* bytes, cudaStream_t s);
bool newton_supported(int nb, int m);
// arithmetic of the Newton linear solves: FP64; FP32 on the CUDA cores; TF32 tensor-core
// block updates with FP32 pivot inverses (both mixed forms keep the residual in FP64)
enum NewtonPrec { kNewtonF64 = 0, kNewtonF32 = 1, kNewtonTF32 = 2 };
// CTAs of the persistent Newton kernel and the scratch each needs (bytes)
int newton_grid(int nb, int m, int flux_kind, int prec);
size_t newton_scratch_per_cta(int nb, int m, int prec, const NlPlan& plan);
// One instance of a batched Newton launch (a device-resident table, sorted by cell0): the
// launch's regions run over all its instances, region eg belonging to the last instance
// whose cell0 <= eg.
struct NlInst {
  const double* Q;
  double* W;
  long long cell0;                  // first global region of the instance
  int nx, ny;
  double lam[2];                    // dt / h_d
  int* stats;                       // [0] unconverged, [1] largest iteration count, [2] flags,
                                    // [7..22] regions by iteration count (15 = 15 or more)
  unsigned long long* iters_total;  // iterations summed over the instance's regions
};
struct NewtonArgs {
  NlDev tb;
  NlPlan plan;
  const double* Q;
  double* W;         // centre prediction, cells x m x theta_T
  int nx, ny;
  long long ncell;
  double lam[2];     // dt / h_d
  double gamma;
  int max_iters;
  double tol;
  void* scratch;     // per-CTA block storage
  size_t scratch_per_cta;
  int* counter;      // work counter (zeroed before the launch)
  int* stats;        // [0] unconverged regions, [1] largest iteration count, [2] flags,
                     // [7..22] regions by iteration count (15 = 15 or more)
  unsigned long long* iters_total;  // Newton iterations summed over regions
  const NlInst* inst;  // batched launch: instance table (ncell = total regions), else nullptr
  int ninst;
};
cudaError_t launch_newton(int nb, int m, int flux_kind, int prec, const NewtonArgs& a, int grid,
                          cudaStream_t s);
// The batched Burgers ensemble's Newton prediction in one launch: the degrees' region queues
// a[0 .. count) (nb[g] = degree + 1, 2..5), highest degree first; every CTA works through
// the queues in that order.  CTAs per SM of that launch for the precision.
struct NewtonMulti {
  NewtonArgs a[4];
  int nb[4];
  int count;
};
// (m: the arguments in host memory; dev: their device copy, which the kernel reads)
cudaError_t launch_newton_multi(int prec, const NewtonMulti& m, const NewtonMulti* dev, int grid,
                                cudaStream_t s);
int newton_multi_ctas_per_sm(int prec);
// Every instance's correction of a batched Burgers ensemble in one launch (one block per
// cell of the concatenated instances, sorted by cell0); tb[nb - 2]: the degree's tables.
struct CorrInst {
  double* Q;
  const double* W;
  long long cell0;
  int nx, ny, nb;
  double lamx, lamy;
};
struct CorrMulti {
  NlDev tb[4];
  const CorrInst* inst;
  int ninst;
};
cudaError_t launch_nl_correct_multi(const CorrMulti& m, long long cells, cudaStream_t s);
cudaError_t launch_nl_correct(int nb, int m, int flux_kind, const NlDev& tb, double* Q,
                              const double* W, int nx, int ny, long long ncell, double lamx,
                              double lamy, double gamma, cudaStream_t s);
// largest wave speed of Q over a 6 x 6 equispaced grid of every cell -> *out (as bits)
cudaError_t launch_max_speed(int nb, int m, int flux_kind, const NlDev& tb, const double* Q,
                             long long ncell, double gamma, unsigned long long* out,
                             cudaStream_t s);

// ---- diagnostics (k_diag.cu) ----
// partial sums (per block) of q[e, r, 0], r < m  -> out[block * m + r]
cudaError_t launch_mass_partials(const double* Q, long long ncell, int m, int thS, double* out,
                                 int nblocks, cudaStream_t s);
// partial sums of the numerator / denominator of eq. l2relerror -> out[block * 2 + {0,1}]
cudaError_t launch_l2_partials(const double* Q, const double* X, long long ncell, int m, int dim,
                               int nb, double* out, int nblocks, cudaStream_t s);
// flag[0] |= 1 if any entry of q is not finite
cudaError_t launch_finite_check(const double* q, long long count, int* flag, cudaStream_t s);
// dev[0..count) = host[0..count) read by the SMs from a pinned (device-accessible) host buffer,
// *flag |= 1 if any value is not finite; both pointers 16-byte aligned
cudaError_t launch_ingest(const double* host, double* dev, long long count, int* flag,
                          cudaStream_t s);

}  // namespace ridg

struct ridg_handle {
  // problem
  int dim = 0, n[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, h[3] = {1, 1, 1};
  int M = 0, nb = 1, thS = 1, thT = 1, m = 1, nR = 1, K = 1;  // K = box.n theta_S
  ridg::RegionBox box;  // linear flux: the upwind region cells the prediction reads
  long long ncell = 0;
  ridg_flux flux{};
  double cfl = 0;
  ridg_options opt{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // time
  double dt = 0, t = 0;
  long long steps = 0;
  bool dt_fixed = false, have_pred = false;
  // device buffers
  double* Q = nullptr;      // state, canonical layout
  double* W = nullptr;      // last full prediction (cells * m * theta_T)
  double* Wbar = nullptr;   // time-mean prediction used by the step (cells * m * theta_S)
  double* P = nullptr;      // linear operator, theta_T x K (time-mean rows first)
  double* red = nullptr;    // reduction partials
  int* status = nullptr;    // device status word(s)
  int red_blocks = 256;
  ridg::MixedOp mixed;       // fused step operator [V; u_x; u_y] P-bar (2D)
  ridg::MixedOp mixed_pred;  // full prediction operator P
  ridg::MixedOp mixed3_pred[4];  // 3D: P's theta_T rows in blocks of mixed3_pred_rows
  int mixed3_pred_rows = 0;
  bool mixed3_fused = false;     // 3D: mixed is the fused step operator (else P-bar)
  double* Y = nullptr;       // fused outputs of the mixed step (cells * nout pairs)
  ridg::MixedState ms;       // digit planes and exponent bookkeeping of the mixed path
  int ny_out = 0;
  // host copy of the operator
  std::vector<double> P_host;
  // graphs: key = number of steps
  std::map<int, cudaGraphExec_t> graphs;
  std::map<int, cudaGraph_t> graph_defs;
  // nonlinear flux: tables, elimination plan, per-CTA block storage of the Newton kernel
  ridg::NlDevTables nl;
  ridg::NlPlan plan{};
  ridg::Nl3Dev nl3{};          // 3D nonlinear flux: tables (in nl3_mem)
  void* nl3_mem = nullptr;
  void* nl_scratch = nullptr;
  size_t nl_scratch_cta = 0;
  int nl_grid = 0;        // CTAs of the persistent Newton launch (autotuned)
  int nl_grid_max = 0;    // CTAs the block storage is allocated for
  int tune_gemm3_slots = 0;   // 3D GEMM plane-operand ring depth (0: as many as fit)
  int tune_corr3_block = 128; // 3D correction block size
  bool nl_scratch_shared = false;  // block storage owned by the batch
  int* nl_words = nullptr;  // [0] work counter, [1..3] Newton statistics, [4..5] max speed
                            // bits, [6..7] total Newton iterations, [8..23] iteration histogram
  long long newton_iters_total = 0;
  // Newton statistics of the last prediction
  long long newton_unconverged = 0;
  int newton_iters_max = 0;
  long long newton_hist[16] = {0};
  unsigned long long gen = 0;  // bumped whenever the operator is rebuilt
  std::string err;
  bool batch_owned = false;
};
