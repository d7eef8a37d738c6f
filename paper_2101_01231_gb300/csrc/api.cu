// C ABI of the RIDG library (include/ridg.h): handle lifecycle, state transfer, the
// prediction / correction / step entry points, diagnostics and the batched ensemble.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "nl3.h"
#include "ridg_internal.h"
#include "tune.h"
#include "tables.h"

using ridg::CorrParams;
using ridg::Grid;

namespace {

int set_err(ridg_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define RIDG_CUDA(h, call)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return set_err((h), RIDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void* dev_alloc(ridg_t* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (h->opt.alloc) return h->opt.alloc(bytes, h->opt.alloc_user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}

void dev_free(ridg_t* h, void* p) {
  if (!p) return;
  if (h->opt.free)
    h->opt.free(p, h->opt.alloc_user);
  else
    cudaFree(p);
}

int max_nb(int dim) { return dim == 1 ? 12 : 6; }

Grid grid_of(const ridg_t* h) {
  Grid g;
  g.dim = h->dim;
  g.n[0] = h->n[0];
  g.n[1] = h->n[1];
  g.n[2] = h->n[2];
  g.ncell = h->ncell;
  g.box = h->box;
  return g;
}

bool is_linear(const ridg_t* h) { return h->flux.kind == RIDG_FLUX_ADVECTION; }

// the split-digit tensor-core form of the linear path (BF16 or FP16 digit operands)
bool is_mixed_linear(const ridg_t* h) {
  return h->opt.precision == RIDG_PREC_MIXED_BF16 || h->opt.precision == RIDG_PREC_MIXED_FP16;
}

bool digits_f16(const ridg_t* h) { return h->opt.precision == RIDG_PREC_MIXED_FP16; }

// autotuner keys: the kernel family and the configuration a choice was timed on
std::string key_gemm3(const ridg_t* h) {
  return "gemm3.slots nb" + std::to_string(h->nb) + " S" + std::to_string(h->opt.slices) +
         " box" + std::to_string(h->box.n);
}
std::string key_corr3(const ridg_t* h) {
  return "corr3.block nb" + std::to_string(h->nb) + " S" + std::to_string(h->opt.slices);
}
std::string key_batch(const ridg_t* h) {
  return "batch.schedule flux" + std::to_string(h->flux.kind) + " prec" +
         std::to_string(h->opt.precision);
}
std::string key_newton(const ridg_t* h) {
  return "newton.grid nb" + std::to_string(h->nb) + " m" + std::to_string(h->m) + " flux" +
         std::to_string(h->flux.kind) + " prec" + std::to_string(h->opt.precision);
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

// the Newton grid for a tuned value q (CTAs per 4 SMs), within the allocated block storage
int newton_grid_of(const ridg_t* h, int q) {
  const int g = q * sm_count() / 4;
  return std::max(1, std::min(g, h->nl_grid_max));
}

int newton_prec(const ridg_t* h) {
  return h->opt.precision == RIDG_PREC_MIXED_TF32   ? ridg::kNewtonTF32
         : h->opt.precision == RIDG_PREC_MIXED_FP32 ? ridg::kNewtonF32
                                                    : ridg::kNewtonF64;
}

void drop_graphs(ridg_t* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : h->graph_defs) cudaGraphDestroy(kv.second);
  h->graphs.clear();
  h->graph_defs.clear();
}

CorrParams corr_params(const ridg_t* h) {
  CorrParams cp;
  std::memset(&cp, 0, sizeof(cp));
  ridg::Tables1D t = ridg::tables1d(h->nb);
  for (int b = 0; b < h->nb; ++b) {
    cp.ep[b] = t.ep[b];
    cp.em[b] = t.em[b];
    cp.eph[b] = (float)t.ep[b];
    cp.epl[b] = (float)(t.ep[b] - (double)cp.eph[b]);
    for (int c = 0; c < h->nb; ++c) cp.D[b * ridg::kMaxNB + c] = t.D[b * h->nb + c];
  }
  for (int d = 0; d < 3; ++d) {
    double nu = d < h->dim ? h->flux.vel[d] * h->dt / h->h[d] : 0.0;
    cp.nu[d] = nu;
    cp.nup[d] = nu > 0 ? nu : 0.0;
    cp.num[d] = nu < 0 ? nu : 0.0;
  }
  auto split = [](double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  for (int i = 0; i < ridg::kMaxNB * ridg::kMaxNB; ++i) split(cp.D[i], cp.Dh[i], cp.Dl[i]);
  for (int d = 0; d < 3; ++d) {
    split(cp.nu[d], cp.nuh[d], cp.nul[d]);
    split(cp.nup[d], cp.nph[d], cp.npl[d]);
    split(cp.num[d], cp.nmh[d], cp.nml[d]);
    for (int a = 0; a < ridg::kMaxNB; ++a)
      split(a >= 1 && a < h->nb ? cp.nu[d] * cp.D[a * ridg::kMaxNB + a - 1] : 0.0, cp.vdh[d][a],
            cp.vdl[d][a]);
    for (int b = 0; b < ridg::kMaxNB; ++b)
      split(b < h->nb ? cp.nu[d] * (cp.nu[d] > 0 ? cp.ep[b] : cp.em[b]) : 0.0, cp.tch[d][b],
            cp.tcl[d][b]);
  }
  return cp;
}

// exponent words of the mixed path: [2] = 1 for FP16 digit operands (read by the kernels)
cudaError_t init_exps(ridg_t* h) {
  static const int zero[4] = {0, 0, 0, 0}, one[4] = {0, 0, 1, 0};
  return cudaMemcpyAsync(h->ms.exps, digits_f16(h) ? one : zero, 4 * sizeof(int),
                         cudaMemcpyHostToDevice, h->stream);
}

// (Re)build the linear operator for the current dt and upload it.
int rebuild_linear(ridg_t* h) {
  double nu[3] = {0, 0, 0};
  for (int d = 0; d < h->dim; ++d) nu[d] = h->flux.vel[d] * h->dt / h->h[d];
  if (!ridg::linear_operator(h->dim, h->M, nu, h->box, h->P_host))
    return set_err(h, RIDG_EINVAL, "region system is singular for this dt");
  RIDG_CUDA(h, cudaMemcpyAsync(h->P, h->P_host.data(), sizeof(double) * h->P_host.size(),
                               cudaMemcpyHostToDevice, h->stream));
  if (is_mixed_linear(h) && h->dim == 3) {
    // 3D: the step's operator -- the fused step operator C P-bar where its digits fit (rows:
    // the volume term sum_d nu_d (D along d) W-bar, then the upwind face trace nu_d tr(W-bar)
    // of every line of modes along d), else the time-mean rows P-bar (first theta_S rows of
    // P) --, and for ridg_predict P's theta_T rows in blocks of 64 (32 where slices x 64
    // columns exceed the GEMM's 256), each its own digit operator
    const int nb = h->nb, K = h->K;
    h->mixed3_fused = ridg::mixed3_fused_fits(nb, h->opt.slices);
    h->mixed3_pred_rows = h->opt.slices * 64 <= 256 ? 64 : 32;
    const int nchunks = (h->thT + h->mixed3_pred_rows - 1) / h->mixed3_pred_rows;
    if (nchunks > 4) return set_err(h, RIDG_EINVAL, "3D prediction blocks");
    for (int a = 0; a <= nchunks; ++a) {
      ridg::MixedOp& op = a == 0 ? h->mixed : h->mixed3_pred[a - 1];
      const int r0 = a == 0 ? 0 : (a - 1) * h->mixed3_pred_rows;
      const int nr = a == 0 ? h->thS : std::min(h->mixed3_pred_rows, h->thT - r0);
      std::vector<double> rows(h->P_host.begin() + (size_t)r0 * h->K,
                               h->P_host.begin() + (size_t)(r0 + nr) * h->K);
      int nout = nr;
      if (a == 0 && h->mixed3_fused) {
        nout = ridg::mixed3_fused_nout(nb);
        std::vector<double> G;
        ridg::fused_step_operator(3, nb, nu, rows, K, G);
        rows.swap(G);
      }
      std::vector<unsigned short> digits;
      std::vector<double> rscale;
      std::vector<float> rowmul;
      int rc = ridg::mixed_build(3, h->nb, rows, nout, h->opt.slices, h->box, digits, rscale,
                                 rowmul, op, digits_f16(h));
      if (rc != RIDG_OK) return set_err(h, rc, "3D mixed operator build failed");
      if (!op.b_slices) {
        op.b_slices = dev_alloc(h, digits.size() * sizeof(unsigned short));
        op.row_scale = (double*)dev_alloc(h, rscale.size() * sizeof(double));
        op.row_mul = (float*)dev_alloc(h, rowmul.size() * sizeof(float));
        if (!op.b_slices || !op.row_scale || !op.row_mul)
          return set_err(h, RIDG_ENOMEM, "mixed operator allocation failed");
      }
      RIDG_CUDA(h, cudaMemcpyAsync(op.row_mul, rowmul.data(), rowmul.size() * sizeof(float),
                                   cudaMemcpyHostToDevice, h->stream));
      RIDG_CUDA(h, cudaMemcpyAsync(op.b_slices, digits.data(),
                                   digits.size() * sizeof(unsigned short), cudaMemcpyHostToDevice,
                                   h->stream));
      RIDG_CUDA(h, cudaMemcpyAsync(op.row_scale, rscale.data(), rscale.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, h->stream));
      RIDG_CUDA(h, cudaStreamSynchronize(h->stream));  // host vectors go out of scope
    }
    if (!h->ms.planes) {
      Grid g = grid_of(h);
      // float2 pairs: the step's outputs, or a block of ridg_predict's
      int ny = std::max(h->thS, h->mixed.nout);
      for (int c = 0; c < nchunks; ++c) ny = std::max(ny, h->mixed3_pred[c].nout);
      h->Y = (double*)dev_alloc(h, (size_t)h->ncell * ny * sizeof(double));
      if (!h->Y) return set_err(h, RIDG_ENOMEM, "mixed-path allocation failed");
      const size_t pb = ridg::mixed3_plane_bytes(g, h->nb, h->opt.slices);
      h->ms.planes = dev_alloc(h, pb);
      h->ms.exps = (int*)dev_alloc(h, 4 * sizeof(int));
      h->ms.maxbits = (unsigned long long*)dev_alloc(h, 2 * sizeof(unsigned long long));
      if (!h->ms.planes || !h->ms.exps || !h->ms.maxbits)
        return set_err(h, RIDG_ENOMEM, "mixed-path allocation failed");
      RIDG_CUDA(h, init_exps(h));
      RIDG_CUDA(h, cudaMemsetAsync(h->ms.planes, 0, pb, h->stream));
      if (ridg::mixed3_make_map(g, h->nb, h->opt.slices, h->ms.planes, h->ms.map) != RIDG_OK)
        return set_err(h, RIDG_ECUDA, "tensor map creation failed");
      h->ms.status = h->status;
    }
    h->ms.valid = false;
  } else if (is_mixed_linear(h)) {
    // fused step operator: rows [V; u_x; u_y] = C P-bar with C mapping the time mean W-bar to
    // the volume term sum_d nu_d (D along d) W-bar and the upwind face traces nu_d tr(W-bar)
    const int nout = h->thS + 2 * h->nb;
    std::vector<double> Pbar(h->P_host.begin(), h->P_host.begin() + (size_t)h->thS * h->K);
    std::vector<double> G;
    ridg::fused_step_operator(2, h->nb, nu, Pbar, h->K, G);
    struct Pending { ridg::MixedOp* op; const std::vector<double>* g; int nout; };
    Pending todo[2] = {{&h->mixed, &G, nout}, {&h->mixed_pred, &h->P_host, h->thT}};
    for (auto& p : todo) {
      std::vector<unsigned short> digits;
      std::vector<double> rscale;
      std::vector<float> rowmul;
      int rc = ridg::mixed_build(h->dim, h->nb, *p.g, p.nout, h->opt.slices, h->box, digits,
                                 rscale, rowmul, *p.op, digits_f16(h));
      if (rc != RIDG_OK) return set_err(h, rc, "mixed operator build failed");
      if (!p.op->b_slices) {
        p.op->b_slices = dev_alloc(h, digits.size() * sizeof(unsigned short));
        p.op->row_scale = (double*)dev_alloc(h, rscale.size() * sizeof(double));
        p.op->row_mul = (float*)dev_alloc(h, rowmul.size() * sizeof(float));
        if (!p.op->b_slices || !p.op->row_scale || !p.op->row_mul)
          return set_err(h, RIDG_ENOMEM, "mixed operator allocation failed");
      }
      RIDG_CUDA(h, cudaMemcpyAsync(p.op->row_mul, rowmul.data(), rowmul.size() * sizeof(float),
                                   cudaMemcpyHostToDevice, h->stream));
      RIDG_CUDA(h, cudaMemcpyAsync(p.op->b_slices, digits.data(),
                                   digits.size() * sizeof(unsigned short), cudaMemcpyHostToDevice,
                                   h->stream));
      RIDG_CUDA(h, cudaMemcpyAsync(p.op->row_scale, rscale.data(), rscale.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, h->stream));
      RIDG_CUDA(h, cudaStreamSynchronize(h->stream));  // host vectors go out of scope
    }
    h->ny_out = nout;
    if (!h->Y) {
      Grid g = grid_of(h);
      h->Y = (double*)dev_alloc(h, (size_t)h->ncell * nout * sizeof(double));
      h->ms.planes = dev_alloc(h, ridg::mixed_plane_bytes(g, h->nb, h->opt.slices));
      h->ms.exps = (int*)dev_alloc(h, 4 * sizeof(int));
      h->ms.maxbits = (unsigned long long*)dev_alloc(h, 2 * sizeof(unsigned long long));
      if (!h->Y || !h->ms.planes || !h->ms.exps || !h->ms.maxbits)
        return set_err(h, RIDG_ENOMEM, "mixed-path allocation failed");
      RIDG_CUDA(h, init_exps(h));
      RIDG_CUDA(h, cudaMemsetAsync(h->ms.planes, 0, ridg::mixed_plane_bytes(g, h->nb, h->opt.slices),
                                   h->stream));
      if (ridg::mixed_make_map(g, h->nb, h->opt.slices, nout, h->ms.planes, h->ms.map) != RIDG_OK ||
          ridg::mixed_make_map(g, h->nb, h->opt.slices, h->thT, h->ms.planes, h->ms.map_pred) !=
              RIDG_OK)
        return set_err(h, RIDG_ECUDA, "tensor map creation failed");
      h->ms.status = h->status;
    }
    h->ms.valid = false;
  }
  RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
  drop_graphs(h);
  h->gen += 1;
  return RIDG_OK;
}

int sign_of(double v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }

// Mixed path: make the digit planes describe the current state (outside graph capture).
int ensure_digits(ridg_t* h) {
  if (!is_mixed_linear(h) || h->ms.valid) return RIDG_OK;
  if (h->dim == 3)
    RIDG_CUDA(h, ridg::launch_mixed3_refresh(grid_of(h), h->nb, h->opt.slices, h->Q, h->ms, h->stream));
  else
    RIDG_CUDA(h, ridg::launch_mixed_refresh(grid_of(h), h->nb, h->opt.slices, h->Q, h->ms, h->stream));
  h->ms.valid = true;
  return RIDG_OK;
}

// Newton prediction of every cell's centre W (nonlinear flux).
int enqueue_newton3(ridg_t* h) {
  ridg::Newton3Args a;
  std::memset(&a, 0, sizeof(a));
  a.tb = h->nl3;
  a.Q = h->Q;
  a.W = h->W;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = h->n[d];
    a.lam[d] = h->dt / h->h[d];
  }
  a.ncell = h->ncell;
  a.max_iters = h->opt.newton_max_iters;
  a.tol = h->opt.newton_tol;
  a.scratch = h->nl_scratch;
  a.scratch_per_cta = h->nl_scratch_cta;
  a.counter = h->nl_words;
  a.stats = h->nl_words + 1;
  a.iters_total = (unsigned long long*)(h->nl_words + 6);
  RIDG_CUDA(h, ridg::launch_newton3(h->nb, newton_prec(h) != ridg::kNewtonF64, a, h->nl_grid,
                                    h->stream));
  return RIDG_OK;
}

int enqueue_newton(ridg_t* h) {
  if (h->dim == 3) return enqueue_newton3(h);
  ridg::NewtonArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tb = h->nl.tb;
  a.plan = h->plan;
  a.Q = h->Q;
  a.W = h->W;
  a.nx = h->n[0];
  a.ny = h->n[1];
  a.ncell = h->ncell;
  a.lam[0] = h->dt / h->h[0];
  a.lam[1] = h->dt / h->h[1];
  a.gamma = h->flux.gamma;
  a.max_iters = h->opt.newton_max_iters;
  a.tol = h->opt.newton_tol;
  a.scratch = h->nl_scratch;
  a.scratch_per_cta = h->nl_scratch_cta;
  a.counter = h->nl_words;
  a.stats = h->nl_words + 1;
  a.iters_total = (unsigned long long*)(h->nl_words + 6);
  RIDG_CUDA(h, ridg::launch_newton(h->nb, h->m, h->flux.kind, newton_prec(h), a, h->nl_grid,
                                   h->stream));
  return RIDG_OK;
}

int enqueue_nl_correct(ridg_t* h) {
  if (h->dim == 3) {
    double lam[3];
    for (int d = 0; d < 3; ++d) lam[d] = h->dt / h->h[d];
    RIDG_CUDA(h, ridg::launch_nl3_correct(h->nb, h->nl3, h->Q, h->W, h->n, h->ncell, lam,
                                          h->stream));
    return RIDG_OK;
  }
  RIDG_CUDA(h, ridg::launch_nl_correct(h->nb, h->m, h->flux.kind, h->nl.tb, h->Q, h->W, h->n[0],
                                       h->n[1], h->ncell, h->dt / h->h[0], h->dt / h->h[1],
                                       h->flux.gamma, h->stream));
  return RIDG_OK;
}

// The step's prediction: FP64 time mean into Wbar, or (mixed) the fused outputs into Y; for
// a nonlinear flux the Newton prediction.
int enqueue_predict_mean(ridg_t* h) {
  if (!is_linear(h)) return enqueue_newton(h);
  Grid g = grid_of(h);
  if (is_mixed_linear(h) && h->dim == 3) {
    RIDG_CUDA(h, ridg::launch_mixed3_gemm(g, h->nb, h->mixed, h->ms, h->Y, h->tune_gemm3_slots,
                                          h->stream, true));
  } else if (is_mixed_linear(h)) {
    RIDG_CUDA(h, ridg::launch_mixed_gemm(g, h->nb, h->mixed, h->ms, h->Y, 1, h->ncell, true,
                                         h->stream));
  } else {
    RIDG_CUDA(h, ridg::launch_predict_fp64(g, h->nb, h->Q, h->P, h->thS, h->Wbar, h->thS,
                                           h->stream));
  }
  return RIDG_OK;
}

int enqueue_correct_after_mean(ridg_t* h) {
  if (!is_linear(h)) return enqueue_nl_correct(h);
  CorrParams cp = corr_params(h);
  if (is_mixed_linear(h) && h->dim == 3) {
    // double-float correction from the time means, with the new state's digit planes
    RIDG_CUDA(h, ridg::launch_mixed3_correct(grid_of(h), h->nb, h->opt.slices, h->Q, h->Y,
                                             h->mixed.gmax, cp, h->ms, h->tune_corr3_block,
                                             h->mixed3_fused,
                                             h->stream));
  } else if (is_mixed_linear(h)) {
    RIDG_CUDA(h, ridg::launch_mixed_correct(grid_of(h), h->nb, h->opt.slices, h->Q, h->Y,
                                            h->mixed.gmax, cp, sign_of(h->flux.vel[0]),
                                            sign_of(h->flux.vel[1]), h->ms, h->stream));
  } else {
    RIDG_CUDA(h, ridg::launch_correct_linear(grid_of(h), h->nb, h->Q, h->Wbar, h->thS, cp,
                                             h->stream));
  }
  return RIDG_OK;
}

// Small 1D FP64 meshes run a whole sequence of steps in one launch.
bool use_run1d(const ridg_t* h) {
  return is_linear(h) && h->opt.precision == RIDG_PREC_FP64 && ridg::run1d_fits(grid_of(h), h->nb);
}

int enqueue_run1d(ridg_t* h, int n) {
  const CorrParams cp = corr_params(h);
  RIDG_CUDA(h, ridg::launch_run1d_fp64(grid_of(h), h->nb, h->Q, h->P, n, cp, h->stream));
  return RIDG_OK;
}

int enqueue_step(ridg_t* h) {
  int rc = enqueue_predict_mean(h);
  if (rc) return rc;
  return enqueue_correct_after_mean(h);
}

cudaError_t clear_newton_stats(ridg_t* h) {
  cudaError_t e = cudaMemsetAsync(h->nl_words + 1, 0, 3 * sizeof(int), h->stream);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(h->nl_words + 6, 0, 18 * sizeof(int), h->stream);
}

// Newton statistics since they were last cleared: regions at the iteration cap, largest
// iteration count, flags (1: zero pivot, 2: non-finite update, 4: tensor-core wait timed out).
int read_newton_stats(ridg_t* h) {
  int w[24] = {0};
  RIDG_CUDA(h, cudaMemcpyAsync(w, h->nl_words, sizeof(w), cudaMemcpyDeviceToHost, h->stream));
  RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
  const int unconverged = w[1], iters_max = w[2], flags = w[3];
  unsigned long long total = 0;
  std::memcpy(&total, w + 6, sizeof(total));
  h->newton_unconverged = unconverged;
  h->newton_iters_max = iters_max;
  h->newton_iters_total = (long long)total;
  for (int k = 0; k < 16; ++k) h->newton_hist[k] = w[8 + k];
  if (flags & 4) return set_err(h, RIDG_ETIMEOUT, "a bounded tensor-core wait in the Newton solve gave up");
  if (flags & 2) return set_err(h, RIDG_ENONFINITE, "Newton produced a non-finite update");
  if (flags & 1) return set_err(h, RIDG_ENONFINITE, "zero pivot in a Newton block solve");
  if (unconverged > 0)
    return set_err(h, RIDG_ENOCONV, std::to_string(unconverged) + " regions hit the Newton iteration cap");
  return RIDG_OK;
}

int read_status(ridg_t* h) {
  int st = 0;
  RIDG_CUDA(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
  if (st & 2) return set_err(h, RIDG_ETIMEOUT, "a bounded tensor-core wait gave up");
  if (st & 4)
    return set_err(h, RIDG_ENONFINITE, "state outgrew the mixed-precision digit range in a step");
  if (!is_linear(h)) return read_newton_stats(h);
  return RIDG_OK;
}

int check_handle(const ridg_t* h) { return h ? RIDG_OK : RIDG_EINVAL; }

}  // namespace

extern "C" {

const char* ridg_strerror(int status) {
  switch (status) {
    case RIDG_OK: return "ok";
    case RIDG_EINVAL: return "invalid argument";
    case RIDG_ENOMEM: return "out of memory";
    case RIDG_ECUDA: return "CUDA error";
    case RIDG_ENONFINITE: return "non-finite value in the state";
    case RIDG_ENOCONV: return "Newton iteration cap reached";
    case RIDG_ETIMEOUT: return "bounded device wait timed out";
    case RIDG_ESTATE: return "call out of order";
    case RIDG_ETOOBIG: return "problem larger than the fixed scratch of the no-allocation entry point";
    default: return "unknown status";
  }
}

const char* ridg_last_error(const ridg_t* h) { return h ? h->err.c_str() : "null handle"; }

int ridg_create(const ridg_mesh* mesh, int order, const ridg_flux* flux, double cfl,
                const ridg_options* opt, ridg_t** out) {
  if (!mesh || !flux || !out) return RIDG_EINVAL;
  *out = nullptr;
  if (mesh->dim < 1 || mesh->dim > 3 || order < 0 || order + 1 > max_nb(mesh->dim) || !(cfl > 0))
    return RIDG_EINVAL;
  const int prec = opt ? opt->precision : RIDG_PREC_FP64;
  int m = 1;
  if (flux->kind == RIDG_FLUX_ADVECTION) {
    if (prec != RIDG_PREC_FP64 && prec != RIDG_PREC_MIXED_BF16 && prec != RIDG_PREC_MIXED_FP16)
      return RIDG_EINVAL;
  } else if (flux->kind == RIDG_FLUX_BURGERS || flux->kind == RIDG_FLUX_EULER) {
    m = flux->kind == RIDG_FLUX_EULER ? 4 : 1;
    if (mesh->dim == 3) {
      // 3D: Burgers at degree 1, FP64 or FP32 region solves (dense per-region LU)
      if (flux->kind != RIDG_FLUX_BURGERS || !ridg::newton3_supported(order + 1) ||
          (prec != RIDG_PREC_FP64 && prec != RIDG_PREC_MIXED_FP32))
        return RIDG_EINVAL;
    } else if (mesh->dim != 2 || !ridg::newton_supported(order + 1, m)) {
      return RIDG_EINVAL;
    }
    if (prec != RIDG_PREC_FP64 && prec != RIDG_PREC_MIXED_FP32 && prec != RIDG_PREC_MIXED_TF32)
      return RIDG_EINVAL;
    if (flux->kind == RIDG_FLUX_EULER && !(flux->gamma > 1.0)) return RIDG_EINVAL;
  } else {
    return RIDG_EINVAL;
  }
  ridg_t* h = new ridg_t();
  if (opt) h->opt = *opt;
  if (h->opt.slices <= 0) h->opt.slices = 6;
  if (h->opt.newton_max_iters <= 0) h->opt.newton_max_iters = 4;
  if (!(h->opt.newton_tol > 0)) h->opt.newton_tol = 1e-10;
  h->dim = mesh->dim;
  h->ncell = 1;
  for (int d = 0; d < 3; ++d) {
    h->n[d] = d < mesh->dim ? mesh->n[d] : 1;
    h->lo[d] = d < mesh->dim ? mesh->lo[d] : 0.0;
    h->hi[d] = d < mesh->dim ? mesh->hi[d] : 1.0;
    if (d < mesh->dim && (h->n[d] < 3 || !(h->hi[d] > h->lo[d]))) {
      delete h;
      return RIDG_EINVAL;
    }
    h->h[d] = (h->hi[d] - h->lo[d]) / h->n[d];
    h->ncell *= h->n[d];
  }
  if (h->ncell >= (1LL << 31)) {  // the kernels index cells with 32-bit arithmetic
    delete h;
    return RIDG_EINVAL;
  }
  h->M = order;
  h->nb = order + 1;
  h->thS = 1;
  for (int d = 0; d < h->dim; ++d) h->thS *= h->nb;
  h->thT = h->thS * h->nb;
  h->nR = 1;
  for (int d = 0; d < h->dim; ++d) h->nR *= 3;
  h->m = m;
  h->flux = *flux;
  if (is_linear(h)) h->box = ridg::upwind_box(h->dim, h->flux.vel);
  h->K = h->box.n * h->thS;
  h->cfl = cfl;
  if (is_mixed_linear(h) &&
      (h->dim == 3 ? !ridg::mixed3_supported(h->nb, h->opt.slices)
                   : (!ridg::mixed_supported(h->dim, h->nb, h->thT) || h->opt.slices < 2 ||
                      h->opt.slices > 7))) {
    delete h;
    return RIDG_EINVAL;
  }
  if (is_mixed_linear(h) && h->dim == 3) {
    h->tune_gemm3_slots = ridg::tune_get(key_gemm3(h), 0);
    h->tune_corr3_block = ridg::tune_get(key_corr3(h), 128);
  }
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return RIDG_ECUDA;
  }
  if (h->opt.stream) {
    h->stream = (cudaStream_t)h->opt.stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return RIDG_ECUDA;
    }
    h->own_stream = true;
  }
  // dt from the CFL number (Sec. 5: dt = nu dx / max wave speed)
  double hmin = h->h[0];
  double amax = 0.0;
  for (int d = 0; d < h->dim; ++d) {
    hmin = std::min(hmin, h->h[d]);
    amax = std::max(amax, std::fabs(flux->vel[d]));
  }
  // linear flux: the speed is known now; nonlinear flux: dt is set from the state
  h->dt = is_linear(h) ? cfl * hmin / (amax > 0 ? amax : 1.0) : 0.0;
  const size_t nQ = (size_t)h->ncell * h->m * h->thS;
  h->Q = (double*)dev_alloc(h, nQ * sizeof(double));
  h->W = (double*)dev_alloc(h, (size_t)h->ncell * h->m * h->thT * sizeof(double));
  h->red = (double*)dev_alloc(h, (size_t)h->red_blocks * 4 * sizeof(double));
  h->status = (int*)dev_alloc(h, 16 * sizeof(int));
  if (is_linear(h)) {
    h->Wbar = (double*)dev_alloc(h, nQ * sizeof(double));
    h->P = (double*)dev_alloc(h, (size_t)h->thT * h->K * sizeof(double));
  }
  if (!h->Q || !h->W || !h->red || !h->status || (is_linear(h) && (!h->Wbar || !h->P))) {
    ridg_destroy(h);
    return RIDG_ENOMEM;
  }
  if (!is_linear(h) && h->dim == 3) {
    size_t tb_bytes = 0;
    ridg::nl3_tables_upload(h->nb, h->nl3, nullptr, &tb_bytes, h->stream);
    h->nl3_mem = dev_alloc(h, tb_bytes);
    h->nl_grid = sm_count();  // one persistent CTA per SM (the region Jacobian lives in HBM)
    h->nl_grid_max = 0;       // (nothing for the autotuner here)
    h->nl_scratch_cta = ridg::newton3_scratch_per_cta(h->nb, newton_prec(h) != ridg::kNewtonF64);
    h->nl_scratch = h->nl_grid > 0 ? dev_alloc(h, h->nl_scratch_cta * (size_t)h->nl_grid) : nullptr;
    h->nl_words = (int*)dev_alloc(h, 24 * sizeof(int));
    if (!h->nl3_mem || !h->nl_scratch || !h->nl_words) {
      ridg_destroy(h);
      return RIDG_ENOMEM;
    }
    int rc = ridg::nl3_tables_upload(h->nb, h->nl3, h->nl3_mem, &tb_bytes, h->stream);
    if (rc == RIDG_OK && cudaMemsetAsync(h->nl_words, 0, 24 * sizeof(int), h->stream) != cudaSuccess)
      rc = RIDG_ECUDA;
    if (rc != RIDG_OK) {
      ridg_destroy(h);
      return rc;
    }
  } else if (!is_linear(h)) {
    size_t tb_bytes = 0;
    ridg::nl_tables_upload(h->nb, h->nl, nullptr, &tb_bytes, h->stream);
    void* tb_mem = dev_alloc(h, tb_bytes);
    h->plan = ridg::build_elim_plan();
    h->nl_grid_max = ridg::newton_grid(h->nb, h->m, h->flux.kind, newton_prec(h));
    h->nl_grid = h->nl_grid_max;
    const int q = ridg::tune_get(key_newton(h), 0);
    if (q > 0 && h->nl_grid_max > 0) h->nl_grid = newton_grid_of(h, q);
    h->nl_scratch_cta = ridg::newton_scratch_per_cta(h->nb, h->m, newton_prec(h), h->plan);
    const size_t scratch = h->nl_scratch_cta * (size_t)h->nl_grid_max;
    h->nl_scratch = h->nl_grid_max > 0 ? dev_alloc(h, scratch) : nullptr;
    h->nl_words = (int*)dev_alloc(h, 24 * sizeof(int));
    if (!tb_mem || !h->nl_scratch || !h->nl_words) {
      dev_free(h, tb_mem);
      ridg_destroy(h);
      return RIDG_ENOMEM;
    }
    int rc = ridg::nl_tables_upload(h->nb, h->nl, tb_mem, &tb_bytes, h->stream);
    if (rc != RIDG_OK) {
      dev_free(h, tb_mem);
      ridg_destroy(h);
      return rc;
    }
    // the blocks' zero padding is never written again
    if (cudaMemsetAsync(h->nl_scratch, 0, scratch, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->nl_words, 0, 24 * sizeof(int), h->stream) != cudaSuccess) {
      ridg_destroy(h);
      return RIDG_ECUDA;
    }
  }
  if (cudaMemsetAsync(h->Q, 0, nQ * sizeof(double), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->status, 0, 16 * sizeof(int), h->stream) != cudaSuccess) {
    ridg_destroy(h);
    return RIDG_ECUDA;
  }
  if (is_linear(h)) {
    int rc = rebuild_linear(h);
    if (rc != RIDG_OK) {
      ridg_destroy(h);
      return rc;
    }
  } else if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    ridg_destroy(h);
    return RIDG_ECUDA;
  }
  *out = h;
  return RIDG_OK;
}

void ridg_destroy(ridg_t* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  dev_free(h, h->Q);
  dev_free(h, h->W);
  dev_free(h, h->Wbar);
  dev_free(h, h->P);
  dev_free(h, h->red);
  dev_free(h, h->status);
  dev_free(h, h->mixed.b_slices);
  dev_free(h, h->mixed.row_scale);
  dev_free(h, h->mixed.row_mul);
  dev_free(h, h->mixed_pred.b_slices);
  dev_free(h, h->mixed_pred.row_scale);
  dev_free(h, h->mixed_pred.row_mul);
  for (auto& op : h->mixed3_pred) {
    dev_free(h, op.b_slices);
    dev_free(h, op.row_scale);
    dev_free(h, op.row_mul);
  }
  dev_free(h, h->Y);
  dev_free(h, h->ms.planes);
  dev_free(h, h->ms.exps);
  dev_free(h, h->ms.maxbits);
  dev_free(h, h->nl.mem);
  if (!h->nl_scratch_shared) dev_free(h, h->nl_scratch);
  dev_free(h, h->nl_words);
  dev_free(h, h->nl3_mem);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// A host pointer the device can dereference as it stands: page-locked memory under unified
// addressing (cudaHostAlloc, cudaHostRegister, torch's pin_memory).
static bool pinned_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA pointer: clear the sticky-free error state
    return false;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}
static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

int ridg_set_state(ridg_t* h, const double* q, int on_device) {
  if (check_handle(h) || !q) return RIDG_EINVAL;
  const size_t bytes = (size_t)h->ncell * h->m * h->thS * sizeof(double);
  const long long count = (long long)(bytes / sizeof(double));
  RIDG_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  if (!on_device && pinned_host(q) && aligned16(q) && aligned16(h->Q)) {
    // pinned host memory: the SMs read it over C2C, copy and finite check in one pass
    RIDG_CUDA(h, ridg::launch_ingest(q, h->Q, count, h->status, h->stream));
  } else {
    RIDG_CUDA(h, cudaMemcpyAsync(h->Q, q, bytes,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 h->stream));
    RIDG_CUDA(h, ridg::launch_finite_check(h->Q, count, h->status, h->stream));
  }
  int flag = 0;
  RIDG_CUDA(h, cudaMemcpyAsync(&flag, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
  h->t = 0.0;
  h->steps = 0;
  h->have_pred = false;
  h->ms.valid = false;
  if (flag) return set_err(h, RIDG_ENONFINITE, "state contains NaN or Inf");
  if (!is_linear(h) && !h->dt_fixed) {
    // Sec. 5: dt = cfl h_min / (largest wave speed of the state)
    unsigned long long bits = 0;
    if (h->dim == 3)
      RIDG_CUDA(h, ridg::launch_max_speed3(h->nb, h->Q, h->ncell,
                                           (unsigned long long*)(h->nl_words + 4), h->stream));
    else
    RIDG_CUDA(h, ridg::launch_max_speed(h->nb, h->m, h->flux.kind, h->nl.tb, h->Q, h->ncell,
                                        h->flux.gamma, (unsigned long long*)(h->nl_words + 4),
                                        h->stream));
    RIDG_CUDA(h, cudaMemcpyAsync(&bits, h->nl_words + 4, sizeof(bits), cudaMemcpyDeviceToHost,
                                 h->stream));
    RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
    double smax = 0.0;
    std::memcpy(&smax, &bits, sizeof(smax));
    if (!(smax > 0.0) || !std::isfinite(smax))
      return set_err(h, RIDG_EINVAL, "the state has no positive finite wave speed; set dt");
    double hmin = std::min(h->h[0], h->h[1]);
    if (h->dim == 3) hmin = std::min(hmin, h->h[2]);
    h->dt = h->cfl * hmin / smax;
    drop_graphs(h);
    h->gen += 1;
  }
  return RIDG_OK;
}

int ridg_get_state(ridg_t* h, double* q, int on_device) {
  if (check_handle(h) || !q) return RIDG_EINVAL;
  const size_t bytes = (size_t)h->ncell * h->m * h->thS * sizeof(double);
  RIDG_CUDA(h, cudaMemcpyAsync(q, h->Q, bytes,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               h->stream));
  RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
  return RIDG_OK;
}

int ridg_set_dt(ridg_t* h, double dt) {
  if (check_handle(h) || !(dt > 0) || !std::isfinite(dt)) return RIDG_EINVAL;
  h->dt = dt;
  h->dt_fixed = true;
  if (is_linear(h)) return rebuild_linear(h);
  drop_graphs(h);
  h->gen += 1;
  return RIDG_OK;
}

int ridg_set_final_time(ridg_t* h, double T, long long* nsteps) {
  if (check_handle(h) || !(T > 0) || !(h->dt > 0)) return RIDG_EINVAL;
  long long N = (long long)std::ceil(T / h->dt - 1e-9);
  if (N < 1) N = 1;
  if (nsteps) *nsteps = N;
  return ridg_set_dt(h, T / (double)N);
}

int ridg_predict(ridg_t* h, double* w_out, int on_device) {
  if (check_handle(h)) return RIDG_EINVAL;
  Grid g = grid_of(h);
  if (!is_linear(h)) {
    if (!(h->dt > 0)) return set_err(h, RIDG_ESTATE, "no dt yet: call ridg_set_state first");
    RIDG_CUDA(h, clear_newton_stats(h));
    int rc = enqueue_newton(h);
    if (rc) return rc;
    h->have_pred = true;
    if (w_out) {
      const size_t bytes = (size_t)h->ncell * h->m * h->thT * sizeof(double);
      RIDG_CUDA(h, cudaMemcpyAsync(w_out, h->W, bytes,
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   h->stream));
    }
    return read_newton_stats(h);
  } else if (is_mixed_linear(h) && h->dim == 2) {
    int rc = ensure_digits(h);
    if (rc) return rc;
    RIDG_CUDA(h, ridg::launch_mixed_gemm(g, h->nb, h->mixed_pred, h->ms, h->W, h->thT, 1, false,
                                         h->stream));
  } else if (is_mixed_linear(h) && h->dim == 3) {
    // P's theta_T rows on the tensor cores in blocks (without the step's exponent
    // bookkeeping).  A block of up to 32 rows is written into its columns of W (FP64) by the
    // GEMM's epilogue; a wider one leaves double-float pairs in Y (coalesced) for a tiled
    // conversion: 64 doubles per cell written row-wise by each epilogue thread cost more in
    // partial-sector stores than the round trip (measured at 96^3 Q2, 3 slices: 0.73 ms for
    // the whole prediction this way, 0.97 ms with every block direct; at 6 slices the 32-row
    // blocks direct: 1.19 ms against 1.50 ms with a conversion pass each)
    int rc = ensure_digits(h);
    if (rc) return rc;
    for (int r0 = 0, c = 0; r0 < h->thT; r0 += h->mixed3_pred_rows, ++c) {
      const ridg::MixedOp& op = h->mixed3_pred[c];
      if (op.nout <= 32) {
        RIDG_CUDA(h, ridg::launch_mixed3_predict(g, h->nb, op, h->ms, h->W, h->thT, r0,
                                                 h->tune_gemm3_slots, h->stream));
      } else {
        RIDG_CUDA(h, ridg::launch_mixed3_gemm(g, h->nb, op, h->ms, h->Y, h->tune_gemm3_slots,
                                              h->stream, false));
        RIDG_CUDA(h, ridg::launch_mixed3_to_w(g, op.nout, r0, h->thT, h->Y, op.gmax, h->ms,
                                              h->W, h->stream));
      }
    }
  } else {
    RIDG_CUDA(h, ridg::launch_predict_fp64(g, h->nb, h->Q, h->P, h->thT, h->W, h->thT, h->stream));
  }
  h->have_pred = true;
  if (w_out) {
    const size_t bytes = (size_t)h->ncell * h->m * h->thT * sizeof(double);
    RIDG_CUDA(h, cudaMemcpyAsync(w_out, h->W, bytes,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 h->stream));
    if (!on_device) RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return RIDG_OK;
}

int ridg_correct(ridg_t* h) {
  if (check_handle(h)) return RIDG_EINVAL;
  if (!h->have_pred) return set_err(h, RIDG_ESTATE, "ridg_correct needs a prediction first");
  if (!is_linear(h)) {
    int rc = enqueue_nl_correct(h);
    if (rc) return rc;
  } else {
    CorrParams cp = corr_params(h);
    RIDG_CUDA(h, ridg::launch_correct_linear(grid_of(h), h->nb, h->Q, h->W, h->thT, cp, h->stream));
  }
  h->ms.valid = false;
  h->have_pred = false;
  h->t += h->dt;
  h->steps += 1;
  return RIDG_OK;
}

int ridg_step(ridg_t* h, int n) {
  if (check_handle(h) || n < 1) return RIDG_EINVAL;
  if (!(h->dt > 0)) return set_err(h, RIDG_ESTATE, "no dt yet: call ridg_set_state first");
  int rc0 = ensure_digits(h);
  if (rc0) return rc0;
  if (!is_linear(h))  // Newton statistics of this call's steps (read by ridg_sync)
    RIDG_CUDA(h, clear_newton_stats(h));
  auto it = h->graphs.find(n);
  if (it == h->graphs.end()) {
    cudaGraph_t graph = nullptr;
    RIDG_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = RIDG_OK;
    if (use_run1d(h))
      rc = enqueue_run1d(h, n);
    else
      for (int i = 0; i < n && rc == RIDG_OK; ++i) rc = enqueue_step(h);
    cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    if (rc != RIDG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    RIDG_CUDA(h, ce);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(graph);
      RIDG_CUDA(h, ie);
    }
    h->graphs[n] = exec;
    h->graph_defs[n] = graph;
    it = h->graphs.find(n);
  }
  RIDG_CUDA(h, cudaGraphLaunch(it->second, h->stream));
  h->have_pred = false;
  h->t += n * h->dt;
  h->steps += n;
  return RIDG_OK;
}


int ridg_sync(ridg_t* h) {
  if (check_handle(h)) return RIDG_EINVAL;
  RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
  return read_status(h);
}

int ridg_profile_step(ridg_t* h, int n, ridg_profile_t* out) {
  if (check_handle(h) || n < 1 || !out) return RIDG_EINVAL;
  if (!(h->dt > 0)) return set_err(h, RIDG_ESTATE, "no dt yet: call ridg_set_state first");
  int rc0 = ensure_digits(h);
  if (rc0) return rc0;
  if (!is_linear(h)) RIDG_CUDA(h, clear_newton_stats(h));
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i) RIDG_CUDA(h, cudaEventCreate(&ev[i]));
  double tp = 0, tc = 0;
  int rc = RIDG_OK;
  for (int i = 0; i < n && rc == RIDG_OK; ++i) {
    cudaEventRecord(ev[0], h->stream);
    rc = enqueue_predict_mean(h);
    if (rc) break;
    cudaEventRecord(ev[1], h->stream);
    rc = enqueue_correct_after_mean(h);
    if (rc) break;
    cudaEventRecord(ev[2], h->stream);
    cudaError_t e = cudaEventSynchronize(ev[2]);
    if (e != cudaSuccess) {
      rc = set_err(h, RIDG_ECUDA, cudaGetErrorString(e));
      break;
    }
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    tp += a;
    tc += b;
    h->t += h->dt;
    h->steps += 1;
  }
  for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  if (rc) return rc;
  out->predict_ms = tp / n;
  out->correct_ms = tc / n;
  out->step_ms = (tp + tc) / n;
  out->launches_per_step = 2;
  h->have_pred = false;
  if (!is_linear(h)) return read_newton_stats(h);
  return RIDG_OK;
}

int ridg_autotune(ridg_t* h, const char* cache_path) {
  if (check_handle(h)) return RIDG_EINVAL;
  if (!(h->dt > 0)) return set_err(h, RIDG_ESTATE, "no dt yet: call ridg_set_state first");
  const bool mixed3 = is_linear(h) && is_mixed_linear(h) && h->dim == 3;
  const bool newton = !is_linear(h) && h->nl_grid_max > 0;
  if (mixed3 || newton) {
    // the candidates run real steps from the current state, which is put back afterwards
    const size_t nQ = (size_t)h->ncell * h->m * h->thS;
    double* save = (double*)dev_alloc(h, nQ * sizeof(double));
    if (!save) return set_err(h, RIDG_ENOMEM, "autotune state copy");
    const double t0 = h->t;
    const long long s0 = h->steps;
    int rc = RIDG_OK;
    auto restore = [&]() -> int {
      RIDG_CUDA(h, cudaMemcpyAsync(h->Q, save, nQ * sizeof(double), cudaMemcpyDeviceToDevice,
                                   h->stream));
      RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
      h->t = t0;
      h->steps = s0;
      h->ms.valid = false;
      h->have_pred = false;
      return RIDG_OK;
    };
    // average prediction / correction device time of n steps (after one untimed step)
    auto measure = [&](int n, double* tp, double* tc) -> int {
      int r = restore();
      if (r) return r;
      ridg_profile_t p;
      r = ridg_profile_step(h, 1, &p);
      if (r && r != RIDG_ENOCONV) return r;
      r = ridg_profile_step(h, n, &p);
      if (r && r != RIDG_ENOCONV) return r;
      *tp = p.predict_ms;
      *tc = p.correct_ms;
      return RIDG_OK;
    };
    if (cudaMemcpyAsync(save, h->Q, nQ * sizeof(double), cudaMemcpyDeviceToDevice, h->stream) !=
        cudaSuccess)
      rc = set_err(h, RIDG_ECUDA, "autotune state copy");
    if (!rc && mixed3) {
      // the GEMM's plane-operand ring depth, then the correction's block size; candidates
      // are interleaved over two rounds of 8 steps and each keeps its better round
      std::vector<int> caps;
      int last_na = -1;
      for (int cap : {3, 4, 5, 6, 8}) {
        const int na = ridg::mixed3_gemm_slots(h->nb, h->opt.slices, h->mixed.npad, h->box, cap);
        if (na < 2 || na == last_na) continue;
        last_na = na;
        caps.push_back(cap);
      }
      std::vector<double> tg(caps.size(), 1e300);
      for (int round = 0; round < 2 && !rc; ++round)
        for (size_t i = 0; i < caps.size() && !rc; ++i) {
          h->tune_gemm3_slots = caps[i];
          double tp = 0, tc = 0;
          if (!(rc = measure(8, &tp, &tc))) tg[i] = std::min(tg[i], tp);
        }
      if (!caps.empty())
        h->tune_gemm3_slots = caps[std::min_element(tg.begin(), tg.end()) - tg.begin()];
      const int blocks[3] = {64, 128, 256};
      double tb[3] = {1e300, 1e300, 1e300};
      for (int round = 0; round < 2 && !rc; ++round)
        for (int i = 0; i < 3 && !rc; ++i) {
          h->tune_corr3_block = blocks[i];
          double tp = 0, tc = 0;
          if (!(rc = measure(8, &tp, &tc))) tb[i] = std::min(tb[i], tc);
        }
      h->tune_corr3_block = blocks[std::min_element(tb, tb + 3) - tb];
      if (!rc) {
        ridg::tune_put(key_gemm3(h), h->tune_gemm3_slots);
        ridg::tune_put(key_corr3(h), h->tune_corr3_block);
      }
    }
    if (!rc && newton) {
      // the persistent Newton grid in CTAs per 4 SMs: fewer CTAs keep more of their block
      // storage in L2, more hide the latency of the pivot chains
      const int per4 = std::max(1, h->nl_grid_max * 4 / std::max(1, sm_count()));
      int best_q = per4;
      double best = 1e300;
      for (int q : {1, 2, 4, 8}) {
        if (q > per4) break;
        h->nl_grid = newton_grid_of(h, q);
        double tp = 0, tc = 0;
        if ((rc = measure(1, &tp, &tc))) break;
        if (tp < best) {
          best = tp;
          best_q = q;
        }
      }
      h->nl_grid = newton_grid_of(h, best_q);
      if (!rc) ridg::tune_put(key_newton(h), best_q);
    }
    const int rr = restore();
    dev_free(h, save);
    drop_graphs(h);
    if (rc) return rc;
    if (rr) return rr;
  }
  if (cache_path && !ridg::tune_save(cache_path))
    return set_err(h, RIDG_EINVAL, std::string("cannot write the tuning cache ") + cache_path);
  return RIDG_OK;
}

int ridg_get_tuning(ridg_t* h, int* gemm3_slots, int* corr3_block, int* newton_grid) {
  if (check_handle(h)) return RIDG_EINVAL;
  if (gemm3_slots) *gemm3_slots = h->tune_gemm3_slots;
  if (corr3_block) *corr3_block = h->tune_corr3_block;
  if (newton_grid) *newton_grid = h->nl_grid;
  return RIDG_OK;
}

int ridg_tune_load(const char* cache_path) {
  if (!cache_path) return RIDG_EINVAL;
  return ridg::tune_load(cache_path) ? RIDG_OK : RIDG_EINVAL;
}

int ridg_tune_lookup(const char* key, int* value) {
  if (!key || !value) return RIDG_EINVAL;
  const int missing = -2147483647;
  const int v = ridg::tune_get(key, missing);
  if (v == missing) return RIDG_EINVAL;
  *value = v;
  return RIDG_OK;
}

int ridg_info(ridg_t* h, ridg_info_t* info) {
  if (check_handle(h) || !info) return RIDG_EINVAL;
  info->dim = h->dim;
  info->order = h->M;
  info->m = h->m;
  info->theta_s = h->thS;
  info->theta_t = h->thT;
  info->cells = h->ncell;
  info->dt = h->dt;
  info->t = h->t;
  info->steps = h->steps;
  info->newton_unconverged = h->newton_unconverged;
  info->newton_iters_max = h->newton_iters_max;
  info->newton_iters_total = h->newton_iters_total;
  info->precision = h->opt.precision;
  info->slices = h->opt.slices;
  for (int k = 0; k < 16; ++k) info->newton_hist[k] = h->newton_hist[k];
  for (int r = 0; r < 4; ++r) info->mass[r] = 0.0;
  return ridg_mass(h, info->mass);
}

int ridg_mass(ridg_t* h, double* mass) {
  if (check_handle(h) || !mass) return RIDG_EINVAL;
  RIDG_CUDA(h, ridg::launch_mass_partials(h->Q, h->ncell, h->m, h->thS, h->red, h->red_blocks,
                                          h->stream));
  std::vector<double> part((size_t)h->red_blocks * h->m);
  RIDG_CUDA(h, cudaMemcpyAsync(part.data(), h->red, part.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
  RIDG_CUDA(h, cudaStreamSynchronize(h->stream));
  double vol = 1.0;
  for (int d = 0; d < h->dim; ++d) vol *= h->h[d];
  for (int r = 0; r < h->m; ++r) {
    double s = 0.0;
    for (int b = 0; b < h->red_blocks; ++b) s += part[(size_t)b * h->m + r];
    mass[r] = s * vol;
  }
  return RIDG_OK;
}

int ridg_l2_error(ridg_t* h, const double* x, int on_device, double* err) {
  if (check_handle(h) || !x || !err) return RIDG_EINVAL;
  size_t nx = (size_t)h->ncell * h->m;
  for (int d = 0; d < h->dim; ++d) nx *= (h->nb + 1);
  const double* xd = x;
  double* tmp = nullptr;
  if (!on_device) {
    tmp = (double*)dev_alloc(h, nx * sizeof(double));
    if (!tmp) return set_err(h, RIDG_ENOMEM, "l2 error buffer");
    cudaError_t e = cudaMemcpyAsync(tmp, x, nx * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      dev_free(h, tmp);
      RIDG_CUDA(h, e);
    }
    xd = tmp;
  }
  std::vector<double> part((size_t)h->red_blocks * 2);
  cudaError_t e = ridg::launch_l2_partials(h->Q, xd, h->ncell, h->m, h->dim, h->nb, h->red,
                                           h->red_blocks, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), h->red, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (tmp) dev_free(h, tmp);
  RIDG_CUDA(h, e);
  double num = 0, den = 0;
  for (int b = 0; b < h->red_blocks; ++b) {
    num += part[2 * b];
    den += part[2 * b + 1];
  }
  *err = den > 0 ? std::sqrt(num / den) : 0.0;
  return RIDG_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// batched ensemble: independent instances sharing one stream; n steps of all of them are
// captured into a single graph and replayed.
// ------------------------------------------------------------------------------------------
// Instances of a nonlinear batch with the same degree: one persistent Newton launch covers
// all their regions (instance table on the device, one region counter).
struct NlGroup {
  std::vector<int> idx;                // instances of the group, in batch order
  std::vector<ridg::NlInst> host;      // the table, refreshed before every batch launch
  ridg::NlInst* table = nullptr;       // device copy
  int* counter = nullptr;              // region counter of the group's launch
  long long regions = 0;
  size_t scratch_off = 0;              // the degree's block storage in the batch's
};

struct ridg_batch {
  std::vector<ridg_t*> inst;
  std::vector<NlGroup> groups;
  void* nl_scratch = nullptr;  // Newton block storage shared by the launches (run in turn)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::map<int, cudaGraphExec_t> graphs;
  std::map<int, cudaGraph_t> defs;
  std::vector<unsigned long long> gens;  // operator generation of each instance at capture
  // nonlinear flux: one Newton launch over every degree's regions and one correction launch
  // over every instance's cells (schedule 1, the default) or one launch per degree and per
  // instance (schedule 0); the autotuner may pick either
  int schedule = 1;
  std::vector<ridg::CorrInst> corr_host;  // all instances, cell0 increasing
  ridg::CorrInst* corr_table = nullptr;
  long long corr_cells = 0;
  ridg::NewtonMulti multi_host{};           // the single Newton launch's arguments
  ridg::NewtonMulti* multi_dev = nullptr;   // and their device copy (read by the kernel)
};

namespace {

// Copy the groups' instance tables (state pointers, meshes, dt / h, statistics words) to the
// device on the batch stream, ahead of the batch graph that reads them.
int refresh_nl_tables(ridg_batch_t* b) {
  for (NlGroup& g : b->groups) {
    long long cell0 = 0;
    for (size_t j = 0; j < g.idx.size(); ++j) {
      ridg_t* h = b->inst[g.idx[j]];
      ridg::NlInst& t = g.host[j];
      t.Q = h->Q;
      t.W = h->W;
      t.cell0 = cell0;
      t.nx = h->n[0];
      t.ny = h->n[1];
      t.lam[0] = h->dt / h->h[0];
      t.lam[1] = h->dt / h->h[1];
      t.stats = h->nl_words + 1;
      t.iters_total = (unsigned long long*)(h->nl_words + 6);
      cell0 += h->ncell;
    }
    g.regions = cell0;
    if (cudaMemcpyAsync(g.table, g.host.data(), g.host.size() * sizeof(ridg::NlInst),
                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return RIDG_ECUDA;
  }
  if (b->corr_table) {
    long long cell0 = 0;
    for (size_t i = 0; i < b->inst.size(); ++i) {
      ridg_t* h = b->inst[i];
      ridg::CorrInst& c = b->corr_host[i];
      c.Q = h->Q;
      c.W = h->W;
      c.cell0 = cell0;
      c.nx = h->n[0];
      c.ny = h->n[1];
      c.nb = h->nb;
      c.lamx = h->dt / h->h[0];
      c.lamy = h->dt / h->h[1];
      cell0 += h->ncell;
    }
    b->corr_cells = cell0;
    if (cudaMemcpyAsync(b->corr_table, b->corr_host.data(),
                        b->corr_host.size() * sizeof(ridg::CorrInst), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess)
      return RIDG_ECUDA;
  }
  return RIDG_OK;
}

// The arguments of a Newton launch over every region of the group's instances.
ridg::NewtonArgs group_args(ridg_batch_t* b, const NlGroup& g) {
  ridg_t* h = b->inst[g.idx[0]];
  ridg::NewtonArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tb = h->nl.tb;
  a.plan = h->plan;
  a.Q = h->Q;
  a.W = h->W;
  a.nx = h->n[0];
  a.ny = h->n[1];
  a.ncell = g.regions;
  a.lam[0] = h->dt / h->h[0];
  a.lam[1] = h->dt / h->h[1];
  a.gamma = h->flux.gamma;
  a.max_iters = h->opt.newton_max_iters;
  a.tol = h->opt.newton_tol;
  a.scratch = (char*)b->nl_scratch + g.scratch_off;
  a.scratch_per_cta = h->nl_scratch_cta;
  a.counter = g.counter;
  a.stats = h->nl_words + 1;
  a.iters_total = (unsigned long long*)(h->nl_words + 6);
  a.inst = g.table;
  a.ninst = (int)g.idx.size();
  return a;
}

// One persistent Newton launch over every region of the group's instances.
int enqueue_newton_group(ridg_batch_t* b, const NlGroup& g) {
  ridg_t* h = b->inst[g.idx[0]];
  const ridg::NewtonArgs a = group_args(b, g);
  RIDG_CUDA(h, ridg::launch_newton(h->nb, h->m, h->flux.kind, newton_prec(h), a, h->nl_grid,
                                   b->stream));
  return RIDG_OK;
}

// The whole ensemble's Newton prediction in one launch (the degrees' queues, highest degree
// first), then every instance's correction in one launch.
int upload_batch_multi(ridg_batch_t* b) {
  ridg::NewtonMulti& m = b->multi_host;
  std::memset(&m, 0, sizeof(m));
  std::vector<const NlGroup*> order;
  for (const NlGroup& g : b->groups) order.push_back(&g);
  std::sort(order.begin(), order.end(), [&](const NlGroup* x, const NlGroup* y) {
    return b->inst[x->idx[0]]->nb > b->inst[y->idx[0]]->nb;
  });
  for (const NlGroup* g : order) {
    m.a[m.count] = group_args(b, *g);
    m.nb[m.count] = b->inst[g->idx[0]]->nb;
    m.count += 1;
  }
  return cudaMemcpyAsync(b->multi_dev, &m, sizeof(m), cudaMemcpyHostToDevice, b->stream) ==
                 cudaSuccess
             ? RIDG_OK
             : RIDG_ECUDA;
}

int enqueue_batch_multi(ridg_batch_t* b) {
  ridg_t* h0 = b->inst[0];
  const int grid = ridg::newton_multi_ctas_per_sm(newton_prec(h0)) * sm_count();
  RIDG_CUDA(h0, ridg::launch_newton_multi(newton_prec(h0), b->multi_host, b->multi_dev, grid,
                                          b->stream));
  ridg::CorrMulti c;
  std::memset(&c, 0, sizeof(c));
  for (const NlGroup& g : b->groups) {
    ridg_t* h = b->inst[g.idx[0]];
    c.tb[h->nb - 2] = h->nl.tb;
  }
  c.inst = b->corr_table;
  c.ninst = (int)b->inst.size();
  RIDG_CUDA(h0, ridg::launch_nl_correct_multi(c, b->corr_cells, b->stream));
  return RIDG_OK;
}

}  // namespace

extern "C" {

int ridg_batch_create(int count, const ridg_mesh* meshes, const int* orders, const ridg_flux* flux,
                      double cfl, const ridg_options* opt, ridg_batch_t** out) {
  if (count < 1 || !meshes || !orders || !flux || !out) return RIDG_EINVAL;
  if (flux->kind != RIDG_FLUX_ADVECTION)
    for (int i = 0; i < count; ++i)
      if (meshes[i].dim != 2) return RIDG_EINVAL;  // the batched Newton launch is 2D
  *out = nullptr;
  ridg_batch_t* b = new ridg_batch_t();
  ridg_options o{};
  if (opt) o = *opt;
  if (o.stream) {
    b->stream = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return RIDG_ECUDA;
    }
    b->own_stream = true;
    o.stream = b->stream;
  }
  for (int i = 0; i < count; ++i) {
    ridg_t* h = nullptr;
    int rc = ridg_create(&meshes[i], orders[i], flux, cfl, &o, &h);
    if (rc != RIDG_OK) {
      ridg_batch_destroy(b);
      return rc;
    }
    h->batch_owned = true;
    b->inst.push_back(h);
  }
  if (flux->kind != RIDG_FLUX_ADVECTION) {
    std::map<int, int> gi;  // degree -> group
    for (int i = 0; i < count; ++i) {
      const int nb = b->inst[i]->nb;
      if (!gi.count(nb)) {
        gi[nb] = (int)b->groups.size();
        b->groups.emplace_back();
      }
      b->groups[gi[nb]].idx.push_back(i);
    }
    // one block storage per degree, shared by the degree's instances (their Newton regions
    // run from one queue): the degrees' block layouts differ, and in the single-launch
    // schedule a CTA's slot of one degree is in use while another CTA works on the next
    // degree, so the degrees never share bytes.  Zeroed once: the blocks' padding is never
    // written again.
    const int multi_grid = flux->kind == RIDG_FLUX_BURGERS
                               ? ridg::newton_multi_ctas_per_sm(newton_prec(b->inst[0])) * sm_count()
                               : 0;
    size_t need = 0;
    for (NlGroup& g : b->groups) {
      ridg_t* h = b->inst[g.idx[0]];
      g.scratch_off = need;
      need += h->nl_scratch_cta * (size_t)std::max(h->nl_grid_max, multi_grid);
    }
    b->nl_scratch = dev_alloc(b->inst[0], need);
    const int rc = !b->nl_scratch ? RIDG_ENOMEM
                   : cudaMemsetAsync(b->nl_scratch, 0, need, b->stream) != cudaSuccess ? RIDG_ECUDA
                                                                                       : RIDG_OK;
    if (rc != RIDG_OK) {
      ridg_batch_destroy(b);
      return rc;
    }
    for (const NlGroup& g : b->groups)
      for (int i : g.idx) {
        ridg_t* h = b->inst[i];
        dev_free(h, h->nl_scratch);
        h->nl_scratch = (char*)b->nl_scratch + g.scratch_off;
        h->nl_scratch_shared = true;
      }
    for (NlGroup& g : b->groups) {
      g.host.resize(g.idx.size());
      g.table = (ridg::NlInst*)dev_alloc(b->inst[0], g.idx.size() * sizeof(ridg::NlInst));
      g.counter = (int*)dev_alloc(b->inst[0], 4 * sizeof(int));
      if (!g.table || !g.counter) {
        ridg_batch_destroy(b);
        return RIDG_ENOMEM;
      }
    }
    // the single-launch schedule (Burgers: the multi-degree kernels are built for one
    // conserved variable); the autotuner's choice, if recorded, decides
    if (flux->kind == RIDG_FLUX_BURGERS) {
      b->corr_host.resize(count);
      b->corr_table = (ridg::CorrInst*)dev_alloc(b->inst[0], count * sizeof(ridg::CorrInst));
      b->multi_dev = (ridg::NewtonMulti*)dev_alloc(b->inst[0], sizeof(ridg::NewtonMulti));
      if (!b->corr_table || !b->multi_dev) {
        ridg_batch_destroy(b);
        return RIDG_ENOMEM;
      }
      b->schedule = ridg::tune_get(key_batch(b->inst[0]), 1);
    } else {
      b->schedule = 0;
    }
  }
  *out = b;
  return RIDG_OK;
}

void ridg_batch_destroy(ridg_batch_t* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : b->defs) cudaGraphDestroy(kv.second);
  if (b->nl_scratch && !b->inst.empty()) dev_free(b->inst[0], b->nl_scratch);
  for (NlGroup& g : b->groups) {
    if (g.table) dev_free(b->inst[0], g.table);
    if (g.counter) dev_free(b->inst[0], g.counter);
  }
  if (b->corr_table) dev_free(b->inst[0], b->corr_table);
  if (b->multi_dev) dev_free(b->inst[0], b->multi_dev);
  for (ridg_t* h : b->inst) ridg_destroy(h);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

ridg_t* ridg_batch_instance(ridg_batch_t* b, int i) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return nullptr;
  return b->inst[i];
}

int ridg_batch_set_state(ridg_batch_t* b, int i, const double* q, int on_device) {
  ridg_t* h = ridg_batch_instance(b, i);
  return h ? ridg_set_state(h, q, on_device) : RIDG_EINVAL;
}

int ridg_batch_get_state(ridg_batch_t* b, int i, double* q, int on_device) {
  ridg_t* h = ridg_batch_instance(b, i);
  return h ? ridg_get_state(h, q, on_device) : RIDG_EINVAL;
}

int ridg_batch_step(ridg_batch_t* b, int n) {
  if (!b || n < 1) return RIDG_EINVAL;
  for (ridg_t* h : b->inst) {
    if (!(h->dt > 0)) return set_err(h, RIDG_ESTATE, "no dt yet: call ridg_set_state first");
    if (!is_linear(h) && clear_newton_stats(h) != cudaSuccess) return RIDG_ECUDA;
  }
  // a rebuilt operator (changed dt) of any instance invalidates the batch graphs
  bool stale = b->gens.size() != b->inst.size();
  for (size_t i = 0; !stale && i < b->inst.size(); ++i) stale = b->gens[i] != b->inst[i]->gen;
  if (stale) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : b->defs) cudaGraphDestroy(kv.second);
    b->graphs.clear();
    b->defs.clear();
    b->gens.clear();
    for (ridg_t* h : b->inst) b->gens.push_back(h->gen);
  }
  // the instance tables (and the groups' region counts the graphs are captured with)
  if (!b->groups.empty()) {
    int rc = refresh_nl_tables(b);
    if (!rc && b->schedule == 1 && b->corr_table) rc = upload_batch_multi(b);
    if (rc) return rc;
  }
  auto it = b->graphs.find(n);
  if (it == b->graphs.end()) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return RIDG_ECUDA;
    int rc = RIDG_OK;
    for (int i = 0; i < n && rc == RIDG_OK; ++i) {
      if (b->groups.empty()) {
        for (ridg_t* h : b->inst) {
          rc = enqueue_step(h);
          if (rc) break;
        }
      } else {
        // nonlinear flux: the whole ensemble in two launches, or one Newton launch per
        // degree over all its instances, then the instances' corrections
        if (b->schedule == 1 && b->corr_table) {
          rc = enqueue_batch_multi(b);
          continue;
        }
        for (const NlGroup& g : b->groups) {
          rc = enqueue_newton_group(b, g);
          if (rc) break;
          for (int j : g.idx) {
            rc = enqueue_nl_correct(b->inst[j]);
            if (rc) break;
          }
          if (rc) break;
        }
      }
    }
    cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    if (rc != RIDG_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc ? rc : RIDG_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      cudaGraphDestroy(graph);
      return RIDG_ECUDA;
    }
    b->graphs[n] = exec;
    b->defs[n] = graph;
    it = b->graphs.find(n);
  }
  if (cudaGraphLaunch(it->second, b->stream) != cudaSuccess) return RIDG_ECUDA;
  for (ridg_t* h : b->inst) {
    h->t += n * h->dt;
    h->steps += n;
  }
  return RIDG_OK;
}

int ridg_batch_schedule(ridg_batch_t* b, int* schedule, int* launches_per_step) {
  if (!b) return RIDG_EINVAL;
  const bool multi = b->schedule == 1 && b->corr_table;
  if (schedule) *schedule = multi ? 1 : 0;
  if (launches_per_step)
    *launches_per_step = b->groups.empty() ? 2 * (int)b->inst.size()
                         : multi          ? 2
                                          : (int)(b->groups.size() + b->inst.size());
  return RIDG_OK;
}

int ridg_batch_autotune(ridg_batch_t* b, const char* cache_path) {
  if (!b || b->inst.empty()) return RIDG_EINVAL;
  if (b->corr_table) {
    // one step in each schedule from the instances' current states (put back afterwards)
    std::vector<double*> save(b->inst.size(), nullptr);
    std::vector<double> t0(b->inst.size());
    std::vector<long long> s0(b->inst.size());
    int rc = RIDG_OK;
    for (size_t i = 0; i < b->inst.size() && !rc; ++i) {
      ridg_t* h = b->inst[i];
      const size_t bytes = (size_t)h->ncell * h->m * h->thS * sizeof(double);
      save[i] = (double*)dev_alloc(h, bytes);
      if (!save[i]) rc = RIDG_ENOMEM;
      else if (cudaMemcpyAsync(save[i], h->Q, bytes, cudaMemcpyDeviceToDevice, b->stream) !=
               cudaSuccess)
        rc = RIDG_ECUDA;
      t0[i] = h->t;
      s0[i] = h->steps;
    }
    auto restore = [&]() {
      for (size_t i = 0; i < b->inst.size(); ++i) {
        ridg_t* h = b->inst[i];
        if (save[i])
          cudaMemcpyAsync(h->Q, save[i], (size_t)h->ncell * h->m * h->thS * sizeof(double),
                          cudaMemcpyDeviceToDevice, b->stream);
        h->t = t0[i];
        h->steps = s0[i];
      }
    };
    double best = 1e300;
    int best_s = b->schedule;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
      rc = RIDG_ECUDA;
    for (int sch = 1; sch >= 0 && !rc; --sch) {
      b->schedule = sch;
      for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
      for (auto& kv : b->defs) cudaGraphDestroy(kv.second);
      b->graphs.clear();
      b->defs.clear();
      for (int rep = 0; rep < 2 && !rc; ++rep) {  // the first run captures the graph
        restore();
        cudaEventRecord(e0, b->stream);
        rc = ridg_batch_step(b, 1);
        cudaEventRecord(e1, b->stream);
        if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = RIDG_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && rep == 1 && ms < best) {
          best = ms;
          best_s = sch;
        }
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    restore();
    cudaStreamSynchronize(b->stream);
    for (size_t i = 0; i < b->inst.size(); ++i) dev_free(b->inst[i], save[i]);
    b->schedule = best_s;
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : b->defs) cudaGraphDestroy(kv.second);
    b->graphs.clear();
    b->defs.clear();
    if (rc && rc != RIDG_ENOCONV) return rc;
    ridg::tune_put(key_batch(b->inst[0]), best_s);
  }
  if (cache_path && !ridg::tune_save(cache_path)) return RIDG_EINVAL;
  return RIDG_OK;
}

int ridg_batch_sync(ridg_batch_t* b) {
  if (!b) return RIDG_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return RIDG_ECUDA;
  // every instance's device status (and Newton statistics); the most severe one is returned
  // (ENOCONV only when nothing worse happened), each instance keeps its own message / info
  int worst = RIDG_OK;
  for (ridg_t* h : b->inst) {
    const int rc = read_status(h);
    if (rc != RIDG_OK && (worst == RIDG_OK || worst == RIDG_ENOCONV)) worst = rc;
  }
  return worst;
}

}  // extern "C"
