// Nonlinear flux in 2D: host tables on the device, the block elimination plan of the
// 3 x 3 region Jacobian, the correction step (Sec. 2.3) with quadrature, and the wave-speed
// reduction that sets dt.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "k_nlflux.cuh"
#include "nl_tables.h"
#include "ridg_internal.h"
#include "tables.h"

namespace ridg {

// ---------------------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------------------
int nl_tables_upload(int nb, NlDevTables& out, void* mem, size_t* bytes, cudaStream_t s) {
  NlHostTables t = build_nl_tables(nb - 1);
  // 6 x 6 equispaced points of the wave-speed estimate
  std::vector<double> eq(6);
  for (int i = 0; i < 6; ++i) eq[i] = -1.0 + 2.0 * i / 5.0;
  std::vector<double> phieq((size_t)t.thS * 36);
  {
    std::vector<double> v(nb), dv(nb);
    std::vector<double> V((size_t)nb * 6);
    for (int i = 0; i < 6; ++i) {
      phi_values(nb, eq[i], v.data(), dv.data());
      for (int b = 0; b < nb; ++b) V[(size_t)b * 6 + i] = v[b];
    }
    for (int s2 = 0; s2 < t.thS; ++s2)
      for (int iy = 0; iy < 6; ++iy)
        for (int ix = 0; ix < 6; ++ix)
          phieq[(size_t)s2 * 36 + iy * 6 + ix] = V[(size_t)(s2 % nb) * 6 + ix] * V[(size_t)(s2 / nb) * 6 + iy];
  }
  struct Piece {
    const void* src;
    size_t n;
    size_t off;
  };
  std::vector<Piece> pieces;
  size_t off = 0;
  auto add = [&](const void* src, size_t nbytes) {
    off = (off + 255) & ~(size_t)255;
    pieces.push_back({src, nbytes, off});
    off += nbytes;
    return pieces.size() - 1;
  };
  auto addd = [&](const std::vector<double>& v) { return add(v.data(), v.size() * sizeof(double)); };
  auto addi = [&](const std::vector<int>& v) { return add(v.data(), v.size() * sizeof(int)); };
  const size_t iMt = addd(t.Mt), iem = addd(t.em), iPsiV = addd(t.PsiV), idPsiV = addd(t.dPsiV),
               iwV = addd(t.wV), iPsiF = addd(t.PsiF), iwF = addd(t.wF), iPhiV = addd(t.PhiV),
               idPhiV = addd(t.dPhiV), iPhiF = addd(t.PhiF), iPsiAtP = addd(t.PsiAtP),
               iPsiAtFP = addd(t.PsiAtFP), iP1 = addd(t.P1), iPhiEq = addd(phieq);
  const size_t iV1 = addd(t.V1), iV1T = addd(t.V1T), idV1 = addd(t.dV1), iep1 = addd(t.ep1),
               iem1 = addd(t.em1);
  size_t ib[2][3], ig[8][3];
  for (int d = 0; d < 2; ++d) {
    ib[d][0] = addi(t.beta[d].ptr);
    ib[d][1] = addi(t.beta[d].p);
    ib[d][2] = addd(t.beta[d].val);
  }
  for (int d = 0; d < 2; ++d)
    for (int sk = 0; sk < 2; ++sk)
      for (int sl = 0; sl < 2; ++sl) {
        const SparseTriple& G = t.gamma[d][sk][sl];
        const int g = d * 4 + sk * 2 + sl;
        ig[g][0] = addi(G.ptr);
        ig[g][1] = addi(G.p);
        ig[g][2] = addd(G.val);
      }
  // merged assembly lists, packed per precision
  NlAsmLists L = build_asm_lists(t);
  struct EntD { int off; int pad; double c; };
  struct EntF { int off; float c; };
  auto packd = [](const std::vector<int>& o, const std::vector<double>& v) {
    std::vector<EntD> e(o.size());
    for (size_t i = 0; i < o.size(); ++i) e[i] = {o[i], 0, v[i]};
    return e;
  };
  auto packf = [](const std::vector<int>& o, const std::vector<double>& v) {
    std::vector<EntF> e(o.size());
    for (size_t i = 0; i < o.size(); ++i) e[i] = {o[i], (float)v[i]};
    return e;
  };
  std::vector<EntD> dd_ = packd(L.doff, L.dval);
  std::vector<EntF> df_ = packf(L.doff, L.dval);
  std::vector<EntD> od_[4];
  std::vector<EntF> of_[4];
  for (int f = 0; f < 4; ++f) {
    od_[f] = packd(L.ooff[f], L.oval[f]);
    of_[f] = packf(L.ooff[f], L.oval[f]);
  }
  const size_t idptr = addi(L.dptr), identd = add(dd_.data(), dd_.size() * sizeof(EntD)),
               identf = add(df_.data(), df_.size() * sizeof(EntF));
  size_t ioptr[4], ioentd[4], ioentf[4];
  for (int f = 0; f < 4; ++f) {
    ioptr[f] = addi(L.optr[f]);
    ioentd[f] = add(od_[f].data(), od_[f].size() * sizeof(EntD));
    ioentf[f] = add(of_[f].data(), of_[f].size() * sizeof(EntF));
  }
  auto tof = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
  std::vector<float> Mtf = tof(t.Mt), PsiAtPf = tof(t.PsiAtP), PsiAtFPf = tof(t.PsiAtFP), P1f = tof(t.P1);
  std::vector<float> T0f = tof(t.T0), T1f = tof(t.T1), ep1f = tof(t.ep1), em1f = tof(t.em1);
  const size_t iMtf = add(Mtf.data(), Mtf.size() * 4), iPsiAtPf = add(PsiAtPf.data(), PsiAtPf.size() * 4),
               iPsiAtFPf = add(PsiAtFPf.data(), PsiAtFPf.size() * 4), iP1f = add(P1f.data(), P1f.size() * 4);
  const size_t iT0f = add(T0f.data(), T0f.size() * 4), iT1f = add(T1f.data(), T1f.size() * 4),
               iep1f = add(ep1f.data(), ep1f.size() * 4), iem1f = add(em1f.data(), em1f.size() * 4);
  const size_t total = (off + 255) & ~(size_t)255;
  if (!mem) {
    *bytes = total;
    return RIDG_OK;
  }
  if (*bytes < total) return RIDG_EINVAL;
  char* base = (char*)mem;
  for (const Piece& p : pieces)
    if (p.n && cudaMemcpyAsync(base + p.off, p.src, p.n, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return RIDG_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RIDG_ECUDA;  // host vectors go away
  auto D = [&](size_t i) { return (const double*)(base + pieces[i].off); };
  auto I = [&](size_t i) { return (const int*)(base + pieces[i].off); };
  NlDev& tb = out.tb;
  tb.Mt = D(iMt);
  tb.em = D(iem);
  tb.PsiV = D(iPsiV);
  tb.dPsiV = D(idPsiV);
  tb.wV = D(iwV);
  tb.PsiF = D(iPsiF);
  tb.wF = D(iwF);
  tb.PhiV = D(iPhiV);
  tb.dPhiV = D(idPhiV);
  tb.PhiF = D(iPhiF);
  tb.PsiAtP = D(iPsiAtP);
  tb.PsiAtFP = D(iPsiAtFP);
  tb.P1 = D(iP1);
  tb.PhiEq = D(iPhiEq);
  tb.V1 = D(iV1);
  tb.V1T = D(iV1T);
  tb.dV1 = D(idV1);
  tb.ep1 = D(iep1);
  tb.em1 = D(iem1);
  for (int d = 0; d < 2; ++d) {
    tb.bptr[d] = I(ib[d][0]);
    tb.bp[d] = I(ib[d][1]);
    tb.bval[d] = D(ib[d][2]);
  }
  for (int g = 0; g < 8; ++g) {
    tb.gptr[g] = I(ig[g][0]);
    tb.gp[g] = I(ig[g][1]);
    tb.gval[g] = D(ig[g][2]);
  }
  tb.dptr = I(idptr);
  tb.dent_d = base + pieces[identd].off;
  tb.dent_f = base + pieces[identf].off;
  for (int f = 0; f < 4; ++f) {
    tb.optr[f] = I(ioptr[f]);
    tb.oent_d[f] = base + pieces[ioentd[f]].off;
    tb.oent_f[f] = base + pieces[ioentf[f]].off;
  }
  auto F = [&](size_t i) { return (const float*)(base + pieces[i].off); };
  tb.Mt_f = F(iMtf);
  tb.PsiAtP_f = F(iPsiAtPf);
  tb.PsiAtFP_f = F(iPsiAtFPf);
  tb.P1_f = F(iP1f);
  tb.T0_f = F(iT0f);
  tb.T1_f = F(iT1f);
  tb.ep1_f = F(iep1f);
  tb.em1_f = F(iem1f);
  out.mem = mem;
  out.bytes = total;
  return RIDG_OK;
}

namespace {

// ---------------------------------------------------------------------------------------
// correction (Sec. 2.3): Q += volume term - surface term, every face flux evaluated from the
// same traces in the same order by both cells that share it (so both see the same bits)
// ---------------------------------------------------------------------------------------
constexpr int kCorrThreads = 128;

// the correction of cell e of one mesh (a block of kCorrThreads threads); shared memory
// carved from `sh` (nl_corr_smem<NB, MV>() bytes)
template <int NB, int MV>
constexpr size_t nl_corr_smem() {
  constexpr int THT = NB * NB * NB, BS = MV * THT, NQ = (3 * (NB - 1) + 2) / 2;
  constexpr int QV = NQ * NQ * NQ, QF = NQ * NQ;
  return sizeof(double) * (5 * BS + 2 * MV * QV + 3 * 4 * MV * QF + 4 * QF);
}

template <int NB, int MV, int FLUX>
__device__ void nl_correct_cell(const NlDev& tb, double* __restrict__ Q, const double* __restrict__ W,
                                int nx, int ny, double lamx, double lamy, double gamma,
                                long long e, double* sh) {
  constexpr int THS = NB * NB, THT = NB * THS, BS = MV * THT;
  constexpr int NQ = (3 * (NB - 1) + 2) / 2, QV = NQ * NQ * NQ, QF = NQ * NQ;
  auto Wc = (double(*)[BS])sh;                               // own, +x, -x, +y, -y neighbours
  auto G = (double(*)[MV][QV])(sh + 5 * BS);                 // sc_d w_q F_d(w), volume points
  auto TL = (double(*)[MV][QF])(sh + 5 * BS + 2 * MV * QV);  // left / right traces per face
  auto TR = (double(*)[MV][QF])(sh + 5 * BS + 2 * MV * QV + 4 * MV * QF);
  auto FH = (double(*)[MV][QF])(sh + 5 * BS + 2 * MV * QV + 8 * MV * QF);  // sc w F-hat
  auto spd = (double(*)[QF])(sh + 5 * BS + 2 * MV * QV + 12 * MV * QF);
  const int tid = threadIdx.x;
  const unsigned ue = (unsigned)e, uy = ue / (unsigned)nx;
  const int ix = (int)(ue - uy * (unsigned)nx), iy = (int)uy;
  const long long nbr[5] = {e, (long long)iy * nx + (ix + 1) % nx, (long long)iy * nx + (ix + nx - 1) % nx,
                            (long long)((iy + 1) % ny) * nx + ix, (long long)((iy + ny - 1) % ny) * nx + ix};
  for (int i = tid; i < 5 * BS; i += kCorrThreads) Wc[i / BS][i % BS] = W[nbr[i / BS] * BS + i % BS];
  __syncthreads();
  const double sc[2] = {0.25 * lamx, 0.25 * lamy};
  for (int q = tid; q < QV; q += kCorrThreads) {
    double w[MV], f[MV];
    for (int j = 0; j < MV; ++j) {
      double acc = 0.0;
      for (int k = 0; k < THT; ++k) acc = fma(tb.PsiV[k * QV + q], Wc[0][j * THT + k], acc);
      w[j] = acc;
    }
    for (int dd = 0; dd < 2; ++dd) {
      nlflux::F<FLUX>(w, dd, f, gamma);
      for (int j = 0; j < MV; ++j) G[dd][j][q] = sc[dd] * tb.wV[q] * f[j];
    }
  }
  // face f = dd * 2 + si (si 0: the +1 face, 1: the -1 face).  Left / right states:
  //   +1 face: L = own trace at +1, R = the +dd neighbour's trace at -1
  //   -1 face: L = the -dd neighbour's trace at +1, R = own trace at -1
  for (int i = tid; i < 4 * QF; i += kCorrThreads) {
    const int f = i / QF, q = i % QF, dd = f >> 1, si = f & 1;
    const double* tp = tb.PsiF + (size_t)(dd * 2 + 0) * THT * QF;  // +1 side table
    const double* tm = tb.PsiF + (size_t)(dd * 2 + 1) * THT * QF;  // -1 side table
    const double* wl = si == 0 ? Wc[0] : Wc[2 + 2 * dd];
    const double* wr = si == 0 ? Wc[1 + 2 * dd] : Wc[0];
    double a[MV], b[MV];
    for (int j = 0; j < MV; ++j) {
      double sl = 0.0, sr = 0.0;
      for (int k = 0; k < THT; ++k) {
        sl = fma(tp[k * QF + q], wl[j * THT + k], sl);
        sr = fma(tm[k * QF + q], wr[j * THT + k], sr);
      }
      a[j] = sl;
      b[j] = sr;
      TL[f][j][q] = sl;
      TR[f][j][q] = sr;
    }
    spd[f][q] = fmax(nlflux::speed<FLUX>(a, dd, gamma), nlflux::speed<FLUX>(b, dd, gamma));
  }
  __syncthreads();
  for (int i = tid; i < 4 * QF; i += kCorrThreads) {
    const int f = i / QF, q = i % QF, dd = f >> 1;
    double alpha = 0.0;
    for (int p = 0; p < QF; ++p) alpha = fmax(alpha, spd[f][p]);
    double a[MV], b[MV], fa[MV], fb[MV];
    for (int j = 0; j < MV; ++j) {
      a[j] = TL[f][j][q];
      b[j] = TR[f][j][q];
    }
    nlflux::F<FLUX>(a, dd, fa, gamma);
    nlflux::F<FLUX>(b, dd, fb, gamma);
    const double wq = sc[dd] * tb.wF[dd * QF + q];
    for (int j = 0; j < MV; ++j) FH[f][j][q] = wq * (0.5 * (fa[j] + fb[j]) - 0.5 * alpha * (b[j] - a[j]));
  }
  __syncthreads();
  for (int i = tid; i < MV * THS; i += kCorrThreads) {
    const int j = i / THS, s2 = i % THS;
    double acc = 0.0;
    for (int dd = 0; dd < 2; ++dd)
      for (int q = 0; q < QV; ++q) acc = fma(tb.dPhiV[(dd * THS + s2) * QV + q], G[dd][j][q], acc);
    for (int f = 0; f < 4; ++f) {
      const double sg = (f & 1) ? 1.0 : -1.0;  // -(flux out at +1) + (flux in at -1)
      const double* ph = tb.PhiF + (size_t)(f * THS + s2) * QF;
      double fs = 0.0;
      for (int q = 0; q < QF; ++q) fs = fma(ph[q], FH[f][j][q], fs);
      acc = fma(sg, fs, acc);
    }
    Q[e * MV * THS + i] += acc;
  }
  __syncthreads();  // the shared arrays are reused by the block's next cell
}

template <int NB, int MV, int FLUX>
__global__ void __launch_bounds__(kCorrThreads) nl_correct_kernel(NlDev tb, double* __restrict__ Q,
                                                                  const double* __restrict__ W,
                                                                  int nx, int ny, double lamx,
                                                                  double lamy, double gamma) {
  __shared__ double sh[nl_corr_smem<NB, MV>() / sizeof(double)];
  nl_correct_cell<NB, MV, FLUX>(tb, Q, W, nx, ny, lamx, lamy, gamma, blockIdx.x, sh);
}

// Every instance's correction of a batched Burgers ensemble in one launch: block b takes the
// cell b of the concatenated instances (the instance of the last table entry whose first
// cell is <= b, found by bisection) and runs that instance's degree.
__global__ void __launch_bounds__(kCorrThreads) nl_correct_multi_kernel(const CorrMulti m) {
  __shared__ double sh[nl_corr_smem<5, 1>() / sizeof(double)];  // the largest degree
  const long long b = blockIdx.x;
  int lo = 0, hi = m.ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (m.inst[mid].cell0 <= b) lo = mid; else hi = mid - 1;
  }
  const CorrInst& in = m.inst[lo];
  const long long e = b - in.cell0;
  switch (in.nb) {
    case 2: nl_correct_cell<2, 1, RIDG_FLUX_BURGERS>(m.tb[0], in.Q, in.W, in.nx, in.ny, in.lamx, in.lamy, 0.0, e, sh); break;
    case 3: nl_correct_cell<3, 1, RIDG_FLUX_BURGERS>(m.tb[1], in.Q, in.W, in.nx, in.ny, in.lamx, in.lamy, 0.0, e, sh); break;
    case 4: nl_correct_cell<4, 1, RIDG_FLUX_BURGERS>(m.tb[2], in.Q, in.W, in.nx, in.ny, in.lamx, in.lamy, 0.0, e, sh); break;
    case 5: nl_correct_cell<5, 1, RIDG_FLUX_BURGERS>(m.tb[3], in.Q, in.W, in.nx, in.ny, in.lamx, in.lamy, 0.0, e, sh); break;
    default: break;
  }
}

template <int NB, int MV, int FLUX>
__global__ void max_speed_kernel(NlDev tb, const double* __restrict__ Q, long long ncell,
                                 double gamma, unsigned long long* out) {
  constexpr int THS = NB * NB;
  double best = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncell * 36;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / 36;
    const int pnt = (int)(i % 36);
    double w[MV];
    for (int j = 0; j < MV; ++j) {
      double acc = 0.0;
      for (int s2 = 0; s2 < THS; ++s2) acc = fma(tb.PhiEq[s2 * 36 + pnt], Q[(e * MV + j) * THS + s2], acc);
      w[j] = acc;
    }
    for (int dd = 0; dd < 2; ++dd) best = fmax(best, nlflux::speed<FLUX>(w, dd, gamma));
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  // speeds are >= 0, so their bit patterns order like their values (a NaN state is refused
  // by the finite check before this runs)
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

}  // namespace

#define RIDG_NL_SWITCH(NB_, M_, KIND_, CALL)                                               \
  do {                                                                                    \
    if (KIND_ == RIDG_FLUX_BURGERS && M_ == 1) {                                          \
      switch (NB_) {                                                                      \
        case 2: { constexpr int NB = 2, MV = 1, FL = RIDG_FLUX_BURGERS; CALL; } break;    \
        case 3: { constexpr int NB = 3, MV = 1, FL = RIDG_FLUX_BURGERS; CALL; } break;    \
        case 4: { constexpr int NB = 4, MV = 1, FL = RIDG_FLUX_BURGERS; CALL; } break;    \
        case 5: { constexpr int NB = 5, MV = 1, FL = RIDG_FLUX_BURGERS; CALL; } break;    \
        default: return cudaErrorInvalidValue;                                            \
      }                                                                                   \
    } else if (KIND_ == RIDG_FLUX_EULER && M_ == 4) {                                     \
      switch (NB_) {                                                                      \
        case 2: { constexpr int NB = 2, MV = 4, FL = RIDG_FLUX_EULER; CALL; } break;      \
        case 3: { constexpr int NB = 3, MV = 4, FL = RIDG_FLUX_EULER; CALL; } break;      \
        default: return cudaErrorInvalidValue;                                            \
      }                                                                                   \
    } else {                                                                              \
      return cudaErrorInvalidValue;                                                       \
    }                                                                                     \
  } while (0)

cudaError_t launch_newton_f64(int nb, int m, int kind, const NewtonArgs& a, int grid,
                              cudaStream_t s);
cudaError_t launch_newton_f32(int nb, int m, int kind, const NewtonArgs& a, int grid,
                              cudaStream_t s);
cudaError_t launch_newton_tf32(int nb, int m, int kind, const NewtonArgs& a, int grid,
                               cudaStream_t s);

bool newton_supported(int nb, int m) { return (m == 1 && nb >= 2 && nb <= 5) || (m == 4 && nb >= 2 && nb <= 3); }

int newton_ctas_per_sm_f64(int nb, int m, int kind);
int newton_ctas_per_sm_f32(int nb, int m, int kind);
int newton_ctas_per_sm_tf32(int nb, int m, int kind);

int newton_grid(int nb, int m, int kind, int prec) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return 0;
  const int per = prec == kNewtonTF32  ? newton_ctas_per_sm_tf32(nb, m, kind)
                  : prec == kNewtonF32 ? newton_ctas_per_sm_f32(nb, m, kind)
                                       : newton_ctas_per_sm_f64(nb, m, kind);
  return per > 0 ? per * sms : 0;  // a persistent grid: every resident CTA slot filled once
}

size_t newton_scratch_per_cta(int nb, int m, int prec, const NlPlan& plan) {
  const int bs = m * nb * nb * nb, bp = (bs + 15) / 16 * 16;
  const size_t bytes =
      (size_t)plan.nslots * bp * bp * (prec == kNewtonF64 ? sizeof(double) : sizeof(float));
  return (bytes + 255) & ~(size_t)255;
}

cudaError_t launch_newton(int nb, int m, int flux_kind, int prec, const NewtonArgs& a, int grid,
                          cudaStream_t s) {
  switch (prec) {
    case kNewtonF64: return launch_newton_f64(nb, m, flux_kind, a, grid, s);
    case kNewtonF32: return launch_newton_f32(nb, m, flux_kind, a, grid, s);
    case kNewtonTF32: return launch_newton_tf32(nb, m, flux_kind, a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_newton_multi_f64(const NewtonMulti& m, const NewtonMulti* dev, int grid,
                                 cudaStream_t s);
cudaError_t launch_newton_multi_f32(const NewtonMulti& m, const NewtonMulti* dev, int grid,
                                 cudaStream_t s);
cudaError_t launch_newton_multi_tf32(const NewtonMulti& m, const NewtonMulti* dev, int grid,
                                 cudaStream_t s);
int newton_multi_ctas_per_sm_f64();
int newton_multi_ctas_per_sm_f32();
int newton_multi_ctas_per_sm_tf32();

cudaError_t launch_newton_multi(int prec, const NewtonMulti& m, const NewtonMulti* dev, int grid,
                                cudaStream_t s) {
  switch (prec) {
    case kNewtonF64: return launch_newton_multi_f64(m, dev, grid, s);
    case kNewtonF32: return launch_newton_multi_f32(m, dev, grid, s);
    case kNewtonTF32: return launch_newton_multi_tf32(m, dev, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int newton_multi_ctas_per_sm(int prec) {
  switch (prec) {
    case kNewtonF64: return newton_multi_ctas_per_sm_f64();
    case kNewtonF32: return newton_multi_ctas_per_sm_f32();
    case kNewtonTF32: return newton_multi_ctas_per_sm_tf32();
    default: return 0;
  }
}

cudaError_t launch_nl_correct(int nb, int m, int flux_kind, const NlDev& tb, double* Q,
                              const double* W, int nx, int ny, long long ncell, double lamx,
                              double lamy, double gamma, cudaStream_t s) {
  RIDG_NL_SWITCH(nb, m, flux_kind,
                 (nl_correct_kernel<NB, MV, FL><<<(unsigned)ncell, kCorrThreads, 0, s>>>(
                     tb, Q, W, nx, ny, lamx, lamy, gamma)));
  return cudaGetLastError();
}

cudaError_t launch_nl_correct_multi(const CorrMulti& m, long long cells, cudaStream_t s) {
  nl_correct_multi_kernel<<<(unsigned)cells, kCorrThreads, 0, s>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_max_speed(int nb, int m, int flux_kind, const NlDev& tb, const double* Q,
                             long long ncell, double gamma, unsigned long long* out,
                             cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const long long work = ncell * 36;
  const unsigned blocks = (unsigned)std::min<long long>((work + 255) / 256, 4096);
  RIDG_NL_SWITCH(nb, m, flux_kind,
                 (max_speed_kernel<NB, MV, FL><<<blocks, 256, 0, s>>>(tb, Q, ncell, gamma, out)));
  return cudaGetLastError();
}

}  // namespace ridg
