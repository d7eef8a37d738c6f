// ridg_l2_error_noalloc: the relative L2 error for callers that cannot allocate device
// memory.  Some callers are not allowed to call cudaMalloc at the point where they need
// this diagnostic: code whose device memory is owned entirely by a pool or arena that must
// see every allocation, and time-critical loops that cannot afford the implicit device
// synchronisation of cudaMalloc / cudaFree.  This entry point therefore allocates nothing:
// its scratch (one pair of partial sums per 256 cells, plus the final pair) lives in a
// file-scope __device__ array of fixed size that every GPU loading the library keeps until
// exit.  The call reads its result back and waits on the caller's stream, so that stream
// must not be capturing a CUDA graph; a capturing stream is refused before any work.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "ridg_internal.h"

namespace {

constexpr int kThreads = 256;                  // cells per partial
constexpr long long kMaxPartials = 65536;      // scratch: 65536 pairs -> 16,777,216 cells
constexpr int kMaxDevices = 64;

// partial (numerator, denominator) pairs, then the final pair at [2 * kMaxPartials]
static __device__ __align__(256) double g_l2_scratch[2 * kMaxPartials + 2];

double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// one partial pair per block of 256 cells (every pair is written: nothing accumulates
// across calls)
__global__ void l2_partials_kernel(const double* __restrict__ Q, const double* __restrict__ X,
                                   long long ncell, int m, int dim, int nb,
                                   double* __restrict__ part) {
  __shared__ double sh[kThreads];
  const int nb2 = nb + 1;
  int thS = 1, thS2 = 1;
  for (int d = 0; d < dim; ++d) {
    thS *= nb;
    thS2 *= nb2;
  }
  double num = 0.0, den = 0.0;
  const long long e = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (e < ncell) {
    for (int r = 0; r < m; ++r) {
      const double* x = X + (e * m + r) * thS2;
      const double* q = Q + (e * m + r) * thS;
      for (int s2 = 0; s2 < thS2; ++s2) {
        const int bx = s2 % nb2;
        const int by = dim > 1 ? (s2 / nb2) % nb2 : 0;
        const int bz = dim > 2 ? s2 / (nb2 * nb2) : 0;
        const double xv = x[s2];
        den += xv * xv;
        if (bx < nb && by < nb && bz < nb) {
          const double dv = xv - q[bx + nb * (by + nb * bz)];
          num += dv * dv;
        } else {
          num += xv * xv;  // the Q(M+1) modes beyond Q(M): dominant truncation term
        }
      }
    }
  }
  const double sn = block_sum(num, sh);
  const double sd = block_sum(den, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sn;
    part[2 * blockIdx.x + 1] = sd;
  }
}

// the partials summed in a fixed order by one block -> part[2 * kMaxPartials .. + 1]
__global__ void l2_final_kernel(double* __restrict__ part, long long nparts) {
  __shared__ double sh[kThreads];
  double num = 0.0, den = 0.0;
  for (long long b = threadIdx.x; b < nparts; b += kThreads) {
    num += part[2 * b];
    den += part[2 * b + 1];
  }
  const double sn = block_sum(num, sh);
  const double sd = block_sum(den, sh);
  if (threadIdx.x == 0) {
    part[2 * kMaxPartials] = sn;
    part[2 * kMaxPartials + 1] = sd;
  }
}

// the device address of the scratch array on the current device, looked up once per device
// with that device current; a cudaDeviceReset (which tears the module down) makes the cached
// address stale, so a process that resets a device must not call this entry point after it
double* scratch_for_current_device(int* status) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *status = RIDG_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_l2_scratch) != cudaSuccess || !p) {
      *status = RIDG_ECUDA;
      return nullptr;
    }
    g_scratch_ptr[dev] = p;
  }
  *status = RIDG_OK;
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" int ridg_l2_error_noalloc(const double* q, const double* x, long long cells, int m,
                                     int dim, int order, void* stream, double* err) {
  if (!q || !x || !err || cells < 1 || m < 1 || dim < 1 || dim > 3 || order < 0)
    return RIDG_EINVAL;
  const long long nparts = (cells + kThreads - 1) / kThreads;
  if (nparts > kMaxPartials) return RIDG_ETOOBIG;
  cudaStream_t s = (cudaStream_t)stream;
  // the read-back and the wait below are illegal on a capturing stream (and on the legacy
  // stream while another stream captures in global mode): refuse before touching anything
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    if (ce != cudaSuccess) cudaGetLastError();  // not sticky; keep it out of later calls
    return RIDG_ESTATE;
  }
  int st = RIDG_OK;
  double* part = scratch_for_current_device(&st);
  if (!part) return st;
  l2_partials_kernel<<<(unsigned)nparts, kThreads, 0, s>>>(q, x, cells, m, dim, order + 1, part);
  l2_final_kernel<<<1, kThreads, 0, s>>>(part, nparts);
  if (cudaGetLastError() != cudaSuccess) return RIDG_ECUDA;
  double fin[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(fin, part + 2 * kMaxPartials, sizeof(fin), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RIDG_ECUDA;
  *err = fin[1] > 0 ? std::sqrt(fin[0] / fin[1]) : 0.0;
  return RIDG_OK;
}
