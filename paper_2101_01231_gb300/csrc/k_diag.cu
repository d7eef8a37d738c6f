// Diagnostic reductions of the RIDG state: cell-average mass, the relative L2 error of
// eq. l2relerror, and a finiteness check.  Every reduction writes one partial per block
// in a fixed order (grid-stride loop, then a fixed shared-memory tree); the host sums the
// partials in block order, so results are run-to-run deterministic.
#include <cuda_runtime.h>

#include "k_tcgen05.cuh"
#include "ridg_internal.h"

namespace ridg {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void mass_kernel(const double* __restrict__ Q, long long ncell, int m, int thS,
                            double* __restrict__ out) {
  __shared__ double sh[kThreads];
  for (int r = 0; r < m; ++r) {
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * kThreads + threadIdx.x; e < ncell;
         e += (long long)gridDim.x * kThreads)
      acc += Q[(e * m + r) * thS];
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x * m + r] = s;
  }
}

// X holds (M+2)^d modes per cell and variable; Q holds (M+1)^d.
__global__ void l2_kernel(const double* __restrict__ Q, const double* __restrict__ X,
                          long long ncell, int m, int dim, int nb, double* __restrict__ out) {
  __shared__ double sh[kThreads];
  const int nb2 = nb + 1;
  int thS = 1, thS2 = 1;
  for (int d = 0; d < dim; ++d) { thS *= nb; thS2 *= nb2; }
  double num = 0.0, den = 0.0;
  for (long long e = (long long)blockIdx.x * kThreads + threadIdx.x; e < ncell;
       e += (long long)gridDim.x * kThreads) {
    for (int r = 0; r < m; ++r) {
      const double* x = X + (e * m + r) * thS2;
      const double* q = Q + (e * m + r) * thS;
      for (int s2 = 0; s2 < thS2; ++s2) {
        int bx = s2 % nb2, by = (s2 / nb2) % nb2, bz = s2 / (nb2 * nb2);
        if (dim < 2) by = 0;
        if (dim < 3) bz = 0;
        const double xv = x[s2];
        den += xv * xv;
        if (bx < nb && by < nb && bz < nb) {
          const int s = bx + nb * (by + nb * bz);
          const double dv = xv - q[s];
          num += dv * dv;
        } else {
          num += xv * xv;
        }
      }
    }
  }
  double sn = block_sum(num, sh);
  double sd = block_sum(den, sh);
  if (threadIdx.x == 0) {
    out[blockIdx.x * 2 + 0] = sn;
    out[blockIdx.x * 2 + 1] = sd;
  }
}

__global__ void finite_kernel(const double* __restrict__ q, long long count, int* flag) {
  int bad = 0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count;
       i += (long long)gridDim.x * kThreads)
    bad |= !isfinite(q[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// A bounded mbarrier wait (the helper every tensor-core kernel uses) on an arrival that
// never comes: the wait must give up by itself and report it (status 1), the way the
// kernels stop on a timeout.  status 0 would mean the wait completed, which cannot happen.
__global__ void bounded_wait_probe_kernel(int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    status[0] = mbar_wait(b, 0) ? 0 : 1;
  }
}

// set_state from a pinned host buffer: the SMs read it over the coherent C2C link themselves
// (16-byte loads, four in flight per thread per iteration), write the device state and raise
// *flag on a value that is not finite -- the copy and the finite check in one pass (measured
// on GB300: 61 us against 73 us for a copy-engine copy followed by the check, 256^2 Q3).
__global__ void __launch_bounds__(256) ingest_kernel(const double* __restrict__ src,
                                                     double* __restrict__ dst, long long n,
                                                     int* __restrict__ flag) {
  const long long n2 = n / 2, stride = (long long)gridDim.x * blockDim.x;
  const double2* s2 = (const double2*)src;
  double2* d2 = (double2*)dst;
  bool bad = false;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n2; i += 4 * stride) {
    const double2 a = s2[i], b = s2[i + stride], c = s2[i + 2 * stride], d = s2[i + 3 * stride];
    d2[i] = a;
    d2[i + stride] = b;
    d2[i + 2 * stride] = c;
    d2[i + 3 * stride] = d;
    bad |= !(isfinite(a.x) && isfinite(a.y) && isfinite(b.x) && isfinite(b.y) &&
             isfinite(c.x) && isfinite(c.y) && isfinite(d.x) && isfinite(d.y));
  }
  for (; i < n2; i += stride) {
    const double2 a = s2[i];
    d2[i] = a;
    bad |= !(isfinite(a.x) && isfinite(a.y));
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const double v = src[n - 1];
    dst[n - 1] = v;
    bad |= !isfinite(v);
  }
  if (bad) atomicOr(flag, 1);
}

}  // namespace

cudaError_t launch_bounded_wait_probe(int* status, cudaStream_t s) {
  bounded_wait_probe_kernel<<<1, 32, 0, s>>>(status);
  return cudaGetLastError();
}

cudaError_t launch_mass_partials(const double* Q, long long ncell, int m, int thS, double* out,
                                 int nblocks, cudaStream_t s) {
  mass_kernel<<<nblocks, kThreads, 0, s>>>(Q, ncell, m, thS, out);
  return cudaGetLastError();
}

cudaError_t launch_l2_partials(const double* Q, const double* X, long long ncell, int m, int dim,
                               int nb, double* out, int nblocks, cudaStream_t s) {
  l2_kernel<<<nblocks, kThreads, 0, s>>>(Q, X, ncell, m, dim, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_ingest(const double* host, double* dev, long long count, int* flag,
                          cudaStream_t s) {
  int d = 0, sms = 0;
  cudaGetDevice(&d);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
  ingest_kernel<<<sms * 4, 256, 0, s>>>(host, dev, count, flag);
  return cudaGetLastError();
}

cudaError_t launch_finite_check(const double* q, long long count, int* flag, cudaStream_t s) {
  finite_kernel<<<256, kThreads, 0, s>>>(q, count, flag);
  return cudaGetLastError();
}

}  // namespace ridg

extern "C" int ridg_check_bounded_wait(void* stream, double* seconds) {
  cudaStream_t s = (cudaStream_t)stream;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return RIDG_ENOMEM;
  int status = -1;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int rc = RIDG_ECUDA;
  if (cudaMemsetAsync(d, 0xFF, sizeof(int), s) == cudaSuccess &&
      cudaEventCreate(&ev[0]) == cudaSuccess && cudaEventCreate(&ev[1]) == cudaSuccess &&
      cudaEventRecord(ev[0], s) == cudaSuccess &&
      ridg::launch_bounded_wait_probe(d, s) == cudaSuccess &&
      cudaEventRecord(ev[1], s) == cudaSuccess &&
      cudaMemcpyAsync(&status, d, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaStreamSynchronize(s) == cudaSuccess) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (seconds) *seconds = ms * 1e-3;
    rc = status == 1 ? RIDG_ETIMEOUT : (status == 0 ? RIDG_OK : RIDG_ECUDA);
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  cudaFree(d);
  return rc;
}

