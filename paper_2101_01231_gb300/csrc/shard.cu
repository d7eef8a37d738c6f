// A linear-advection mesh sharded into slabs along its slowest axis (the paper's domain
// decomposition of RIDG, Sec. 5, carried to GPUs): slab i owns a contiguous range of layers
// and is an ordinary handle on its own device and stream, whose local mesh is the slab plus
// the halo layers upstream of it along the slab axis, periodic locally.
//
// With upwind face values a cell's prediction reads only the region cells upstream of it,
// and its correction only its own and its upstream neighbours' time means.  So the step of
// a slab's first interior layer needs the state of the two layers upstream of it: one for
// the prediction of the layer below it (whose time mean its correction reads), one more for
// that layer's own upwind box.  Those two layers are the halo; each step starts by copying
// them from the upstream slab's last two interior layers (one contiguous peer copy: in the
// canonical layout a layer of the slowest axis is contiguous).  The slab's local periodic
// wrap then only reaches halo cells, whose results are discarded, so every interior cell
// computes exactly what the unsharded step computes (the same operands in the same order:
// the FP64 path is bit-identical).  For a zero velocity component along the axis the slabs
// do not interact and carry no halo.
//
// Ordering per step (events, no host waits): slab i's copy waits for the upstream slab's
// previous step; slab j's step waits for the copy that reads its state; then it runs its
// captured step graph.  Slabs on different devices copy with cudaMemcpyPeerAsync.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ridg_internal.h"

struct ridg_shard {
  int count = 0, axis = 0, halo = 0, dir = 0;  // dir: +1 halo below (a > 0), -1 above
  long long layer = 0;                           // doubles per layer (whole problem)
  int n_axis = 0, m = 1, ths = 1;
  std::vector<ridg_t*> h;
  std::vector<int> first, nloc, dev;
  std::vector<cudaEvent_t> stepped, copied;
  bool primed = false;
};

namespace {

// the slab receiving slab i's interior (its downstream neighbour) and the one it reads
int upstream(const ridg_shard* s, int i) {
  return s->dir > 0 ? (i - 1 + s->count) % s->count : (i + 1) % s->count;
}
int downstream(const ridg_shard* s, int i) {
  return s->dir > 0 ? (i + 1) % s->count : (i - 1 + s->count) % s->count;
}

// local layer index of global layer offset k within slab i (k = 0: first interior layer)
int local_of(const ridg_shard* s, int k) { return (s->dir > 0 ? s->halo : 0) + k; }

void destroy_events(ridg_shard* s) {
  for (size_t i = 0; i < s->h.size(); ++i) {
    if (!s->h[i]) continue;
    cudaSetDevice(s->dev[i]);
    if (i < s->stepped.size() && s->stepped[i]) cudaEventDestroy(s->stepped[i]);
    if (i < s->copied.size() && s->copied[i]) cudaEventDestroy(s->copied[i]);
  }
}

}  // namespace

extern "C" {

void ridg_shard_destroy(ridg_shard_t* s) {
  if (!s) return;
  int cur = 0;
  cudaGetDevice(&cur);
  destroy_events(s);
  for (size_t i = 0; i < s->h.size(); ++i) {
    if (!s->h[i]) continue;
    cudaSetDevice(s->dev[i]);
    ridg_destroy(s->h[i]);
  }
  cudaSetDevice(cur);
  delete s;
}

int ridg_shard_create(const ridg_mesh* mesh, int order, const ridg_flux* flux, double cfl,
                      const ridg_options* opt, int count, const int* devices,
                      ridg_shard_t** out) {
  if (!mesh || !flux || !out || count < 1) return RIDG_EINVAL;
  *out = nullptr;
  if (flux->kind != RIDG_FLUX_ADVECTION || mesh->dim < 1 || mesh->dim > 3) return RIDG_EINVAL;
  if (opt && opt->stream) return RIDG_EINVAL;  // every slab runs on a stream of its own
  const int axis = mesh->dim - 1;
  const int n = mesh->n[axis];
  const double a = flux->vel[axis];
  auto* s = new ridg_shard();
  s->count = count;
  s->axis = axis;
  s->n_axis = n;
  s->dir = a > 0 ? 1 : (a < 0 ? -1 : 0);
  s->halo = s->dir ? 2 : 0;
  // layers per slab: as even as possible; each at least 2 (the halo is one slab's two
  // outermost layers) and, with its halo, at least 3 (the smallest mesh a handle takes)
  const int base = n / count, extra = n % count;
  int g = 0;
  for (int i = 0; i < count; ++i) {
    const int k = base + (i < extra ? 1 : 0);
    s->first.push_back(g);
    s->nloc.push_back(k);
    g += k;
    if (k < 2 || k + s->halo < 3) {
      delete s;
      return RIDG_EINVAL;
    }
  }
  int cur = 0;
  cudaGetDevice(&cur);
  s->dev.assign(count, cur);
  if (devices)
    for (int i = 0; i < count; ++i) s->dev[i] = devices[i];
  const double hx = (mesh->hi[axis] - mesh->lo[axis]) / n;
  s->h.assign(count, nullptr);
  s->stepped.assign(count, nullptr);
  s->copied.assign(count, nullptr);
  int rc = RIDG_OK;
  for (int i = 0; i < count && rc == RIDG_OK; ++i) {
    if (cudaSetDevice(s->dev[i]) != cudaSuccess) {
      rc = RIDG_ECUDA;
      break;
    }
    ridg_mesh lm = *mesh;
    lm.n[axis] = s->nloc[i] + s->halo;
    const int l0 = s->first[i] - (s->dir > 0 ? s->halo : 0);  // global layer of local 0
    lm.lo[axis] = mesh->lo[axis] + l0 * hx;
    lm.hi[axis] = lm.lo[axis] + lm.n[axis] * hx;
    rc = ridg_create(&lm, order, flux, cfl, opt, &s->h[i]);
    if (rc == RIDG_OK) {
      // the slab's cell sizes and step exactly as the whole mesh's (recomputed from the
      // slab's own extent they could differ in the last bit, and so would the operator)
      ridg_t* hs = s->h[i];
      double hmin = 0.0, amax = 0.0;
      for (int d = 0; d < mesh->dim; ++d) {
        hs->h[d] = (mesh->hi[d] - mesh->lo[d]) / mesh->n[d];
        hmin = d == 0 ? hs->h[0] : std::min(hmin, hs->h[d]);
        amax = std::max(amax, std::fabs(flux->vel[d]));
      }
      rc = ridg_set_dt(hs, cfl * hmin / (amax > 0 ? amax : 1.0));
      hs->dt_fixed = false;  // as the unsharded handle: ridg_set_final_time may change it
    }
    if (rc == RIDG_OK &&
        (cudaEventCreateWithFlags(&s->stepped[i], cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&s->copied[i], cudaEventDisableTiming) != cudaSuccess))
      rc = RIDG_ECUDA;
  }
  cudaSetDevice(cur);
  if (rc != RIDG_OK) {
    ridg_shard_destroy(s);
    return rc;
  }
  // peer access between the slabs' devices where they differ (already enabled is fine)
  for (int i = 0; i < count; ++i) {
    const int j = upstream(s, i);
    if (s->dev[i] == s->dev[j]) continue;
    int ok = 0;
    cudaDeviceCanAccessPeer(&ok, s->dev[i], s->dev[j]);
    if (ok) {
      cudaSetDevice(s->dev[i]);
      const cudaError_t e = cudaDeviceEnablePeerAccess(s->dev[j], 0);
      if (e == cudaErrorPeerAccessAlreadyEnabled) cudaGetLastError();
    }
  }
  cudaSetDevice(cur);
  s->m = s->h[0]->m;
  s->ths = s->h[0]->thS;
  s->layer = (long long)s->m * s->ths;
  for (int d = 0; d < axis; ++d) s->layer *= mesh->n[d];
  *out = s;
  return RIDG_OK;
}

ridg_t* ridg_shard_slab(ridg_shard_t* s, int i) {
  if (!s || i < 0 || i >= s->count) return nullptr;
  return s->h[i];
}

// q: the whole problem's state in the canonical layout (host, or device memory of the
// current device if on_device)
int ridg_shard_set_state(ridg_shard_t* s, const double* q, int on_device) {
  if (!s || !q) return RIDG_EINVAL;
  const size_t lb = (size_t)s->layer * sizeof(double);
  std::vector<double> host;
  const double* src = q;
  if (on_device) {
    host.resize((size_t)s->layer * s->n_axis);
    if (cudaMemcpy(host.data(), q, host.size() * sizeof(double), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return RIDG_ECUDA;
    src = host.data();
  }
  int cur = 0;
  cudaGetDevice(&cur);
  int rc = RIDG_OK;
  for (int i = 0; i < s->count && rc == RIDG_OK; ++i) {
    const int nl = s->nloc[i] + s->halo;
    const int l0 = s->first[i] - (s->dir > 0 ? s->halo : 0);
    std::vector<double> loc((size_t)s->layer * nl);
    for (int l = 0; l < nl; ++l) {
      const int gl = ((l0 + l) % s->n_axis + s->n_axis) % s->n_axis;  // periodic
      std::memcpy(loc.data() + (size_t)l * s->layer, src + (size_t)gl * s->layer, lb);
    }
    cudaSetDevice(s->dev[i]);
    rc = ridg_set_state(s->h[i], loc.data(), 0);
  }
  cudaSetDevice(cur);
  s->primed = false;
  return rc;
}

int ridg_shard_get_state(ridg_shard_t* s, double* q, int on_device) {
  if (!s || !q) return RIDG_EINVAL;
  const size_t lb = (size_t)s->layer * sizeof(double);
  std::vector<double> host((size_t)s->layer * s->n_axis);
  int cur = 0;
  cudaGetDevice(&cur);
  int rc = RIDG_OK;
  for (int i = 0; i < s->count && rc == RIDG_OK; ++i) {
    const int nl = s->nloc[i] + s->halo;
    std::vector<double> loc((size_t)s->layer * nl);
    cudaSetDevice(s->dev[i]);
    rc = ridg_get_state(s->h[i], loc.data(), 0);
    for (int k = 0; k < s->nloc[i] && rc == RIDG_OK; ++k)
      std::memcpy(host.data() + (size_t)(s->first[i] + k) * s->layer,
                  loc.data() + (size_t)local_of(s, k) * s->layer, lb);
  }
  cudaSetDevice(cur);
  if (rc) return rc;
  if (on_device)
    return cudaMemcpy(q, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice) ==
                   cudaSuccess
               ? RIDG_OK
               : RIDG_ECUDA;
  std::memcpy(q, host.data(), host.size() * sizeof(double));
  return RIDG_OK;
}

int ridg_shard_step(ridg_shard_t* s, int n) {
  if (!s || n < 1) return RIDG_EINVAL;
  int cur = 0;
  cudaGetDevice(&cur);
  const size_t hb = (size_t)s->halo * s->layer * sizeof(double);
  int rc = RIDG_OK;
  for (int k = 0; k < n && rc == RIDG_OK; ++k) {
    if (s->halo > 0) {
      // halo exchange: slab i's two halo layers <- the upstream slab's outermost interior
      for (int i = 0; i < s->count && rc == RIDG_OK; ++i) {
        const int j = upstream(s, i);
        ridg_t* hi = s->h[i];
        ridg_t* hj = s->h[j];
        cudaSetDevice(s->dev[i]);
        if (s->primed && cudaStreamWaitEvent(hi->stream, s->stepped[j], 0) != cudaSuccess) {
          rc = RIDG_ECUDA;
          break;
        }
        // source: slab j's last two interior layers (a > 0) or its first two (a < 0);
        // destination: slab i's halo, below (local 0, 1) or above (after its interior)
        const int src_l = s->dir > 0 ? local_of(s, s->nloc[j] - 2) : local_of(s, 0);
        const int dst_l = s->dir > 0 ? 0 : s->nloc[i];
        const double* src = hj->Q + (size_t)src_l * s->layer;
        double* dst = hi->Q + (size_t)dst_l * s->layer;
        const cudaError_t e =
            s->dev[i] == s->dev[j]
                ? cudaMemcpyAsync(dst, src, hb, cudaMemcpyDeviceToDevice, hi->stream)
                : cudaMemcpyPeerAsync(dst, s->dev[i], src, s->dev[j], hb, hi->stream);
        if (e != cudaSuccess || cudaEventRecord(s->copied[i], hi->stream) != cudaSuccess) {
          rc = RIDG_ECUDA;
          break;
        }
        hi->ms.valid = false;  // the mixed path's digit planes no longer match the halo
      }
    }
    for (int j = 0; j < s->count && rc == RIDG_OK; ++j) {
      ridg_t* hj = s->h[j];
      cudaSetDevice(s->dev[j]);
      // slab j's state must not change before its downstream neighbour has copied it
      if (s->halo > 0 &&
          cudaStreamWaitEvent(hj->stream, s->copied[downstream(s, j)], 0) != cudaSuccess) {
        rc = RIDG_ECUDA;
        break;
      }
      rc = ridg_step(hj, 1);
      if (rc == RIDG_OK && cudaEventRecord(s->stepped[j], hj->stream) != cudaSuccess)
        rc = RIDG_ECUDA;
    }
    s->primed = true;
  }
  cudaSetDevice(cur);
  return rc;
}

int ridg_shard_sync(ridg_shard_t* s) {
  if (!s) return RIDG_EINVAL;
  int cur = 0;
  cudaGetDevice(&cur);
  int rc = RIDG_OK;
  for (int i = 0; i < s->count; ++i) {
    cudaSetDevice(s->dev[i]);
    const int r = ridg_sync(s->h[i]);
    if (rc == RIDG_OK) rc = r;
  }
  cudaSetDevice(cur);
  return rc;
}

}  // extern "C"
