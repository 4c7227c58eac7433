// Batched (continuous-batching) execution of many independent simulations of
// uneven size: the serving path.  Each simulation is the paper's KDK leapfrog
// (Eq. 5-7) over the Eq. 1-2 force sum, with its own N, softening, G, time
// step and precision mode (FP64, MIXED or F64E).
//
// All resident simulations share one device pool of `capacity` particles.
// A simulation occupies a contiguous range of it; ranges are handed out first
// fit and returned on eviction, so admission is decided by free device memory
// (a free range of n particles) and a free slot.  One tick advances every
// resident simulation by one step with at most three force launches (MIXED
// prep, MIXED force, FP64 force) over work-unit tables that never let a tile
// cross from one simulation into another, plus one epilogue launch that sums
// each simulation's j-segments in a fixed order and applies its KDK update.
//
// Per simulation (pool range [off, off+n)):
//   R  (x, y, z, m) state positions at the step boundary
//   F  (x, y, z, m) positions of the next force evaluation (KDK predictor)
//   V  velocity at the step boundary; VB = (v + vt)/2 (Eq. 5/7); A = (a, pot) at R
// A newly admitted simulation is first packed into R, V (its raw input is
// staged in its own, still unused VB/A range), then its first tick evaluates
// a(t0) and the predictor (Eq. 5 needs a(t0)); every later tick is one step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nbody_internal.cuh"

using nb::d4;

namespace {

constexpr int SMAX = 16;       // most j-segments per simulation
constexpr int ALIGN = 64;      // pool ranges start on 64-particle boundaries
constexpr int FL_ACTIVE = 1, FL_INIT = 2;
constexpr int NCLS = 3;  // kernel classes: FP64, MIXED, F64E
int cls_of(int mode) { return mode == NBODY_MIXED ? 1 : mode == NBODY_F64E ? 2 : 0; }

struct SimDesc {
  int64_t off, n, part;
  double G, dt, hdt;
  int32_t S, flags;
};

struct SimHost {
  bool used = false, active = false, init = false;
  int mode = NBODY_FP64;
  int64_t off = 0, n = 0;
  double eps = 0, G = 1, dt = 0;
  int64_t steps = 0;
};

thread_local char g_msg[512] = "";

int bfail(int code, const char *what, cudaError_t ce = cudaSuccess) {
  if (ce != cudaSuccess)
    snprintf(g_msg, sizeof g_msg, "%s: %s (%s)", nbody_strerror(code), what, cudaGetErrorString(ce));
  else
    snprintf(g_msg, sizeof g_msg, "%s: %s", nbody_strerror(code), what);
  return code;
}

#define BCK(call)                                                    \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return bfail(NBODY_ECUDA, #call, e_);     \
  } while (0)

// ---------------------------------------------------------------- kernels
__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// After the force launches of a tick: a = G sum_k part, then either the
// first-step set-up (a(t0), predictor) or the corrector of Eq. 7 followed by
// the next predictor (Eq. 5-6), per particle of every active simulation.
__global__ void k_batch_kdk(const int32_t *__restrict__ sim_of, const SimDesc *__restrict__ sims,
                            int64_t hi, const d4 *__restrict__ part, d4 *__restrict__ R,
                            d4 *__restrict__ F, d4 *__restrict__ V, d4 *__restrict__ VB,
                            d4 *__restrict__ A) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < hi;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int s = sim_of[g];
    if (s < 0) continue;
    const SimDesc d = sims[s];
    if (!(d.flags & FL_ACTIVE)) continue;
    const int64_t i = g - d.off;
    const d4 p0 = part[d.part + i];
    double x = p0.x, y = p0.y, z = p0.z, w = p0.w;
    for (int k = 1; k < d.S; k++) {
      const d4 p = part[d.part + (int64_t)k * d.n + i];
      x = __dadd_rn(x, p.x);
      y = __dadd_rn(y, p.y);
      z = __dadd_rn(z, p.z);
      w = __dadd_rn(w, p.w);
    }
    const double ax = __dmul_rn(d.G, x), ay = __dmul_rn(d.G, y), az = __dmul_rn(d.G, z);
    A[g] = d4{ax, ay, az, -__dmul_rn(d.G, w)};
    d4 v, r;
    if (d.flags & FL_INIT) {
      v = V[g];
      r = R[g];
    } else {
      const d4 vb = VB[g];
      v = d4{__dadd_rn(vb.x, __dmul_rn(d.hdt, ax)), __dadd_rn(vb.y, __dmul_rn(d.hdt, ay)),
             __dadd_rn(vb.z, __dmul_rn(d.hdt, az)), 0.0};
      V[g] = v;
      r = F[g];
      R[g] = r;
    }
    const double tx = __dadd_rn(v.x, __dmul_rn(d.dt, ax));
    const double ty = __dadd_rn(v.y, __dmul_rn(d.dt, ay));
    const double tz = __dadd_rn(v.z, __dmul_rn(d.dt, az));
    VB[g] = d4{__dmul_rn(__dadd_rn(v.x, tx), 0.5), __dmul_rn(__dadd_rn(v.y, ty), 0.5),
               __dmul_rn(__dadd_rn(v.z, tz), 0.5), 0.0};
    F[g] = d4{__dadd_rn(r.x, __dmul_rn(d.hdt, __dadd_rn(tx, v.x))),
              __dadd_rn(r.y, __dmul_rn(d.hdt, __dadd_rn(ty, v.y))),
              __dadd_rn(r.z, __dmul_rn(d.hdt, __dadd_rn(tz, v.z))), r.w};
  }
}

}  // namespace

// ---------------------------------------------------------------- the pool
struct nbody_batch {
  cudaStream_t st = nullptr;  // the caller's stream: every copy and launch of the pool
  int device = 0, sms = 0;
  int64_t cap = 0;
  int max_sims = 0;
  d4 *R = nullptr, *F = nullptr, *V = nullptr, *VB = nullptr, *A = nullptr, *part = nullptr;
  float4 *fpos = nullptr, *fposff = nullptr, *anchor = nullptr;  // MIXED / F64E staging
  int32_t *sim_of = nullptr;
  double *diag_blocks = nullptr, *diag_out = nullptr, *h_diag = nullptr;
  double *stage = nullptr;  // device scratch for unpacking (cap x 6 doubles)
  // tables, double-buffered: [buffer] device + pinned host
  nb::Unit *d_units[2] = {nullptr, nullptr}, *h_units[2] = {nullptr, nullptr};
  nb::PrepUnit *d_prep[2] = {nullptr, nullptr}, *h_prep[2] = {nullptr, nullptr};
  SimDesc *d_sims[2] = {nullptr, nullptr}, *h_sims[2] = {nullptr, nullptr};
  cudaEvent_t tab_ev[2] = {nullptr, nullptr};
  int64_t units_cap = 0, prep_cap = 0;
  int tb = 0;
  bool dirty = true;
  int64_t n64 = 0, nmx = 0, nfe = 0, nprep = 0, nprepfe = 0, hi = 0;  // table sizes, pool high-water mark
  // admission staging (pinned host ring)
  static constexpr int RING = 4;
  double *h_in[RING] = {};
  size_t h_in_cap[RING] = {};
  cudaEvent_t in_ev[RING] = {};
  int ring = 0;
  // host state
  std::vector<SimHost> sims;
  std::map<int64_t, int64_t> free_ranges;  // offset -> length
  int r_mode[3] = {2, 2, 2};                 // R per kernel class (FP64, MIXED, F64E)
  int fp64_per_sm = 2;                       // resident FP64 force blocks per SM (persistent grid)
  int64_t seg_mode[3] = {4096, 8192, 4096};  // target j-segment length per class
  // profiling
  std::vector<cudaEvent_t> evs;  // 8 per tick: tick start/end, then start/end per class
  size_t ev_used = 0;
  std::vector<double> tick_inter[3];
  int64_t launches = 0;
  bool prof = false;
};

namespace {

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

bool take_range(nbody_batch *b, int64_t n, int64_t *off) {
  const int64_t need = round_up(n, ALIGN);
  for (auto it = b->free_ranges.begin(); it != b->free_ranges.end(); ++it) {
    if (it->second >= need) {
      *off = it->first;
      const int64_t rest = it->second - need, at = it->first + need;
      b->free_ranges.erase(it);
      if (rest > 0) b->free_ranges[at] = rest;
      return true;
    }
  }
  return false;
}

void give_range(nbody_batch *b, int64_t off, int64_t n) {
  int64_t len = round_up(n, ALIGN);
  auto nx = b->free_ranges.lower_bound(off);
  if (nx != b->free_ranges.end() && off + len == nx->first) {
    len += nx->second;
    b->free_ranges.erase(nx);
  }
  auto pv = b->free_ranges.lower_bound(off);
  if (pv != b->free_ranges.begin()) {
    --pv;
    if (pv->first + pv->second == off) {
      pv->second += len;
      return;
    }
  }
  b->free_ranges[off] = len;
}

int grow_pinned(void **p, size_t *cap, size_t need) {
  if (*cap >= need) return NBODY_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost(p, need) != cudaSuccess) return bfail(NBODY_ENOMEM, "pinned staging");
  *cap = need;
  return NBODY_OK;
}

int ensure_tables(nbody_batch *b, int64_t nunits, int64_t nprep) {
  if (nunits > b->units_cap) {
    const int64_t c = std::max<int64_t>(nunits, 2 * b->units_cap);
    for (int k = 0; k < 2; k++) {
      BCK(cudaEventSynchronize(b->tab_ev[k]));
      if (b->d_units[k]) cudaFree(b->d_units[k]);
      if (b->h_units[k]) cudaFreeHost(b->h_units[k]);
      b->d_units[k] = nullptr;
      b->h_units[k] = nullptr;
      if (cudaMalloc(&b->d_units[k], c * sizeof(nb::Unit)) != cudaSuccess ||
          cudaMallocHost(&b->h_units[k], c * sizeof(nb::Unit)) != cudaSuccess)
        return bfail(NBODY_ENOMEM, "unit tables");
    }
    b->units_cap = c;
  }
  if (nprep > b->prep_cap) {
    const int64_t c = std::max<int64_t>(nprep, 2 * b->prep_cap);
    for (int k = 0; k < 2; k++) {
      BCK(cudaEventSynchronize(b->tab_ev[k]));
      if (b->d_prep[k]) cudaFree(b->d_prep[k]);
      if (b->h_prep[k]) cudaFreeHost(b->h_prep[k]);
      b->d_prep[k] = nullptr;
      b->h_prep[k] = nullptr;
      if (cudaMalloc(&b->d_prep[k], c * sizeof(nb::PrepUnit)) != cudaSuccess ||
          cudaMallocHost(&b->h_prep[k], c * sizeof(nb::PrepUnit)) != cudaSuccess)
        return bfail(NBODY_ENOMEM, "prep tables");
    }
    b->prep_cap = c;
  }
  return NBODY_OK;
}

// Rebuild the work-unit tables of the resident simulations into the spare
// buffer and upload them (stream-ordered before the next tick).
int build_tables(nbody_batch *b) {
  std::vector<nb::Unit> uc[NCLS];
  std::vector<nb::PrepUnit> prep, prepfe;
  const int nsl = b->max_sims;
  const int nb_buf = 1 - b->tb;
  BCK(cudaEventSynchronize(b->tab_ev[nb_buf]));  // its previous upload has been consumed
  SimDesc *hs = b->h_sims[nb_buf];
  int64_t pbase = 0, abase = 0, hi = 0;
  for (int s = 0; s < nsl; s++) {
    const SimHost &h = b->sims[s];
    SimDesc d = {};
    if (h.used && h.active) {
      const int m = cls_of(h.mode);
      const int bt = nb::force_block_threads(h.mode), T = nb::force_tile(h.mode);
      const int64_t pb = (int64_t)bt * b->r_mode[m];
      int64_t seg = std::max<int64_t>(T, round_up(b->seg_mode[m], T));
      if ((h.n + seg - 1) / seg > SMAX) seg = round_up((h.n + SMAX - 1) / SMAX, T);
      const int S = (int)((h.n + seg - 1) / seg);
      d.off = h.off;
      d.n = h.n;
      d.part = pbase;
      d.G = h.G;
      d.dt = h.dt;
      d.hdt = h.dt / 2;
      d.S = S;
      d.flags = FL_ACTIVE | (h.init ? FL_INIT : 0);
      for (int64_t ib = 0; ib < h.n; ib += pb)
        for (int k = 0; k < S; k++) {
          nb::Unit u;
          u.i0 = h.off + ib;
          u.ni = (int32_t)std::min<int64_t>(pb, h.n - ib);
          u.j0 = h.off + (int64_t)k * seg;
          u.nj = (int32_t)std::min<int64_t>(seg, h.n - (int64_t)k * seg);
          u.out = pbase + (int64_t)k * h.n + ib;
          u.anchor = abase + (int64_t)k * seg / T;
          u.eps2 = h.eps * h.eps;
          uc[m].push_back(u);
        }
      if (m) {
        for (int64_t t = 0; t * T < h.n; t++) {
          nb::PrepUnit p;
          p.j0 = h.off + t * T;
          p.cnt = (int32_t)std::min<int64_t>(T, h.n - t * T);
          p.anchor = abase + t;
          p.pad = 0;
          (m == 1 ? prep : prepfe).push_back(p);
        }
        abase += (h.n + T - 1) / T;
      }
      pbase += (int64_t)S * h.n;
      hi = std::max(hi, h.off + h.n);
    }
    hs[s] = d;
  }
  // largest units first, so that the tail of the launch is made of small ones
  auto by_work = [](const nb::Unit &a, const nb::Unit &c) {
    return (int64_t)a.ni * a.nj > (int64_t)c.ni * c.nj;
  };
  for (int m = 0; m < NCLS; m++) std::stable_sort(uc[m].begin(), uc[m].end(), by_work);
  const int64_t nu = (int64_t)(uc[0].size() + uc[1].size() + uc[2].size());
  const int64_t np = (int64_t)(prep.size() + prepfe.size());
  int rc = ensure_tables(b, nu, np);
  if (rc) return rc;
  nb::Unit *hu = b->h_units[nb_buf];
  int64_t at = 0;
  for (int m = 0; m < NCLS; m++) {
    std::copy(uc[m].begin(), uc[m].end(), hu + at);
    at += (int64_t)uc[m].size();
  }
  std::copy(prep.begin(), prep.end(), b->h_prep[nb_buf]);
  std::copy(prepfe.begin(), prepfe.end(), b->h_prep[nb_buf] + prep.size());
  if (nu) BCK(cudaMemcpyAsync(b->d_units[nb_buf], hu, nu * sizeof(nb::Unit), cudaMemcpyHostToDevice, b->st));
  if (np)
    BCK(cudaMemcpyAsync(b->d_prep[nb_buf], b->h_prep[nb_buf], np * sizeof(nb::PrepUnit),
                        cudaMemcpyHostToDevice, b->st));
  BCK(cudaMemcpyAsync(b->d_sims[nb_buf], hs, nsl * sizeof(SimDesc), cudaMemcpyHostToDevice, b->st));
  BCK(cudaEventRecord(b->tab_ev[nb_buf], b->st));
  b->tb = nb_buf;
  b->n64 = (int64_t)uc[0].size();
  b->nmx = (int64_t)uc[1].size();
  b->nfe = (int64_t)uc[2].size();
  b->nprep = (int64_t)prep.size();
  b->nprepfe = (int64_t)prepfe.size();
  b->hi = hi;
  b->dirty = false;
  return NBODY_OK;
}

cudaEvent_t next_event(nbody_batch *b) {
  if (b->ev_used == b->evs.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    b->evs.push_back(e);
  }
  return b->evs[b->ev_used++];
}

int check_slot(nbody_batch *b, int slot) {
  if (!b) return bfail(NBODY_EINVAL, "NULL batch");
  if (slot < 0 || slot >= b->max_sims || !b->sims[slot].used) return bfail(NBODY_EINVAL, "bad slot");
  return NBODY_OK;
}

void free_batch(nbody_batch *b) {
  void *dp[] = {b->R, b->F, b->V, b->VB, b->A, b->part, b->fpos, b->fposff, b->anchor, b->sim_of,
                b->diag_blocks, b->diag_out, b->stage, b->d_units[0], b->d_units[1],
                b->d_prep[0], b->d_prep[1], b->d_sims[0], b->d_sims[1]};
  for (void *p : dp)
    if (p) cudaFree(p);
  void *hp[] = {b->h_diag, b->h_units[0], b->h_units[1], b->h_prep[0], b->h_prep[1],
                b->h_sims[0], b->h_sims[1]};
  for (void *p : hp)
    if (p) cudaFreeHost(p);
  for (int k = 0; k < nbody_batch::RING; k++) {
    if (b->h_in[k]) cudaFreeHost(b->h_in[k]);
    if (b->in_ev[k]) cudaEventDestroy(b->in_ev[k]);
  }
  for (int k = 0; k < 2; k++)
    if (b->tab_ev[k]) cudaEventDestroy(b->tab_ev[k]);
  for (auto e : b->evs) cudaEventDestroy(e);
}

}  // namespace

extern "C" {

const char *nbody_batch_last_error(void) { return g_msg; }

int64_t nbody_batch_bytes_per_particle(void) {
  return 5 * (int64_t)sizeof(d4) + SMAX * (int64_t)sizeof(d4) + 3 * (int64_t)sizeof(float4) +
         (int64_t)sizeof(int32_t) + 6 * (int64_t)sizeof(double);
}

int nbody_batch_create(nbody_batch **out, int64_t capacity, int max_sims, void *cuda_stream) {
  if (!out) return bfail(NBODY_EINVAL, "out is NULL");
  *out = nullptr;
  if (capacity < 1 || max_sims < 1 || max_sims > (1 << 20))
    return bfail(NBODY_EINVAL, "capacity and max_sims must be >= 1");
  nbody_batch *b = new (std::nothrow) nbody_batch;
  if (!b) return bfail(NBODY_ENOMEM, "batch");
  b->cap = round_up(capacity, ALIGN);
  b->max_sims = max_sims;
  b->st = (cudaStream_t)cuda_stream;
  b->sims.assign(max_sims, SimHost());
  b->free_ranges[0] = b->cap;
  cudaError_t ce = cudaGetDevice(&b->device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (ce != cudaSuccess) {
    delete b;
    return bfail(NBODY_ECUDA, "no CUDA device", ce);
  }
  const size_t c = (size_t)b->cap;
  const int64_t tiles = b->cap / 256 + max_sims + 1;
  bool ok = cudaMalloc(&b->R, c * sizeof(d4)) == cudaSuccess &&
            cudaMalloc(&b->F, c * sizeof(d4)) == cudaSuccess &&
            cudaMalloc(&b->V, c * sizeof(d4)) == cudaSuccess &&
            cudaMalloc(&b->VB, c * sizeof(d4)) == cudaSuccess &&
            cudaMalloc(&b->A, c * sizeof(d4)) == cudaSuccess &&
            cudaMalloc(&b->part, c * SMAX * sizeof(d4)) == cudaSuccess &&
            cudaMalloc(&b->fpos, c * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&b->fposff, 2 * c * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&b->anchor, (size_t)tiles * 2 * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&b->sim_of, c * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&b->stage, c * 6 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->diag_blocks, (size_t)nb::diag_blocks(b->cap) * 8 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->diag_out, 16 * sizeof(double)) == cudaSuccess &&
            cudaMallocHost(&b->h_diag, 16 * sizeof(double)) == cudaSuccess;
  for (int k = 0; ok && k < 2; k++)
    ok = cudaMalloc(&b->d_sims[k], max_sims * sizeof(SimDesc)) == cudaSuccess &&
         cudaMallocHost(&b->h_sims[k], max_sims * sizeof(SimDesc)) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->tab_ev[k], cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < nbody_batch::RING; k++)
    ok = cudaEventCreateWithFlags(&b->in_ev[k], cudaEventDisableTiming) == cudaSuccess;
  if (ok) {
    k_fill_i32<<<256, 256, 0, b->st>>>(b->sim_of, b->cap, -1);
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(b->st) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_batch(b);
    delete b;
    return bfail(NBODY_ENOMEM, "batch pool");
  }
  *out = b;
  return NBODY_OK;
}

int nbody_batch_destroy(nbody_batch *b) {
  if (!b) return NBODY_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->st);
  free_batch(b);
  delete b;
  return NBODY_OK;
}

int nbody_batch_admit(nbody_batch *b, int64_t n, int mode, double eps, double G, double dt,
                      const double *pos, const double *vel, const double *mass, int on_device,
                      int *slot) {
  if (!b || !slot) return bfail(NBODY_EINVAL, "NULL argument");
  *slot = -1;
  if (n < 1) return bfail(NBODY_EINVAL, "n < 1");
  if (mode != NBODY_FP64 && mode != NBODY_MIXED && mode != NBODY_F64E)
    return bfail(NBODY_EINVAL, "batch modes: FP64, MIXED or F64E");
  if (!(eps >= 0) || !std::isfinite(eps) || !std::isfinite(G)) return bfail(NBODY_EINVAL, "eps or G");
  if (!(dt > 0) || !std::isfinite(dt)) return bfail(NBODY_EINVAL, "dt must be finite and > 0");
  if (!pos || !mass) return bfail(NBODY_EINVAL, "NULL pos or mass");
  BCK(cudaSetDevice(b->device));
  if (!on_device) {  // reject bad input before it occupies anything
    for (int64_t k = 0; k < 3 * n; k++)
      if (!std::isfinite(pos[k]) || (vel && !std::isfinite(vel[k])))
        return bfail(NBODY_EINVAL, "non-finite position or velocity");
    for (int64_t k = 0; k < n; k++)
      if (!std::isfinite(mass[k]) || mass[k] < 0) return bfail(NBODY_EINVAL, "bad mass");
  }
  int s = -1;
  for (int k = 0; k < b->max_sims; k++)
    if (!b->sims[k].used) {
      s = k;
      break;
    }
  if (s < 0) return bfail(NBODY_ENOSPC, "no free slot");
  int64_t off = 0;
  if (!take_range(b, n, &off)) return bfail(NBODY_ENOSPC, "no free range of n particles");
  // Host input is staged in this simulation's own VB range (pos then mass, 4n doubles)
  // and A range (vel, 3n doubles): both are unused until its first tick.  The copies
  // are ordered on the pool's stream after every tick already queued, so a reused
  // range is never overwritten while an earlier simulation's tick still reads it.
  double *raw = (double *)(b->VB + off);
  double *raw_pos = raw, *raw_vel = (double *)(b->A + off), *raw_mass = raw + 3 * n;
  const double *ppos = pos, *pvel = vel, *pmass = mass;
  if (!on_device) {
    const int k = b->ring;
    b->ring = (b->ring + 1) % nbody_batch::RING;
    cudaError_t ce = cudaEventSynchronize(b->in_ev[k]);
    if (ce != cudaSuccess) {
      give_range(b, off, n);
      return bfail(NBODY_ECUDA, "staging event", ce);
    }
    const size_t need = sizeof(double) * 7 * (size_t)n;
    int rc = grow_pinned((void **)&b->h_in[k], &b->h_in_cap[k], need);
    if (rc) {
      give_range(b, off, n);
      return rc;
    }
    double *h = b->h_in[k];
    memcpy(h, pos, 3 * n * sizeof(double));
    memcpy(h + 3 * n, mass, n * sizeof(double));
    if (vel) memcpy(h + 4 * n, vel, 3 * n * sizeof(double));
    BCK(cudaMemcpyAsync(raw_pos, h, 4 * n * sizeof(double), cudaMemcpyHostToDevice, b->st));
    if (vel) BCK(cudaMemcpyAsync(raw_vel, h + 4 * n, 3 * n * sizeof(double), cudaMemcpyHostToDevice, b->st));
    BCK(cudaEventRecord(b->in_ev[k], b->st));  // the pinned ring slot is reusable after this
    ppos = raw_pos;
    pmass = raw_mass;
    pvel = vel ? raw_vel : nullptr;
  }
  BCK(nb::launch_pack(NBODY_FP64, ppos, pvel, pmass, n, b->R + off, b->V + off, nullptr, b->st));
  BCK(cudaMemcpyAsync(b->F + off, b->R + off, n * sizeof(d4), cudaMemcpyDeviceToDevice, b->st));
  k_fill_i32<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, b->st>>>(b->sim_of + off, n, s);
  BCK(cudaGetLastError());
  b->launches += 2;
  SimHost &h = b->sims[s];
  h = SimHost();
  h.used = h.active = h.init = true;
  h.mode = mode;
  h.off = off;
  h.n = n;
  h.eps = eps;
  h.G = G;
  h.dt = dt;
  b->dirty = true;
  *slot = s;
  return NBODY_OK;
}

int nbody_batch_evict(nbody_batch *b, int slot) {
  int rc = check_slot(b, slot);
  if (rc) return rc;
  BCK(cudaSetDevice(b->device));
  SimHost &h = b->sims[slot];
  k_fill_i32<<<(unsigned)std::min<int64_t>((h.n + 255) / 256, 1024), 256, 0, b->st>>>(b->sim_of + h.off, h.n, -1);
  BCK(cudaGetLastError());
  b->launches++;
  give_range(b, h.off, h.n);
  h = SimHost();
  b->dirty = true;
  return NBODY_OK;
}

static int batch_step_impl(nbody_batch *b, int64_t nticks);

int nbody_batch_step(nbody_batch *b, int64_t nticks) {
  if (!b || nticks < 0) return bfail(NBODY_EINVAL, "batch step");
  BCK(cudaSetDevice(b->device));
  nvtxRangePushA("nbody_batch_step");
  const int rc = batch_step_impl(b, nticks);
  nvtxRangePop();
  return rc;
}

static int batch_step_impl(nbody_batch *b, int64_t nticks) {
  for (int64_t t = 0; t < nticks; t++) {
    if (b->dirty) {
      int rc = build_tables(b);
      if (rc) return rc;
    }
    if (b->n64 + b->nmx + b->nfe == 0) return NBODY_OK;
    cudaEvent_t e[2 + 2 * NCLS] = {};
    if (b->prof)
      for (int k = 0; k < 2 + 2 * NCLS; k++)
        if (!(e[k] = next_event(b))) return bfail(NBODY_ECUDA, "event");
    const int tb = b->tb;
    if (b->prof) BCK(cudaEventRecord(e[0], b->st));
    if (b->nmx) {
      if (b->prof) BCK(cudaEventRecord(e[4], b->st));
      BCK(nb::launch_mixed_prep_units(b->F, b->d_prep[tb], b->nprep, b->fpos, b->anchor, b->st));
      BCK(nb::launch_force_units(NBODY_MIXED, b->F, b->fpos, b->anchor, b->d_units[tb] + b->n64,
                                 b->nmx, b->r_mode[1], b->part, 0, b->st));
      if (b->prof) BCK(cudaEventRecord(e[5], b->st));
      b->launches += 2;
    }
    if (b->nfe) {
      if (b->prof) BCK(cudaEventRecord(e[6], b->st));
      BCK(nb::launch_mixed_prep_units(b->F, b->d_prep[tb] + b->nprep, b->nprepfe, b->fposff,
                                      b->anchor, b->st, true));
      BCK(nb::launch_force_units(NBODY_F64E, b->F, b->fposff, b->anchor,
                                 b->d_units[tb] + b->n64 + b->nmx, b->nfe, b->r_mode[2], b->part, 0,
                                 b->st));
      if (b->prof) BCK(cudaEventRecord(e[7], b->st));
      b->launches += 2;
    }
    if (b->n64) {
      if (b->prof) BCK(cudaEventRecord(e[2], b->st));
      // FP64 blocks are long and need few warps to keep the FP64 pipe busy: a
      // persistent grid of fp64_per_sm blocks per SM leaves the rest of each
      // SM to FP32-bound work running on other streams (another pool's ticks)
      BCK(nb::launch_force_units(NBODY_FP64, b->F, nullptr, nullptr, b->d_units[tb], b->n64,
                                 b->r_mode[0], b->part, (int64_t)b->fp64_per_sm * b->sms, b->st));
      if (b->prof) BCK(cudaEventRecord(e[3], b->st));
      b->launches++;
    }
    const unsigned g = (unsigned)std::min<int64_t>((b->hi + 255) / 256, (int64_t)b->sms * 32);
    k_batch_kdk<<<g, 256, 0, b->st>>>(b->sim_of, b->d_sims[tb], b->hi, b->part, b->R, b->F, b->V,
                                      b->VB, b->A);
    BCK(cudaGetLastError());
    b->launches++;
    if (b->prof) BCK(cudaEventRecord(e[1], b->st));
    // bookkeeping: every active simulation advanced one step, except first ticks (a(t0) only)
    bool any_init = false;
    double inter[NCLS] = {0, 0, 0};
    for (auto &h : b->sims) {
      if (!(h.used && h.active)) continue;
      inter[cls_of(h.mode)] += (double)h.n * (double)h.n;
      if (h.init) {
        h.init = false;
        any_init = true;
      } else {
        h.steps++;
      }
    }
    if (b->prof) {
      b->tick_inter[0].push_back(b->n64 ? inter[0] : 0);
      b->tick_inter[1].push_back(b->nmx ? inter[1] : 0);
      b->tick_inter[2].push_back(b->nfe ? inter[2] : 0);
    }
    if (any_init) b->dirty = true;  // the INIT flags must be cleared in the device table
  }
  return NBODY_OK;
}

int nbody_batch_query(nbody_batch *b) {
  if (!b) return bfail(NBODY_EINVAL, "NULL batch");
  BCK(cudaSetDevice(b->device));
  const cudaError_t e = cudaStreamQuery(b->st);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return bfail(NBODY_ECUDA, "cudaStreamQuery", e);
}

int nbody_batch_sync(nbody_batch *b) {
  if (!b) return bfail(NBODY_EINVAL, "NULL batch");
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(b->st));
  return NBODY_OK;
}

int nbody_batch_get_state(nbody_batch *b, int slot, double *pos, double *vel, double *t,
                          int64_t *step, int on_device) {
  int rc = check_slot(b, slot);
  if (rc) return rc;
  BCK(cudaSetDevice(b->device));
  const SimHost &h = b->sims[slot];
  const size_t n = (size_t)h.n;
  if (pos || vel) {
    double *dp = on_device ? pos : (pos ? b->stage : nullptr);
    double *dv = on_device ? vel : (vel ? b->stage + 3 * n : nullptr);
    BCK(nb::launch_unpack_state(NBODY_FP64, b->R + h.off, b->V + h.off, h.n, dp, dv, b->st));
    b->launches++;
    if (!on_device) {
      if (pos) BCK(cudaMemcpyAsync(pos, b->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, b->st));
      if (vel) BCK(cudaMemcpyAsync(vel, b->stage + 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, b->st));
    }
  }
  if (t) *t = (double)h.steps * h.dt;
  if (step) *step = h.steps;
  BCK(cudaStreamSynchronize(b->st));
  return NBODY_OK;
}

int nbody_batch_get_accel(nbody_batch *b, int slot, double *acc, double *pot, int on_device) {
  int rc = check_slot(b, slot);
  if (rc) return rc;
  BCK(cudaSetDevice(b->device));
  const SimHost &h = b->sims[slot];
  if (h.init) return bfail(NBODY_ESTATE, "no force evaluated yet for this slot");
  const size_t n = (size_t)h.n;
  double *da = on_device ? acc : (acc ? b->stage : nullptr);
  double *dq = on_device ? pot : (pot ? b->stage + 3 * n : nullptr);
  BCK(nb::launch_unpack_acc(NBODY_FP64, b->A + h.off, h.n, da, dq, b->st));
  b->launches++;
  if (!on_device) {
    if (acc) BCK(cudaMemcpyAsync(acc, b->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, b->st));
    if (pot) BCK(cudaMemcpyAsync(pot, b->stage + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost, b->st));
  }
  BCK(cudaStreamSynchronize(b->st));
  return NBODY_OK;
}

int nbody_batch_diagnostics(nbody_batch *b, int slot, double *E, double *K, double *W, double *P,
                            double *L) {
  int rc = check_slot(b, slot);
  if (rc) return rc;
  BCK(cudaSetDevice(b->device));
  const SimHost &h = b->sims[slot];
  if (h.init) return bfail(NBODY_ESTATE, "no force evaluated yet for this slot");
  const int nbk = nb::diag_blocks(h.n);
  BCK(nb::launch_diag(NBODY_FP64, b->R + h.off, b->V + h.off, b->A + h.off, h.n, b->diag_blocks, nbk,
                      b->diag_out, b->st));
  b->launches += 2;
  BCK(cudaMemcpyAsync(b->h_diag, b->diag_out, 9 * sizeof(double), cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  const double *o = b->h_diag;
  if (E) *E = o[0];
  if (K) *K = o[1];
  if (W) *W = o[2];
  if (P) memcpy(P, o + 3, 3 * sizeof(double));
  if (L) memcpy(L, o + 6, 3 * sizeof(double));
  return NBODY_OK;
}

int nbody_batch_info(nbody_batch *b, int *active, int64_t *used, int64_t *largest_free) {
  if (!b) return bfail(NBODY_EINVAL, "NULL batch");
  int a = 0;
  int64_t u = 0, lf = 0;
  for (auto &h : b->sims)
    if (h.used) {
      a++;
      u += round_up(h.n, ALIGN);
    }
  for (auto &r : b->free_ranges) lf = std::max(lf, r.second);
  if (active) *active = a;
  if (used) *used = u;
  if (largest_free) *largest_free = lf;
  return NBODY_OK;
}

int nbody_batch_slot_info(nbody_batch *b, int slot, int64_t *n, int *mode, int64_t *steps) {
  int rc = check_slot(b, slot);
  if (rc) return rc;
  const SimHost &h = b->sims[slot];
  if (n) *n = h.n;
  if (mode) *mode = h.mode;
  if (steps) *steps = h.steps;
  return NBODY_OK;
}

int nbody_batch_set_launch(nbody_batch *b, int mode, int ipt, int64_t seg) {
  if (!b) return bfail(NBODY_EINVAL, "NULL batch");
  if (mode != NBODY_FP64 && mode != NBODY_MIXED && mode != NBODY_F64E) return bfail(NBODY_EINVAL, "mode");
  if (ipt != 1 && ipt != 2 && ipt != 4 && ipt != 8) return bfail(NBODY_EINVAL, "ipt");
  if (seg < 1) return bfail(NBODY_EINVAL, "seg");
  const int m = cls_of(mode);
  if (b->r_mode[m] != ipt || b->seg_mode[m] != seg) {
    b->r_mode[m] = ipt;
    b->seg_mode[m] = seg;
    b->dirty = true;
  }
  return NBODY_OK;
}

int nbody_batch_set_fp64_residency(nbody_batch *b, int blocks_per_sm) {
  if (!b || blocks_per_sm < 0 || blocks_per_sm > 64) return bfail(NBODY_EINVAL, "blocks_per_sm");
  b->fp64_per_sm = blocks_per_sm;
  return NBODY_OK;
}

int nbody_batch_profile(nbody_batch *b, int enable) {
  if (!b) return bfail(NBODY_EINVAL, "NULL batch");
  b->prof = enable != 0;
  return NBODY_OK;
}

// Per-tick timings since the last read (synchronises): up to `cap` ticks of
// tick_ms (whole tick), force_ms[3*k..3*k+2] (FP64, MIXED, F64E force
// launches, 0 when absent) and inter[3*k..] (interactions of each class in
// tick k).  *nticks receives the number of ticks recorded (all are consumed).
int nbody_batch_profile_read(nbody_batch *b, int64_t cap, double *tick_ms, double *force_ms,
                             double *inter, int64_t *nticks) {
  if (!b) return bfail(NBODY_EINVAL, "NULL batch");
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(b->st));
  const int64_t nt = (int64_t)b->tick_inter[0].size();
  for (int64_t k = 0; k < nt && k < cap; k++) {
    cudaEvent_t *e = &b->evs[(2 + 2 * NCLS) * k];
    float ms = 0;
    BCK(cudaEventElapsedTime(&ms, e[0], e[1]));
    if (tick_ms) tick_ms[k] = ms;
    for (int m = 0; m < NCLS; m++) {
      float f = 0;
      if (b->tick_inter[m][k] > 0) BCK(cudaEventElapsedTime(&f, e[2 + 2 * m], e[3 + 2 * m]));
      if (force_ms) force_ms[NCLS * k + m] = f;
      if (inter) inter[NCLS * k + m] = b->tick_inter[m][k];
    }
  }
  if (nticks) *nticks = nt;
  for (int m = 0; m < NCLS; m++) b->tick_inter[m].clear();
  b->ev_used = 0;
  return NBODY_OK;
}

int64_t nbody_batch_launch_count(const nbody_batch *b) { return b ? b->launches : 0; }

}  // extern "C"
