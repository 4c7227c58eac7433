// C ABI of the library (declared in include/nbody.h): simulation contexts,
// state transfer, the Eq. 1-2 force call, KDK (Eq. 5-7) and RK4 stepping, and
// the Eq. 8-10 diagnostics.  All device work is issued on the context's
// stream; nothing here computes on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nbody_internal.cuh"

using nb::d4;

struct nbody_ctx {
  int64_t n = 0;
  int mode = NBODY_FP64;
  double eps = 0, G = 1;
  cudaStream_t st = nullptr;
  int device = 0;
  int num_sms = 0;
  void *posm[2] = {nullptr, nullptr};
  int cur = 0;
  void *vel = nullptr, *vbar = nullptr, *acc = nullptr;
  void *part = nullptr;
  int part_slices = 0;
  void *rk_vs = nullptr, *rk_sr = nullptr, *rk_sv = nullptr;
  void *tmp_posm = nullptr, *tmp_acc = nullptr;
  float4 *fpos = nullptr, *anchor = nullptr;
  double *diag_blocks = nullptr, *diag_out = nullptr, *h_diag = nullptr;
  int *d_flag = nullptr, *h_flag = nullptr;
  double *stage = nullptr;  // device staging of host arrays (n x 7 doubles)
  bool has_state = false, acc_valid = false, pred_valid = false;
  double pred_dt = 0;
  double t = 0;
  int64_t step = 0;
  nb::Shape shape;
  double timeout_s = 0;
  int64_t launches = 0;
  bool prof = false;
  // FP64 each-pair-once path: -1 auto, 0 off, 1 on; diagonal-block units,
  // per-diagonal row/column buffers (2 x sym_d x n entries)
  int sym = -1;
  nb::Unit *sym_units = nullptr;
  int sym_units_m = 0;
  void *sym_buf = nullptr;
  int sym_d = 0;
  // particle order of the force sum: 0 = input order, 1 = spatial (Morton)
  // order; order scratch, sorted-to-input permutation, sorted positions and
  // the sorted partial sums (alt_slices slices of n)
  int order = 0;
  void *ord_scratch = nullptr;
  int32_t *perm = nullptr;
  d4 *sposm = nullptr;
  void *part_alt = nullptr;
  int alt_slices = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;  // all created events
  size_t ev_used = 0;                                          // pairs recorded since last read
};

// ---------------------------------------------------------------- errors
static thread_local char g_last[512] = "";

static int fail(int code, const char *what, cudaError_t ce = cudaSuccess) {
  if (ce != cudaSuccess)
    snprintf(g_last, sizeof g_last, "%s: %s (%s)", nbody_strerror(code), what,
             cudaGetErrorString(ce));
  else
    snprintf(g_last, sizeof g_last, "%s: %s", nbody_strerror(code), what);
  return code;
}

int nb::record_error(int code, const char *what, cudaError_t ce) { return fail(code, what, ce); }

#define CK(call)                                                         \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return fail(NBODY_ECUDA, #call, e_);          \
  } while (0)

// ---------------------------------------------------------------- helpers
static size_t r4(const nbody_ctx *c) { return 4 * nb::real_bytes(c->mode); }
static size_t part_r4(const nbody_ctx *c) {
  return c->mode == NBODY_FP32 ? sizeof(float4) : sizeof(d4);
}

static int sync(nbody_ctx *c) {
  if (c->timeout_s <= 0) {
    CK(cudaStreamSynchronize(c->st));
    return NBODY_OK;
  }
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(c->st);
    if (e == cudaSuccess) return NBODY_OK;
    if (e != cudaErrorNotReady) return fail(NBODY_ECUDA, "cudaStreamQuery", e);
    double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > c->timeout_s) return fail(NBODY_ETIMEOUT, "stream did not finish within the timeout");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// Default launch shape: enough thread blocks to fill every SM several times.
static void default_shape(nbody_ctx *c, nb::Shape &sh, int r_req, int s_req) {
  sh = nb::Shape();
  sh.bt = nb::force_block_threads(c->mode);
  sh.t = nb::force_tile(c->mode);
  // measured on GB300: FP64 is FP64-pipe bound at any R; the packed FP32 and
  // float-float kernels keep enough warps resident only at R = 2
  int r = r_req ? r_req : (c->mode == NBODY_FP64 ? 4 : 2);
  if (c->mode == NBODY_F64E && r > 4) r = 4;
  while (!r_req && r > 1 && (int64_t)sh.bt * r * c->num_sms > c->n) r >>= 1;
  sh.r = r;
  const int64_t bx = (c->n + (int64_t)sh.bt * r - 1) / ((int64_t)sh.bt * r);
  const int64_t smax = (c->n + sh.t - 1) / sh.t;
  int64_t s = s_req;
  if (!s) {
    int occ = nb::force_max_blocks_per_sm(c->mode, sh);
    if (occ < 1) occ = 1;
    const int64_t target = 8LL * c->num_sms * occ;
    s = (target + bx - 1) / bx;
  }
  if (s > smax) s = smax;
  if (s > 64) s = 64;
  if (s < 1) s = 1;
  sh.s = (int)s;
}

// segment length (a multiple of the tile) and the segment count it implies
static int64_t seg_len(const nbody_ctx *c, int &S) {
  int64_t seg = (c->n + c->shape.s - 1) / c->shape.s;
  seg = (seg + c->shape.t - 1) / c->shape.t * c->shape.t;
  S = (int)((c->n + seg - 1) / seg);
  return seg;
}

static int ensure_slices(nbody_ctx *c, void **buf, int *have, int S) {
  if (S <= *have) return NBODY_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  if (cudaMalloc(buf, (size_t)S * c->n * part_r4(c)) != cudaSuccess)
    return fail(NBODY_ENOMEM, "j-segment partial buffer");
  *have = S;
  return NBODY_OK;
}

// S slices of partial sums in c->part and, with the spatial order, as many in
// c->part_alt (the force kernels write there; the slices are then moved to
// input order in c->part).
static int ensure_part(nbody_ctx *c, int S) {
  int rc = ensure_slices(c, &c->part, &c->part_slices, S);
  if (!rc && c->order) rc = ensure_slices(c, &c->part_alt, &c->alt_slices, S);
  return rc;
}

// The force kernels' output slices for this evaluation.
static void *force_out(const nbody_ctx *c) { return c->order ? c->part_alt : c->part; }

// Blocks (of sym_block_particles()) below which the automatic choice keeps
// the one-sided kernel: with few blocks the diagonals hold too few work items
// to fill the GPU (measured on GB300 with blocks of 512: 43.6 against 55.9
// Gint/s at 32 blocks, N = 2^14; 68.5 against 56.6 at 64 blocks, N = 2^15).
static const int SYM_AUTO_MIN_BLOCKS = 64;

static int sym_block(const nbody_ctx *c) {
  return c->mode == NBODY_F64E ? nb::sym_block_particles_ff() : nb::sym_block_particles();
}

static int sym_blocks(const nbody_ctx *c) {
  const int B = sym_block(c);
  return (int)((c->n + B - 1) / B);
}

static bool use_sym(const nbody_ctx *c) {
  if ((c->mode != NBODY_FP64 && c->mode != NBODY_F64E) || c->sym == 0) return false;
  return c->sym == 1 ? sym_blocks(c) >= 2 : sym_blocks(c) >= SYM_AUTO_MIN_BLOCKS;
}

// FP64 and F64E, each pair once: slices 0..P-1 of c->part = pairs inside each
// block (the one-sided kernel on the M diagonal blocks, each block's j range in
// P parts), slice P = row sums and slice P+1 = column sums of the M (M - 1) / 2
// pairs of distinct blocks, added over the block diagonals in order.  F64E
// blocks are its float-float tiles.
static int force_sym(nbody_ctx *c, const void *posm_in, int &S) {
  const bool ff = c->mode == NBODY_F64E;
  const int B = sym_block(c);
  const int M = sym_blocks(c);
  const int nd = M / 2;
  // pairs inside the diagonal blocks: each block's j range in P parts (one
  // unit each, partial sums in slices 0..P-1) so that the one-sided launch has
  // at least two work items per resident block slot
  const int ur = ff ? nb::sym_r_ff() : nb::sym_units_r();  // one-sided R covering a block
  const int per_sm_1 = nb::force_max_blocks_per_sm(c->mode, nb::Shape{nb::force_block_threads(c->mode),
                                                                      ur, nb::force_tile(c->mode), 1});
  const int64_t slots_1 = (int64_t)c->num_sms * std::max(1, per_sm_1);
  const int64_t want = (2 * slots_1 + M - 1) / M;
  int P = 1;  // a power of two dividing the block size
  while (P < want && P < (ff ? 2 : 4)) P *= 2;
  int rc = ensure_part(c, P + 2);
  if (rc) return rc;
  void *out = force_out(c);  // only after ensure_part, which may (re)allocate it
  if (c->sym_units_m != M * P) {
    if (c->sym_units) cudaFree(c->sym_units);
    c->sym_units = nullptr;
    c->sym_units_m = 0;
    std::vector<nb::Unit> u((size_t)M * P);
    const int64_t len = B / P;
    for (int I = 0; I < M; I++)
      for (int q = 0; q < P; q++) {
        nb::Unit &v = u[(size_t)q * M + I];
        v.i0 = (int64_t)I * B;
        v.ni = (int32_t)std::min<int64_t>(B, c->n - v.i0);
        v.j0 = v.i0 + q * len;
        const int64_t part_len = q == P - 1 ? B - q * len : len;  // the last part takes any remainder
        v.nj = (int32_t)std::max<int64_t>(0, std::min<int64_t>(part_len, c->n - v.j0));
        v.out = (int64_t)q * c->n + v.i0;
        v.anchor = ff ? I : 0;  // F64E: block I is float-float tile I
        v.eps2 = c->eps * c->eps;
      }
    if (cudaMalloc(&c->sym_units, sizeof(nb::Unit) * M * P) != cudaSuccess)
      return fail(NBODY_ENOMEM, "diagonal-block units");
    CK(cudaMemcpy(c->sym_units, u.data(), sizeof(nb::Unit) * M * P, cudaMemcpyHostToDevice));
    c->sym_units_m = M * P;
  }
  if (!c->sym_d && nd > 0) {
    // enough work items per launch for ~32 waves, within 1 GiB of buffers
    const int per_sm = ff ? nb::sym_blocks_per_sm_ff() : nb::sym_blocks_per_sm();
    const int64_t slots = (int64_t)c->num_sms * std::max(1, per_sm);
    int64_t D = (32 * slots + M - 1) / M;
    const int64_t cap = std::max<int64_t>(1, ((int64_t)1 << 30) / (64 * c->n));
    D = std::max<int64_t>(1, std::min<int64_t>({D, cap, (int64_t)nd}));
    if (cudaMalloc(&c->sym_buf, (size_t)2 * D * c->n * sizeof(nb::d4)) != cudaSuccess)
      return fail(NBODY_ENOMEM, "row/column buffers");
    c->sym_d = (int)D;
  }
  if (ff) {
    CK(nb::launch_mixed_prep((const nb::d4 *)posm_in, c->n, nb::force_tile(NBODY_F64E), c->fpos,
                             c->anchor, c->st, true));
    c->launches++;
  }
  CK(nb::launch_force_units(c->mode, posm_in, c->fpos, c->anchor, c->sym_units, (int64_t)M * P, ur,
                            out, 0, c->st));
  c->launches++;
  S = P;
  if (nd == 0) return NBODY_OK;
  nb::d4 *part = (nb::d4 *)out + (int64_t)(P - 1) * c->n;  // rows in slice P, columns in P + 1
  nb::d4 *rows = (nb::d4 *)c->sym_buf, *cols = rows + (int64_t)c->sym_d * c->n;
  for (int d0 = 1; d0 <= nd; d0 += c->sym_d) {
    const int D = std::min(c->sym_d, nd - d0 + 1);
    if (ff)
      CK(nb::launch_force_f64e_sym((const nb::d4 *)posm_in, c->fpos, c->anchor, c->n,
                                   c->eps * c->eps, M, d0, D, rows, cols, c->st));
    else
      CK(nb::launch_force_f64_sym((const nb::d4 *)posm_in, c->n, c->eps * c->eps, M, d0, D, rows,
                                  cols, c->st));
    CK(nb::launch_sym_combine(rows, cols, D, c->n, part + c->n, part + 2 * c->n, d0 == 1, c->st));
    c->launches += 2;
  }
  S = P + 2;
  return NBODY_OK;
}

static int ensure_order(nbody_ctx *c) {
  if (c->perm) return NBODY_OK;
  if (cudaMalloc(&c->ord_scratch, nb::order_scratch_bytes(c->n)) != cudaSuccess ||
      cudaMalloc(&c->perm, sizeof(int32_t) * c->n) != cudaSuccess ||
      cudaMalloc(&c->sposm, sizeof(d4) * c->n) != cudaSuccess) {
    cudaGetLastError();
    return fail(NBODY_ENOMEM, "spatial order buffers");
  }
  return NBODY_OK;
}

static int force_sums(nbody_ctx *c, const void *posm_in, int &S);

// Raw force sums of the positions in posm_in into c->part (input order);
// returns the number of partial slices written through S.  With the spatial
// order the particles are sorted along a Morton curve first, the force
// kernels run on the sorted copy, and their slices are scattered back.
static int force(nbody_ctx *c, const void *posm_in, int &S) {
  if (!c->order) return force_sums(c, posm_in, S);
  int rc = ensure_order(c);
  if (rc) return rc;
  CK(nb::launch_spatial_order((const d4 *)posm_in, c->n, c->ord_scratch, c->perm, c->sposm, c->st));
  c->launches += 4;
  rc = force_sums(c, c->sposm, S);
  if (rc) return rc;
  CK(nb::launch_unpermute((const d4 *)c->part_alt, c->perm, S, c->n, (d4 *)c->part, c->st));
  c->launches++;
  return NBODY_OK;
}

// The force kernels on posm_in, partial slices into force_out(c).
static int force_sums(nbody_ctx *c, const void *posm_in, int &S) {
  std::pair<cudaEvent_t, cudaEvent_t> *ev = nullptr;
  if (c->prof) {
    if (c->ev_used == c->ev_pool.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> p;
      CK(cudaEventCreate(&p.first));
      CK(cudaEventCreate(&p.second));
      c->ev_pool.push_back(p);
    }
    ev = &c->ev_pool[c->ev_used++];
  }
  if (use_sym(c)) {
    if (ev) CK(cudaEventRecord(ev->first, c->st));
    int rc = force_sym(c, posm_in, S);
    if (rc) return rc;
    if (ev) CK(cudaEventRecord(ev->second, c->st));
    return NBODY_OK;
  }
  const int64_t seg = seg_len(c, S);
  int rc = ensure_part(c, S);
  if (rc) return rc;
  if (c->mode == NBODY_MIXED || c->mode == NBODY_F64E) {
    CK(nb::launch_mixed_prep((const d4 *)posm_in, c->n, c->shape.t, c->fpos, c->anchor, c->st,
                             c->mode == NBODY_F64E));
    c->launches++;
  }
  nb::ForceIn in;
  in.posm = posm_in;
  in.fpos = c->fpos;
  in.anchor = c->anchor;
  in.n = c->n;
  in.eps2 = c->eps * c->eps;
  in.seg = seg;
  in.part = force_out(c);
  nb::Shape sh = c->shape;
  sh.s = S;
  if (ev) CK(cudaEventRecord(ev->first, c->st));
  CK(nb::launch_force(c->mode, in, sh, c->st));
  c->launches++;
  if (ev) CK(cudaEventRecord(ev->second, c->st));
  return NBODY_OK;
}

static nb::EpiIn epi(const nbody_ctx *c, int S) {
  nb::EpiIn e;
  e.n = c->n;
  e.S = S;
  e.part = c->part;
  e.G = c->G;
  return e;
}

static int ensure_acc(nbody_ctx *c) {
  if (c->acc_valid) return NBODY_OK;
  int S = 0;
  int rc = force(c, c->posm[c->cur], S);
  if (rc) return rc;
  CK(nb::launch_store_acc(c->mode, epi(c, S), c->acc, c->st));
  c->launches++;
  c->acc_valid = true;
  return NBODY_OK;
}

static int ensure_stage(nbody_ctx *c) {
  if (c->stage) return NBODY_OK;
  if (cudaMalloc(&c->stage, sizeof(double) * 7 * (size_t)c->n) != cudaSuccess)
    return fail(NBODY_ENOMEM, "host staging buffer");
  return NBODY_OK;
}

static void free_all(nbody_ctx *c) {
  for (auto &p : c->ev_pool) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  c->ev_pool.clear();
  void *ptrs[] = {c->posm[0], c->posm[1], c->vel, c->vbar, c->acc, c->part, c->rk_vs, c->rk_sr,
                  c->rk_sv, c->tmp_posm, c->tmp_acc, c->fpos, c->anchor, c->diag_blocks,
                  c->diag_out, c->d_flag, c->stage, c->sym_units, c->sym_buf,
                  c->ord_scratch, c->perm, c->sposm, c->part_alt};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->h_diag) cudaFreeHost(c->h_diag);
  if (c->h_flag) cudaFreeHost(c->h_flag);
}

// ---------------------------------------------------------------- ABI
extern "C" {

int nbody_version(void) { return 100; }

const char *nbody_strerror(int code) {
  switch (code) {
    case NBODY_OK: return "ok";
    case NBODY_EINVAL: return "invalid argument";
    case NBODY_ENOMEM: return "out of memory";
    case NBODY_ECUDA: return "CUDA error";
    case NBODY_ETIMEOUT: return "timed out";
    case NBODY_ESTATE: return "state not set";
    case NBODY_ENOSPC: return "no free slot or memory";
    default: return "unknown error";
  }
}

const char *nbody_last_error(void) { return g_last; }

int nbody_create(nbody_ctx **out, int64_t n, int mode, double eps, double G, void *cuda_stream) {
  if (!out) return fail(NBODY_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1) return fail(NBODY_EINVAL, "n < 1");
  if (mode != NBODY_FP64 && mode != NBODY_MIXED && mode != NBODY_FP32 && mode != NBODY_F64E)
    return fail(NBODY_EINVAL, "unknown mode");
  if (!(eps >= 0) || !std::isfinite(eps)) return fail(NBODY_EINVAL, "eps must be finite and >= 0");
  if (!std::isfinite(G)) return fail(NBODY_EINVAL, "G must be finite");
  if (mode == NBODY_FP32 && eps * eps < 1.1754943508222875e-38 && eps != 0)
    return fail(NBODY_EINVAL, "eps^2 underflows binary32");
  nbody_ctx *c = new (std::nothrow) nbody_ctx;
  if (!c) return fail(NBODY_ENOMEM, "context");
  c->n = n;
  c->mode = mode;
  c->eps = eps;
  c->G = G;
  c->st = (cudaStream_t)cuda_stream;
  cudaError_t ce = cudaGetDevice(&c->device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (ce != cudaSuccess) {
    delete c;
    return fail(NBODY_ECUDA, "no CUDA device", ce);
  }
  const size_t b4 = (size_t)n * r4(c);
  bool ok = cudaMalloc(&c->posm[0], b4) == cudaSuccess && cudaMalloc(&c->posm[1], b4) == cudaSuccess &&
            cudaMalloc(&c->vel, b4) == cudaSuccess && cudaMalloc(&c->vbar, b4) == cudaSuccess &&
            cudaMalloc(&c->acc, b4) == cudaSuccess && cudaMalloc(&c->d_flag, sizeof(int)) == cudaSuccess &&
            cudaMallocHost(&c->h_flag, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->diag_out, 16 * sizeof(double)) == cudaSuccess &&
            cudaMallocHost(&c->h_diag, 16 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->diag_blocks, (size_t)nb::diag_blocks(n) * 8 * sizeof(double)) == cudaSuccess;
  if (ok && (mode == NBODY_MIXED || mode == NBODY_F64E)) {
    const int64_t tiles = (n + 255) / 256;
    const size_t per = mode == NBODY_F64E ? 2 : 1;  // float4 per particle
    ok = cudaMalloc(&c->fpos, (size_t)n * per * sizeof(float4)) == cudaSuccess &&
         cudaMalloc(&c->anchor, (size_t)tiles * 2 * sizeof(float4)) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return fail(NBODY_ENOMEM, "device state");
  }
  default_shape(c, c->shape, 0, 0);
  c->order = (mode == NBODY_MIXED || mode == NBODY_F64E) ? 1 : 0;
  *out = c;
  return NBODY_OK;
}

int nbody_destroy(nbody_ctx *c) {
  if (!c) return NBODY_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->st);
  free_all(c);
  delete c;
  return NBODY_OK;
}

int nbody_set_timeout(nbody_ctx *c, double seconds) {
  if (!c || !(seconds >= 0)) return fail(NBODY_EINVAL, "timeout");
  c->timeout_s = seconds;
  return NBODY_OK;
}

// pos/vel/mass into dst_posm/dst_vel (device layout), validated; host arrays
// go through the staging buffer.
static int load_arrays(nbody_ctx *c, const double *pos, const double *vel, const double *mass,
                       int on_device, void *dst_posm, void *dst_vel, bool check) {
  const double *dp = pos, *dv = vel, *dm = mass;
  const size_t n = (size_t)c->n;
  if (!on_device) {
    int rc = ensure_stage(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->stage, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->stage + 3 * n, mass, n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    dp = c->stage;
    dm = c->stage + 3 * n;
    if (vel) {
      CK(cudaMemcpyAsync(c->stage + 4 * n, vel, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->st));
      dv = c->stage + 4 * n;
    }
  }
  if (check) CK(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->st));
  CK(nb::launch_pack(c->mode, dp, dv, dm, c->n, dst_posm, dst_vel, check ? c->d_flag : nullptr, c->st));
  c->launches++;
  if (check) {
    CK(cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    int rc = sync(c);
    if (rc) return rc;
    if (*c->h_flag) return fail(NBODY_EINVAL, "non-finite position/velocity/mass or negative mass");
  }
  return NBODY_OK;
}

int nbody_set_state(nbody_ctx *c, const double *pos, const double *vel, const double *mass,
                    int on_device) {
  if (!c || !pos || !mass) return fail(NBODY_EINVAL, "NULL argument");
  CK(cudaSetDevice(c->device));
  // load into the spare buffer first so that a rejected input keeps the old
  // state; the spare buffer held the next KDK predictor, rebuilt on demand
  c->pred_valid = false;
  const int spare = 1 - c->cur;
  void *vtmp = c->vbar;  // vbar is rebuilt by the next KDK step anyway
  int rc = load_arrays(c, pos, vel, mass, on_device, c->posm[spare], vtmp, true);
  if (rc) return rc;
  c->cur = spare;
  CK(cudaMemcpyAsync(c->vel, vtmp, (size_t)c->n * r4(c), cudaMemcpyDeviceToDevice, c->st));
  c->has_state = true;
  c->acc_valid = false;
  c->pred_valid = false;
  c->t = 0;
  c->step = 0;
  return sync(c);
}

int nbody_set_clock(nbody_ctx *c, double t, int64_t step) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (!std::isfinite(t) || step < 0) return fail(NBODY_EINVAL, "t must be finite and step >= 0");
  c->t = t;
  c->step = step;
  return NBODY_OK;
}

int nbody_get_state(nbody_ctx *c, double *pos, double *vel, double *t, int64_t *step,
                    int on_device) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (!c->has_state) return fail(NBODY_ESTATE, "get_state before set_state");
  CK(cudaSetDevice(c->device));
  const size_t n = (size_t)c->n;
  if (pos || vel) {
    if (on_device) {
      CK(nb::launch_unpack_state(c->mode, c->posm[c->cur], c->vel, c->n, pos, vel, c->st));
      c->launches++;
    } else {
      int rc = ensure_stage(c);
      if (rc) return rc;
      CK(nb::launch_unpack_state(c->mode, c->posm[c->cur], c->vel, c->n, pos ? c->stage : nullptr,
                                 vel ? c->stage + 3 * n : nullptr, c->st));
      c->launches++;
      if (pos) CK(cudaMemcpyAsync(pos, c->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      if (vel)
        CK(cudaMemcpyAsync(vel, c->stage + 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    }
  }
  if (t) *t = c->t;
  if (step) *step = c->step;
  return sync(c);
}

static int copy_acc_out(nbody_ctx *c, const void *accbuf, double *acc, double *pot, int on_device,
                        int64_t count = -1) {
  const size_t n = (size_t)(count < 0 ? c->n : count);
  if (on_device) {
    CK(nb::launch_unpack_acc(c->mode, accbuf, (int64_t)n, acc, pot, c->st));
    c->launches++;
  } else {
    int rc = ensure_stage(c);
    if (rc) return rc;
    CK(nb::launch_unpack_acc(c->mode, accbuf, (int64_t)n, acc ? c->stage : nullptr,
                             pot ? c->stage + 3 * n : nullptr, c->st));
    c->launches++;
    if (acc) CK(cudaMemcpyAsync(acc, c->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (pot) CK(cudaMemcpyAsync(pot, c->stage + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  return sync(c);
}

int nbody_accel(nbody_ctx *c, const double *pos, const double *mass, double *acc, double *pot,
                int on_device) {
  if (!c || !pos || !mass || !acc) return fail(NBODY_EINVAL, "NULL argument");
  CK(cudaSetDevice(c->device));
  if (!c->tmp_posm) {
    if (cudaMalloc(&c->tmp_posm, (size_t)c->n * r4(c)) != cudaSuccess ||
        cudaMalloc(&c->tmp_acc, (size_t)c->n * r4(c)) != cudaSuccess)
      return fail(NBODY_ENOMEM, "accel buffers");
  }
  nvtxRangePushA("nbody_accel");
  int rc = load_arrays(c, pos, nullptr, mass, on_device, c->tmp_posm, nullptr, false);
  int S = 0;
  if (!rc) rc = force(c, c->tmp_posm, S);
  nvtxRangePop();
  if (rc) return rc;
  CK(nb::launch_store_acc(c->mode, epi(c, S), c->tmp_acc, c->st));
  c->launches++;
  return copy_acc_out(c, c->tmp_acc, acc, pot, on_device);
}

int nbody_accel_rows(nbody_ctx *c, int64_t i0, int64_t ni, const double *pos, const double *mass,
                     double *acc, double *pot, int on_device) {
  if (!c || !pos || !mass || !acc) return fail(NBODY_EINVAL, "NULL argument");
  if (i0 < 0 || ni < 1 || i0 > c->n - ni) return fail(NBODY_EINVAL, "rows outside [0, n)");
  CK(cudaSetDevice(c->device));
  if (!c->tmp_posm) {
    if (cudaMalloc(&c->tmp_posm, (size_t)c->n * r4(c)) != cudaSuccess ||
        cudaMalloc(&c->tmp_acc, (size_t)c->n * r4(c)) != cudaSuccess)
      return fail(NBODY_ENOMEM, "accel buffers");
  }
  nvtxRangePushA("nbody_accel_rows");
  int rc = load_arrays(c, pos, nullptr, mass, on_device, c->tmp_posm, nullptr, false);
  int S = 0;
  const int64_t seg = seg_len(c, S);
  if (!rc) rc = ensure_part(c, S);
  nvtxRangePop();
  if (rc) return rc;
  // the one-sided kernels in input order, in the context's launch shape: the
  // rows come out as those rows of nbody_accel with the each-pair-once path
  // off and NBODY_ORDER_INPUT, bit for bit
  if (c->mode == NBODY_MIXED || c->mode == NBODY_F64E) {
    CK(nb::launch_mixed_prep((const d4 *)c->tmp_posm, c->n, c->shape.t, c->fpos, c->anchor, c->st,
                             c->mode == NBODY_F64E));
    c->launches++;
  }
  nb::ForceIn in;
  in.posm = c->tmp_posm;
  in.fpos = c->fpos;
  in.anchor = c->anchor;
  in.n = c->n;
  in.eps2 = c->eps * c->eps;
  in.seg = seg;
  in.part = c->part;
  in.i0 = i0;
  in.rows = ni;
  nb::Shape sh = c->shape;
  sh.s = S;
  CK(nb::launch_force(c->mode, in, sh, c->st));
  nb::EpiIn e = epi(c, S);
  e.n = ni;
  CK(nb::launch_store_acc(c->mode, e, c->tmp_acc, c->st));
  c->launches += 2;
  return copy_acc_out(c, c->tmp_acc, acc, pot, on_device, ni);
}

int nbody_get_accel(nbody_ctx *c, double *acc, double *pot, int on_device) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (!c->has_state) return fail(NBODY_ESTATE, "get_accel before set_state");
  CK(cudaSetDevice(c->device));
  int rc = ensure_acc(c);
  if (rc) return rc;
  if (!acc && !pot) return sync(c);
  return copy_acc_out(c, c->acc, acc, pot, on_device);
}

// nsteps steps of size dt, each a sequence of nh KDK steps (Eq. 5-7) of sizes
// h[0..nh-1] (KDK: one of dt; FR4: w1 dt, w0 dt, w1 dt).  Each force
// evaluation is followed by one fused kernel: the corrector of the KDK step
// that ended and the predictor of the next one.
static int step_kdk_seq(nbody_ctx *c, const double *h, int nh, double dt, int64_t nsteps) {
  int rc = ensure_acc(c);
  if (rc) return rc;
  const int nxt = 1 - c->cur;
  if (!(c->pred_valid && c->pred_dt == h[0])) {
    CK(nb::launch_kdk_predict(c->mode, c->n, h[0], c->posm[c->cur], c->vel, c->acc, c->vbar,
                              c->posm[nxt], c->st));
    c->launches++;
    c->pred_valid = true;
    c->pred_dt = h[0];
  }
  for (int64_t k = 0; k < nsteps; k++) {
    for (int s = 0; s < nh; s++) {
      const int a = c->cur, b = 1 - c->cur;  // posm[b] holds the predicted positions
      int S = 0;
      rc = force(c, c->posm[b], S);
      if (rc) return rc;
      CK(nb::launch_kdk_correct_predict(c->mode, epi(c, S), h[s], h[(s + 1) % nh], c->acc,
                                        c->posm[b], c->vel, c->vbar, c->posm[a], c->st));
      c->launches++;
      c->cur = b;
    }
    c->t += dt;
    c->step++;
  }
  return NBODY_OK;
}

static int step_kdk(nbody_ctx *c, double dt, int64_t nsteps) {
  return step_kdk_seq(c, &dt, 1, dt, nsteps);
}

// Fourth-order composition (Yoshida 1990; Forest and Ruth 1990): the weights
// are the binary64 roundings of 1/(2 - 2^(1/3)) and -2^(1/3)/(2 - 2^(1/3)).
static int step_fr4(nbody_ctx *c, double dt, int64_t nsteps) {
  const double w1 = 0x1.59e8b6eb96338p+0, w0 = -0x1.b3d16dd72c671p+0;
  const double h[3] = {w1 * dt, w0 * dt, w1 * dt};
  return step_kdk_seq(c, h, 3, dt, nsteps);
}

static int step_rk4(nbody_ctx *c, double dt, int64_t nsteps) {
  if (!c->rk_vs) {
    const size_t b4 = (size_t)c->n * r4(c);
    if (cudaMalloc(&c->rk_vs, b4) != cudaSuccess || cudaMalloc(&c->rk_sr, b4) != cudaSuccess ||
        cudaMalloc(&c->rk_sv, b4) != cudaSuccess)
      return fail(NBODY_ENOMEM, "RK4 stage buffers");
  }
  const int stg = 1 - c->cur;
  for (int64_t k = 0; k < nsteps; k++) {
    for (int stage = 1; stage <= 4; stage++) {
      int S = 0;
      int rc = force(c, stage == 1 ? c->posm[c->cur] : c->posm[stg], S);
      if (rc) return rc;
      CK(nb::launch_rk4_stage(c->mode, epi(c, S), stage, dt, c->posm[c->cur], c->vel, c->rk_vs,
                              c->rk_sr, c->rk_sv, c->posm[stg], c->st));
      c->launches++;
    }
    c->t += dt;
    c->step++;
  }
  if (nsteps > 0) {
    c->acc_valid = false;
    c->pred_valid = false;
  }
  return NBODY_OK;
}

int nbody_step(nbody_ctx *c, int scheme, double dt, int64_t nsteps) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (scheme != NBODY_KDK && scheme != NBODY_RK4 && scheme != NBODY_FR4)
    return fail(NBODY_EINVAL, "unknown scheme");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(NBODY_EINVAL, "dt must be finite and > 0");
  if (nsteps < 0) return fail(NBODY_EINVAL, "nsteps < 0");
  if (!c->has_state) return fail(NBODY_ESTATE, "step before set_state");
  CK(cudaSetDevice(c->device));
  nvtxRangePushA(scheme == NBODY_KDK ? "nbody_step KDK"
                 : scheme == NBODY_RK4 ? "nbody_step RK4" : "nbody_step FR4");
  const int rc = scheme == NBODY_KDK   ? step_kdk(c, dt, nsteps)
                 : scheme == NBODY_RK4 ? step_rk4(c, dt, nsteps)
                                       : step_fr4(c, dt, nsteps);
  nvtxRangePop();
  return rc;
}

int nbody_diagnostics_ext(nbody_ctx *c, double *E, double *K, double *W, double *P, double *L) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (!c->has_state) return fail(NBODY_ESTATE, "diagnostics before set_state");
  CK(cudaSetDevice(c->device));
  int rc = ensure_acc(c);
  if (rc) return rc;
  const int nbk = nb::diag_blocks(c->n);
  CK(nb::launch_diag(c->mode, c->posm[c->cur], c->vel, c->acc, c->n, c->diag_blocks, nbk,
                     c->diag_out, c->st));
  c->launches += 2;
  CK(cudaMemcpyAsync(c->h_diag, c->diag_out, 9 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  rc = sync(c);
  if (rc) return rc;
  const double *o = c->h_diag;
  if (E) *E = o[0];
  if (K) *K = o[1];
  if (W) *W = o[2];
  if (P) memcpy(P, o + 3, 3 * sizeof(double));
  if (L) memcpy(L, o + 6, 3 * sizeof(double));
  return NBODY_OK;
}

int nbody_diagnostics(nbody_ctx *c, double *E, double *P, double *L) {
  return nbody_diagnostics_ext(c, E, nullptr, nullptr, P, L);
}

int nbody_set_launch(nbody_ctx *c, int ipt, int jsplit) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (ipt != 0 && ipt != 1 && ipt != 2 && ipt != 4 && ipt != 8) return fail(NBODY_EINVAL, "ipt");
  if (jsplit < 0 || jsplit > 64) return fail(NBODY_EINVAL, "jsplit");
  CK(cudaSetDevice(c->device));
  default_shape(c, c->shape, ipt, jsplit);
  return NBODY_OK;
}

int nbody_get_launch(nbody_ctx *c, int *ipt, int *jsplit, int *threads, int *tile) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  int S = 0;
  seg_len(c, S);
  if (ipt) *ipt = c->shape.r;
  if (jsplit) *jsplit = S;
  if (threads) *threads = c->shape.bt;
  if (tile) *tile = c->shape.t;
  return NBODY_OK;
}

int nbody_set_symmetric(nbody_ctx *c, int mode) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (mode < -1 || mode > 1) return fail(NBODY_EINVAL, "symmetric mode must be -1, 0 or 1");
  if (mode == 1 && c->mode != NBODY_FP64 && c->mode != NBODY_F64E)
    return fail(NBODY_EINVAL, "each-pair-once path is FP64 and F64E only");
  c->sym = mode;
  return NBODY_OK;
}

int nbody_set_order(nbody_ctx *c, int order) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (order != NBODY_ORDER_INPUT && order != NBODY_ORDER_SPATIAL)
    return fail(NBODY_EINVAL, "order must be NBODY_ORDER_INPUT or NBODY_ORDER_SPATIAL");
  if (order == NBODY_ORDER_SPATIAL && c->mode == NBODY_FP32)
    return fail(NBODY_EINVAL, "the spatial order is not offered in NBODY_FP32");
  c->order = order;
  return NBODY_OK;
}

int nbody_get_order(const nbody_ctx *c, int *order) {
  if (!c || !order) return fail(NBODY_EINVAL, "NULL argument");
  *order = c->order;
  return NBODY_OK;
}

int nbody_get_symmetric(const nbody_ctx *c, int *mode, int *active) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  if (mode) *mode = c->sym;
  if (active) *active = use_sym(c) ? 1 : 0;
  return NBODY_OK;
}

int64_t nbody_launch_count(const nbody_ctx *c) { return c ? c->launches : 0; }

int nbody_profile(nbody_ctx *c, int enable) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  c->prof = enable != 0;
  return NBODY_OK;
}

int nbody_profile_read(nbody_ctx *c, double *force_ms, int64_t *force_launches) {
  if (!c) return fail(NBODY_EINVAL, "NULL context");
  CK(cudaSetDevice(c->device));
  int rc = sync(c);
  if (rc) return rc;
  double tot = 0;
  for (size_t k = 0; k < c->ev_used; k++) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->ev_pool[k].first, c->ev_pool[k].second));
    tot += ms;
  }
  if (force_ms) *force_ms = tot;
  if (force_launches) *force_launches = (int64_t)c->ev_used;
  c->ev_used = 0;
  return NBODY_OK;
}

}  // extern "C"
