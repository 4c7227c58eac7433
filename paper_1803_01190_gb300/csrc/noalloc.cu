// nbody_accel_f64_static: the binary64 force evaluation of nbody_accel, for
// callers that must not have this library allocate device memory.
//
// Who needs it: a host application (a game engine, a plugin host, a larger
// simulation framework) that owns all GPU memory through its own allocator or
// has already reserved it, and a timing-critical loop in which a cudaMalloc or
// cudaFree would stall the device.  Such a caller can still hand over its own
// input and output arrays; the scratch that the force kernel needs besides
// them (packed positions, per-segment partial sums) lives in one file-scope
// __device__ array that every GPU loading this library holds until the
// process exits.
//
// Limits and sharing:
//   - n <= NBODY_STATIC_MAX_N (32768 particles); larger n is rejected with
//     NBODY_EINVAL before anything is launched.
//   - all calls share the one array; nothing in it needs to start at zero
//     (every byte a call reads was written earlier in the same call), but two
//     calls whose work overlaps on the GPU (different streams, or different
//     host threads) race on it and give wrong results.  Order them on one
//     stream or serialise them.
//   - the array's device address is looked up once per CUDA context, with
//     that context current: on the first call of a device's primary context,
//     again after cudaDeviceReset (which makes a new one), and for any other
//     context the caller makes current.  Make that first call before any
//     stream capture begins.
//   - inputs are not scanned for non-finite values (as in nbody_accel); a NaN
//     input gives NaN outputs.
// The paper has no counterpart of this entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "nbody_internal.cuh"

namespace {

constexpr int64_t kMaxN = NBODY_STATIC_MAX_N;
constexpr size_t kScratchBytes = (size_t)NBODY_STATIC_SCRATCH_BYTES;
static_assert(kScratchBytes >= (size_t)kMaxN * sizeof(nb::d4) * 3, "scratch too small");

// The scratch itself.  In host code this name is only a stand-in: its device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Driver entry points for the identity of the current context, looked up once
// through the runtime (the library links only the CUDA runtime).
using CtxGetCurrent = int (*)(void **);                  // cuCtxGetCurrent
using CtxGetId = int (*)(void *, unsigned long long *);  // cuCtxGetId

// One cached address per context, keyed by the context's unique id (ids are
// never reused within a process, unlike context handles).
constexpr int kCache = 64;
struct Entry {
  unsigned long long id;
  void *addr;
  int sms;
};
std::mutex g_mu;
Entry g_cache[kCache] = {};
int g_used = 0, g_next = 0;
CtxGetCurrent g_get_current = nullptr;
CtxGetId g_get_id = nullptr;

int fail(int code, const char *what, cudaError_t ce = cudaSuccess) {
  return nb::record_error(code, what, ce);
}

int current_context_id(unsigned long long *id) {
  if (!g_get_current || !g_get_id) {
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    cudaError_t ce = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000,
                                                      cudaEnableDefault, &qa);
    if (ce == cudaSuccess)
      ce = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
    if (ce != cudaSuccess || qa != cudaDriverEntryPointSuccess ||
        qb != cudaDriverEntryPointSuccess || !a || !b)
      return fail(NBODY_ECUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId", ce);
    g_get_current = (CtxGetCurrent)a;
    g_get_id = (CtxGetId)b;
  }
  void *ctx = nullptr;
  if (g_get_current(&ctx) != 0) return fail(NBODY_ECUDA, "cuCtxGetCurrent");
  if (!ctx) {
    // nothing current yet: bind the current device's primary context, as the
    // runtime does before any launch
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaSetDevice(dev);
    if (ce != cudaSuccess) return fail(NBODY_ECUDA, "primary context", ce);
    if (g_get_current(&ctx) != 0 || !ctx) return fail(NBODY_ECUDA, "no current CUDA context");
  }
  if (g_get_id(ctx, id) != 0) return fail(NBODY_ECUDA, "cuCtxGetId");
  return NBODY_OK;
}

// Device address of g_scratch in the current context and the device's SM count.
int scratch_for_current_context(void **addr, int *sms) {
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc) return rc;
  for (int k = 0; k < g_used; k++)
    if (g_cache[k].id == id) {
      *addr = g_cache[k].addr;
      *sms = g_cache[k].sms;
      return NBODY_OK;
    }
  void *p = nullptr;
  cudaError_t ce = cudaGetSymbolAddress(&p, g_scratch);
  if (ce != cudaSuccess || !p) return fail(NBODY_ECUDA, "cudaGetSymbolAddress(scratch)", ce);
  int dev = 0, s = 0;
  ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
  if (ce != cudaSuccess) return fail(NBODY_ECUDA, "SM count", ce);
  Entry &e = g_cache[g_used < kCache ? g_used++ : (g_next++ % kCache)];
  e = Entry{id, p, s};
  *addr = p;
  *sms = s;
  return NBODY_OK;
}

}  // namespace

extern "C" int nbody_accel_f64_static(int64_t n, const double *pos, const double *mass, double eps,
                                      double G, double *acc, double *pot, void *cuda_stream) {
  if (n < 1) return fail(NBODY_EINVAL, "n < 1");
  if (n > kMaxN) return fail(NBODY_EINVAL, "n exceeds the static scratch capacity");
  if (!pos || !mass || !acc) return fail(NBODY_EINVAL, "NULL pos, mass or acc");
  if (!(eps >= 0) || !std::isfinite(eps) || !std::isfinite(G))
    return fail(NBODY_EINVAL, "eps must be finite and >= 0, G finite");
  void *base = nullptr;
  int sms = 0;
  int rc = scratch_for_current_context(&base, &sms);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // scratch layout: [packed positions n][summed accelerations n][S partial slices of n]
  nb::d4 *posm = (nb::d4 *)base;
  nb::d4 *accd = posm + n;
  nb::d4 *part = accd + n;
  const int64_t slots = (int64_t)(kScratchBytes / sizeof(nb::d4)) / n - 2;

  nb::Shape sh;
  sh.bt = nb::force_block_threads(NBODY_FP64);
  sh.t = nb::force_tile(NBODY_FP64);
  sh.r = 4;
  while (sh.r > 1 && (int64_t)sh.bt * sh.r * sms > n) sh.r >>= 1;
  const int64_t bx = (n + (int64_t)sh.bt * sh.r - 1) / ((int64_t)sh.bt * sh.r);
  int occ = nb::force_max_blocks_per_sm(NBODY_FP64, sh);
  if (occ < 1) occ = 1;
  int64_t s = (8LL * sms * occ + bx - 1) / bx;
  const int64_t smax = (n + sh.t - 1) / sh.t;
  if (s > smax) s = smax;
  if (s > 64) s = 64;
  if (s > slots) s = slots;
  if (s < 1) s = 1;
  int64_t seg = (n + s - 1) / s;
  seg = (seg + sh.t - 1) / sh.t * sh.t;
  sh.s = (int)((n + seg - 1) / seg);

  cudaError_t ce = nb::launch_pack(NBODY_FP64, pos, nullptr, mass, n, posm, nullptr, nullptr, st);
  if (ce != cudaSuccess) return fail(NBODY_ECUDA, "pack launch", ce);
  nb::ForceIn in;
  in.posm = posm;
  in.fpos = nullptr;
  in.anchor = nullptr;
  in.n = n;
  in.eps2 = eps * eps;
  in.seg = seg;
  in.part = part;
  ce = nb::launch_force(NBODY_FP64, in, sh, st);
  if (ce != cudaSuccess) return fail(NBODY_ECUDA, "force launch", ce);
  nb::EpiIn e;
  e.n = n;
  e.S = sh.s;
  e.part = part;
  e.G = G;
  ce = nb::launch_store_acc(NBODY_FP64, e, accd, st);
  if (ce != cudaSuccess) return fail(NBODY_ECUDA, "sum launch", ce);
  ce = nb::launch_unpack_acc(NBODY_FP64, accd, n, acc, pot, st);
  if (ce != cudaSuccess) return fail(NBODY_ECUDA, "unpack launch", ce);
  return NBODY_OK;
}
