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
//   - the first call on a device looks up the array's device address with that
//     device current (a one-time set-up per device); make that first call
//     before any stream capture begins.
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

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Errors are reported by code only (the codes of include/nbody.h).
int fail(int code, const char *, cudaError_t = cudaSuccess) { return code; }

// Device address of g_scratch on the current device, looked up once per device.
int scratch_for_current_device(void **addr, int *sms) {
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(NBODY_ECUDA, "cudaGetDevice", ce);
  if (dev < 0 || dev >= kMaxDevices) return fail(NBODY_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    ce = cudaGetSymbolAddress(&p, g_scratch);
    if (ce != cudaSuccess || !p) return fail(NBODY_ECUDA, "cudaGetSymbolAddress(scratch)", ce);
    int s = 0;
    ce = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return fail(NBODY_ECUDA, "cudaDeviceGetAttribute", ce);
    g_addr[dev] = p;
    g_sms[dev] = s;
  }
  *addr = g_addr[dev];
  *sms = g_sms[dev];
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
  int rc = scratch_for_current_device(&base, &sms);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // scratch layout: [packed positions n][summed accelerations n][S partial slices of n]
  nb::d4 *posm = (nb::d4 *)base;
  nb::d4 *accd = posm + n;
  nb::d4 *part = accd + n;
  const int64_t slots = (int64_t)(kScratchBytes / sizeof(nb::d4)) / n - 2;

  nb::Shape sh;
  sh.bt = 128;
  sh.t = 128;
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
