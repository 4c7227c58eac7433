// Spatial (Morton, Z-curve) ordering of the particles before the force sum.
//
// The mixed kernel evaluates Eq. 2 in binary32 on coordinates re-centred on
// an anchor per j-tile: x_j - c and x_i - c are each rounded once to binary32,
// so a pair's difference carries an error of about 2^-24 |x - c|.  For a
// close pair (|d| near the softening) that is a relative error of
// 2^-24 |x - c| / |d|, and with particles in input order a tile spans the
// whole system, |x - c| ~ its radius.  Sorting the particles along a
// space-filling curve first makes every tile of consecutive particles
// spatially compact, so |x - c| is the tile's own size wherever a pair is
// close, and the binary32 coordinates keep their digits.
//
// The order is a deterministic function of the positions alone: the bounding
// box is an exact min/max (order independent), the key of a particle is the
// bit interleave of its three 21-bit cell indices in that box, and the sort
// is a stable radix sort on (key, input index), so equal keys keep input
// order.  Results therefore stay bit-reproducible (a resumed run recomputes
// the same order from the same positions).
//
// Steps (one force evaluation): bbox partials -> bbox + keys -> sort ->
// gather of the positions into sorted order; after the force kernels, the
// j-segment partial sums are scattered back to input order.
#include <cuda_runtime.h>

#include <algorithm>

#include <cub/device/device_radix_sort.cuh>

#include "nbody_internal.cuh"

namespace nb {

namespace {

constexpr int kBT = 256;
constexpr int kBboxBlocks = 256;  // partial boxes reduced by one block afterwards
constexpr int kCellBits = 21;     // per coordinate; 63-bit keys

// Per-block min/max of each coordinate over a grid-stride share of [0, n).
__global__ void __launch_bounds__(kBT) k_bbox_partial(const d4 *__restrict__ posm, int64_t n,
                                                      double *__restrict__ part) {
  __shared__ double s[6][kBT];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)kBT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBT) {
    const d4 p = posm[i];
    lo[0] = fmin(lo[0], p.x);
    lo[1] = fmin(lo[1], p.y);
    lo[2] = fmin(lo[2], p.z);
    hi[0] = fmax(hi[0], p.x);
    hi[1] = fmax(hi[1], p.y);
    hi[2] = fmax(hi[2], p.z);
  }
  for (int c = 0; c < 3; c++) {
    s[c][threadIdx.x] = lo[c];
    s[3 + c][threadIdx.x] = hi[c];
  }
  __syncthreads();
  for (int h = kBT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int c = 0; c < 3; c++) {
        s[c][threadIdx.x] = fmin(s[c][threadIdx.x], s[c][threadIdx.x + h]);
        s[3 + c][threadIdx.x] = fmax(s[3 + c][threadIdx.x], s[3 + c][threadIdx.x + h]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

// Spread the low 21 bits of v to every third bit of a 64-bit word.
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

// Every block reduces the partial boxes itself (a few KB, L2-resident), then
// writes the keys and the identity permutation of its particles.
__global__ void __launch_bounds__(kBT) k_morton_keys(const d4 *__restrict__ posm, int64_t n,
                                                     const double *__restrict__ part, int nparts,
                                                     uint64_t *__restrict__ keys,
                                                     int32_t *__restrict__ idx) {
  __shared__ double box[6];
  if (threadIdx.x < 6) {
    const int c = threadIdx.x;
    double v = part[c];
    for (int b = 1; b < nparts; b++)
      v = c < 3 ? fmin(v, part[b * 6 + c]) : fmax(v, part[b * 6 + c]);
    box[c] = v;
  }
  __syncthreads();
  const double span = fmax(fmax(box[3] - box[0], box[4] - box[1]), box[5] - box[2]);
  const double cells = (double)((1u << kCellBits) - 1);
  const double scale = span > 0 ? cells / span : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kBT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBT) {
    const d4 p = posm[i];
    const double q[3] = {(p.x - box[0]) * scale, (p.y - box[1]) * scale, (p.z - box[2]) * scale};
    uint64_t key = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const double f = fmin(fmax(floor(q[c]), 0.0), cells);  // in [0, cells]; NaN gives 0
      key |= spread3((uint64_t)f) << c;
    }
    keys[i] = key;
    idx[i] = (int32_t)i;
  }
}

__global__ void __launch_bounds__(kBT) k_gather_posm(const d4 *__restrict__ posm,
                                                     const int32_t *__restrict__ perm, int64_t n,
                                                     d4 *__restrict__ sposm) {
  for (int64_t s = blockIdx.x * (int64_t)kBT + threadIdx.x; s < n; s += (int64_t)gridDim.x * kBT)
    sposm[s] = posm[perm[s]];
}

// part[k n + perm[s]] = sorted[k n + s] for every slice k.
__global__ void __launch_bounds__(kBT) k_unpermute(const d4 *__restrict__ sorted,
                                                   const int32_t *__restrict__ perm, int S,
                                                   int64_t n, d4 *__restrict__ part) {
  for (int64_t s = blockIdx.x * (int64_t)kBT + threadIdx.x; s < n; s += (int64_t)gridDim.x * kBT) {
    const int64_t i = perm[s];
    for (int k = 0; k < S; k++) part[(int64_t)k * n + i] = sorted[(int64_t)k * n + s];
  }
}

unsigned grid(int64_t n) {
  int64_t g = (n + kBT - 1) / kBT;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t sort_temp_bytes(int64_t n) {
  size_t bytes = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr,
                                  (const int32_t *)nullptr, (int32_t *)nullptr, (int)n, 0,
                                  3 * kCellBits);
  return bytes;
}

}  // namespace

// Scratch layout: bbox partials | keys in | keys out | identity indices | sort temp.
size_t order_scratch_bytes(int64_t n) {
  return align256(sizeof(double) * 6 * kBboxBlocks) + 2 * align256(sizeof(uint64_t) * n) +
         align256(sizeof(int32_t) * n) + align256(sort_temp_bytes(n));
}

cudaError_t launch_spatial_order(const d4 *posm, int64_t n, void *scratch, int32_t *perm,
                                 d4 *sposm, cudaStream_t st) {
  if (n > 0x7fffffff) return cudaErrorInvalidValue;
  char *p = (char *)scratch;
  double *bb = (double *)p;
  p += align256(sizeof(double) * 6 * kBboxBlocks);
  uint64_t *kin = (uint64_t *)p;
  p += align256(sizeof(uint64_t) * n);
  uint64_t *kout = (uint64_t *)p;
  p += align256(sizeof(uint64_t) * n);
  int32_t *idx = (int32_t *)p;
  p += align256(sizeof(int32_t) * n);
  size_t tb = sort_temp_bytes(n);
  const int nb = (int)std::min<int64_t>(kBboxBlocks, (n + kBT - 1) / kBT);
  k_bbox_partial<<<nb, kBT, 0, st>>>(posm, n, bb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_morton_keys<<<grid(n), kBT, 0, st>>>(posm, n, bb, nb, kin, idx);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cub::DeviceRadixSort::SortPairs(p, tb, kin, kout, idx, perm, (int)n, 0, 3 * kCellBits, st);
  if (e != cudaSuccess) return e;
  k_gather_posm<<<grid(n), kBT, 0, st>>>(posm, perm, n, sposm);
  return cudaGetLastError();
}

cudaError_t launch_unpermute(const d4 *sorted, const int32_t *perm, int S, int64_t n, d4 *part,
                             cudaStream_t st) {
  k_unpermute<<<grid(n), kBT, 0, st>>>(sorted, perm, S, n, part);
  return cudaGetLastError();
}

}  // namespace nb
