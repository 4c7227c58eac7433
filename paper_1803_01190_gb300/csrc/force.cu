// Force kernels: Eq. 1-2 of the paper (section 1), the O(N^2) sum over all
// pairs of softened gravitational accelerations
//     a_i = G sum_{j != i} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
// and potentials pot_i = -G sum_{j != i} m_j / (|r_j - r_i|^2 + eps^2)^{1/2}.
//
// One thread block owns BT*R i-particles (R per thread, in registers) and one
// j-segment; it walks the segment in tiles of T j-particles staged through
// shared memory (the paper's GFC kernel stages i and j data in shared memory,
// section 2; here only j is staged: i stays in registers).  Every thread reads
// the same tile entry at the same time, a shared-memory broadcast.  The self
// pair j == i is excluded by a select in the few tiles that overlap the
// block's own i-range; all other tiles run without a predicate.
//
// The kernels write raw sums (no G, positive potential sum) per j-segment;
// the epilogue kernels in update.cu sum the segments in a fixed order, apply
// G and the update of the integrator.
//
// Three arithmetics:
//   f64   binary64 pair arithmetic.  GB300 issues binary64 at about 1/64 of the
//         binary32 rate, so the kernel is bound by the FP64 pipe and its cost
//         is its count of FP64 instructions per pair: 18 (3 DADD for d,
//         3 DFMA for |d|^2 + eps^2, 5 for the reciprocal square root, 3 DMUL,
//         3 DFMA and 1 DADD for the sums).  The reciprocal square root takes
//         its seed from the binary32 special-function unit through integer
//         bit moves (no FP64 conversion instruction) and refines it with one
//         third-order step in binary64.
//   mixed binary32 pair arithmetic on coordinates re-centred on an anchor (the
//         per-coordinate median) per j-tile, with the i coordinates held as float-float pairs so that the
//         per-tile shift costs three binary32 operations per coordinate and no
//         FP64 instruction; per-tile binary32 partial sums are folded into
//         float-float (compensated, TwoSum) accumulators, returned as binary64.
//   f32   binary32 throughout with plain binary32 accumulation: the paper's SP.
#include <cuda_runtime.h>

#include "nbody_internal.cuh"

namespace nb {

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/sqrt(x) in binary64, accurate to about half an ulp for x in [2^-126, 2^128).
// Seed: the top 23 mantissa bits of x are re-biased into a binary32 (exponent
// 1023 -> 127) by integer moves, sent through the SFU reciprocal square root,
// and moved back the same way.  The seed y0 has 24 significant bits and a
// relative error below 2^-21, so t = y0^2 is exact and the residual
// e = 1 - x y0^2 satisfies |e| < 2^-20.  Then 1/sqrt(x) = y0 (1 - e)^{-1/2}
// = y0 (1 + e/2 + 3e^2/8 + 5e^3/16 + ...); truncating after e^2 leaves a
// relative error below 5/16 |e|^3 < 2^-61.  Outside the range (zero,
// negative, huge, non-finite) it falls back to 1.0 / sqrt(x).
__device__ __forceinline__ double rsqrt_f64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  if (hi - 0x38100000u >= 0x47F00000u - 0x38100000u) return 1.0 / sqrt(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned fb = __funnelshift_l(lo, hi - 0x38000000u, 3);
  const unsigned yb = __float_as_uint(rsqrt_approx(__uint_as_float(fb)));
  const double y0 = __hiloint2double((int)((yb >> 3) + 0x38000000u), (int)(yb << 29));
  const double t = y0 * y0;
  const double e = fma(-x, t, 1.0);
  const double c = fma(e, 0.375, 0.5);
  const double d = y0 * e;
  return fma(d, c, y0);
}

// float-float accumulation a += b (Knuth's TwoSum; exact error term).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b) {
  const float s = __fadd_rn(hi, b);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// ---------------------------------------------------------------- binary64
template <bool MASK>
__device__ __forceinline__ void body_f64(const d4 &pj, double xi, double yi, double zi,
                                         double eps2, double &ax, double &ay, double &az,
                                         double &pt, bool self) {
  const double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
  double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
  double m = pj.w;
  if (MASK && self) {
    r2 = 1.0;
    m = 0.0;
  }
  const double y = rsqrt_f64(r2);
  const double my = m * y;
  const double f = my * (y * y);
  ax = fma(dx, f, ax);
  ay = fma(dy, f, ay);
  az = fma(dz, f, az);
  pt += my;
}

template <int BT, int R, int T>
__global__ void __launch_bounds__(BT) k_force_f64(const d4 *__restrict__ posm, int64_t n,
                                                  double eps2, int64_t seg,
                                                  d4 *__restrict__ part) {
  __shared__ d4 tile[T];
  const int tid = threadIdx.x;
  const int64_t ib = (int64_t)blockIdx.x * (BT * R);
  const int64_t j0 = (int64_t)blockIdx.y * seg;
  const int64_t j1 = min(n, j0 + seg);
  double xi[R], yi[R], zi[R], ax[R], ay[R], az[R], pt[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = ib + r * BT + tid;
    const d4 p = posm[i < n ? i : n - 1];
    xi[r] = p.x;
    yi[r] = p.y;
    zi[r] = p.z;
    ax[r] = ay[r] = az[r] = pt[r] = 0.0;
  }
  for (int64_t jt = j0; jt < j1; jt += T) {
    const int cnt = (int)min((int64_t)T, j1 - jt);
    __syncthreads();
    for (int k = tid; k < cnt; k += BT) tile[k] = posm[jt + k];
    __syncthreads();
    const bool diag = (jt < ib + BT * R) && (jt + cnt > ib);
    if (cnt == T && !diag) {
#pragma unroll 2
      for (int k = 0; k < T; k++) {
        const d4 pj = tile[k];
#pragma unroll
        for (int r = 0; r < R; r++)
          body_f64<false>(pj, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pt[r], false);
      }
    } else {
      for (int k = 0; k < cnt; k++) {
        const d4 pj = tile[k];
        const int64_t j = jt + k;
#pragma unroll
        for (int r = 0; r < R; r++)
          body_f64<true>(pj, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pt[r],
                         j == ib + r * BT + tid);
      }
    }
  }
  d4 *out = part + (int64_t)blockIdx.y * n;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = ib + r * BT + tid;
    if (i < n) out[i] = d4{ax[r], ay[r], az[r], pt[r]};
  }
}

// ---------------------------------------------------------------- binary32 pair body
// REFINE: one Newton step y = y0 + y0 (1 - r2 y0^2) / 2 on the SFU result.  The
// SFU approximation's error has a systematic part that adds up coherently
// over the N terms of a sum; the Newton step (4 more binary32 instructions)
// leaves an error of about one rounding, which averages out instead.
template <bool MASK, bool REFINE>
__device__ __forceinline__ void body_f32(const float4 &pj, float xi, float yi, float zi,
                                         float eps2, float &ax, float &ay, float &az, float &pt,
                                         bool self) {
  const float dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
  float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
  float m = pj.w;
  if (MASK && self) {
    r2 = 1.0f;
    m = 0.0f;
  }
  float y = rsqrt_approx(r2);
  if (REFINE) {
    const float e = fmaf(-(r2 * y), y, 1.0f);
    y = fmaf(y * 0.5f, e, y);
  }
  const float my = m * y;
  const float f = my * (y * y);
  ax = fmaf(dx, f, ax);
  ay = fmaf(dy, f, ay);
  az = fmaf(dz, f, az);
  pt += my;
}

// ---------------------------------------------------------------- mixed
// fpos[j] = (x_j - c_t, y_j - c_t, z_j - c_t, m_j) in binary32, c_t the anchor of
// j's tile; anchor[2t] = float hi part of c_t, anchor[2t+1] = float lo part.
template <int BT, int R, int T>
__global__ void __launch_bounds__(BT) k_force_mixed(const d4 *__restrict__ posm,
                                                    const float4 *__restrict__ fpos,
                                                    const float4 *__restrict__ anchor, int64_t n,
                                                    float eps2, int64_t seg,
                                                    d4 *__restrict__ part) {
  __shared__ float4 tile[T];
  const int tid = threadIdx.x;
  const int64_t ib = (int64_t)blockIdx.x * (BT * R);
  const int64_t j0 = (int64_t)blockIdx.y * seg;
  const int64_t j1 = min(n, j0 + seg);
  float xh[R], yh[R], zh[R], xl[R], yl[R], zl[R];
  float axh[R], axl[R], ayh[R], ayl[R], azh[R], azl[R], pth[R], ptl[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = ib + r * BT + tid;
    const d4 p = posm[i < n ? i : n - 1];
    xh[r] = __double2float_rn(p.x);
    yh[r] = __double2float_rn(p.y);
    zh[r] = __double2float_rn(p.z);
    xl[r] = __double2float_rn(p.x - (double)xh[r]);
    yl[r] = __double2float_rn(p.y - (double)yh[r]);
    zl[r] = __double2float_rn(p.z - (double)zh[r]);
    axh[r] = axl[r] = ayh[r] = ayl[r] = azh[r] = azl[r] = pth[r] = ptl[r] = 0.0f;
  }
  for (int64_t jt = j0; jt < j1; jt += T) {
    const int cnt = (int)min((int64_t)T, j1 - jt);
    __syncthreads();
    for (int k = tid; k < cnt; k += BT) tile[k] = fpos[jt + k];
    __syncthreads();
    const int64_t tt = jt / T;
    const float4 ch = anchor[2 * tt], cl = anchor[2 * tt + 1];
    float xr[R], yr[R], zr[R], sx[R], sy[R], sz[R], sp[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      xr[r] = __fadd_rn(__fsub_rn(xh[r], ch.x), __fsub_rn(xl[r], cl.x));
      yr[r] = __fadd_rn(__fsub_rn(yh[r], ch.y), __fsub_rn(yl[r], cl.y));
      zr[r] = __fadd_rn(__fsub_rn(zh[r], ch.z), __fsub_rn(zl[r], cl.z));
      sx[r] = sy[r] = sz[r] = sp[r] = 0.0f;
    }
    const float e2 = eps2;
    const bool diag = (jt < ib + BT * R) && (jt + cnt > ib);
    if (cnt == T && !diag) {
#pragma unroll 4
      for (int k = 0; k < T; k++) {
        const float4 pj = tile[k];
#pragma unroll
        for (int r = 0; r < R; r++)
          body_f32<false, true>(pj, xr[r], yr[r], zr[r], e2, sx[r], sy[r], sz[r], sp[r], false);
      }
    } else {
      for (int k = 0; k < cnt; k++) {
        const float4 pj = tile[k];
        const int64_t j = jt + k;
#pragma unroll
        for (int r = 0; r < R; r++)
          body_f32<true, true>(pj, xr[r], yr[r], zr[r], e2, sx[r], sy[r], sz[r], sp[r],
                         j == ib + r * BT + tid);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      two_sum_acc(axh[r], axl[r], sx[r]);
      two_sum_acc(ayh[r], ayl[r], sy[r]);
      two_sum_acc(azh[r], azl[r], sz[r]);
      two_sum_acc(pth[r], ptl[r], sp[r]);
    }
  }
  d4 *out = part + (int64_t)blockIdx.y * n;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = ib + r * BT + tid;
    if (i < n)
      out[i] = d4{(double)axh[r] + (double)axl[r], (double)ayh[r] + (double)ayl[r],
                  (double)azh[r] + (double)azl[r], (double)pth[r] + (double)ptl[r]};
  }
}

// One block per j-tile: anchor c = the per-coordinate median of the tile's
// positions (binary64), fpos[j] = float(r_j - c), float(m_j); anchor[2t],
// anchor[2t+1] = float-float c.  The median follows the bulk of the tile: for
// a spatially compact tile it lies inside it, and for an unsorted tile it
// stays near the centre of the particle distribution even when a few members
// sit far out in a halo (a bounding-box centre would be pulled out there and
// cost every coordinate relative to it several digits).  It is found with a
// bitonic sort of each coordinate in shared memory (tile = block = 256).
template <int BT>
__global__ void __launch_bounds__(BT) k_mixed_prep(const d4 *__restrict__ posm, int64_t n,
                                                   int tile, float4 *__restrict__ fpos,
                                                   float4 *__restrict__ anchor) {
  static_assert((BT & (BT - 1)) == 0, "bitonic sort needs a power-of-two block");
  __shared__ double v[BT];
  const int64_t t = blockIdx.x;
  const int64_t j0 = t * tile;
  const int cnt = (int)min((int64_t)tile, n - j0);
  const int tid = threadIdx.x;
  d4 p = {0, 0, 0, 0};
  if (tid < cnt) p = posm[j0 + tid];
  double c[3];
  for (int q = 0; q < 3; q++) {
    __syncthreads();
    v[tid] = tid < cnt ? (q == 0 ? p.x : q == 1 ? p.y : p.z) : 1e308;
    __syncthreads();
    for (int k = 2; k <= BT; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int o = tid ^ j;
        if (o > tid) {
          const double a = v[tid], b = v[o];
          const bool up = (tid & k) == 0;
          if ((a > b) == up) {
            v[tid] = b;
            v[o] = a;
          }
        }
        __syncthreads();
      }
    }
    c[q] = v[(cnt - 1) / 2];
  }
  if (tid < cnt)
    fpos[j0 + tid] = make_float4(__double2float_rn(p.x - c[0]), __double2float_rn(p.y - c[1]),
                                 __double2float_rn(p.z - c[2]), __double2float_rn(p.w));
  if (tid == 0) {
    const float hx = __double2float_rn(c[0]), hy = __double2float_rn(c[1]),
                hz = __double2float_rn(c[2]);
    anchor[2 * t] = make_float4(hx, hy, hz, 0.0f);
    anchor[2 * t + 1] = make_float4(__double2float_rn(c[0] - (double)hx),
                                    __double2float_rn(c[1] - (double)hy),
                                    __double2float_rn(c[2] - (double)hz), 0.0f);
  }
}

// ---------------------------------------------------------------- binary32 (paper's SP)
template <int BT, int R, int T>
__global__ void __launch_bounds__(BT) k_force_f32(const float4 *__restrict__ posm, int64_t n,
                                                  float eps2, int64_t seg,
                                                  float4 *__restrict__ part) {
  __shared__ float4 tile[T];
  const int tid = threadIdx.x;
  const int64_t ib = (int64_t)blockIdx.x * (BT * R);
  const int64_t j0 = (int64_t)blockIdx.y * seg;
  const int64_t j1 = min(n, j0 + seg);
  float xi[R], yi[R], zi[R], ax[R], ay[R], az[R], pt[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = ib + r * BT + tid;
    const float4 p = posm[i < n ? i : n - 1];
    xi[r] = p.x;
    yi[r] = p.y;
    zi[r] = p.z;
    ax[r] = ay[r] = az[r] = pt[r] = 0.0f;
  }
  for (int64_t jt = j0; jt < j1; jt += T) {
    const int cnt = (int)min((int64_t)T, j1 - jt);
    __syncthreads();
    for (int k = tid; k < cnt; k += BT) tile[k] = posm[jt + k];
    __syncthreads();
    const bool diag = (jt < ib + BT * R) && (jt + cnt > ib);
    if (cnt == T && !diag) {
#pragma unroll 4
      for (int k = 0; k < T; k++) {
        const float4 pj = tile[k];
#pragma unroll
        for (int r = 0; r < R; r++)
          body_f32<false, false>(pj, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pt[r], false);
      }
    } else {
      for (int k = 0; k < cnt; k++) {
        const float4 pj = tile[k];
        const int64_t j = jt + k;
#pragma unroll
        for (int r = 0; r < R; r++)
          body_f32<true, false>(pj, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pt[r],
                         j == ib + r * BT + tid);
      }
    }
  }
  float4 *out = part + (int64_t)blockIdx.y * n;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = ib + r * BT + tid;
    if (i < n) out[i] = make_float4(ax[r], ay[r], az[r], pt[r]);
  }
}

// ---------------------------------------------------------------- dispatch
// Fixed block and tile sizes per arithmetic; R is chosen at run time.
constexpr int BT_F64 = 128, T_F64 = 128;
constexpr int BT_F32 = 256, T_F32 = 256;

bool shape_supported(int mode, const Shape &sh) {
  if (sh.r != 1 && sh.r != 2 && sh.r != 4 && sh.r != 8) return false;
  if (sh.s < 1 || sh.s > 65535) return false;
  if (mode == NBODY_FP64) return sh.bt == BT_F64 && sh.t == T_F64;
  return sh.bt == BT_F32 && sh.t == T_F32;
}

template <int R>
static const void *kernel_for(int mode) {
  switch (mode) {
    case NBODY_FP64: return (const void *)k_force_f64<BT_F64, R, T_F64>;
    case NBODY_MIXED: return (const void *)k_force_mixed<BT_F32, R, T_F32>;
    default: return (const void *)k_force_f32<BT_F32, R, T_F32>;
  }
}

static const void *kernel_ptr(int mode, int r) {
  switch (r) {
    case 1: return kernel_for<1>(mode);
    case 2: return kernel_for<2>(mode);
    case 4: return kernel_for<4>(mode);
    default: return kernel_for<8>(mode);
  }
}

int force_max_blocks_per_sm(int mode, const Shape &sh) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_ptr(mode, sh.r), sh.bt, 0) !=
      cudaSuccess)
    return 0;
  return nb;
}

template <int R>
static void launch_r(int mode, const ForceIn &in, dim3 grid, cudaStream_t st) {
  if (mode == NBODY_FP64) {
    k_force_f64<BT_F64, R, T_F64><<<grid, BT_F64, 0, st>>>(
        (const d4 *)in.posm, in.n, in.eps2, in.seg, (d4 *)in.part);
  } else if (mode == NBODY_MIXED) {
    k_force_mixed<BT_F32, R, T_F32><<<grid, BT_F32, 0, st>>>(
        (const d4 *)in.posm, in.fpos, in.anchor, in.n, (float)in.eps2, in.seg, (d4 *)in.part);
  } else {
    k_force_f32<BT_F32, R, T_F32><<<grid, BT_F32, 0, st>>>(
        (const float4 *)in.posm, in.n, (float)in.eps2, in.seg, (float4 *)in.part);
  }
}

cudaError_t launch_force(int mode, const ForceIn &in, const Shape &sh, cudaStream_t st) {
  if (!shape_supported(mode, sh) || in.n < 1) return cudaErrorInvalidValue;
  const int64_t per_block = (int64_t)sh.bt * sh.r;
  const int64_t gx = (in.n + per_block - 1) / per_block;
  if (gx > 0x7fffffff) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)gx, (unsigned)sh.s);
  switch (sh.r) {
    case 1: launch_r<1>(mode, in, grid, st); break;
    case 2: launch_r<2>(mode, in, grid, st); break;
    case 4: launch_r<4>(mode, in, grid, st); break;
    default: launch_r<8>(mode, in, grid, st); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_mixed_prep(const d4 *posm, int64_t n, int tile, float4 *fpos, float4 *anchor,
                              cudaStream_t st) {
  if (tile != 256) return cudaErrorInvalidValue;  // one thread per tile member
  const int64_t nt = (n + tile - 1) / tile;
  k_mixed_prep<256><<<(unsigned)nt, 256, 0, st>>>(posm, n, tile, fpos, anchor);
  return cudaGetLastError();
}

}  // namespace nb
