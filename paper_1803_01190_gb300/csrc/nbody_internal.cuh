// Internal declarations of the GB300 direct-summation N-body library.
//
// Device layout of one simulation (n particles, all arrays length n unless
// stated; `real` is double for FP64/MIXED and float for FP32):
//   posm[2]  real4 (x, y, z, m)   ping-pong positions+mass; posm[cur] is the
//                                 state at the step boundary, posm[nxt] the
//                                 positions of the next force evaluation
//   vel      real4 (vx, vy, vz, -) velocity at the step boundary
//   vbar     real4                 KDK half-sum (v + vt)/2 of Eq. 5/7
//   acc      real4 (ax, ay, az, pot) Eq. 1-2 at posm[cur]
//   part     real4 x S x n         j-segment partial sums of the force kernel
//   rk_*     real4                 RK4 stage velocity and running sums
//   fpos     float4 x n, anchor    MIXED only: j coordinates re-centred per tile
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nbody.h"

namespace nb {

struct __align__(32) d4 {
  double x, y, z, w;
};

template <typename real>
struct vec4;
template <>
struct vec4<double> {
  using type = d4;
};
template <>
struct vec4<float> {
  using type = float4;
};
template <typename real>
using real4 = typename vec4<real>::type;

// Force-kernel shape.  BT threads per block, R i-particles per thread, T
// j-particles per shared-memory tile; grid = (ceil(n / (BT*R)), S).
struct Shape {
  int bt = 128;
  int r = 4;
  int t = 128;
  int s = 1;
};

// One thread block's share of a force evaluation: i-particles [i0, i0+ni)
// against j-particles [j0, j0+nj) of the same system (pool indices), raw
// partial sums written to part[out + (i - i0)].  anchor: MIXED tile-anchor
// index of the tile that starts at j0.  eps2: that system's softening^2.
struct Unit {
  int64_t i0, j0, out, anchor;
  double eps2;
  int32_t ni, nj;
};

// One MIXED prep block: the tile [j0, j0+cnt) with anchor index `anchor`.
struct PrepUnit {
  int64_t j0, anchor;
  int32_t cnt, pad;
};

// Raw force sums written by the force kernels, per j-segment s:
//   part[s*n + i] = ( sum_j m_j (x_j - x_i) / w_ij, ..y.., ..z..,
//                     sum_j m_j / sqrt(|d_ij|^2 + eps^2) )
// over j != i in segment s.  G and the sign of the potential are applied by
// the epilogue kernels.
struct ForceIn {
  const void *posm;      // real4 (FP64, FP32) or d4 (MIXED) positions+mass
  const float4 *fpos;    // MIXED: re-centred j coordinates + float mass
  const float4 *anchor;  // MIXED: per tile (hi.xyz, lo.xyz) float-float anchors, 2 per tile
  int64_t n;
  double eps2;
  int64_t seg;           // j-segment length (multiple of the tile)
  void *part;            // S * rows entries
  int64_t i0 = 0;        // the rows [i0, i0 + rows) are summed against all n
  int64_t rows = -1;     // -1: all n
};

// launchers (force.cu); return cudaError_t of the launch
cudaError_t launch_force(int mode, const ForceIn &in, const Shape &sh, cudaStream_t st);
// varlen: blocks run the units of `units` (device array), R i-particles per
// thread; at most max_blocks blocks (0 = one per unit), each looping over units
cudaError_t launch_force_units(int mode, const void *posm, const float4 *fpos,
                               const float4 *anchor, const Unit *units, int64_t nunits, int r,
                               void *part, int64_t max_blocks, cudaStream_t st);
cudaError_t launch_mixed_prep_units(const d4 *posm, const PrepUnit *units, int64_t nunits,
                                    float4 *fpos, float4 *anchor, cudaStream_t st, bool ff = false);
int force_block_threads(int mode);
int force_tile(int mode);
// ff: write float-float re-centred coordinates (F64E, two float4 per particle)
cudaError_t launch_mixed_prep(const d4 *posm, int64_t n, int tile, float4 *fpos, float4 *anchor,
                              cudaStream_t st, bool ff = false);
int force_max_blocks_per_sm(int mode, const Shape &sh);
// FP64, each pair once (Newton's third law): blocks of sym_block_particles()
// particles (the one-sided kernel with R = sym_units_r() runs the pairs inside
// each block); launch D diagonals d0 .. d0+D-1 of the M x M block pairs, row
// sums of diagonal d0+k into rows[k*n ..], column sums into cols[k*n ..];
// launch_sym_combine adds them (in diagonal order) into acc_rows / acc_cols
// (overwriting them when first).
int sym_block_particles();
int sym_r();
int sym_units_r();
int sym_blocks_per_sm();
cudaError_t launch_force_f64_sym(const d4 *posm, int64_t n, double eps2, int M, int d0, int D,
                                 d4 *rows, d4 *cols, cudaStream_t st);
cudaError_t launch_sym_combine(const d4 *rows, const d4 *cols, int D, int64_t n, d4 *acc_rows,
                               d4 *acc_cols, bool first, cudaStream_t st);
// F64E, each pair once: blocks of sym_block_particles_ff() particles (one
// float-float tile each); jff / anchor from launch_mixed_prep(..., ff = true)
int sym_block_particles_ff();
int sym_r_ff();
int sym_blocks_per_sm_ff();
cudaError_t launch_force_f64e_sym(const d4 *posm, const float4 *jff, const float4 *anchor,
                                  int64_t n, double eps2, int M, int d0, int D, d4 *rows,
                                  d4 *cols, cudaStream_t st);

bool shape_supported(int mode, const Shape &sh);

// update / epilogue kernels (update.cu)
struct EpiIn {
  int64_t n;
  int S;
  const void *part;  // S * n raw sums (real4 for FP64/FP32; d4 for MIXED)
  double G;
};
cudaError_t launch_pack(int mode, const double *pos, const double *vel, const double *mass,
                        int64_t n, void *posm, void *velv, int *flag, cudaStream_t st);
cudaError_t launch_unpack_state(int mode, const void *posm, const void *velv, int64_t n,
                                double *pos, double *vel, cudaStream_t st);
cudaError_t launch_store_acc(int mode, const EpiIn &e, void *acc, cudaStream_t st);
cudaError_t launch_unpack_acc(int mode, const void *acc, int64_t n, double *acc3, double *pot,
                              cudaStream_t st);
cudaError_t launch_kdk_predict(int mode, int64_t n, double dt, const void *posm_cur,
                               const void *vel, const void *acc, void *vbar, void *posm_nxt,
                               cudaStream_t st);
cudaError_t launch_kdk_correct_predict(int mode, const EpiIn &e, double dt, double dt_next,
                                       void *acc, void *posm_new, void *vel, void *vbar,
                                       void *posm_pred, cudaStream_t st);
cudaError_t launch_rk4_stage(int mode, const EpiIn &e, int stage, double dt, const void *posm0,
                             void *vel0, void *rk_vs, void *rk_sr, void *rk_sv, void *posm_stage,
                             cudaStream_t st);
cudaError_t launch_diag(int mode, const void *posm, const void *vel, const void *acc, int64_t n,
                        double *blocks, int nblocks, double *out9, cudaStream_t st);
int diag_blocks(int64_t n);

// Spatial (Morton) order of the particles (order.cu).  launch_spatial_order
// writes perm (sorted position -> input index) and sposm[s] = posm[perm[s]],
// using `scratch` of order_scratch_bytes(n); launch_unpermute scatters S
// slices of sorted partial sums back to input order: part[k n + perm[s]] =
// sorted[k n + s].
size_t order_scratch_bytes(int64_t n);
cudaError_t launch_spatial_order(const d4 *posm, int64_t n, void *scratch, int32_t *perm,
                                 d4 *sposm, cudaStream_t st);
cudaError_t launch_unpermute(const d4 *sorted, const int32_t *perm, int S, int64_t n, d4 *part,
                             cudaStream_t st);

// Records the detail that nbody_last_error() returns on this thread and
// returns `code` (api.cu); every entry point reports its failures through it.
int record_error(int code, const char *what, cudaError_t ce = cudaSuccess);

inline size_t real_bytes(int mode) { return mode == NBODY_FP32 ? sizeof(float) : sizeof(double); }

}  // namespace nb
