// O(N) kernels around the force sum: packing of the caller's arrays into the
// device layout, the epilogues that sum the force kernel's j-segments in a
// fixed order and apply the integrator (the paper's US kernel, section 2,
// fused with the segment sum), and the Eq. 8-10 reductions.
//
// The integrator arithmetic uses explicitly rounded operations (no fused
// multiply-add contraction) in the order the paper writes the formulas, so
// that a step differs from a plain sequential evaluation only through the
// accelerations it is given.
#include <cuda_runtime.h>

#include "nbody_internal.cuh"

namespace nb {

template <typename real>
struct ops;
template <>
struct ops<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
};
template <>
struct ops<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
};

template <typename real>
__device__ __forceinline__ real4<real> mk4(real x, real y, real z, real w) {
  real4<real> v;
  v.x = x;
  v.y = y;
  v.z = z;
  v.w = w;
  return v;
}

// Sum of the S j-segment partials of particle i in segment order, with G and
// the sign of the potential applied: returns (a_x, a_y, a_z, pot).
template <typename real, typename P>
__device__ __forceinline__ real4<real> gather_acc(const P *part, int S, int64_t n, int64_t i,
                                                  real G) {
  using O = ops<real>;
  const P p0 = part[i];
  real x = (real)p0.x, y = (real)p0.y, z = (real)p0.z, w = (real)p0.w;
  for (int s = 1; s < S; s++) {
    const P p = part[(int64_t)s * n + i];
    x = O::add(x, (real)p.x);
    y = O::add(y, (real)p.y);
    z = O::add(z, (real)p.z);
    w = O::add(w, (real)p.w);
  }
  return mk4<real>(O::mul(G, x), O::mul(G, y), O::mul(G, z), -O::mul(G, w));
}

// ---------------------------------------------------------------- pack / unpack
template <typename real>
__global__ void k_pack(const double *__restrict__ pos, const double *__restrict__ vel,
                       const double *__restrict__ mass, int64_t n, real4<real> *__restrict__ posm,
                       real4<real> *__restrict__ velv, int *__restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], m = mass[i];
    double vx = 0, vy = 0, vz = 0;
    if (vel) {
      vx = vel[3 * i];
      vy = vel[3 * i + 1];
      vz = vel[3 * i + 2];
    }
    const bool ok = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(m) && m >= 0.0 &&
                    isfinite(vx) && isfinite(vy) && isfinite(vz);
    if (!ok && flag) atomicOr(flag, 1);
    posm[i] = mk4<real>((real)x, (real)y, (real)z, (real)m);
    if (velv) velv[i] = mk4<real>((real)vx, (real)vy, (real)vz, (real)0);
  }
}

template <typename real>
__global__ void k_unpack_state(const real4<real> *__restrict__ posm,
                               const real4<real> *__restrict__ velv, int64_t n,
                               double *__restrict__ pos, double *__restrict__ vel) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (pos) {
      const real4<real> p = posm[i];
      pos[3 * i] = p.x;
      pos[3 * i + 1] = p.y;
      pos[3 * i + 2] = p.z;
    }
    if (vel) {
      const real4<real> v = velv[i];
      vel[3 * i] = v.x;
      vel[3 * i + 1] = v.y;
      vel[3 * i + 2] = v.z;
    }
  }
}

template <typename real, typename P>
__global__ void k_store_acc(const P *__restrict__ part, int S, int64_t n, real G,
                            real4<real> *__restrict__ acc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc[i] = gather_acc<real, P>(part, S, n, i, G);
}

template <typename real>
__global__ void k_unpack_acc(const real4<real> *__restrict__ acc, int64_t n,
                             double *__restrict__ acc3, double *__restrict__ pot) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const real4<real> a = acc[i];
    if (acc3) {
      acc3[3 * i] = a.x;
      acc3[3 * i + 1] = a.y;
      acc3[3 * i + 2] = a.z;
    }
    if (pot) pot[i] = a.w;
  }
}

// ---------------------------------------------------------------- KDK, Eq. 5-7
// Predictor and drift for the step that starts at (r, v, a):
//   vt = v + dt a                      (Eq. 5)
//   r' = r + dt/2 (vt + v)             (Eq. 6)     -> posm_nxt (mass copied)
//   vbar = (v + vt) / 2                (first term of Eq. 7, kept for the corrector)
template <typename real>
__device__ __forceinline__ void kdk_predict_one(real dt, real hdt, const real4<real> &r,
                                                const real4<real> &v, const real4<real> &a,
                                                real4<real> &vbar, real4<real> &rn) {
  using O = ops<real>;
  const real tx = O::add(v.x, O::mul(dt, a.x));
  const real ty = O::add(v.y, O::mul(dt, a.y));
  const real tz = O::add(v.z, O::mul(dt, a.z));
  rn = mk4<real>(O::add(r.x, O::mul(hdt, O::add(tx, v.x))), O::add(r.y, O::mul(hdt, O::add(ty, v.y))),
                 O::add(r.z, O::mul(hdt, O::add(tz, v.z))), r.w);
  vbar = mk4<real>(O::mul(O::add(v.x, tx), (real)0.5), O::mul(O::add(v.y, ty), (real)0.5),
                   O::mul(O::add(v.z, tz), (real)0.5), (real)0);
}

template <typename real>
__global__ void k_kdk_predict(int64_t n, real dt, real hdt, const real4<real> *__restrict__ posm,
                              const real4<real> *__restrict__ vel,
                              const real4<real> *__restrict__ acc, real4<real> *__restrict__ vbar,
                              real4<real> *__restrict__ posm_nxt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    real4<real> vb, rn;
    kdk_predict_one<real>(dt, hdt, posm[i], vel[i], acc[i], vb, rn);
    vbar[i] = vb;
    posm_nxt[i] = rn;
  }
}

// After the force at r(t+dt): a' = G sum(parts); corrector
//   v(t+dt) = vbar + dt/2 a'           (Eq. 7, chdt = dt/2 of the step just ended)
// then the predictor and drift of the next step, of size dt_next (the same dt
// for KDK; the next substep's for the fourth-order composition), into posm_pred.
template <typename real, typename P>
__global__ void k_kdk_correct_predict(const P *__restrict__ part, int S, int64_t n, real G,
                                      real chdt, real dt, real hdt, real4<real> *__restrict__ acc,
                                      const real4<real> *__restrict__ posm_new,
                                      real4<real> *__restrict__ vel, real4<real> *__restrict__ vbar,
                                      real4<real> *__restrict__ posm_pred) {
  using O = ops<real>;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const real4<real> a = gather_acc<real, P>(part, S, n, i, G);
    acc[i] = a;
    const real4<real> vb = vbar[i];
    const real4<real> v = mk4<real>(O::add(vb.x, O::mul(chdt, a.x)), O::add(vb.y, O::mul(chdt, a.y)),
                                    O::add(vb.z, O::mul(chdt, a.z)), (real)0);
    vel[i] = v;
    real4<real> nvb, rn;
    kdk_predict_one<real>(dt, hdt, posm_new[i], v, a, nvb, rn);
    vbar[i] = nvb;
    posm_pred[i] = rn;
  }
}

// ---------------------------------------------------------------- RK4
// Classical Runge-Kutta on (r, v) with running sums in the order
//   r(t+dt) = r + dt/6 (((v + 2 v2) + 2 v3) + v4)
//   v(t+dt) = v + dt/6 (((a1 + 2 a2) + 2 a3) + a4)
// where v2 = v + dt/2 a1, v3 = v + dt/2 a2, v4 = v + dt a3 and the stage
// positions are r + dt/2 v, r + dt/2 v2, r + dt v3.  Stage k runs after the
// force evaluation a_k.
template <typename real, typename P>
__global__ void k_rk4_stage(const P *__restrict__ part, int S, int64_t n, real G, int stage,
                            real dt, real hdt, real dt6, real4<real> *__restrict__ posm0,
                            real4<real> *__restrict__ vel0, real4<real> *__restrict__ vs,
                            real4<real> *__restrict__ sr, real4<real> *__restrict__ sv,
                            real4<real> *__restrict__ posm_stage) {
  using O = ops<real>;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const real4<real> a = gather_acc<real, P>(part, S, n, i, G);
    const real4<real> r0 = posm0[i];
    const real4<real> v0 = vel0[i];
    if (stage == 1) {
      const real4<real> v2 = mk4<real>(O::add(v0.x, O::mul(hdt, a.x)), O::add(v0.y, O::mul(hdt, a.y)),
                                       O::add(v0.z, O::mul(hdt, a.z)), (real)0);
      sv[i] = mk4<real>(a.x, a.y, a.z, (real)0);
      sr[i] = mk4<real>(O::add(v0.x, O::mul((real)2, v2.x)), O::add(v0.y, O::mul((real)2, v2.y)),
                        O::add(v0.z, O::mul((real)2, v2.z)), (real)0);
      vs[i] = v2;
      posm_stage[i] = mk4<real>(O::add(r0.x, O::mul(hdt, v0.x)), O::add(r0.y, O::mul(hdt, v0.y)),
                                O::add(r0.z, O::mul(hdt, v0.z)), r0.w);
    } else if (stage == 2 || stage == 3) {
      const real c = stage == 2 ? hdt : dt;  // v3 = v + dt/2 a2 ; v4 = v + dt a3
      const real4<real> vp = vs[i];          // v2 (stage 2) or v3 (stage 3)
      const real4<real> vn = mk4<real>(O::add(v0.x, O::mul(c, a.x)), O::add(v0.y, O::mul(c, a.y)),
                                       O::add(v0.z, O::mul(c, a.z)), (real)0);
      real4<real> s = sv[i];
      s = mk4<real>(O::add(s.x, O::mul((real)2, a.x)), O::add(s.y, O::mul((real)2, a.y)),
                    O::add(s.z, O::mul((real)2, a.z)), (real)0);
      sv[i] = s;
      real4<real> q = sr[i];
      const real w = stage == 2 ? (real)2 : (real)1;  // + 2 v3 ; + v4
      q = mk4<real>(O::add(q.x, O::mul(w, vn.x)), O::add(q.y, O::mul(w, vn.y)),
                    O::add(q.z, O::mul(w, vn.z)), (real)0);
      sr[i] = q;
      vs[i] = vn;
      // stage positions r + dt/2 v2 (after a2) and r + dt v3 (after a3)
      posm_stage[i] = mk4<real>(O::add(r0.x, O::mul(c, vp.x)), O::add(r0.y, O::mul(c, vp.y)),
                                O::add(r0.z, O::mul(c, vp.z)), r0.w);
    } else {
      const real4<real> s = sv[i];
      const real4<real> q = sr[i];
      const real sx = O::add(s.x, a.x), sy = O::add(s.y, a.y), sz = O::add(s.z, a.z);
      posm0[i] = mk4<real>(O::add(r0.x, O::mul(dt6, q.x)), O::add(r0.y, O::mul(dt6, q.y)),
                           O::add(r0.z, O::mul(dt6, q.z)), r0.w);
      vel0[i] = mk4<real>(O::add(v0.x, O::mul(dt6, sx)), O::add(v0.y, O::mul(dt6, sy)),
                          O::add(v0.z, O::mul(dt6, sz)), (real)0);
    }
  }
}

// ---------------------------------------------------------------- Eq. 8-10
constexpr int DIAG_BT = 256;

int diag_blocks(int64_t n) {
  int64_t b = (n + DIAG_BT - 1) / DIAG_BT;
  return (int)(b < 1024 ? b : 1024);
}

// Per-block sums of (K, W, Px, Py, Pz, Lx, Ly, Lz) with
//   K = m |v|^2 / 2, W = m pot / 2 (pot carries -G sum_j m_j / |r_ij + eps|),
//   P = m v (Eq. 9), L = m r x v (Eq. 10 is L_z),
// each block striding over particles in a fixed order and reducing in a
// fixed tree: the result is deterministic for a given n.
template <typename real>
__global__ void __launch_bounds__(DIAG_BT) k_diag_blocks(const real4<real> *__restrict__ posm,
                                                         const real4<real> *__restrict__ vel,
                                                         const real4<real> *__restrict__ acc,
                                                         int64_t n, double *__restrict__ blocks) {
  __shared__ double sh[8][DIAG_BT];
  double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)DIAG_BT + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * DIAG_BT) {
    const real4<real> p = posm[i];
    const real4<real> v = vel[i];
    const double m = p.w, x = p.x, y = p.y, z = p.z, vx = v.x, vy = v.y, vz = v.z;
    const double pot = acc[i].w;
    q[0] += m * (vx * vx + vy * vy + vz * vz) * 0.5;
    q[1] += m * pot * 0.5;
    q[2] += m * vx;
    q[3] += m * vy;
    q[4] += m * vz;
    q[5] += m * (y * vz - z * vy);
    q[6] += m * (z * vx - x * vz);
    q[7] += m * (x * vy - y * vx);
  }
  for (int c = 0; c < 8; c++) sh[c][threadIdx.x] = q[c];
  __syncthreads();
  for (int w = DIAG_BT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 8; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 8) blocks[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// out9 = (E, K, W, Px, Py, Pz, Lx, Ly, Lz) from nb block sums, fixed order.
__global__ void __launch_bounds__(DIAG_BT) k_diag_final(const double *__restrict__ blocks, int nb,
                                                        double *__restrict__ out9) {
  __shared__ double sh[8][DIAG_BT];
  double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nb; b += DIAG_BT)
    for (int c = 0; c < 8; c++) q[c] += blocks[b * 8 + c];
  for (int c = 0; c < 8; c++) sh[c][threadIdx.x] = q[c];
  __syncthreads();
  for (int w = DIAG_BT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 8; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out9[0] = sh[0][0] + sh[1][0];
    for (int c = 0; c < 8; c++) out9[1 + c] = sh[c][0];
  }
}

// ---------------------------------------------------------------- launchers
static unsigned grid_for(int64_t n, int bt = 256) {
  int64_t g = (n + bt - 1) / bt;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)(g < 1 ? 1 : g);
}

cudaError_t launch_pack(int mode, const double *pos, const double *vel, const double *mass,
                        int64_t n, void *posm, void *velv, int *flag, cudaStream_t st) {
  if (mode == NBODY_FP32)
    k_pack<float><<<grid_for(n), 256, 0, st>>>(pos, vel, mass, n, (float4 *)posm, (float4 *)velv,
                                               flag);
  else
    k_pack<double><<<grid_for(n), 256, 0, st>>>(pos, vel, mass, n, (d4 *)posm, (d4 *)velv, flag);
  return cudaGetLastError();
}

cudaError_t launch_unpack_state(int mode, const void *posm, const void *velv, int64_t n,
                                double *pos, double *vel, cudaStream_t st) {
  if (mode == NBODY_FP32)
    k_unpack_state<float><<<grid_for(n), 256, 0, st>>>((const float4 *)posm,
                                                       (const float4 *)velv, n, pos, vel);
  else
    k_unpack_state<double><<<grid_for(n), 256, 0, st>>>((const d4 *)posm, (const d4 *)velv, n,
                                                        pos, vel);
  return cudaGetLastError();
}

cudaError_t launch_store_acc(int mode, const EpiIn &e, void *acc, cudaStream_t st) {
  if (mode == NBODY_FP32)
    k_store_acc<float, float4><<<grid_for(e.n), 256, 0, st>>>((const float4 *)e.part, e.S, e.n,
                                                              (float)e.G, (float4 *)acc);
  else
    k_store_acc<double, d4><<<grid_for(e.n), 256, 0, st>>>((const d4 *)e.part, e.S, e.n, e.G,
                                                           (d4 *)acc);
  return cudaGetLastError();
}

cudaError_t launch_unpack_acc(int mode, const void *acc, int64_t n, double *acc3, double *pot,
                              cudaStream_t st) {
  if (mode == NBODY_FP32)
    k_unpack_acc<float><<<grid_for(n), 256, 0, st>>>((const float4 *)acc, n, acc3, pot);
  else
    k_unpack_acc<double><<<grid_for(n), 256, 0, st>>>((const d4 *)acc, n, acc3, pot);
  return cudaGetLastError();
}

cudaError_t launch_kdk_predict(int mode, int64_t n, double dt, const void *posm_cur,
                               const void *vel, const void *acc, void *vbar, void *posm_nxt,
                               cudaStream_t st) {
  if (mode == NBODY_FP32)
    k_kdk_predict<float><<<grid_for(n), 256, 0, st>>>(
        n, (float)dt, (float)(dt / 2), (const float4 *)posm_cur, (const float4 *)vel,
        (const float4 *)acc, (float4 *)vbar, (float4 *)posm_nxt);
  else
    k_kdk_predict<double><<<grid_for(n), 256, 0, st>>>(n, dt, dt / 2, (const d4 *)posm_cur,
                                                       (const d4 *)vel, (const d4 *)acc,
                                                       (d4 *)vbar, (d4 *)posm_nxt);
  return cudaGetLastError();
}

cudaError_t launch_kdk_correct_predict(int mode, const EpiIn &e, double dt, double dt_next,
                                       void *acc, void *posm_new, void *vel, void *vbar,
                                       void *posm_pred, cudaStream_t st) {
  if (mode == NBODY_FP32)
    k_kdk_correct_predict<float, float4><<<grid_for(e.n), 256, 0, st>>>(
        (const float4 *)e.part, e.S, e.n, (float)e.G, (float)(dt / 2), (float)dt_next,
        (float)(dt_next / 2), (float4 *)acc, (const float4 *)posm_new, (float4 *)vel,
        (float4 *)vbar, (float4 *)posm_pred);
  else
    k_kdk_correct_predict<double, d4><<<grid_for(e.n), 256, 0, st>>>(
        (const d4 *)e.part, e.S, e.n, e.G, dt / 2, dt_next, dt_next / 2, (d4 *)acc,
        (const d4 *)posm_new, (d4 *)vel, (d4 *)vbar, (d4 *)posm_pred);
  return cudaGetLastError();
}

cudaError_t launch_rk4_stage(int mode, const EpiIn &e, int stage, double dt, const void *posm0,
                             void *vel0, void *rk_vs, void *rk_sr, void *rk_sv, void *posm_stage,
                             cudaStream_t st) {
  if (mode == NBODY_FP32)
    k_rk4_stage<float, float4><<<grid_for(e.n), 256, 0, st>>>(
        (const float4 *)e.part, e.S, e.n, (float)e.G, stage, (float)dt, (float)(dt / 2),
        (float)(dt / 6), (float4 *)posm0, (float4 *)vel0, (float4 *)rk_vs, (float4 *)rk_sr,
        (float4 *)rk_sv, (float4 *)posm_stage);
  else
    k_rk4_stage<double, d4><<<grid_for(e.n), 256, 0, st>>>(
        (const d4 *)e.part, e.S, e.n, e.G, stage, dt, dt / 2, dt / 6, (d4 *)posm0, (d4 *)vel0,
        (d4 *)rk_vs, (d4 *)rk_sr, (d4 *)rk_sv, (d4 *)posm_stage);
  return cudaGetLastError();
}

cudaError_t launch_diag(int mode, const void *posm, const void *vel, const void *acc, int64_t n,
                        double *blocks, int nblocks, double *out9, cudaStream_t st) {
  if (mode == NBODY_FP32)
    k_diag_blocks<float><<<nblocks, DIAG_BT, 0, st>>>((const float4 *)posm, (const float4 *)vel,
                                                      (const float4 *)acc, n, blocks);
  else
    k_diag_blocks<double><<<nblocks, DIAG_BT, 0, st>>>((const d4 *)posm, (const d4 *)vel,
                                                       (const d4 *)acc, n, blocks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_diag_final<<<1, DIAG_BT, 0, st>>>(blocks, nblocks, out9);
  return cudaGetLastError();
}

}  // namespace nb
