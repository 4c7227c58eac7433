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
// Four arithmetics:
//   f64   binary64 pair arithmetic.  GB300 issues binary64 at about 1/72 of the
//         binary32 rate, so the kernel is bound by the FP64 pipe and its cost
//         is its count of FP64 instructions per pair: 9 (3 DADD for d,
//         3 DFMA for |d|^2 + eps^2, 3 DFMA for the acceleration sums).  The
//         rest runs on the otherwise idle integer and FP32 pipes: 1/r and
//         1/r^2 within 0.52 ulp (SFU seed, exact integer residual), the
//         products m/r and (m/r)/r^2 by a correctly rounded integer binary64
//         multiply, and the potential sum by a correctly rounded integer
//         binary64 add.  From 64 blocks of 384 particles the FP64 path
//         evaluates each pair once for both particles (k_force_f64_sym:
//         12 FP64 instructions per pair, 6 per interaction).
//   mixed binary32 pair arithmetic (packed: two j per instruction, SFU
//         reciprocal square root) on coordinates re-centred on an anchor (the
//         per-coordinate median) per j-tile, with the i coordinates held as
//         float-float pairs so that the per-tile shift costs three binary32
//         operations per coordinate and no FP64 instruction; per-tile binary32
//         partial sums are folded into float-float (compensated, TwoSum)
//         accumulators, returned as binary64.
//   f64e  binary64-class accuracy on the binary32 pipes: float-float (about 48
//         significant bits) pair arithmetic on coordinates re-centred per
//         j-tile, float-float tile partials folded into binary64 per tile.
//         About 160 binary32 instructions per pair, but on pipes 64 times
//         faster than GB300's FP64 pipe.  From 64 blocks of 256 particles it
//         evaluates each pair once for both particles (k_force_f64e_sym).
//   f32   binary32 throughout (packed pairs, SFU reciprocal square root) with
//         plain binary32 accumulation: the paper's SP.  The two halves of a
//         thread's packed accumulators (even and odd j) are added at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "nbody_internal.cuh"

namespace nb {

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/sqrt(x) and 1/x in binary64 (each within about 0.52 ulp) for x in
// [2^-60, 2^60), without any FP64 instruction: GB300's FP64 pipe is the
// bottleneck of the FP64 force kernel, while its FP32 and integer pipes are
// idle there.  Inputs are the two halves of x; outputs are the 53-bit
// significands (in [2^52, 2^53)) and biased binary64 exponents.
//  1. x = xh + xl in binary32: xh = the top 24 significant bits of x moved
//     into a float by integer operations (exponent 1023 -> 127), xl = the
//     next 29 bits converted and scaled (relative error 2^-47 of x).
//  2. Seed y0 = SFU rsqrt(xh) (relative error below 2^-21), improved on the
//     FP32 pipe: e0 = 1 - x y0^2 from exact products (TwoProd by FMA);
//     g = e0 (1/2 + 3 e0/8), the second-order correction.
//  3. s = y0 (1 + g) as an integer significand S in [2^30, 2^31) with a
//     binary64 exponent E: s = S 2^(E - 1053), |x s^2 - 1| < 2^-29.
//  4. Exact residual in integers: with X the 53-bit significand of x,
//     P = X S^2 is within 2^(K-29) of 2^K, K = 3181 - Ex - 2E; the low 96 bits
//     of P (three 32x32 products and the high half of the fourth) give
//     T = (P - 2^K) / 2^32 exactly as a signed 64-bit integer, and
//     e = 1 - x s^2 = -T 2^(32-K).
//  5. 1/sqrt(x) = s (1 + e/2 + 3e^2/8 + ...) and 1/x = s^2 (1 + e + e^2 ...);
//     e^2 < 2^-58 is below the rounding, so the significands are
//     S 2^22 - S T 2^(53-K) and S^2 / 2^sh - (S^2 / 2^32) T 2^(64-K-sh), formed
//     with 8 fraction bits, renormalised by one bit if they left [2^52, 2^53)
//     and rounded to nearest.
__device__ __forceinline__ void rsqrt_recip_sig(unsigned hi, unsigned lo, uint64_t &R, int &ER,
                                                uint64_t &Q, int &EQ) {
  // 1-2: binary32 seed and second-order correction
  const float xh = __uint_as_float(__funnelshift_l(lo, hi - 0x38000000u, 3));
  const float scale = __uint_as_float(((hi >> 20) - 948u) << 23);  // 2^(Ex - 1075)
  const float xl = __uint2float_rn(lo & 0x1FFFFFFFu) * scale;
  const float y0 = rsqrt_approx(xh);
  const float th = y0 * y0, tl = fmaf(y0, y0, -th);
  const float u = xh * th, ue = fmaf(xh, th, -u);
  const float e0 = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, u), ue), fmaf(xh, tl, xl * th));
  const float g = e0 * fmaf(e0, 0.375f, 0.5f);
  // 3: S = y0's significand at a 2^30 scale plus y0 g rounded at that scale
  const unsigned yb = __float_as_uint(y0);
  const float y0m = __uint_as_float((yb & 0x7FFFFFu) | 0x3F800000u);  // y0's significand in [1, 2)
  const int ci = __float2int_rn(y0m * (g * 1073741824.0f));
  unsigned S = (((yb & 0x7FFFFFu) | 0x800000u) << 7) + (unsigned)ci;
  int E = (int)((yb >> 23) & 0xFFu) + 896;
  if (S >= 0x80000000u) {
    S >>= 1;
    E += 1;
  } else if (S < 0x40000000u) {
    S <<= 1;
    E -= 1;
  }
  // 4: T = (X S^2 - 2^K) / 2^32 from the low 96 bits of the product
  const int Ex = (int)(hi >> 20);
  const unsigned a1 = (hi & 0xFFFFFu) | 0x100000u;
  const uint64_t S2 = (uint64_t)S * S;
  const unsigned b1 = (unsigned)(S2 >> 32), b0 = (unsigned)S2;
  uint64_t Tu = (uint64_t)a1 * b0 + __umulhi(lo, b0);
  Tu += (uint64_t)lo * b1;
  Tu += (uint64_t)(a1 * b1) << 32;
  const int Th = (int)(Tu >> 32);
  const unsigned Tl = (unsigned)Tu;
  // 5a: 1/sqrt(x)
  const int64_t ST = (int64_t)(int)S * Th + (int64_t)__umulhi(S, Tl);  // S T / 2^32
  const int64_t Rf = (int64_t)((uint64_t)S << 30) - (ST >> (3088 - Ex - 2 * E));
  const int sR = 8 + (Rf >= (int64_t)1 << 61) - (Rf < (int64_t)1 << 60);
  R = (uint64_t)(Rf + ((int64_t)1 << (sR - 1))) >> sR;
  ER = E + sR - 8;
  // 5b: 1/x
  const int sh = 8 + (b1 >= 0x20000000u);
  const int64_t BT = (int64_t)b1 * Th + (int64_t)__umulhi(b1, Tl);  // (S^2 / 2^32) T / 2^32
  const int64_t Qf = (int64_t)(S2 >> (sh - 8)) - (BT >> (3077 - Ex - 2 * E + sh));
  const int sQ = 8 + (Qf >= (int64_t)1 << 61) - (Qf < (int64_t)1 << 60);
  Q = (uint64_t)(Qf + ((int64_t)1 << (sQ - 1))) >> sQ;
  EQ = sh + 2 * E - 1031 + sQ - 8;
}

// Binary64 multiplication on the integer pipes, correctly rounded (to nearest,
// ties to even): significands A in [2^52, 2^53] and B in [2^52, 2^53) with
// biased exponents ea, eb; the caller guarantees a normal result.  The 106-bit
// product comes from four 32x32 products; U = its top 64 bits (in [2^62, 2^64)),
// the bits below form the sticky bit.  Returns the significand (2^53 after a
// rounding carry, which the packing below absorbs into the exponent) and the
// biased exponent.
__device__ __forceinline__ uint64_t mul_sig(uint64_t A, int ea, uint64_t B, int eb, int &e) {
  const unsigned a1 = (unsigned)(A >> 32), a0 = (unsigned)A;
  const unsigned b1 = (unsigned)(B >> 32), b0 = (unsigned)B;
  const uint64_t lo = (uint64_t)a0 * b0;
  uint64_t V = (uint64_t)a1 * b0 + (lo >> 32);
  V += (uint64_t)a0 * b1;
  const uint64_t U = (((uint64_t)a1 * b1) << 22) + (V >> 10);
  const int n = (int)(U >> 63);
  const int sft = 10 + n;
  const uint64_t sig = U >> sft;
  const uint64_t rb = (U >> (sft - 1)) & 1u;
  const bool st = ((U & (((uint64_t)1 << (sft - 1)) - 1u)) | (V & 0x3FFu) | (unsigned)lo) != 0;
  e = ea + eb - 1023 + n;
  return sig + (rb & (uint64_t)(st | (bool)(sig & 1u)));
}
__device__ __forceinline__ double pack_f64(uint64_t sig, int e) {
  return __longlong_as_double((long long)((((uint64_t)(e - 1)) << 52) + sig));
}

// Binary64 addition of two non-negative numbers on the integer pipes (the
// potential sum of the one-sided kernel), correctly rounded to nearest even and
// bit-identical to DADD: significands at bit 62 of a 64-bit word, the smaller
// one shifted right by the exponent difference with a sticky bit, at most a
// one-bit normalisation after a carry, rounded at bit 10.  ok = false for a
// subnormal or overflowing result or a negative operand, where the caller adds
// in binary64 out of line.  It costs about 40 ALU-pipe instructions, less ALU
// time than the FP64 pipe time of one DADD (one FP64 instruction takes the
// pipe as long as 32 ALU instructions): +12 % measured in the one-sided
// kernel, and in the each-pair-once kernel, for both of its potential sums,
// +22 % together with the block shape that makes room for the registers.
__device__ __forceinline__ uint64_t add_pos_bits(uint64_t a, uint64_t b, bool &ok) {
  const uint64_t M52 = 0xFFFFFFFFFFFFFull;
  const bool sw = b > a;
  const uint64_t X = sw ? b : a, Y = sw ? a : b;
  const int eX = (int)(X >> 52), eY = (int)(Y >> 52);
  const uint64_t MX = ((X & M52) | ((uint64_t)1 << 52)) << 10;
  const uint64_t MY0 = ((Y & M52) | ((uint64_t)(eY != 0) << 52)) << 10;
  const int dc = min(eX - eY, 63);
  const uint64_t st = (MY0 & (((uint64_t)1 << dc) - 1u)) != 0;
  const uint64_t S = (MX + (MY0 >> dc)) | st;
  const int c = (int)(S >> 63);
  const uint64_t N = (S >> c) | (S & (uint64_t)c);
  uint64_t sig = N >> 10;
  sig += ((N >> 9) & 1u) & (uint64_t)(((N & 0x1FFu) != 0) | (bool)(sig & 1u));
  const int E = eX + c;
  ok = (E <= 2046 && !(eY == 0 && Y != 0) && eX != 0 && ((a | b) >> 63) == 0) || X == 0;
  return X == 0 ? 0 : ((uint64_t)(E - 1) << 52) + sig;
}
__device__ __noinline__ uint64_t add_pos_slow(uint64_t a, uint64_t b) {
  return (uint64_t)__double_as_longlong(__longlong_as_double((long long)a) +
                                        __longlong_as_double((long long)b));
}
// acc += v for the bit pattern acc of a non-negative binary64 sum
__device__ __forceinline__ void acc_pos(uint64_t &acc, double v) {
  bool ok;
  const uint64_t vb = (uint64_t)__double_as_longlong(v);
  const uint64_t r = add_pos_bits(acc, vb, ok);
  if (ok)
    acc = r;
  else
    acc = add_pos_slow(acc, vb);
}

// The same quantities in binary64 arithmetic, out of line: for r^2 outside
// [2^-60, 2^60) (and zero or non-finite) and for masses outside
// [2^-895, 2^897) (and zero), where the integer path's ranges do not hold.
__device__ __noinline__ double2 pair_scale_f64_slow(double r2, double m) {
  const double my = m * (1.0 / sqrt(r2));
  return make_double2(my, my * (1.0 / r2));
}

// float-float accumulation a += b (Knuth's TwoSum; exact error term).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b) {
  const float s = __fadd_rn(hi, b);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// ---------------------------------------------------------------- work descriptors
// A kernel runs units k = first(), first() + stride(), ... < count().
// Dense: one system of n particles; block (x, y) = i-block x of the rows
// [i_base, i_base + rows) against j-segment y of all n; the row sums go to
// part[y * rows + (i - i_base)] (all rows: i_base = 0, rows = n).
struct DenseWork {
  int64_t n, seg, i_base, rows;
  double eps2;
  int per_block, tile;
  __device__ __forceinline__ int64_t first() const { return 0; }
  __device__ __forceinline__ int64_t stride() const { return 1; }
  __device__ __forceinline__ int64_t count() const { return 1; }
  __device__ __forceinline__ Unit get(int64_t) const {
    Unit u;
    const int64_t r0 = (int64_t)blockIdx.x * per_block;
    u.i0 = i_base + r0;
    u.ni = (int)min((int64_t)per_block, rows - r0);
    u.j0 = (int64_t)blockIdx.y * seg;
    u.nj = (int)min(seg, n - u.j0);
    u.out = (int64_t)blockIdx.y * rows + r0;
    u.anchor = u.j0 / tile;
    u.eps2 = eps2;
    return u;
  }
};
// Table: block x runs units[x], units[x + gridDim.x], ... (many systems of
// uneven size in one launch; a grid smaller than the table makes the launch
// persistent, which caps how many of its blocks sit on an SM at once).
struct TableWork {
  const Unit *units;
  int64_t n;
  __device__ __forceinline__ int64_t first() const { return blockIdx.x; }
  __device__ __forceinline__ int64_t stride() const { return gridDim.x; }
  __device__ __forceinline__ int64_t count() const { return n; }
  __device__ __forceinline__ Unit get(int64_t k) const { return units[k]; }
};

// ---------------------------------------------------------------- binary64
template <bool MASK>
__device__ __forceinline__ void body_f64(const d4 &pj, double xi, double yi, double zi,
                                         double eps2, double &ax, double &ay, double &az,
                                         uint64_t &pt, bool self) {
  const double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
  double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
  double m = pj.w;
  if (MASK && self) {
    r2 = 1.0;
    m = 0.0;
  }
  // my = m / r and f = my / r^2, both binary64 products correctly rounded
  const unsigned hi = (unsigned)__double2hiint(r2);
  const unsigned mh = (unsigned)__double2hiint(m);
  double my, f;
  if (hi - 0x3C300000u < 0x43B00000u - 0x3C300000u && (mh >> 20) - 128u < 1793u) {
    uint64_t R, Q;
    int ER, EQ, emy, ef;
    rsqrt_recip_sig(hi, (unsigned)__double2loint(r2), R, ER, Q, EQ);
    const uint64_t Am = ((uint64_t)((mh & 0xFFFFFu) | 0x100000u) << 32) | (unsigned)__double2loint(m);
    const uint64_t smy = mul_sig(Am, (int)(mh >> 20), R, ER, emy);
    const uint64_t sf = mul_sig(smy, emy, Q, EQ, ef);
    my = pack_f64(smy, emy);
    f = pack_f64(sf, ef);
  } else {
    const double2 v = pair_scale_f64_slow(r2, m);
    my = v.x;
    f = v.y;
  }
  ax = fma(dx, f, ax);
  ay = fma(dy, f, ay);
  az = fma(dz, f, az);
  acc_pos(pt, my);  // the potential sum: integer pipes
}

template <int BT, int R, int T, class W>
__global__ void __launch_bounds__(BT) k_force_f64(const d4 *__restrict__ posm, W work,
                                                  d4 *__restrict__ part) {
  __shared__ d4 tile[T];
  for (int64_t uk = work.first(); uk < work.count(); uk += work.stride()) {
    const Unit u = work.get(uk);
    const int tid = threadIdx.x;
    const int64_t j1 = u.j0 + u.nj;
    const double eps2 = u.eps2;
    double xi[R], yi[R], zi[R], ax[R], ay[R], az[R];
    uint64_t pt[R];  // bit patterns of the potential sums
  #pragma unroll
    for (int r = 0; r < R; r++) {
      const int li = r * BT + tid;
      const d4 p = posm[u.i0 + (li < u.ni ? li : 0)];
      xi[r] = p.x;
      yi[r] = p.y;
      zi[r] = p.z;
      ax[r] = ay[r] = az[r] = 0.0;
      pt[r] = 0;
    }
    for (int64_t jt = u.j0; jt < j1; jt += T) {
      const int cnt = (int)min((int64_t)T, j1 - jt);
      __syncthreads();
      for (int k = tid; k < cnt; k += BT) tile[k] = posm[jt + k];
      __syncthreads();
      const bool diag = (jt < u.i0 + u.ni) && (jt + cnt > u.i0);
      if (cnt == T && !diag) {
  #pragma unroll 2
        for (int k = 0; k < T; k++) {
          const d4 pj = tile[k];
  #pragma unroll
          for (int r = 0; r < R; r++)
            body_f64<false>(pj, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pt[r], false);
        }
      } else if (cnt == T) {  // a full tile that holds some of this block's own i
  #pragma unroll 2
        for (int k = 0; k < T; k++) {
          const d4 pj = tile[k];
          const int64_t j = jt + k;
  #pragma unroll
          for (int r = 0; r < R; r++)
            body_f64<true>(pj, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pt[r],
                           j == u.i0 + r * BT + tid);
        }
      } else {
        for (int k = 0; k < cnt; k++) {
          const d4 pj = tile[k];
          const int64_t j = jt + k;
  #pragma unroll
          for (int r = 0; r < R; r++)
            body_f64<true>(pj, xi[r], yi[r], zi[r], eps2, ax[r], ay[r], az[r], pt[r],
                           j == u.i0 + r * BT + tid);
        }
      }
    }
  #pragma unroll
    for (int r = 0; r < R; r++) {
      const int li = r * BT + tid;
      if (li < u.ni)
        part[u.out + li] = d4{ax[r], ay[r], az[r], __longlong_as_double((long long)pt[r])};
    }
  }
}

// ---------------------------------------------------------------- binary64, each pair once
// Newton's third law: the pair (i, j) contributes m_j d / w to a_i and
// -m_i d / w to a_j with the same d = r_j - r_i and w = (|d|^2 + eps^2)^{3/2},
// so one evaluation of d, |d|^2 + eps^2, 1/r and 1/r^2 serves both: 12 FP64
// instructions for two interactions instead of 18 (the one-sided kernel's 9 twice).
//
// Particles are cut into M blocks of B = BT*R.  A work item (d, I), d >= 1,
// pairs i-block I with j-block J = (I + d) mod M; d = 1 .. floor(M/2) covers
// every unordered pair of distinct blocks once (for d = M/2 with M even, only
// I < M/2 computes; the other items write zeros).  For a fixed d every block
// is the row block of one item and the column block of one item, so the
// item's row sums (block I) and column sums (block J) each own a slice of the
// per-diagonal buffers rows[dl], cols[dl] without any atomic or race; the
// slices are added in diagonal order afterwards (deterministic).  Pairs
// inside a block (d = 0) run through the one-sided kernel.
//
// Column sums: i stays in registers (R per thread); a j-tile of T particles
// is in shared memory and is walked in chunks of 32.  At step k of a chunk,
// lane l works on j = (l + k) mod 32 with its R i-particles and then hands the
// running sum of that j to lane l - 1, so after 32 steps lane l holds the sum
// over the warp's i-particles of j = l.  The warps' sums are then added in a
// fixed order in shared memory.
__device__ __noinline__ double2 rq_f64_slow(double r2) {
  return make_double2(1.0 / sqrt(r2), 1.0 / r2);
}

struct MassSig {
  uint64_t A;  // 53-bit significand
  int e;       // biased exponent
  bool fast;   // in [2^-895, 2^897): the integer multiply applies
};
__device__ __forceinline__ MassSig mass_sig(double m) {
  const unsigned mh = (unsigned)__double2hiint(m);
  MassSig s;
  s.A = ((uint64_t)((mh & 0xFFFFFu) | 0x100000u) << 32) | (unsigned)__double2loint(m);
  s.e = (int)(mh >> 20);
  s.fast = (mh >> 20) - 128u < 1793u;
  return s;
}

// m/r and (m/r)/r^2 from the integer 1/r, 1/r^2 (or, for masses outside the
// integer range, binary64 products of their packed values)
__device__ __forceinline__ void scale_pair(double m, const MassSig &ms, uint64_t R, int ER,
                                           uint64_t Q, int EQ, double &my, double &f) {
  if (ms.fast) {
    int emy, ef;
    const uint64_t smy = mul_sig(ms.A, ms.e, R, ER, emy);
    const uint64_t sf = mul_sig(smy, emy, Q, EQ, ef);
    my = pack_f64(smy, emy);
    f = pack_f64(sf, ef);
  } else {
    my = m * pack_f64(R, ER);
    f = my * pack_f64(Q, EQ);
  }
}

// Both potential sums, pt (row) and gp (column), are bit patterns added on the
// integer pipes (acc_pos, bit-identical to DADD): 12 FP64 instructions per
// pair, 6 per interaction.
__device__ __forceinline__ void body_f64_sym(const d4 &pj, const MassSig &mj, double xi,
                                             double yi, double zi, double mi,
                                             const MassSig &msi, double eps2, double &ax,
                                             double &ay, double &az, uint64_t &pt, double &gx,
                                             double &gy, double &gz, uint64_t &gp) {
  const double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
  const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
  const unsigned hi = (unsigned)__double2hiint(r2);
  double my, f, myj, fj;
  if (hi - 0x3C300000u < 0x43B00000u - 0x3C300000u) {
    uint64_t R, Q;
    int ER, EQ;
    rsqrt_recip_sig(hi, (unsigned)__double2loint(r2), R, ER, Q, EQ);
    scale_pair(pj.w, mj, R, ER, Q, EQ, my, f);
    scale_pair(mi, msi, R, ER, Q, EQ, myj, fj);
  } else {
    const double2 v = rq_f64_slow(r2);
    my = pj.w * v.x;
    f = my * v.y;
    myj = mi * v.x;
    fj = myj * v.y;
  }
  ax = fma(dx, f, ax);
  ay = fma(dy, f, ay);
  az = fma(dz, f, az);
  acc_pos(pt, my);
  gx = fma(-dx, fj, gx);
  gy = fma(-dy, fj, gy);
  gz = fma(-dz, fj, gz);
  acc_pos(gp, myj);
}

// Padding beyond n: massless and far away (finite r^2, zero contribution).
__device__ __forceinline__ d4 pad_or_load(const d4 *posm, int64_t k, int64_t n) {
  return k < n ? posm[k] : d4{1e30, 1e30, 1e30, 0.0};
}

template <int BT, int R, int T>
__global__ void __launch_bounds__(BT) k_force_f64_sym(const d4 *__restrict__ posm, int64_t n,
                                                      double eps2, int M, int d0,
                                                      d4 *__restrict__ rows,
                                                      d4 *__restrict__ cols) {
  constexpr int B = BT * R, NW = BT / 32;
  static_assert(T == BT && B % T == 0, "one column sum per thread per tile");
  __shared__ d4 tile[T];
  __shared__ d4 colw[NW][T];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int dl = blockIdx.x / M, I = blockIdx.x % M, d = d0 + dl;
  const int J = (I + d) % M;
  const int64_t i0 = (int64_t)I * B, j0 = (int64_t)J * B;
  d4 *rowo = rows + (int64_t)dl * n;
  d4 *colo = cols + (int64_t)dl * n;
  if (2 * d == M && I >= M / 2) {  // the pair of blocks is the item (I - M/2, I)
    for (int k = tid; k < B; k += BT) {
      if (i0 + k < n) rowo[i0 + k] = d4{0.0, 0.0, 0.0, 0.0};
      if (j0 + k < n) colo[j0 + k] = d4{0.0, 0.0, 0.0, 0.0};
    }
    return;
  }
  double xi[R], yi[R], zi[R], mi[R], ax[R], ay[R], az[R];
  uint64_t pt[R];  // bit patterns of the row potential sums
  MassSig msi[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const d4 p = pad_or_load(posm, i0 + r * BT + tid, n);
    xi[r] = p.x;
    yi[r] = p.y;
    zi[r] = p.z;
    mi[r] = p.w;
    msi[r] = mass_sig(p.w);
    ax[r] = ay[r] = az[r] = 0.0;
    pt[r] = 0;
  }
  for (int t0 = 0; t0 < B; t0 += T) {
    const int64_t jt = j0 + t0;
    __syncthreads();
    for (int k = tid; k < T; k += BT) tile[k] = pad_or_load(posm, jt + k, n);
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < T; c += 32) {
      double gx = 0.0, gy = 0.0, gz = 0.0;
      uint64_t gp = 0;  // bit pattern of the column potential sum
      // not unrolled: measured on GB300 at N = 2^18, unroll 2 ran 4 % slower
#pragma unroll 1
      for (int k = 0; k < 32; k++) {
        const d4 pj = tile[c + ((lane + k) & 31)];
        const MassSig mj = mass_sig(pj.w);
#pragma unroll
        for (int r = 0; r < R; r++)
          body_f64_sym(pj, mj, xi[r], yi[r], zi[r], mi[r], msi[r], eps2, ax[r], ay[r], az[r],
                       pt[r], gx, gy, gz, gp);
        const int src = (lane + 1) & 31;
        gx = __shfl_sync(0xFFFFFFFFu, gx, src);
        gy = __shfl_sync(0xFFFFFFFFu, gy, src);
        gz = __shfl_sync(0xFFFFFFFFu, gz, src);
        gp = __shfl_sync(0xFFFFFFFFu, gp, src);
      }
      colw[warp][c + lane] = d4{gx, gy, gz, __longlong_as_double((long long)gp)};
    }
    __syncthreads();
    {
      d4 s = colw[0][tid];
#pragma unroll
      for (int w = 1; w < NW; w++) {
        const d4 v = colw[w][tid];
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
      }
      if (jt + tid < n) colo[jt + tid] = s;
    }
  }
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = i0 + r * BT + tid;
    if (i < n) rowo[i] = d4{ax[r], ay[r], az[r], __longlong_as_double((long long)pt[r])};
  }
}

// acc_rows[i] (+)= rows[0][i] + ... + rows[D-1][i], the same for the columns,
// in diagonal order.
__global__ void k_sym_combine(const d4 *__restrict__ rows, const d4 *__restrict__ cols, int D,
                              int64_t n, d4 *__restrict__ acc_rows, d4 *__restrict__ acc_cols,
                              int first) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    d4 a = first ? d4{0.0, 0.0, 0.0, 0.0} : acc_rows[i];
    d4 b = first ? d4{0.0, 0.0, 0.0, 0.0} : acc_cols[i];
    for (int k = 0; k < D; k++) {
      const d4 u = rows[(int64_t)k * n + i], v = cols[(int64_t)k * n + i];
      a.x += u.x;
      a.y += u.y;
      a.z += u.z;
      a.w += u.w;
      b.x += v.x;
      b.y += v.y;
      b.z += v.z;
      b.w += v.w;
    }
    acc_rows[i] = a;
    acc_cols[i] = b;
  }
}

// ---------------------------------------------------------------- packed binary32 pairs
// Two j-particles per instruction with the packed FP32 instructions of sm_100+
// (one issue slot drives two lanes of FMA-pipe work).  Shared-memory tile
// entry k holds j = 2k and 2k+1 as A = (x0, x1, y0, y1), B = (z0, z1, m0, m1).
// (nx, ny, nz) are the negated i coordinates in both halves.  An odd tail is
// padded with a massless particle at 1e18 (finite r^2, zero contribution).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// REFINE adds one Newton step to the SFU reciprocal square root (4 more FMA-pipe
// operations).  Both packed kernels run without it: measured against the oracle
// on the disk + halo and uniform-sphere workloads, the step changed the RMS force
// error of the mixed kernel by less than 0.2 % (coordinate rounding and
// accumulation dominate) while costing 26 % of its throughput.
template <bool MASK, bool REFINE>
__device__ __forceinline__ void body_pair(const float4 &A, const float4 &B, float2 nx, float2 ny,
                                          float2 nz, float2 e2, float2 &ax, float2 &ay,
                                          float2 &az, float2 &pt, bool self0, bool self1) {
  const float2 dx = __fadd2_rn(f2(A.x, A.y), nx);
  const float2 dy = __fadd2_rn(f2(A.z, A.w), ny);
  const float2 dz = __fadd2_rn(f2(B.x, B.y), nz);
  float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
  float2 m = f2(B.z, B.w);
  if (MASK) {
    if (self0) {
      r2.x = 1.0f;
      m.x = 0.0f;
    }
    if (self1) {
      r2.y = 1.0f;
      m.y = 0.0f;
    }
  }
  float2 y = f2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
  if (REFINE) {  // y += y (1 - r2 y^2) / 2, as (-y/2) (r2 y^2 - 1) + y
    const float2 e = __ffma2_rn(__fmul2_rn(r2, y), y, f2(-1.0f, -1.0f));
    y = __ffma2_rn(__fmul2_rn(y, f2(-0.5f, -0.5f)), e, y);
  }
  const float2 my = __fmul2_rn(m, y);
  const float2 f = __fmul2_rn(my, __fmul2_rn(y, y));
  ax = __ffma2_rn(dx, f, ax);
  ay = __ffma2_rn(dy, f, ay);
  az = __ffma2_rn(dz, f, az);
  pt = __fadd2_rn(pt, my);
}

// Stage j-particles [jt, jt+cnt) of `src` (float4 x, y, z, m) as pairs.
template <int BT, int T>
__device__ __forceinline__ void load_pairs(const float4 *__restrict__ src, int64_t jt, int cnt,
                                           float4 *tA, float4 *tB) {
  const float4 dummy = make_float4(1e18f, 1e18f, 1e18f, 0.0f);
  for (int k = threadIdx.x; 2 * k < cnt; k += BT) {
    const float4 a = src[jt + 2 * k];
    const float4 b = 2 * k + 1 < cnt ? src[jt + 2 * k + 1] : dummy;
    tA[k] = make_float4(a.x, b.x, a.y, b.y);
    tB[k] = make_float4(a.z, b.z, a.w, b.w);
  }
}

// ---------------------------------------------------------------- float-float (F64E)
// Binary64-class arithmetic on the binary32 pipes: every quantity is an
// unevaluated sum hi + lo of two floats (about 48 significant bits), built
// from the error-free transformations TwoSum (Knuth), Fast2Sum (Dekker,
// |a| >= |b|) and TwoProd via FMA; two j-particles per packed instruction.
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  unsigned long long A, B, D;
  memcpy(&A, &a, 8);
  memcpy(&B, &b, 8);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D) : "l"(A), "l"(B));
  float2 d;
  memcpy(&d, &D, 8);
  return d;
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
  s = __fadd2_rn(a, b);
  const float2 bb = fsub2(s, a);
  e = __fadd2_rn(fsub2(a, fsub2(s, bb)), fsub2(b, bb));
}
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
  s = __fadd2_rn(a, b);
  e = fsub2(b, fsub2(s, a));
}
__device__ __forceinline__ void two_prod2(float2 a, float2 b, float2 &p, float2 &e) {
  p = __fmul2_rn(a, b);
  e = __ffma2_rn(a, b, neg2(p));
}
__device__ __forceinline__ void two_sum1(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Exact binary32 -> binary64 by integer moves (zero and subnormal inputs give
// 0, which is far below the precision of any value they are added to).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned mag = b & 0x7fffffffu;
  if (mag < 0x00800000u) return 0.0;
  return __hiloint2double((int)((b & 0x80000000u) | ((mag >> 3) + 0x38000000u)), (int)(b << 29));
}

// One tile entry: j = 2k, 2k+1 as H = (xh0, xh1, yh0, yh1), H2 = (zh0, zh1, mh0, mh1),
// L, L2 the matching low parts.  (nxh, nxl, ...) are the negated float-float
// i coordinates in both halves; the four float-float accumulators get the
// terms m_j d_ij / w_ij (x, y, z) and m_j / sqrt(d^2 + eps^2).
template <bool MASK>
__device__ __forceinline__ void body_ff(const float4 &H, const float4 &H2, const float4 &L,
                                        const float4 &L2, float2 nxh, float2 nxl, float2 nyh,
                                        float2 nyl, float2 nzh, float2 nzl, float2 e2h, float2 e2l,
                                        float2 (&ah)[4], float2 (&al)[4], bool self0, bool self1) {
  float2 dh[3], dl[3];
  {
    const float2 jh[3] = {f2(H.x, H.y), f2(H.z, H.w), f2(H2.x, H2.y)};
    const float2 jl[3] = {f2(L.x, L.y), f2(L.z, L.w), f2(L2.x, L2.y)};
    const float2 ih[3] = {nxh, nyh, nzh}, il[3] = {nxl, nyl, nzl};
#pragma unroll
    for (int c = 0; c < 3; c++) {  // d = (jh + jl) - (ih + il), renormalised
      float2 s, e;
      two_sum2(jh[c], ih[c], s, e);
      const float2 t = __fadd2_rn(__fadd2_rn(jl[c], il[c]), e);
      two_sum2(s, t, dh[c], dl[c]);
    }
  }
  // r2 = |d|^2 + eps^2
  float2 p[3], pe[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    two_prod2(dh[c], dh[c], p[c], pe[c]);
    pe[c] = __ffma2_rn(__fadd2_rn(dh[c], dh[c]), dl[c], pe[c]);
  }
  float2 s1, e1, s2, e2, s3, e3;
  two_sum2(p[0], p[1], s1, e1);
  two_sum2(s1, p[2], s2, e2);
  two_sum2(s2, e2h, s3, e3);
  const float2 lo = __fadd2_rn(__fadd2_rn(__fadd2_rn(pe[0], pe[1]), __fadd2_rn(pe[2], e2l)),
                               __fadd2_rn(__fadd2_rn(e1, e2), e3));
  float2 r2h, r2l;
  fast_two_sum2(s3, lo, r2h, r2l);
  float2 mh = f2(H2.z, H2.w), ml = f2(L2.z, L2.w);
  if (MASK) {
    if (self0) {
      r2h.x = 1.0f;
      r2l.x = 0.0f;
      mh.x = ml.x = 0.0f;
    }
    if (self1) {
      r2h.y = 1.0f;
      r2l.y = 0.0f;
      mh.y = ml.y = 0.0f;
    }
  }
  // y = r2^{-1/2}: SFU seed y0, residual e = 1 - r2 y0^2 in float-float,
  // y = y0 (1 + e/2 + 3 e^2 / 8) = y0 + y0 e (1/2 + 3e/8)
  const float2 y0 = f2(rsqrt_approx(r2h.x), rsqrt_approx(r2h.y));
  float2 th, tl, u, ue;
  two_prod2(y0, y0, th, tl);
  two_prod2(r2h, th, u, ue);
  const float2 cross = __ffma2_rn(r2h, tl, __fmul2_rn(r2l, th));
  const float2 e = fsub2(fsub2(fsub2(f2(1.0f, 1.0f), u), ue), cross);
  const float2 yl = __fmul2_rn(__fmul2_rn(y0, e), __ffma2_rn(e, f2(0.375f, 0.375f), f2(0.5f, 0.5f)));
  // q = y^2, a = m y, b = a q = m y^3
  float2 q, qe, a, ae, b, be;
  two_prod2(y0, y0, q, qe);
  const float2 ql = __ffma2_rn(__fadd2_rn(y0, y0), yl, qe);
  two_prod2(mh, y0, a, ae);
  const float2 al_ = __ffma2_rn(mh, yl, __ffma2_rn(ml, y0, ae));
  two_prod2(a, q, b, be);
  const float2 bl = __ffma2_rn(a, ql, __ffma2_rn(al_, q, be));
  // accumulate d b (three components) and a
#pragma unroll
  for (int c = 0; c < 4; c++) {
    float2 th2, tl2;
    if (c < 3) {
      float2 ce;
      two_prod2(dh[c], b, th2, ce);
      tl2 = __ffma2_rn(dh[c], bl, __ffma2_rn(dl[c], b, ce));
    } else {
      th2 = a;
      tl2 = al_;
    }
    float2 s, es;
    two_sum2(ah[c], th2, s, es);
    fast_two_sum2(s, __fadd2_rn(al[c], __fadd2_rn(es, tl2)), ah[c], al[c]);
  }
}

// Stage j-particles [jt, jt+cnt) of `src` (two float4 per particle: hi
// (x, y, z, m), lo (x, y, z, m)) as pairs; odd tail padded as in load_pairs.
template <int BT, int T>
__device__ __forceinline__ void load_pairs_ff(const float4 *__restrict__ src, int64_t jt, int cnt,
                                              float4 *tH, float4 *tH2, float4 *tL, float4 *tL2) {
  const float4 dh = make_float4(1e18f, 1e18f, 1e18f, 0.0f), dl = make_float4(0, 0, 0, 0);
  for (int k = threadIdx.x; 2 * k < cnt; k += BT) {
    const float4 ah = src[2 * (jt + 2 * k)], alo = src[2 * (jt + 2 * k) + 1];
    const bool hb = 2 * k + 1 < cnt;
    const float4 bh = hb ? src[2 * (jt + 2 * k + 1)] : dh;
    const float4 blo = hb ? src[2 * (jt + 2 * k + 1) + 1] : dl;
    tH[k] = make_float4(ah.x, bh.x, ah.y, bh.y);
    tH2[k] = make_float4(ah.z, bh.z, ah.w, bh.w);
    tL[k] = make_float4(alo.x, blo.x, alo.y, blo.y);
    tL2[k] = make_float4(alo.z, blo.z, alo.w, blo.w);
  }
}

// F64E force: i coordinates re-centred on each j-tile's anchor in float-float
// (from the particle's own float-float and the anchor's), pair terms and
// per-tile partial sums in float-float, folded into binary64 once per tile.
template <int BT, int R, int T, class W>
__global__ void __launch_bounds__(BT) k_force_f64e(const d4 *__restrict__ posm,
                                                   const float4 *__restrict__ jff,
                                                   const float4 *__restrict__ anchor, W work,
                                                   d4 *__restrict__ part) {
  __shared__ float4 tH[T / 2], tH2[T / 2], tL[T / 2], tL2[T / 2];
  for (int64_t uk = work.first(); uk < work.count(); uk += work.stride()) {
    const Unit u = work.get(uk);
    const int tid = threadIdx.x;
    const int64_t j1 = u.j0 + u.nj;
    const float e2hs = (float)u.eps2;
    const float e2ls = (float)(u.eps2 - (double)e2hs);
    const float2 e2h = f2(e2hs, e2hs), e2l = f2(e2ls, e2ls);
    float xh[R][3], xl[R][3];
    double acc[R][4];
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int li = r * BT + tid;
      const d4 p = posm[u.i0 + (li < u.ni ? li : 0)];
      const double c3[3] = {p.x, p.y, p.z};
#pragma unroll
      for (int c = 0; c < 3; c++) {
        xh[r][c] = __double2float_rn(c3[c]);
        xl[r][c] = __double2float_rn(c3[c] - (double)xh[r][c]);
      }
#pragma unroll
      for (int c = 0; c < 4; c++) acc[r][c] = 0.0;
    }
    for (int64_t jt = u.j0; jt < j1; jt += T) {
      const int cnt = (int)min((int64_t)T, j1 - jt);
      __syncthreads();
      load_pairs_ff<BT, T>(jff, jt, cnt, tH, tH2, tL, tL2);
      __syncthreads();
      const int64_t tt = u.anchor + (jt - u.j0) / T;
      const float4 ch = anchor[2 * tt], cl = anchor[2 * tt + 1];
      const float chv[3] = {ch.x, ch.y, ch.z}, clv[3] = {cl.x, cl.y, cl.z};
      float2 nh[R][3], nl[R][3], ah[R][4], al[R][4];
#pragma unroll
      for (int r = 0; r < R; r++) {
#pragma unroll
        for (int c = 0; c < 3; c++) {  // -(x_i - c_t) as float-float
          float s, e;
          two_sum1(xh[r][c], -chv[c], s, e);
          const float t = __fadd_rn(__fsub_rn(xl[r][c], clv[c]), e);
          float h, l;
          two_sum1(s, t, h, l);
          nh[r][c] = f2(-h, -h);
          nl[r][c] = f2(-l, -l);
        }
#pragma unroll
        for (int c = 0; c < 4; c++) ah[r][c] = al[r][c] = f2(0.0f, 0.0f);
      }
      const int np = (cnt + 1) / 2;
      const bool diag = (jt < u.i0 + u.ni) && (jt + cnt > u.i0);
      if (cnt == T && !diag) {
        for (int k = 0; k < T / 2; k++) {
          const float4 H = tH[k], H2 = tH2[k], L = tL[k], L2 = tL2[k];
#pragma unroll
          for (int r = 0; r < R; r++)
            body_ff<false>(H, H2, L, L2, nh[r][0], nl[r][0], nh[r][1], nl[r][1], nh[r][2],
                           nl[r][2], e2h, e2l, ah[r], al[r], false, false);
        }
      } else {
        for (int k = 0; k < np; k++) {
          const float4 H = tH[k], H2 = tH2[k], L = tL[k], L2 = tL2[k];
          const int64_t j = jt + 2 * k;
#pragma unroll
          for (int r = 0; r < R; r++) {
            const int64_t i = u.i0 + r * BT + tid;
            body_ff<true>(H, H2, L, L2, nh[r][0], nl[r][0], nh[r][1], nl[r][1], nh[r][2],
                          nl[r][2], e2h, e2l, ah[r], al[r], j == i, j + 1 == i);
          }
        }
      }
      // fold the tile: even + odd lanes in float-float, then into binary64
#pragma unroll
      for (int r = 0; r < R; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
          float s, e;
          two_sum1(ah[r][c].x, ah[r][c].y, s, e);
          const float l = __fadd_rn(__fadd_rn(al[r][c].x, al[r][c].y), e);
          acc[r][c] += f2d_exact(s) + f2d_exact(l);
        }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int li = r * BT + tid;
      if (li < u.ni) part[u.out + li] = d4{acc[r][0], acc[r][1], acc[r][2], acc[r][3]};
    }
  }
}

// ---------------------------------------------------------------- float-float, each pair once
// The F64E pair body evaluated once for both particles (Newton's third law):
// the difference, |d|^2 + eps^2, y = 1/r and q = y^2 are shared; the i side
// gets m_j y and m_j y q, the j side m_i y and m_i y q with -d.  Two
// j-particles per packed instruction (one tile entry); the j side's four
// float-float sums for an entry are (gh, gl).
__device__ __forceinline__ void body_ff_sym(const float4 &H, const float4 &H2, const float4 &L,
                                            const float4 &L2, float2 nxh, float2 nxl,
                                            float2 nyh, float2 nyl, float2 nzh, float2 nzl,
                                            float2 mih, float2 mil, float2 e2h, float2 e2l,
                                            float2 (&ah)[4], float2 (&al)[4], float2 (&gh)[4],
                                            float2 (&gl)[4]) {
  float2 dh[3], dl[3];
  {
    const float2 jh[3] = {f2(H.x, H.y), f2(H.z, H.w), f2(H2.x, H2.y)};
    const float2 jl[3] = {f2(L.x, L.y), f2(L.z, L.w), f2(L2.x, L2.y)};
    const float2 ih[3] = {nxh, nyh, nzh}, il[3] = {nxl, nyl, nzl};
#pragma unroll
    for (int c = 0; c < 3; c++) {  // d = (jh + jl) - (ih + il), renormalised
      float2 s, e;
      two_sum2(jh[c], ih[c], s, e);
      const float2 t = __fadd2_rn(__fadd2_rn(jl[c], il[c]), e);
      two_sum2(s, t, dh[c], dl[c]);
    }
  }
  float2 p[3], pe[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    two_prod2(dh[c], dh[c], p[c], pe[c]);
    pe[c] = __ffma2_rn(__fadd2_rn(dh[c], dh[c]), dl[c], pe[c]);
  }
  float2 s1, e1, s2, e2, s3, e3;
  two_sum2(p[0], p[1], s1, e1);
  two_sum2(s1, p[2], s2, e2);
  two_sum2(s2, e2h, s3, e3);
  const float2 lo = __fadd2_rn(__fadd2_rn(__fadd2_rn(pe[0], pe[1]), __fadd2_rn(pe[2], e2l)),
                               __fadd2_rn(__fadd2_rn(e1, e2), e3));
  float2 r2h, r2l;
  fast_two_sum2(s3, lo, r2h, r2l);
  const float2 y0 = f2(rsqrt_approx(r2h.x), rsqrt_approx(r2h.y));
  float2 th, tl, u, ue;
  two_prod2(y0, y0, th, tl);
  two_prod2(r2h, th, u, ue);
  const float2 cross = __ffma2_rn(r2h, tl, __fmul2_rn(r2l, th));
  const float2 e = fsub2(fsub2(fsub2(f2(1.0f, 1.0f), u), ue), cross);
  const float2 yl = __fmul2_rn(__fmul2_rn(y0, e), __ffma2_rn(e, f2(0.375f, 0.375f), f2(0.5f, 0.5f)));
  float2 q, qe;
  two_prod2(y0, y0, q, qe);
  const float2 ql = __ffma2_rn(__fadd2_rn(y0, y0), yl, qe);
  // one side: a = m y, b = a q, sums += (sgn d b, a)
  auto side = [&](float2 mh, float2 ml, bool neg, float2(&sh)[4], float2(&sl)[4]) {
    float2 a, ae, b, be;
    two_prod2(mh, y0, a, ae);
    const float2 al_ = __ffma2_rn(mh, yl, __ffma2_rn(ml, y0, ae));
    two_prod2(a, q, b, be);
    const float2 bl = __ffma2_rn(a, ql, __ffma2_rn(al_, q, be));
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float2 th2, tl2;
      if (c < 3) {
        const float2 dhc = neg ? neg2(dh[c]) : dh[c], dlc = neg ? neg2(dl[c]) : dl[c];
        float2 ce;
        two_prod2(dhc, b, th2, ce);
        tl2 = __ffma2_rn(dhc, bl, __ffma2_rn(dlc, b, ce));
      } else {
        th2 = a;
        tl2 = al_;
      }
      float2 s, es;
      two_sum2(sh[c], th2, s, es);
      fast_two_sum2(s, __fadd2_rn(sl[c], __fadd2_rn(es, tl2)), sh[c], sl[c]);
    }
  };
  side(f2(H2.z, H2.w), f2(L2.z, L2.w), false, ah, al);
  side(mih, mil, true, gh, gl);
}

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return f2(__shfl_sync(0xFFFFFFFFu, v.x, src), __shfl_sync(0xFFFFFFFFu, v.y, src));
}

// Work item (d, I) of the block-diagonal schedule of k_force_f64_sym with
// blocks of B = BT*R = T particles: one F64E tile (one anchor) per column
// block.  Row sums into rows[dl], column sums into cols[dl], binary64.
template <int BT, int R, int T>
__global__ void __launch_bounds__(BT) k_force_f64e_sym(const d4 *__restrict__ posm,
                                                       const float4 *__restrict__ jff,
                                                       const float4 *__restrict__ anchor,
                                                       int64_t n, double eps2, int M, int d0,
                                                       d4 *__restrict__ rows,
                                                       d4 *__restrict__ cols) {
  constexpr int B = BT * R, NW = BT / 32, NE = T / 2;  // NE tile entries of 2 j
  static_assert(B == T && NE == BT, "one tile per block, one column entry per thread");
  __shared__ float4 tH[NE], tH2[NE], tL[NE], tL2[NE];
  __shared__ double colw[NW][4][T];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int dl = blockIdx.x / M, I = blockIdx.x % M, d = d0 + dl;
  const int J = (I + d) % M;
  const int64_t i0 = (int64_t)I * B, j0 = (int64_t)J * B;
  d4 *rowo = rows + (int64_t)dl * n;
  d4 *colo = cols + (int64_t)dl * n;
  if (2 * d == M && I >= M / 2) {
    for (int k = tid; k < B; k += BT) {
      if (i0 + k < n) rowo[i0 + k] = d4{0.0, 0.0, 0.0, 0.0};
      if (j0 + k < n) colo[j0 + k] = d4{0.0, 0.0, 0.0, 0.0};
    }
    return;
  }
  const float e2hs = (float)eps2;
  const float e2ls = (float)(eps2 - (double)e2hs);
  const float2 e2h = f2(e2hs, e2hs), e2l = f2(e2ls, e2ls);
  {  // entry tid = j0 + 2 tid, j0 + 2 tid + 1; beyond n massless at 1e18 from the anchor
    const int64_t ja = j0 + 2 * tid, jb = ja + 1;
    const float4 dh = make_float4(1e18f, 1e18f, 1e18f, 0.0f), dz = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float4 ah_ = ja < n ? jff[2 * ja] : dh, alo = ja < n ? jff[2 * ja + 1] : dz;
    const float4 bh_ = jb < n ? jff[2 * jb] : dh, blo = jb < n ? jff[2 * jb + 1] : dz;
    tH[tid] = make_float4(ah_.x, bh_.x, ah_.y, bh_.y);
    tH2[tid] = make_float4(ah_.z, bh_.z, ah_.w, bh_.w);
    tL[tid] = make_float4(alo.x, blo.x, alo.y, blo.y);
    tL2[tid] = make_float4(alo.z, blo.z, alo.w, blo.w);
  }
  const float4 ch = anchor[2 * J], cl = anchor[2 * J + 1];
  const float chv[3] = {ch.x, ch.y, ch.z}, clv[3] = {cl.x, cl.y, cl.z};
  float2 nh[R][3], nl[R][3], ah[R][4], al[R][4], mh[R], ml[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = i0 + r * BT + tid;
    // beyond n: massless, 1e18 from the anchor (finite r^2, zero contribution)
    const d4 pi = i < n ? posm[i] : d4{0.0, 0.0, 0.0, 0.0};
    const double c3[3] = {pi.x, pi.y, pi.z};
#pragma unroll
    for (int c = 0; c < 3; c++) {  // -(x_i - c_J) as float-float
      const float xh = __double2float_rn(c3[c]);
      const float xl = __double2float_rn(c3[c] - (double)xh);
      float s, e;
      two_sum1(xh, -chv[c], s, e);
      const float t = __fadd_rn(__fsub_rn(xl, clv[c]), e);
      float h, l;
      two_sum1(s, t, h, l);
      if (i >= n) h = 1e18f, l = 0.0f;
      nh[r][c] = f2(-h, -h);
      nl[r][c] = f2(-l, -l);
    }
    const float m_h = __double2float_rn(pi.w);
    const float m_l = __double2float_rn(pi.w - (double)m_h);
    mh[r] = f2(m_h, m_h);
    ml[r] = f2(m_l, m_l);
#pragma unroll
    for (int c = 0; c < 4; c++) ah[r][c] = al[r][c] = f2(0.0f, 0.0f);
  }
  __syncthreads();
#pragma unroll 1
  for (int c0 = 0; c0 < NE; c0 += 32) {
    float2 gh[4], gl[4];
#pragma unroll
    for (int c = 0; c < 4; c++) gh[c] = gl[c] = f2(0.0f, 0.0f);
#pragma unroll 1
    for (int k = 0; k < 32; k++) {
      const int ent = c0 + ((lane + k) & 31);
      const float4 H = tH[ent], H2 = tH2[ent], L = tL[ent], L2 = tL2[ent];
#pragma unroll
      for (int r = 0; r < R; r++)
        body_ff_sym(H, H2, L, L2, nh[r][0], nl[r][0], nh[r][1], nl[r][1], nh[r][2], nl[r][2],
                    mh[r], ml[r], e2h, e2l, ah[r], al[r], gh, gl);
      const int src = (lane + 1) & 31;
#pragma unroll
      for (int c = 0; c < 4; c++) {
        gh[c] = shfl2(gh[c], src);
        gl[c] = shfl2(gl[c], src);
      }
    }
    // lane holds entry c0 + lane (j = 2 (c0 + lane) and 2 (c0 + lane) + 1)
#pragma unroll
    for (int c = 0; c < 4; c++) {
      colw[warp][c][2 * (c0 + lane)] = f2d_exact(gh[c].x) + f2d_exact(gl[c].x);
      colw[warp][c][2 * (c0 + lane) + 1] = f2d_exact(gh[c].y) + f2d_exact(gl[c].y);
    }
  }
  __syncthreads();
  for (int k = tid; k < T; k += BT) {
    double v[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      v[c] = colw[0][c][k];
#pragma unroll
      for (int w = 1; w < NW; w++) v[c] += colw[w][c][k];
    }
    if (j0 + k < n) colo[j0 + k] = d4{v[0], v[1], v[2], v[3]};
  }
  // rows: fold even + odd lanes in float-float, then into binary64
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = i0 + r * BT + tid;
    double v[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      float s, e;
      two_sum1(ah[r][c].x, ah[r][c].y, s, e);
      const float l = __fadd_rn(__fadd_rn(al[r][c].x, al[r][c].y), e);
      v[c] = f2d_exact(s) + f2d_exact(l);
    }
    if (i < n) rowo[i] = d4{v[0], v[1], v[2], v[3]};
  }
}

// ---------------------------------------------------------------- mixed
// fpos[j] = (x_j - c_t, y_j - c_t, z_j - c_t, m_j) in binary32, c_t the anchor of
// j's tile; anchor[2t] = float hi part of c_t, anchor[2t+1] = float lo part.
template <int BT, int R, int T, class W>
__global__ void __launch_bounds__(BT) k_force_mixed(const d4 *__restrict__ posm,
                                                    const float4 *__restrict__ fpos,
                                                    const float4 *__restrict__ anchor, W work,
                                                    d4 *__restrict__ part) {
  __shared__ float4 tA[T / 2], tB[T / 2];
  for (int64_t uk = work.first(); uk < work.count(); uk += work.stride()) {
    const Unit u = work.get(uk);
    const int tid = threadIdx.x;
    const int64_t j1 = u.j0 + u.nj;
    const float2 e2 = f2((float)u.eps2, (float)u.eps2);
    float xh[R], yh[R], zh[R], xl[R], yl[R], zl[R];
    float axh[R], axl[R], ayh[R], ayl[R], azh[R], azl[R], pth[R], ptl[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int li = r * BT + tid;
      const d4 p = posm[u.i0 + (li < u.ni ? li : 0)];
      xh[r] = __double2float_rn(p.x);
      yh[r] = __double2float_rn(p.y);
      zh[r] = __double2float_rn(p.z);
      xl[r] = __double2float_rn(p.x - (double)xh[r]);
      yl[r] = __double2float_rn(p.y - (double)yh[r]);
      zl[r] = __double2float_rn(p.z - (double)zh[r]);
      axh[r] = axl[r] = ayh[r] = ayl[r] = azh[r] = azl[r] = pth[r] = ptl[r] = 0.0f;
    }
    for (int64_t jt = u.j0; jt < j1; jt += T) {
      const int cnt = (int)min((int64_t)T, j1 - jt);
      __syncthreads();
      load_pairs<BT, T>(fpos, jt, cnt, tA, tB);
      __syncthreads();
      const int64_t tt = u.anchor + (jt - u.j0) / T;
      const float4 ch = anchor[2 * tt], cl = anchor[2 * tt + 1];
      float2 nx[R], ny[R], nz[R], sx[R], sy[R], sz[R], sp[R];
#pragma unroll
      for (int r = 0; r < R; r++) {
        // x_i - c_t rounded once: TwoSum of the high parts, then the low parts
        float x, y, z, s, e;
        two_sum1(xh[r], -ch.x, s, e);
        x = __fadd_rn(s, __fadd_rn(__fsub_rn(xl[r], cl.x), e));
        two_sum1(yh[r], -ch.y, s, e);
        y = __fadd_rn(s, __fadd_rn(__fsub_rn(yl[r], cl.y), e));
        two_sum1(zh[r], -ch.z, s, e);
        z = __fadd_rn(s, __fadd_rn(__fsub_rn(zl[r], cl.z), e));
        nx[r] = f2(-x, -x);
        ny[r] = f2(-y, -y);
        nz[r] = f2(-z, -z);
        sx[r] = sy[r] = sz[r] = sp[r] = f2(0.0f, 0.0f);
      }
      const int np = (cnt + 1) / 2;
      const bool diag = (jt < u.i0 + u.ni) && (jt + cnt > u.i0);
      if (cnt == T && !diag) {
#pragma unroll 2
        for (int k = 0; k < T / 2; k++) {
          const float4 A = tA[k], B = tB[k];
#pragma unroll
          for (int r = 0; r < R; r++)
            body_pair<false, false>(A, B, nx[r], ny[r], nz[r], e2, sx[r], sy[r], sz[r], sp[r],
                                   false, false);
        }
      } else {
        for (int k = 0; k < np; k++) {
          const float4 A = tA[k], B = tB[k];
          const int64_t j = jt + 2 * k;
#pragma unroll
          for (int r = 0; r < R; r++) {
            const int64_t i = u.i0 + r * BT + tid;
            body_pair<true, false>(A, B, nx[r], ny[r], nz[r], e2, sx[r], sy[r], sz[r], sp[r],
                                  j == i, j + 1 == i);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; r++) {
        two_sum_acc(axh[r], axl[r], __fadd_rn(sx[r].x, sx[r].y));
        two_sum_acc(ayh[r], ayl[r], __fadd_rn(sy[r].x, sy[r].y));
        two_sum_acc(azh[r], azl[r], __fadd_rn(sz[r].x, sz[r].y));
        two_sum_acc(pth[r], ptl[r], __fadd_rn(sp[r].x, sp[r].y));
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int li = r * BT + tid;
      if (li < u.ni)
        part[u.out + li] = d4{(double)axh[r] + (double)axl[r], (double)ayh[r] + (double)ayl[r],
                              (double)azh[r] + (double)azl[r], (double)pth[r] + (double)ptl[r]};
    }
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
struct DensePrep {
  int64_t n;
  int tile;
  __device__ __forceinline__ PrepUnit get() const {
    PrepUnit u;
    u.anchor = blockIdx.x;
    u.j0 = (int64_t)blockIdx.x * tile;
    u.cnt = (int)min((int64_t)tile, n - u.j0);
    u.pad = 0;
    return u;
  }
};
struct TablePrep {
  const PrepUnit *units;
  __device__ __forceinline__ PrepUnit get() const { return units[blockIdx.x]; }
};

// FF = true (F64E): the re-centred coordinates and the mass are written as
// float-float, two float4 per particle (hi x, y, z, m; lo x, y, z, m).
template <int BT, class W, bool FF>
__global__ void __launch_bounds__(BT) k_mixed_prep(const d4 *__restrict__ posm, W work,
                                                   float4 *__restrict__ fpos,
                                                   float4 *__restrict__ anchor) {
  static_assert((BT & (BT - 1)) == 0, "bitonic sort needs a power-of-two block");
  __shared__ double v[BT];
  const PrepUnit pu = work.get();
  const int64_t t = pu.anchor;
  const int64_t j0 = pu.j0;
  const int cnt = pu.cnt;
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
  if (tid < cnt) {
    const double dx = p.x - c[0], dy = p.y - c[1], dz = p.z - c[2];
    const float hx = __double2float_rn(dx), hy = __double2float_rn(dy), hz = __double2float_rn(dz),
                hm = __double2float_rn(p.w);
    if (FF) {
      fpos[2 * (j0 + tid)] = make_float4(hx, hy, hz, hm);
      fpos[2 * (j0 + tid) + 1] =
          make_float4(__double2float_rn(dx - (double)hx), __double2float_rn(dy - (double)hy),
                      __double2float_rn(dz - (double)hz), __double2float_rn(p.w - (double)hm));
    } else {
      fpos[j0 + tid] = make_float4(hx, hy, hz, hm);
    }
  }
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
template <int BT, int R, int T, class W>
__global__ void __launch_bounds__(BT) k_force_f32(const float4 *__restrict__ posm, W work,
                                                  float4 *__restrict__ part) {
  __shared__ float4 tA[T / 2], tB[T / 2];
  for (int64_t uk = work.first(); uk < work.count(); uk += work.stride()) {
    const Unit u = work.get(uk);
    const int tid = threadIdx.x;
    const int64_t j1 = u.j0 + u.nj;
    const float2 e2 = f2((float)u.eps2, (float)u.eps2);
    float2 nx[R], ny[R], nz[R], ax[R], ay[R], az[R], pt[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int li = r * BT + tid;
      const float4 p = posm[u.i0 + (li < u.ni ? li : 0)];
      nx[r] = f2(-p.x, -p.x);
      ny[r] = f2(-p.y, -p.y);
      nz[r] = f2(-p.z, -p.z);
      ax[r] = ay[r] = az[r] = pt[r] = f2(0.0f, 0.0f);
    }
    for (int64_t jt = u.j0; jt < j1; jt += T) {
      const int cnt = (int)min((int64_t)T, j1 - jt);
      __syncthreads();
      load_pairs<BT, T>(posm, jt, cnt, tA, tB);
      __syncthreads();
      const int np = (cnt + 1) / 2;
      const bool diag = (jt < u.i0 + u.ni) && (jt + cnt > u.i0);
      if (cnt == T && !diag) {
#pragma unroll 2
        for (int k = 0; k < T / 2; k++) {
          const float4 A = tA[k], B = tB[k];
#pragma unroll
          for (int r = 0; r < R; r++)
            body_pair<false, false>(A, B, nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r], pt[r],
                                    false, false);
        }
      } else {
        for (int k = 0; k < np; k++) {
          const float4 A = tA[k], B = tB[k];
          const int64_t j = jt + 2 * k;
#pragma unroll
          for (int r = 0; r < R; r++) {
            const int64_t i = u.i0 + r * BT + tid;
            body_pair<true, false>(A, B, nx[r], ny[r], nz[r], e2, ax[r], ay[r], az[r], pt[r],
                                   j == i, j + 1 == i);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int li = r * BT + tid;
      if (li < u.ni)
        part[u.out + li] = make_float4(__fadd_rn(ax[r].x, ax[r].y), __fadd_rn(ay[r].x, ay[r].y),
                                       __fadd_rn(az[r].x, az[r].y), __fadd_rn(pt[r].x, pt[r].y));
    }
  }
}

// ---------------------------------------------------------------- dispatch
// Fixed block and tile sizes per arithmetic; R is chosen at run time.
constexpr int BT_F64 = 128, T_F64 = 128;
constexpr int BT_F32 = 256, T_F32 = 256;
constexpr int BT_FF = 128, T_FF = 256;

int force_block_threads(int mode) {
  return mode == NBODY_FP64 ? BT_F64 : mode == NBODY_F64E ? BT_FF : BT_F32;
}
int force_tile(int mode) { return mode == NBODY_FP64 ? T_F64 : mode == NBODY_F64E ? T_FF : T_F32; }

bool shape_supported(int mode, const Shape &sh) {
  if (sh.r != 1 && sh.r != 2 && sh.r != 4 && sh.r != 8) return false;
  if (mode == NBODY_F64E && sh.r == 8) return false;
  if (sh.s < 1 || sh.s > 65535) return false;
  return sh.bt == force_block_threads(mode) && sh.t == force_tile(mode);
}

template <int R>
static const void *kernel_for(int mode) {
  switch (mode) {
    case NBODY_FP64: return (const void *)k_force_f64<BT_F64, R, T_F64, DenseWork>;
    case NBODY_MIXED: return (const void *)k_force_mixed<BT_F32, R, T_F32, DenseWork>;
    case NBODY_F64E: return (const void *)k_force_f64e<BT_FF, (R < 4 ? R : 4), T_FF, DenseWork>;
    default: return (const void *)k_force_f32<BT_F32, R, T_F32, DenseWork>;
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

template <int R, class W>
static void launch_rw(int mode, const void *posm, const float4 *fpos, const float4 *anchor,
                      const W &w, dim3 grid, void *part, cudaStream_t st) {
  if (mode == NBODY_FP64) {
    k_force_f64<BT_F64, R, T_F64, W><<<grid, BT_F64, 0, st>>>((const d4 *)posm, w, (d4 *)part);
  } else if (mode == NBODY_MIXED) {
    k_force_mixed<BT_F32, R, T_F32, W><<<grid, BT_F32, 0, st>>>((const d4 *)posm, fpos, anchor, w,
                                                                (d4 *)part);
  } else if (mode == NBODY_F64E) {
    constexpr int RF = R < 4 ? R : 4;
    k_force_f64e<BT_FF, RF, T_FF, W><<<grid, BT_FF, 0, st>>>((const d4 *)posm, fpos, anchor, w,
                                                             (d4 *)part);
  } else {
    k_force_f32<BT_F32, R, T_F32, W><<<grid, BT_F32, 0, st>>>((const float4 *)posm, w,
                                                              (float4 *)part);
  }
}

template <class W>
static cudaError_t launch_w(int mode, int r, const void *posm, const float4 *fpos,
                            const float4 *anchor, const W &w, dim3 grid, void *part,
                            cudaStream_t st) {
  switch (r) {
    case 1: launch_rw<1>(mode, posm, fpos, anchor, w, grid, part, st); break;
    case 2: launch_rw<2>(mode, posm, fpos, anchor, w, grid, part, st); break;
    case 4: launch_rw<4>(mode, posm, fpos, anchor, w, grid, part, st); break;
    case 8: launch_rw<8>(mode, posm, fpos, anchor, w, grid, part, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- binary64, each pair once: launches
// R = 3 (blocks of 384): 114 registers, 4 blocks of 4 warps per SM.  Measured on
// GB300 at N = 2^18 (this kernel alone, Gint/s): both potential sums in binary64
// R = 4 (148 registers, 3 blocks) 78.9, R = 3 81.6, R = 2 78.8; the row sum on the
// integer pipes R = 4 73.3, R = 3 85.6, R = 2 83.4; both sums on the integer
// pipes, k-loop not unrolled: R = 3 96.1, R = 2 96.3, R = 1 95.3 (unrolled twice:
// R = 2 92.2).
constexpr int SYM_BT = 128, SYM_R = 3, SYM_T = 128;

int sym_block_particles() { return SYM_BT * SYM_R; }
int sym_r() { return SYM_R; }
// the one-sided kernel's R for the pairs inside the diagonal blocks: the
// smallest supported R whose BT*R covers a block
int sym_units_r() { return SYM_R <= 1 ? 1 : SYM_R <= 2 ? 2 : SYM_R <= 4 ? 4 : 8; }

int sym_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_f64_sym<SYM_BT, SYM_R, SYM_T>,
                                                    SYM_BT, 0) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_force_f64_sym(const d4 *posm, int64_t n, double eps2, int M, int d0, int D,
                                 d4 *rows, d4 *cols, cudaStream_t st) {
  k_force_f64_sym<SYM_BT, SYM_R, SYM_T><<<D * M, SYM_BT, 0, st>>>(posm, n, eps2, M, d0, rows, cols);
  return cudaGetLastError();
}

constexpr int SYMFF_BT = 128, SYMFF_R = 2, SYMFF_T = 256;

int sym_block_particles_ff() { return SYMFF_BT * SYMFF_R; }
int sym_r_ff() { return SYMFF_R; }

int sym_blocks_per_sm_ff() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &nb, k_force_f64e_sym<SYMFF_BT, SYMFF_R, SYMFF_T>, SYMFF_BT, 0) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_force_f64e_sym(const d4 *posm, const float4 *jff, const float4 *anchor,
                                  int64_t n, double eps2, int M, int d0, int D, d4 *rows,
                                  d4 *cols, cudaStream_t st) {
  k_force_f64e_sym<SYMFF_BT, SYMFF_R, SYMFF_T><<<D * M, SYMFF_BT, 0, st>>>(
      posm, jff, anchor, n, eps2, M, d0, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_sym_combine(const d4 *rows, const d4 *cols, int D, int64_t n, d4 *acc_rows,
                               d4 *acc_cols, bool first, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  k_sym_combine<<<(unsigned)blocks, 256, 0, st>>>(rows, cols, D, n, acc_rows, acc_cols,
                                                  first ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_force(int mode, const ForceIn &in, const Shape &sh, cudaStream_t st) {
  const int64_t rows = in.rows < 0 ? in.n : in.rows;
  if (!shape_supported(mode, sh) || in.n < 1 || rows < 1 || in.i0 < 0 || in.i0 + rows > in.n)
    return cudaErrorInvalidValue;
  const int64_t per_block = (int64_t)sh.bt * sh.r;
  const int64_t gx = (rows + per_block - 1) / per_block;
  if (gx > 0x7fffffff) return cudaErrorInvalidValue;
  DenseWork w;
  w.n = in.n;
  w.seg = in.seg;
  w.i_base = in.i0;
  w.rows = rows;
  w.eps2 = in.eps2;
  w.per_block = (int)per_block;
  w.tile = sh.t;
  return launch_w(mode, sh.r, in.posm, in.fpos, in.anchor, w, dim3((unsigned)gx, (unsigned)sh.s),
                  in.part, st);
}

cudaError_t launch_force_units(int mode, const void *posm, const float4 *fpos,
                               const float4 *anchor, const Unit *units, int64_t nunits, int r,
                               void *part, int64_t max_blocks, cudaStream_t st) {
  if (nunits < 1) return cudaErrorInvalidValue;
  TableWork w;
  w.units = units;
  w.n = nunits;
  int64_t g = nunits;
  if (max_blocks > 0 && g > max_blocks) g = max_blocks;
  if (g > 0x7fffffff) g = 0x7fffffff;
  return launch_w(mode, r, posm, fpos, anchor, w, dim3((unsigned)g), part, st);
}

cudaError_t launch_mixed_prep(const d4 *posm, int64_t n, int tile, float4 *fpos, float4 *anchor,
                              cudaStream_t st, bool ff) {
  if (tile != 256) return cudaErrorInvalidValue;  // one thread per tile member
  const int64_t nt = (n + tile - 1) / tile;
  DensePrep w;
  w.n = n;
  w.tile = tile;
  if (ff)
    k_mixed_prep<256, DensePrep, true><<<(unsigned)nt, 256, 0, st>>>(posm, w, fpos, anchor);
  else
    k_mixed_prep<256, DensePrep, false><<<(unsigned)nt, 256, 0, st>>>(posm, w, fpos, anchor);
  return cudaGetLastError();
}

cudaError_t launch_mixed_prep_units(const d4 *posm, const PrepUnit *units, int64_t nunits,
                                    float4 *fpos, float4 *anchor, cudaStream_t st, bool ff) {
  if (nunits < 1 || nunits > 0x7fffffff) return cudaErrorInvalidValue;
  TablePrep w;
  w.units = units;
  if (ff)
    k_mixed_prep<256, TablePrep, true><<<(unsigned)nunits, 256, 0, st>>>(posm, w, fpos, anchor);
  else
    k_mixed_prep<256, TablePrep, false><<<(unsigned)nunits, 256, 0, st>>>(posm, w, fpos, anchor);
  return cudaGetLastError();
}

}  // namespace nb
