// dw_core.cuh -- the plan's per-mechanism records and the double-word arithmetic, shared by
// the library's kernels and by the topology-specialised kernels compiled at run time
// (which see this file through NVRTC, hence no host headers there).
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <stdint.h>

#include <cmath>
#endif

namespace links {

constexpr float kU = 5.9604645e-08f;     // unit roundoff of float32, 2^-24
// Forward error bound of one FP32 dyad (product form): E_k = (E_i + E_j + kAmpErr u R12)
// / sin(gamma) + kAddErr u (R12 + |x_k| + |y_k|).  The first term is the error of the
// slack (distance of the parents, rounding of R12 and the MUFU reciprocal square roots,
// amplified by the conditioning 1/sin(gamma)); the second is the rounding of the new
// position, which is not amplified.  In a float32 emulation with the MUFU error
// modelled the bound exceeded the true error on every step (true/bound <= 0.86).
constexpr float kAmpErr = 3.0f;
constexpr float kAddErr = 2.0f;
// Emitted FP32 positions are used where their forward error bound is below this
// fraction of the bounding-box diagonal (so the true error stays below ~5.2e-6 of it),
// else the step is recomputed in double-word arithmetic.
// Position budget of the emit's certified FP32 path, relative to the bounding-box
// diagonal L: the error bound E of every joint plus the rounding of the absolute
// float32 output (u |p| per coordinate, |p| <= |pivot| + bmax) must stay below it.
struct __align__(16) MechHdr {
  int32_t status;
  uint8_t n, nd, nf, motor_joint;
  uint8_t coupler_slot, pivot_joint, pad0, pad1;  // pad0 = pivot slot
  float ux_h, ux_l, uy_h, uy_l;  // crank vector: actuated joint - pivot (initial)
  float px_h, px_l, py_h, py_l;  // pivot (absolute)
  float bmax;                    // bound of |p - pivot| of any joint during the turn
  float e_motor;                 // FP32 error bound of the actuated joint position
  float e_fixed;                 // FP32 error bound of a fixed joint position
  float lbox;                    // bounding-box diagonal of the initial positions
};
static_assert(sizeof(MechHdr) == 64, "MechHdr must be 64 bytes");

// Dyad record: three float4 per dyad.
//   r0 = {offPij, R12_h, Rm_h, c_h}     FP32 screen
//   r1 = {w2, locc, offK, offEij}       FP32 screen
//   r2 = {r1sq_h, r1sq_l, c_l, slots}   double-word chain, FP64 kernel, export
// with r1 = |p_k - p_i|, r2 = |p_k - p_j|, R12 = r1 + r2, Rm = |r1 - r2|,
// c = r1^2 - r2^2, w2 = 2 r1 r2, locc = local FP32 error constant, and (i, j) ordered
// so that the initial configuration has (p_j - p_i) x (p_k - p_i) >= 0 (the solved
// branch is then always the "+" one).  The off* words hold byte offsets into a
// lane's slot arrays of the screen (positions 256 B per slot, bounds 128 B per slot)
// as two 16-bit halves: offPij = P(i) | P(j) << 16, offK = P(k) | E(k) << 16,
// offEij = E(i) | E(j) << 16; slots = i | j << 8 | k_joint << 16 | k << 24.
struct DyadRec {
  float4 r0, r1, r2;
};

// ---------------------------------------------------------------------------------------
// Double-word ("float-float") arithmetic.  A value is hi + lo with |lo| <= ulp(hi)/2.
// Building blocks: Knuth's TwoSum, Dekker's Fast2Sum, FMA-based TwoProd, and the
// double-word add / multiply algorithms analysed by Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44(2), 2017.  The add is the "sloppy" variant: its error is
// bounded by ~2^-48 (|x| + |y|) in absolute terms, which is what positions need.
// Rounded intrinsics keep the compiler from contracting or reordering the steps.
// ---------------------------------------------------------------------------------------
struct dw {
  float h, l;
};

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float frsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ float fsqrt_rn(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ float fdiv_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float frcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
#else
// Host code is compiled with -ffp-contract=off; fmaf is the correctly rounded C99 fma.
inline float fadd(float a, float b) { return a + b; }
inline float fsub(float a, float b) { return a - b; }
inline float fmul(float a, float b) { return a * b; }
inline float ffma(float a, float b, float c) { return std::fmaf(a, b, c); }
inline float frsqrt(float x) { return 1.0f / std::sqrt(x); }
inline float fsqrt_rn(float x) { return std::sqrt(x); }
inline float fdiv_rn(float a, float b) { return a / b; }
inline float frcp(float x) { return 1.0f / x; }
#endif

#define LINKS_HD __host__ __device__ __forceinline__

LINKS_HD dw two_sum(float a, float b) {
  float s = fadd(a, b);
  float bb = fsub(s, a);
  float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
  return {s, e};
}
LINKS_HD dw fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  float s = fadd(a, b);
  float e = fsub(b, fsub(s, a));
  return {s, e};
}
LINKS_HD dw dw_make(float a) { return {a, 0.0f}; }
LINKS_HD dw dw_from_double(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return {h, l};
}
LINKS_HD double dw_to_double(dw x) { return (double)x.h + (double)x.l; }
LINKS_HD dw dw_neg(dw x) { return {-x.h, -x.l}; }
LINKS_HD dw dw_add(dw x, dw y) {
  dw s = two_sum(x.h, y.h);
  float v = fadd(x.l, y.l);
  float w = fadd(s.l, v);
  return fast_two_sum(s.h, w);
}
LINKS_HD dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
LINKS_HD dw dw_mul(dw x, dw y) {
  float p = fmul(x.h, y.h);
  float e = ffma(x.h, y.h, -p);
  e = ffma(x.h, y.l, e);
  e = ffma(x.l, y.h, e);
  return fast_two_sum(p, e);
}
LINKS_HD dw dw_mul_f(dw x, float y) {
  float p = fmul(x.h, y);
  float e = ffma(x.h, y, -p);
  e = ffma(x.l, y, e);
  return fast_two_sum(p, e);
}
LINKS_HD dw dw_sqr(dw x) {
  float p = fmul(x.h, x.h);
  float e = ffma(x.h, x.h, -p);
  float t = fmul(x.h, x.l);
  e = ffma(2.0f, t, e);
  return fast_two_sum(p, e);
}
LINKS_HD dw dw_scale2(dw x, float pow2) { return {fmul(x.h, pow2), fmul(x.l, pow2)}; }  // exact

// Fused double-word expressions: the exact high products are combined with one
// error-free sum and the low-order terms are accumulated in single precision before
// the final renormalisation (the compensated dot product of Ogita, Rump and Oishi,
// 2005, for two or three terms).  Relative error O(u^2) of the sum of the terms'
// magnitudes, as for the chained operations, in fewer operations.
// x^2 + y^2
LINKS_HD dw dw_sum_sq(dw x, dw y) {
  const float p1 = fmul(x.h, x.h), e1 = ffma(x.h, x.h, -p1);
  const float p2 = fmul(y.h, y.h), e2 = ffma(y.h, y.h, -p2);
  const dw s = two_sum(p1, p2);
  float t = fadd(fadd(e1, e2), s.l);
  t = ffma(fadd(x.h, x.h), x.l, t);
  t = ffma(fadd(y.h, y.h), y.l, t);
  return fast_two_sum(s.h, t);
}
// 4ab - c^2
LINKS_HD dw dw_4ab_minus_sq(dw a, dw b, dw c) {
  const float p = fmul(a.h, b.h);
  float ep = ffma(a.h, b.h, -p);
  ep = ffma(a.h, b.l, ep);
  ep = ffma(a.l, b.h, ep);
  const float q = fmul(c.h, c.h);
  float eq = ffma(c.h, c.h, -q);
  eq = ffma(fadd(c.h, c.h), c.l, eq);
  const dw s = two_sum(fmul(4.0f, p), -q);
  const float t = fsub(ffma(4.0f, ep, s.l), eq);
  return fast_two_sum(s.h, t);
}
// z + a x + sg b y, sg = +1 or -1
LINKS_HD dw dw_axpby(dw z, dw a, dw x, dw b, dw y, float sg) {
  const float p1 = fmul(a.h, x.h), e1 = ffma(a.h, x.h, -p1);
  const float bs = fmul(sg, b.h), bl = fmul(sg, b.l);
  const float p2 = fmul(bs, y.h), e2 = ffma(bs, y.h, -p2);
  const dw s1 = two_sum(p1, p2);
  const dw s2 = two_sum(z.h, s1.h);
  float t = fadd(fadd(fadd(z.l, s1.l), s2.l), fadd(e1, e2));
  t = ffma(a.h, x.l, t);
  t = ffma(a.l, x.h, t);
  t = ffma(bs, y.l, t);
  t = ffma(bl, y.h, t);
  return fast_two_sum(s2.h, t);
}
// sqrt(x) for x > 0: FP32 seed from rsqrt, one Newton correction with an exact residual.
LINKS_HD dw dw_sqrt(dw x) {
  if (!(x.h > 0.0f)) return {0.0f, 0.0f};
  float r = frsqrt(x.h);
  float s = fmul(x.h, r);
  float p = fmul(s, s);
  float e = ffma(s, s, -p);
  float res = fadd(fsub(fsub(x.h, p), e), x.l);
  float corr = fmul(res, fmul(0.5f, r));
  return fast_two_sum(s, corr);
}
// Same with correctly rounded seeds: bit-identical on host and device (plan builder).
LINKS_HD dw dw_sqrt_exact(dw x) {
  if (!(x.h > 0.0f)) return {0.0f, 0.0f};
  float s = fsqrt_rn(x.h);
  float p = fmul(s, s);
  float e = ffma(s, s, -p);
  float res = fadd(fsub(fsub(x.h, p), e), x.l);
  return fast_two_sum(s, fdiv_rn(res, fadd(s, s)));
}
// 1/x: FP32 seed, one Newton correction with an exact residual.
LINKS_HD dw dw_rcp(dw x) {
  float y = frcp(x.h);
  float p = fmul(x.h, y);
  float e = ffma(x.h, y, -p);
  float r = fsub(fsub(fsub(1.0f, p), e), fmul(x.l, y));
  return fast_two_sum(y, fmul(y, r));
}
LINKS_HD float dw_sign(dw x) { return x.h != 0.0f ? x.h : x.l; }

}  // namespace links
