// step.cuh -- the arithmetic of one step of a mechanism shared by the library's kernels
// and the topology-specialised kernels compiled at run time: the FP32 dyad of the
// screens (with its forward error bound) and the double-word chain that rescues the
// steps the FP32 bounds leave uncertain.
#pragma once

#include "dw_core.cuh"

namespace links {

__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3_nan(float a, float b, float c) {  // NaN-propagating
  // two two-input minima: the three-input NaN-propagating form is not one instruction
  float r;
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(r), "f"(c));
  return r;
}

// Reciprocal square root with subnormal inputs flushed to zero (one MUFU operation; the
// same approximation as rsqrtf on normal inputs).  A subnormal distance or discriminant
// then gives an infinite bound or a NaN, which the screens treat as uncertain.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One FP32 dyad in product form, D = (d + R12)(R12 - d)(d - Rm)(d + Rm), for parents
// (pix, piy), (pjx, pjy) with bounds ei, ej and the record's r0 = {., R12, Rm, c},
// r1 = {2 r1 r2, local error constant, ., .}: the joint (kx, ky), its forward error
// bound ek, and the step's running lockw = min over dyads of slack + bound (< 0:
// certainly locked), zmin = min of slack - bound (>= 0 everywhere: certainly free;
// NaN propagates) and isgmax = max 1/sin(gamma).  Every operation is a rounded
// intrinsic, so no compiler contracts or reorders it: each kernel that calls this
// gets the same values.
__device__ __forceinline__ void fp32_dyad_core(float pix, float piy, float pjx, float pjy, float ei, float ej,
                                               const float4& r0, const float4& r1, float& lockw, float& zmin,
                                               float& isgmax, float& kx, float& ky, float& ek) {
  const float R12 = r0.y, Rm = r0.z;
  const float dx = __fsub_rn(pjx, pix), dy = __fsub_rn(pjy, piy);
  const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
  const float rd = rsqrt_ftz(d2);
  const float dd = __fmul_rn(d2, rd);
  const float s2 = __fsub_rn(R12, dd), s3 = __fsub_rn(dd, Rm);
  const float D = __fmul_rn(__fmul_rn(__fadd_rn(dd, R12), s2), __fmul_rn(s3, __fadd_rn(dd, Rm)));
  const float rD = rsqrt_ftz(D);
  const float isg = __fmul_rn(r1.x, rD);
  const float del = __fadd_rn(__fadd_rn(ei, ej), r1.y);
  lockw = min3(lockw, __fadd_rn(s2, del), __fadd_rn(s3, del));
  zmin = min3_nan(zmin, __fsub_rn(s2, del), __fsub_rn(s3, del));
  isgmax = fmaxf(isgmax, isg);
  const float hinv = __fmul_rn(0.5f, __fmul_rn(rd, rd));
  const float a = __fmul_rn(__fadd_rn(d2, r0.w), hinv), bq = __fmul_rn(__fmul_rn(D, rD), hinv);
  kx = __fmaf_rn(a, dx, __fmaf_rn(-bq, dy, pix));
  ky = __fmaf_rn(a, dy, __fmaf_rn(bq, dx, piy));
  ek = __fmaf_rn(del, isg, __fmul_rn(kAddErr * kU, __fadd_rn(R12, __fadd_rn(fabsf(kx), fabsf(ky)))));
}

struct dwp {
  dw x, y;
};

struct LocLocal {  // thread-local array; the fixed slots are copied in
  static constexpr bool kFixInLoc = true;
  dwp* v;
  __device__ dwp get(int s) const { return v[s]; }
  __device__ void set(int s, const dwp& x) const { v[s] = x; }
};
template <class Loc>
__device__ __forceinline__ dwp slot_pos(const Loc& loc, const float4* fix, int nf, int s) {
  if (!Loc::kFixInLoc && s < nf) {
    const float4 f = fix[s];
    return {{f.x, f.y}, {f.z, f.w}};
  }
  return loc.get(s);
}

// Double-word chain of one step into loc[slot], relative to the pivot.  fix holds the
// fixed slots as (x_h, x_l, y_h, y_l).
// Returns true if a dyad locks (D <= 0); *qmin = min q over the dyads solved before
// (qmin may be NULL: the emit needs no q).
// Inlined: as a call it cost the emit 12% (argument passing and saved registers
// around it).
template <class Loc>
__device__ __forceinline__ bool dw_chain(const MechHdr& h, const float4* fix, const DyadRec* __restrict__ dy,
                                         float4 csv, Loc loc, float* qmin) {
  const int nf = h.nf, nd = h.nd;
  if (Loc::kFixInLoc)
    for (int s = 0; s < nf; ++s) {
      float4 f = fix[s];
      loc.set(s, {{f.x, f.y}, {f.z, f.w}});
    }
  dw c = {csv.x, csv.y}, s = {csv.z, csv.w};
  dw ux = {h.ux_h, h.ux_l}, uy = {h.uy_h, h.uy_l};
  dwp m = {dw_sub(dw_mul(c, ux), dw_mul(s, uy)), dw_add(dw_mul(s, ux), dw_mul(c, uy))};
  loc.set(nf, m);
  float q = __int_as_float(0x7f800000);  // +inf
  for (int d = 0; d < nd; ++d) {
    const float c_h = dy[d].r0.w, w2 = dy[d].r1.x;  // records in global or shared memory
    const float4 r2 = dy[d].r2;
    uint32_t sl = __float_as_uint(r2.w);
    const dwp pi = slot_pos(loc, fix, nf, sl & 0xff), pj = slot_pos(loc, fix, nf, (sl >> 8) & 0xff);
    dw dx = dw_sub(pj.x, pi.x), dy_ = dw_sub(pj.y, pi.y);
    dw d2 = dw_sum_sq(dx, dy_);
    dw e = dw_add(d2, dw{c_h, r2.z});
    dw D = dw_4ab_minus_sq(d2, dw{r2.x, r2.y}, e);
    if (!(dw_sign(D) > 0.0f)) {
      if (qmin) *qmin = q;
      return true;
    }
    if (qmin) q = fminf(q, __fdividef(D.h, w2 * w2));
    dw sq = dw_sqrt(D);
    dw hinv = dw_scale2(dw_rcp(d2), 0.5f);
    dw a = dw_mul(e, hinv), bq = dw_mul(sq, hinv);
    dwp pk;
    pk.x = dw_axpby(pi.x, a, dx, bq, dy_, -1.0f);
    pk.y = dw_axpby(pi.y, a, dy_, bq, dx, 1.0f);
    loc.set(sl >> 24, pk);
  }
  if (qmin) *qmin = q;
  return false;
}

}  // namespace links
