// path_core.cuh -- the body of the path normalisation (the configured variant of Sec.
// "Dataset Curation & Processing": centroid, unit RMS radius, principal axis), run by
// paths.cu's kernel and by the serving loop's persistent kernel.  Each including
// translation unit gets its own copy.
#pragma once

#include "links_internal.cuh"

namespace links {
namespace {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Normalisation of curve m (in, out [M, T, 2]; may alias) by one warp: centroid 0, unit
// RMS radius, major axis of the 2x2 covariance on +x with sum(x^3) >= 0; an isotropic
// covariance is not rotated; a curve of equal points maps to zeros.  PL = points per lane.
template <int PL>
__device__ __forceinline__ void normalize_warp(int64_t m, int T, const float2* __restrict__ in, float2* __restrict__ out,
                                               int lane) {
  const float invT = 1.0f / (float)T;
  const float2* src = in + m * T;
  float2 p[PL];
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    int t = lane + 32 * i;
    p[i] = t < T ? __ldcs(src + t) : make_float2(0.f, 0.f);
  }
  // work relative to the first point: smaller magnitudes, and a curve of equal
  // points becomes exactly zero (so it is recognised below)
  const float ox = __shfl_sync(kFull, p[0].x, 0), oy = __shfl_sync(kFull, p[0].y, 0);
  float sx = 0.f, sy = 0.f;
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    if (lane + 32 * i < T) {
      p[i].x -= ox;
      p[i].y -= oy;
      sx += p[i].x;
      sy += p[i].y;
    }
  }
  const float cx = warp_sum(sx) * invT, cy = warp_sum(sy) * invT;
  float r2 = 0.f;
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    if (lane + 32 * i < T) {
      p[i].x -= cx;
      p[i].y -= cy;
      r2 = fmaf(p[i].x, p[i].x, fmaf(p[i].y, p[i].y, r2));
    }
  }
  const float ms = warp_sum(r2) * invT;
  float2* dst = out + m * T;
  if (!(ms > 0.f)) {
#pragma unroll
    for (int i = 0; i < PL; ++i)
      if (lane + 32 * i < T) __stcs(dst + lane + 32 * i, make_float2(0.f, 0.f));
    return;
  }
  const float inv = rsqrtf(ms);
  float a = 0.f, bxy = 0.f, c = 0.f;
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    if (lane + 32 * i < T) {
      p[i].x *= inv;
      p[i].y *= inv;
      a = fmaf(p[i].x, p[i].x, a);
      bxy = fmaf(p[i].x, p[i].y, bxy);
      c = fmaf(p[i].y, p[i].y, c);
    }
  }
  const float sxx = warp_sum(a) * invT, sxy = warp_sum(bxy) * invT, syy = warp_sum(c) * invT;
  const float dxy = sxx - syy;
  const float gap = sqrtf(fmaf(dxy, dxy, 4.f * sxy * sxy));
  float cs = 1.f, sn = 0.f;
  if (gap > 1e-9f * (sxx + syy)) sincosf(0.5f * atan2f(2.f * sxy, dxy), &sn, &cs);
  float s3 = 0.f;
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    if (lane + 32 * i < T) {
      float xr = fmaf(cs, p[i].x, sn * p[i].y);
      float yr = fmaf(-sn, p[i].x, cs * p[i].y);
      p[i] = make_float2(xr, yr);
      s3 = fmaf(xr * xr, xr, s3);
    }
  }
  const float sg = warp_sum(s3) < 0.f ? -1.f : 1.f;
#pragma unroll
  for (int i = 0; i < PL; ++i)
    if (lane + 32 * i < T) __stcs(dst + lane + 32 * i, make_float2(sg * p[i].x, sg * p[i].y));
}

}  // namespace
}  // namespace links
