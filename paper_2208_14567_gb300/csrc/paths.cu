// paths.cu -- path normalisation and bidirectional chamfer top-k retrieval
// (LINKS, Sec. "Dataset Curation & Processing" and Sec. "A Case Study of Mechanism
// Retrieval").
//
// normalize: per curve of T points, subtract the centroid, scale to unit RMS radius,
//   rotate the major axis of the 2x2 covariance onto +x, and of the two rotations
//   that do this take the one with sum(x^3) >= 0; an isotropic covariance
//   (lambda1 - lambda2 <= 1e-9 (lambda1 + lambda2)) is not rotated; a curve of equal
//   points maps to zeros.  One warp per curve, points in registers: HBM-bound.
// chamfer top-k: CD(P, C) = mean_p min_c |p - c| + mean_c min_p |c - p| (Euclidean),
//   the k smallest per query, ascending, ties to the lower database index.  Each
//   warp owns one query; its four 8-lane groups take four database curves at a time
//   from a shared-memory stage, each lane holding PL query points in registers; the
//   200 x 200 point pairs are reduced to row minima (registers) and column minima
//   (an 8-lane min per database point).  No tensor cores: the inner dimension is 2.
//   Each warp keeps a running top-k in registers; a second kernel merges the partial
//   lists of the database chunks.
#include <algorithm>

#include "links_internal.cuh"

namespace links {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <int PL>
__global__ void __launch_bounds__(256) normalize_kernel(int64_t M, int T, const float2* __restrict__ in,
                                                        float2* __restrict__ out, const int32_t* __restrict__ M_dev) {
  const int lane = threadIdx.x & 31;
  if (M_dev) M = min(M, (int64_t)*M_dev);
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float invT = 1.0f / (float)T;
  for (int64_t m = w0; m < M; m += nw) {
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
      continue;
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
}

// ------------------------------------------------------------------------- chamfer

constexpr int kCWarps = 8;   // queries per CTA
constexpr int kStage = 32;   // database curves per shared-memory stage
constexpr int kMaxK = 32;
constexpr float kFar = 1e18f;

__device__ __forceinline__ bool lex_less(float d, int i, float d2, int i2) {
  return d < d2 || (d == d2 && i < i2);
}

// Insert (d, id) into the warp's sorted top-k held by lanes 0..k-1.
__device__ __forceinline__ void topk_insert(float& kd, int& ki, int k, float d, int id) {
  const int lane = threadIdx.x & 31;
  float last_d = __shfl_sync(kFull, kd, k - 1);
  int last_i = __shfl_sync(kFull, ki, k - 1);
  if (!lex_less(d, id, last_d, last_i)) return;
  const unsigned gt = __ballot_sync(kFull, lane < k && lex_less(d, id, kd, ki));
  const int pos = __ffs(gt) - 1;  // first entry that the candidate beats
  float up_d = __shfl_up_sync(kFull, kd, 1);
  int up_i = __shfl_up_sync(kFull, ki, 1);
  if (lane < k && lane > pos) { kd = up_d; ki = up_i; }
  if (lane == pos) { kd = d; ki = id; }
}

// Packed float pairs (sm_100+ f32x2 arithmetic): one instruction for two lanes' worth.
using f2 = unsigned long long;
__device__ __forceinline__ f2 pk2(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 up2(f2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// PL (even) query points per lane, held as PL/2 packed pairs; database points are
// taken two at a time, so each block of 2 x 2 point pairs costs 8 packed arithmetic
// instructions and 4 three-input minima.
template <int PL>
__global__ void __launch_bounds__(256) chamfer_kernel(int Q, int64_t M, int T, const float2* __restrict__ qs,
                                                      const float2* __restrict__ db, int k, int64_t chunk,
                                                      float* __restrict__ part_d, int32_t* __restrict__ part_i) {
  static_assert(PL % 2 == 0, "query points are processed in pairs");
  extern __shared__ float2 stage[];  // [kStage][T]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 3, gl = lane & 7;
  const unsigned gmask = 0xffu << (g * 8);
  const int q = blockIdx.x * kCWarps + warp;
  const int64_t c0 = (int64_t)blockIdx.y * chunk;
  const int64_t c1 = min(M, c0 + chunk);
  // this lane's query points p = gl * PL + i; padding points sit far away, so they
  // never give a column minimum, and their row minima are left out of the sum
  f2 QX[PL / 2], QY[PL / 2];
#pragma unroll
  for (int i = 0; i < PL / 2; ++i) {
    int t = gl * PL + 2 * i;
    float2 a = (q < Q && t < T) ? qs[(int64_t)q * T + t] : make_float2(kFar, kFar);
    float2 b = (q < Q && t + 1 < T) ? qs[(int64_t)q * T + t + 1] : make_float2(kFar, kFar);
    QX[i] = pk2(a.x, b.x);
    QY[i] = pk2(a.y, b.y);
  }
  float kd = INFINITY;
  int ki = INT32_MAX;
  const float invT = 1.0f / (float)T;
  for (int64_t base = c0; base < c1; base += kStage) {
    const int nst = c1 - base < kStage ? (int)(c1 - base) : kStage;
    __syncthreads();
    for (int x = threadIdx.x; x < nst * T; x += blockDim.x) stage[x] = db[base * T + x];
    __syncthreads();
    if (q >= Q) continue;
    for (int s0 = 0; s0 < nst; s0 += 4) {
      const int s = s0 + g;
      const bool live = s < nst;
      const float2* cp = stage + (live ? s : 0) * T;
      float rmin[PL];
#pragma unroll
      for (int i = 0; i < PL; ++i) rmin[i] = INFINITY;
      float csum = 0.f;
      for (int j = 0; j < T; j += 2) {
        const float2 ca = cp[j];
        const bool two = j + 1 < T;
        const float2 cb = cp[two ? j + 1 : j];
        const f2 AX = pk2(ca.x, ca.x), AY = pk2(ca.y, ca.y);
        const f2 BX = pk2(cb.x, cb.x), BY = pk2(cb.y, cb.y);
        float ma = INFINITY, mb = INFINITY;
#pragma unroll
        for (int i = 0; i < PL / 2; ++i) {
          f2 dxa = sub2(QX[i], AX), dya = sub2(QY[i], AY);
          f2 dxb = sub2(QX[i], BX), dyb = sub2(QY[i], BY);
          float2 ea = up2(fma2(dya, dya, mul2(dxa, dxa)));
          float2 eb = up2(fma2(dyb, dyb, mul2(dxb, dxb)));
          rmin[2 * i] = min3(rmin[2 * i], ea.x, eb.x);
          rmin[2 * i + 1] = min3(rmin[2 * i + 1], ea.y, eb.y);
          ma = min3(ma, ea.x, ea.y);
          mb = min3(mb, eb.x, eb.y);
        }
        ma = fminf(ma, __shfl_xor_sync(gmask, ma, 1));
        mb = fminf(mb, __shfl_xor_sync(gmask, mb, 1));
        ma = fminf(ma, __shfl_xor_sync(gmask, ma, 2));
        mb = fminf(mb, __shfl_xor_sync(gmask, mb, 2));
        ma = fminf(ma, __shfl_xor_sync(gmask, ma, 4));
        mb = fminf(mb, __shfl_xor_sync(gmask, mb, 4));
        csum += sqrtf(ma) + (two ? sqrtf(mb) : 0.f);
      }
      float rsum = 0.f;
#pragma unroll
      for (int i = 0; i < PL; ++i)
        if (gl * PL + i < T) rsum += sqrtf(rmin[i]);
      rsum += __shfl_xor_sync(gmask, rsum, 1);
      rsum += __shfl_xor_sync(gmask, rsum, 2);
      rsum += __shfl_xor_sync(gmask, rsum, 4);
      const float cd = live ? (rsum + csum) * invT : INFINITY;
      // the four groups' results, inserted in database order
#pragma unroll
      for (int gg = 0; gg < 4; ++gg) {
        float d = __shfl_sync(kFull, cd, gg * 8);
        if (s0 + gg < nst) topk_insert(kd, ki, k, d, (int)(base + s0 + gg));
      }
    }
  }
  if (q < Q && lane < k) {
    int64_t o = ((int64_t)q * gridDim.y + blockIdx.y) * k + lane;
    part_d[o] = kd;
    part_i[o] = ki;
  }
}

// One warp per query: merge nchunk partial lists of k into the final top-k.
__global__ void topk_merge_kernel(int Q, int nchunk, int k, const float* __restrict__ part_d,
                                  const int32_t* __restrict__ part_i, int32_t* __restrict__ idx,
                                  float* __restrict__ dist) {
  const int lane = threadIdx.x & 31;
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= Q) return;
  const int n = nchunk * k;
  const float* d = part_d + (int64_t)q * n;
  const int32_t* ii = part_i + (int64_t)q * n;
  float kd = INFINITY;
  int ki = INT32_MAX;
  for (int x0 = 0; x0 < n; x0 += 32) {
    float cd = x0 + lane < n ? d[x0 + lane] : INFINITY;
    int ci = x0 + lane < n ? ii[x0 + lane] : INT32_MAX;
    for (int l = 0; l < 32 && x0 + l < n; ++l) {
      float dd = __shfl_sync(kFull, cd, l);
      int di = __shfl_sync(kFull, ci, l);
      if (di != INT32_MAX) topk_insert(kd, ki, k, dd, di);
    }
  }
  if (lane < k) {
    idx[(int64_t)q * k + lane] = ki == INT32_MAX ? -1 : ki;
    dist[(int64_t)q * k + lane] = kd;
  }
}

template <int PL>
int launch_chamfer(links_ctx ctx, int Q, int64_t M, int T, const float2* qs, const float2* db, int k,
                   int32_t* idx, float* dist) {
  // database chunks: enough CTAs to fill the GPU a few times over
  const int qtiles = (Q + kCWarps - 1) / kCWarps;
  if (M == 0) {  // nothing to rank: idx = -1, dist = +inf
    KernelScope ks(ctx, "topk_merge");
    topk_merge_kernel<<<(Q * 32 + 255) / 256, 256, 0, ctx->stream>>>(Q, 0, k, nullptr, nullptr, idx, dist);
    LINKS_CUDA(cudaGetLastError());
    return LINKS_OK;
  }
  int64_t want = (int64_t)ctx->num_sms * 8;
  int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>((want + qtiles - 1) / qtiles, (M + kStage - 1) / kStage));
  nchunk = std::min<int64_t>(nchunk, 65535);
  int64_t chunk = (M + nchunk - 1) / nchunk;
  chunk = (chunk + kStage - 1) / kStage * kStage;
  nchunk = (M + chunk - 1) / chunk;
  const size_t need = (size_t)Q * nchunk * k * (sizeof(float) + sizeof(int32_t));
  int st = ensure_workspace(ctx, need);
  if (st) return st;
  float* part_d = reinterpret_cast<float*>(ctx->ws);
  int32_t* part_i = reinterpret_cast<int32_t*>(part_d + (size_t)Q * nchunk * k);
  const size_t smem = (size_t)kStage * T * sizeof(float2);
  LINKS_CUDA(cudaFuncSetAttribute(chamfer_kernel<PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    KernelScope ks(ctx, "chamfer");
    chamfer_kernel<PL><<<dim3(qtiles, (unsigned)nchunk), 256, smem, ctx->stream>>>(Q, M, T, qs, db, k, chunk,
                                                                                  part_d, part_i);
  }
  LINKS_CUDA(cudaGetLastError());
  {
    KernelScope ks(ctx, "topk_merge");
    topk_merge_kernel<<<(Q * 32 + 255) / 256, 256, 0, ctx->stream>>>(Q, (int)nchunk, k, part_d, part_i, idx, dist);
  }
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

}  // namespace

static int normalize_launch(links_ctx ctx, int64_t M, const int32_t* M_dev, int T, const float* in, float* out) {
  if (M == 0) return LINKS_OK;
  int per_sm = 8;
  unsigned grid = (unsigned)std::min<int64_t>((M + 7) / 8, (int64_t)ctx->num_sms * per_sm);
  KernelScope ks(ctx, "normalize");
  const float2* i2 = reinterpret_cast<const float2*>(in);
  float2* o2 = reinterpret_cast<float2*>(out);
  if (T <= 64) normalize_kernel<2><<<grid, 256, 0, ctx->stream>>>(M, T, i2, o2, M_dev);
  else if (T <= 256) normalize_kernel<8><<<grid, 256, 0, ctx->stream>>>(M, T, i2, o2, M_dev);
  else normalize_kernel<32><<<grid, 256, 0, ctx->stream>>>(M, T, i2, o2, M_dev);
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

int normalize_paths(links_ctx ctx, int64_t M, int T, const float* in, float* out) {
  return normalize_launch(ctx, M, nullptr, T, in, out);
}

int normalize_paths_count(links_ctx ctx, const int32_t* M_dev, int64_t M_cap, int T, const float* in, float* out) {
  return normalize_launch(ctx, M_cap, M_dev, T, in, out);
}

int chamfer_topk(links_ctx ctx, int Q, int64_t M, int T, const float* q, const float* db, int k, int32_t* idx,
                 float* dist) {
  if (Q == 0) return LINKS_OK;
  const float2* q2 = reinterpret_cast<const float2*>(q);
  const float2* d2 = reinterpret_cast<const float2*>(db);
  const int pl = (T + 7) / 8;
  if (pl <= 4) return launch_chamfer<4>(ctx, Q, M, T, q2, d2, k, idx, dist);
  if (pl <= 8) return launch_chamfer<8>(ctx, Q, M, T, q2, d2, k, idx, dist);
  if (pl <= 16) return launch_chamfer<16>(ctx, Q, M, T, q2, d2, k, idx, dist);
  if (pl <= 26) return launch_chamfer<26>(ctx, Q, M, T, q2, d2, k, idx, dist);
  return launch_chamfer<32>(ctx, Q, M, T, q2, d2, k, idx, dist);
}

}  // namespace links
