// paths.cu -- path normalisation, dataset curation and chamfer retrieval
// (LINKS, Sec. "Dataset Curation & Processing" and Sec. "A Case Study of Mechanism
// Retrieval").
//
// normalize: per curve of T points, subtract the centroid, scale to unit RMS radius,
//   rotate the major axis of the 2x2 covariance onto +x, and of the two rotations
//   that do this take the one with sum(x^3) >= 0; an isotropic covariance
//   (lambda1 - lambda2 <= 1e-9 (lambda1 + lambda2)) is not rotated; a curve of equal
//   points maps to zeros.  One warp per curve, points in registers: HBM-bound.
// normalize_maxline: the paper's normalisation (farthest pair onto a unit horizontal
//   line, bounding box centred at (0.5, 0.5)) and its circle statistic; one warp per
//   curve, the farthest pair in two passes of packed arithmetic.
// curation: the same per joint path of the simulated rows, arc and circle flags, the
//   keep draws, and an ordered compaction of the kept paths.
// chamfer: CD(P, C) = mean_p min_c |p - c| + mean_c min_p |c - p| (Euclidean).  A CTA
//   takes 16 queries (a warp each) against a chunk of the database staged in shared
//   memory 32 curves at a time; 16-lane groups compute exact CDs with the query's points
//   in registers (packed pairs), after lower bounds (a distance table of the query and
//   runs of 4 database points) drop the curves that cannot qualify.  No tensor cores: the
//   inner dimension is 2.  Top-k mode keeps each query's k smallest (ascending, ties to
//   the lower index), pruning at the k-th distance found so far; first-k mode scans the
//   database in a given order and keeps the first k curves under a cut-off, pruning at
//   the cut-off and skipping positions past the k-th hit.  A second kernel merges the
//   chunks' lists.
#include <cuda_fp16.h>

#include <algorithm>

#include "path_core.cuh"
#include "packed.cuh"

namespace links {
namespace {

template <int PL>
__global__ void __launch_bounds__(256) normalize_kernel(int64_t M, int T, const float2* __restrict__ in,
                                                        float2* __restrict__ out, const int32_t* __restrict__ M_dev) {
  const int lane = threadIdx.x & 31;
  if (M_dev) M = min(M, (int64_t)*M_dev);
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t m = w0; m < M; m += nw) normalize_warp<PL>(m, T, in, out, lane);
}

// The paper's path normalisation (Sec. "Dataset Curation & Processing"): the farthest
// pair of points (a, b), a < b, becomes a horizontal line of length 1 from a to b and
// the bounding box is centred at (0.5, 0.5); the circle statistic is the variance of
// the points' distances from (0.5, 0.5) (the paper's circle test).  One warp per curve,
// staged in shared memory; lane l holds points u = l + 32 i.

// Loads curve src (T points) into the lane's registers and the warp's shared copy.
template <int PL>
__device__ __forceinline__ void load_curve(const float2* __restrict__ src, int T, int lane, float2* sp,
                                           float2 (&p)[PL]) {
  __syncwarp();
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    const int t = lane + 32 * i;
    p[i] = t < T ? src[t] : make_float2(0.f, 0.f);
    sp[t] = p[i];
  }
  __syncwarp();
}

// The farthest pair, first in (a, b) order among equal distances, in two passes:
// (1) each lane keeps, per point u, the largest squared distance to a later point v
// (read as a broadcast from shared memory, two u at a time in packed f32x2 arithmetic,
// blocks with every u > v skipped), and the warp takes the maximum; (2) a is the first
// u whose maximum equals it and b the first v > a at that distance.  Both passes
// evaluate the same expression on the same operands, so the equality test is exact.
// One point gives the pair (0, 0).
template <int PL>
__device__ __forceinline__ void farthest_pair(const float2 (&p)[PL], const float2* sp, int T, int lane, int& ba,
                                              int& bb) {
  static_assert(PL % 2 == 0, "points are paired for the packed arithmetic");
  f2 UX[PL / 2], UY[PL / 2];
  float bu[PL];  // per point u: largest squared distance to a later point (-1: none)
#pragma unroll
  for (int k = 0; k < PL / 2; ++k) {
    UX[k] = pk2(p[2 * k].x, p[2 * k + 1].x);
    UY[k] = pk2(p[2 * k].y, p[2 * k + 1].y);
    bu[2 * k] = bu[2 * k + 1] = -1.0f;
  }
#pragma unroll
  for (int j = 0; j < PL; ++j) {  // v = 32 j + vl
    const int nv = min(32, T - 32 * j);
    for (int vl = 0; vl < nv; ++vl) {
      const float2 c = sp[32 * j + vl];
      const f2 VX = pk2(c.x, c.x), VY = pk2(c.y, c.y);
#pragma unroll
      for (int k = 0; k < PL / 2; ++k) {
        if (2 * k > j) continue;  // u >= 32 (j + 1) > v
        const f2 dx = sub2(VX, UX[k]), dy = sub2(VY, UY[k]);
        const float2 d2 = up2(fma2(dx, dx, mul2(dy, dy)));
        if (2 * k < j) bu[2 * k] = fmaxf(bu[2 * k], d2.x);
        else if (lane < vl) bu[2 * k] = fmaxf(bu[2 * k], d2.x);
        if (2 * k + 1 < j) bu[2 * k + 1] = fmaxf(bu[2 * k + 1], d2.y);
        else if (2 * k + 1 == j && lane < vl) bu[2 * k + 1] = fmaxf(bu[2 * k + 1], d2.y);
      }
    }
  }
  float best = bu[0];
#pragma unroll
  for (int i = 1; i < PL; ++i) best = fmaxf(best, bu[i]);
#pragma unroll
  for (int o = 16; o; o >>= 1) best = fmaxf(best, __shfl_xor_sync(kFull, best, o));
  ba = INT32_MAX;
#pragma unroll
  for (int i = PL - 1; i >= 0; --i)
    if (best >= 0.f && bu[i] == best) ba = lane + 32 * i;
#pragma unroll
  for (int o = 16; o; o >>= 1) ba = min(ba, __shfl_xor_sync(kFull, ba, o));
  if (ba == INT32_MAX) ba = 0;
  const float2 A = sp[ba];
  bb = INT32_MAX;
  const f2 AX = pk2(A.x, A.x), AY = pk2(A.y, A.y);
#pragma unroll
  for (int k = PL / 2 - 1; k >= 0; --k) {  // the first pass's packed operations, v - u
    const f2 dx = sub2(UX[k], AX), dy = sub2(UY[k], AY);
    const float2 d2 = up2(fma2(dx, dx, mul2(dy, dy)));
    const int v0 = lane + 64 * k, v1 = v0 + 32;
    if (v1 > ba && v1 < T && d2.y == best) bb = v1;
    if (v0 > ba && v0 < T && d2.x == best) bb = v0;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) bb = min(bb, __shfl_xor_sync(kFull, bb, o));
  if (bb == INT32_MAX) bb = ba;
}

// Normalises the curve on the pair (ba, bb) (points a and b read from the shared
// copy), writes it to dst when dst is not NULL, and returns the circle statistic
// (the same value in every lane).  Equal points give the centre of the box and 0.
template <int PL>
__device__ __forceinline__ float maxline_apply(float2 (&p)[PL], const float2* sp, int T, int lane, int ba, int bb,
                                               float2* dst) {
  const float invT = 1.0f / (float)T;
  const float ax = sp[ba].x, ay = sp[ba].y;
  const float dx = sp[bb].x - ax, dy = sp[bb].y - ay;
  const float d = sqrtf(fmaf(dx, dx, dy * dy));
  if (!(d > 0.0f)) {
    if (dst) {
#pragma unroll
      for (int i = 0; i < PL; ++i)
        if (lane + 32 * i < T) dst[lane + 32 * i] = make_float2(0.5f, 0.5f);
    }
    return 0.0f;
  }
  const float c = dx / d, s = dy / d, inv = 1.0f / d;
  float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    const float x = p[i].x - ax, y = p[i].y - ay;
    p[i] = make_float2(fmaf(c, x, s * y) * inv, fmaf(c, y, -s * x) * inv);
    if (lane + 32 * i < T) {
      x0 = fminf(x0, p[i].x);
      x1 = fmaxf(x1, p[i].x);
      y0 = fminf(y0, p[i].y);
      y1 = fmaxf(y1, p[i].y);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    x0 = fminf(x0, __shfl_xor_sync(kFull, x0, o));
    x1 = fmaxf(x1, __shfl_xor_sync(kFull, x1, o));
    y0 = fminf(y0, __shfl_xor_sync(kFull, y0, o));
    y1 = fmaxf(y1, __shfl_xor_sync(kFull, y1, o));
  }
  const float sx = 0.5f - 0.5f * (x0 + x1), sy = 0.5f - 0.5f * (y0 + y1);
  float r[PL], rs = 0.f;
#pragma unroll
  for (int i = 0; i < PL; ++i) {
    p[i].x += sx;
    p[i].y += sy;
    r[i] = hypotf(p[i].x - 0.5f, p[i].y - 0.5f);
    if (lane + 32 * i < T) {
      if (dst) dst[lane + 32 * i] = p[i];
      rs += r[i];
    }
  }
  const float mean = warp_sum(rs) * invT;
  float v = 0.f;
#pragma unroll
  for (int i = 0; i < PL; ++i)
    if (lane + 32 * i < T) v = fmaf(r[i] - mean, r[i] - mean, v);
  return warp_sum(v) * invT;
}

template <int PL>
__global__ void __launch_bounds__(256) maxline_kernel(int64_t M, int T, const float2* __restrict__ in,
                                                      float2* __restrict__ out, int32_t* __restrict__ pair,
                                                      float* __restrict__ circ_var) {
  __shared__ float2 curve_s[8][32 * PL];
  const int lane = threadIdx.x & 31;
  float2* sp = curve_s[threadIdx.x >> 5];
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t m = w0; m < M; m += nw) {
    float2 p[PL];
    load_curve<PL>(in + m * T, T, lane, sp, p);
    int ba, bb;
    farthest_pair<PL>(p, sp, T, lane, ba, bb);
    const float v = maxline_apply<PL>(p, sp, T, lane, ba, bb, out + m * T);
    if (lane == 0) {
      if (pair) pair[2 * m] = ba, pair[2 * m + 1] = bb;
      if (circ_var) circ_var[m] = v;
    }
  }
}

// ------------------------------------------------------------------------ curation
//
// The paper's dataset curation (Sec. "Dataset Curation & Processing"): the path of
// every moving joint of every mechanism is normalised; a path is an arc when its joint
// is linked to a fixed joint and a circle when its circle statistic is below a
// threshold; arcs and circles are removed except for a random fraction kept.  The
// keep draw of path (b, j) is output b * n_max + j of the splitmix64 generator (Steele,
// Lea and Flood, OOPSLA 2014; Vigna's constants) started at the seed, as a double in
// [0, 1) from its top 53 bits.

enum : uint8_t { kPathBit = 1, kArcBit = 2, kCircleBit = 4, kKeptBit = 8 };

__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-53;
}

struct CurateArgs {
  int64_t R;                 // rows (mechanisms with trajectories)
  int n_max, T;
  const float2* traj;        // [R, n_max, T]
  const int32_t* row_index;  // [R] mechanism of each row (NULL: row r is mechanism r)
  int64_t B;                 // mechanisms (bound of the row_index entries)
  int32_t* err;              // device error word (bit 2: a row index out of range)
  const int32_t* n_joints;   // [B]
  const uint8_t* adj;        // [B, n_max, n_max]
  const int8_t* type;        // [B, n_max]
  double circle_var, keep_rate;
  uint64_t seed;
  uint8_t* flags;            // [R, n_max]
  float* circ_var;           // [R, n_max] or NULL
  int32_t* pair;             // [R, n_max, 2]
};

// One warp per (row, joint): flags, circle statistic and the normalising pair.
template <int PL>
__global__ void __launch_bounds__(256) curate_flags_kernel(CurateArgs ca) {
  __shared__ float2 curve_s[8][32 * PL];
  const int lane = threadIdx.x & 31;
  float2* sp = curve_s[threadIdx.x >> 5];
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = ca.R * ca.n_max;
  for (int64_t e = w0; e < total; e += nw) {
    const int64_t r = e / ca.n_max;
    const int j = (int)(e - r * ca.n_max);
    const int64_t b = ca.row_index ? ca.row_index[r] : r;
    const bool bad = b < 0 || b >= ca.B;
    if (bad && lane == 0 && j == 0) atomicOr(ca.err, 2);
    const int n = bad ? 0 : min(ca.n_joints[b], ca.n_max);
    const int8_t* tb = ca.type + (bad ? 0 : b) * ca.n_max;
    if (j >= n || tb[j] == 0) {  // padding, a fixed joint or a bad row: no path
      if (lane == 0) {
        ca.flags[e] = 0;
        if (ca.circ_var) ca.circ_var[e] = 0.f;
        ca.pair[2 * e] = ca.pair[2 * e + 1] = 0;
      }
      continue;
    }
    float2 p[PL];
    load_curve<PL>(ca.traj + e * ca.T, ca.T, lane, sp, p);
    int ba, bb;
    farthest_pair<PL>(p, sp, ca.T, lane, ba, bb);
    const float v = maxline_apply<PL>(p, sp, ca.T, lane, ba, bb, nullptr);
    const uint8_t* ab = ca.adj + (b * ca.n_max + j) * ca.n_max;
    bool ground = false;
    for (int k = lane; k < n; k += 32) ground = ground || (ab[k] && tb[k] == 0);
    const bool arc = __any_sync(kFull, ground);
    const bool circle = (double)v < ca.circle_var;
    const bool kept = !(arc || circle) || splitmix_uniform(ca.seed, (uint64_t)(b * ca.n_max + j)) < ca.keep_rate;
    if (lane == 0) {
      ca.flags[e] = kPathBit | (arc ? kArcBit : 0) | (circle ? kCircleBit : 0) | (kept ? kKeptBit : 0);
      if (ca.circ_var) ca.circ_var[e] = v;
      ca.pair[2 * e] = ba;
      ca.pair[2 * e + 1] = bb;
    }
  }
}

// One warp per kept path: its normalised curve at its place in the kept list.
template <int PL>
__global__ void __launch_bounds__(256) curate_write_kernel(int n_max, int T, const float2* __restrict__ traj,
                                                           const int32_t* __restrict__ pair,
                                                           const int32_t* __restrict__ kept_index,
                                                           const int32_t* __restrict__ n_kept, int64_t cap,
                                                           float2* __restrict__ out) {
  __shared__ float2 curve_s[8][32 * PL];
  const int lane = threadIdx.x & 31;
  float2* sp = curve_s[threadIdx.x >> 5];
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = min((int64_t)*n_kept, cap);
  for (int64_t q = w0; q < n; q += nw) {
    const int64_t e = kept_index[q];
    float2 p[PL];
    load_curve<PL>(traj + e * T, T, lane, sp, p);
    maxline_apply<PL>(p, sp, T, lane, pair[2 * e], pair[2 * e + 1], out + q * T);
  }
}

template <int PL>
static int launch_curate(links_ctx ctx, const CurateArgs& ca, int32_t* kept_index, float* kept_paths, int64_t cap,
                         int32_t* n_kept, int32_t* sums) {
  int per_sm = 0;
  LINKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, curate_flags_kernel<PL>, 256, 0));
  const int64_t total = ca.R * ca.n_max;
  unsigned grid = (unsigned)std::min<int64_t>((total + 7) / 8, (int64_t)ctx->num_sms * std::max(per_sm, 1));
  if (grid > 0) {
    KernelScope ks(ctx, "curate_flags");
    curate_flags_kernel<PL><<<grid, 256, 0, ctx->stream>>>(ca);
    LINKS_CUDA(cudaGetLastError());
  }
  {
    KernelScope ks(ctx, "curate_compact");
    int st = compact_flags(ctx->stream, ca.flags, kKeptBit, total, sums, kept_index, cap, n_kept);
    if (st) return st;
  }
  if (kept_paths && cap > 0) {
    LINKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, curate_write_kernel<PL>, 256, 0));
    grid = (unsigned)std::min<int64_t>((std::min(cap, total) + 7) / 8, (int64_t)ctx->num_sms * std::max(per_sm, 1));
    if (grid > 0) {
      KernelScope ks(ctx, "curate_write");
      curate_write_kernel<PL><<<grid, 256, 0, ctx->stream>>>(ca.n_max, ca.T, ca.traj, ca.pair, kept_index, n_kept,
                                                             cap, reinterpret_cast<float2*>(kept_paths));
      LINKS_CUDA(cudaGetLastError());
    }
  }
  return LINKS_OK;
}

// ------------------------------------------------------------------------- chamfer

constexpr int kStage = 32;   // database curves per shared-memory stage
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

// Insertion into a warp's list of the first k hits in scan order: lane i < k holds the
// i-th smallest scan position found so far (INT32_MAX when empty) and its distance.
// Positions are unique, so the order is total.
__device__ __forceinline__ void first_insert(float& kd, int& ki, int k, float d, int pos) {
  const int lane = threadIdx.x & 31;
  if (pos >= __shfl_sync(kFull, ki, k - 1)) return;
  const unsigned gt = __ballot_sync(kFull, lane < k && pos < ki);
  const int at = __ffs(gt) - 1;
  float up_d = __shfl_up_sync(kFull, kd, 1);
  int up_i = __shfl_up_sync(kFull, ki, 1);
  if (lane < k && lane > at) { kd = up_d; ki = up_i; }
  if (lane == at) { kd = d; ki = pos; }
}

// Chamfer distance in FP64 by a 16-lane group (all lanes return the value), for a
// pair whose FP32 distance lies within its rounding band of a threshold, so that the
// decision is the one the FP64 definition takes.  It is that definition evaluated
// step for step: squared distances without fused multiply-adds, the nearest point's
// distance per point, and each term's sum taken in point order (sixteen points at a
// time, one per lane, added in lane order), so the value is the same to the last bit
// as a plain sequential evaluation.
__device__ __noinline__ double chamfer_f64(const float2* __restrict__ qp, const float2* cp, int T, int gl,
                                           unsigned gmask) {
  double sum[2] = {0.0, 0.0};
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {  // 0: query points to the curve, 1: the reverse
    const float2* from = side ? cp : qp;
    const float2* to = side ? qp : cp;
    double s = 0.0;
    for (int t0 = 0; t0 < T; t0 += 16) {
      double v = 0.0;
      if (t0 + gl < T) {
        const double ax = from[t0 + gl].x, ay = from[t0 + gl].y;
        double m = INFINITY;
        for (int j = 0; j < T; ++j) {
          const double dx = ax - (double)to[j].x, dy = ay - (double)to[j].y;
          m = fmin(m, __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        }
        v = sqrt(m);
      }
      const int n = min(16, T - t0);
      for (int l = 0; l < n; ++l) s = __dadd_rn(s, __shfl_sync(gmask, v, l, 16));
    }
    sum[side] = s;
  }
  return __dadd_rn(sum[0] / T, sum[1] / T);
}

__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// ---- exact pruning
//
// Column term.  DT(x) = min over query points p of |x - p| is 1-Lipschitz, so for a
// database point c and any grid node v, min_p |c - p| = DT(c) >= DT(v) - |c - v|.
// The column term of CD (mean over c of DT(c)) is therefore bounded below by the
// mean of max(0, DT(v(c)) - |c - v(c)|), v(c) the node nearest to c: one table
// look-up per database point.  The table holds DT at kNG x kNG nodes over the query's
// bounding square with a margin, rounded down to half precision.
//
// Row term.  The database curve's points are split into runs of kRun consecutive
// points with centre z_g; rho bounds |c - z_g| for every point of every run.  A
// query point p is then at least min_g |p - z_g| - rho from the curve, which costs
// ceil(T/kRun) instead of T distance evaluations per query point.  (Runs of 4 prune
// about twice as many pairs as runs of 8 for twice the cost of this bound, which pays.)

constexpr int kNG = 60;                       // grid nodes per side (7200-byte table)
constexpr int kRun = 4;                       // points per run
constexpr int kMaxG = 64;                     // runs per curve (T <= 256)
constexpr float kLbShrink = 1.0f - 0x1p-20f;  // covers the rounding of computed distances
constexpr float kLbGrow = 1.0f + 0x1p-20f;    // (relative error below 2^-21.9 each)
constexpr float kRound = 12582912.0f;         // 1.5 * 2^23: x + kRound rounds x to an integer

// Hardware reciprocal square root (relative error at most 2^-22.9; +inf at 0, so
// d2 * rsqrt_approx(d2) is NaN there and the caller's fmaxf drops the term, which
// only lowers the bound).
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One CTA per query: node spacing and origin, then DT at every node (brute force).
// Also resets the query's shared pruning distance.
__global__ void __launch_bounds__(256) dt_grid_kernel(int Q, int T, const float2* __restrict__ qs,
                                                      __half* __restrict__ grids, float4* __restrict__ gparam,
                                                      float* __restrict__ gthr) {
  __shared__ float2 pts[256];
  __shared__ float red[4][8];
  const int q = blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  float2 v = t < T ? qs[(int64_t)q * T + t] : make_float2(0.f, 0.f);
  if (t < T) pts[t] = v;
  float lo_x = t < T ? v.x : INFINITY, hi_x = t < T ? v.x : -INFINITY;
  float lo_y = t < T ? v.y : INFINITY, hi_y = t < T ? v.y : -INFINITY;
  for (int o = 16; o > 0; o >>= 1) {
    lo_x = fminf(lo_x, __shfl_xor_sync(kFull, lo_x, o));
    hi_x = fmaxf(hi_x, __shfl_xor_sync(kFull, hi_x, o));
    lo_y = fminf(lo_y, __shfl_xor_sync(kFull, lo_y, o));
    hi_y = fmaxf(hi_y, __shfl_xor_sync(kFull, hi_y, o));
  }
  if (lane == 0) {
    red[0][warp] = lo_x;
    red[1][warp] = hi_x;
    red[2][warp] = lo_y;
    red[3][warp] = hi_y;
  }
  __syncthreads();
  float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
  for (int w = 0; w < 8; ++w) {
    x0 = fminf(x0, red[0][w]);
    x1 = fmaxf(x1, red[1][w]);
    y0 = fminf(y0, red[2][w]);
    y1 = fmaxf(y1, red[3][w]);
  }
  float side = fmaxf(x1 - x0, y1 - y0);
  if (!(side > 0.f)) side = 1.0f;  // one distinct point (or non-finite input)
  const float h = side * 1.3f / (float)(kNG - 1);
  const float ox = 0.5f * (x0 + x1) - 0.65f * side, oy = 0.5f * (y0 + y1) - 0.65f * side;
  if (t == 0) {
    gparam[q] = make_float4(ox, oy, h, 1.0f / h);
    gthr[q] = INFINITY;
  }
  for (int node = t; node < kNG * kNG; node += blockDim.x) {
    const int ix = node % kNG, iy = node / kNG;
    const float nx = fmaf((float)ix, h, ox), ny = fmaf((float)iy, h, oy);
    float m = INFINITY;
    for (int j = 0; j < T; ++j) {
      const float dx = pts[j].x - nx, dy = pts[j].y - ny;
      m = fminf(m, fmaf(dy, dy, dx * dx));
    }
    grids[(int64_t)q * kNG * kNG + node] = __float2half_rd(sqrtf(m) * kLbShrink);
  }
}

// The exact and the bounding computations run on 16-lane groups (two per warp):
// lane gl of a group holds query points gl * PL + i (i < PL), packed in pairs, read
// from global memory (L1) for each pair it takes;
// points past T sit far away, so they never give a column minimum, and their row
// minima are left out of the sums.
template <int PL>
__device__ __forceinline__ void load_query(const float2* qp, int T, int gl, f2* QX, f2* QY) {
#pragma unroll
  for (int i = 0; i < PL / 2; ++i) {
    const int t = gl * PL + 2 * i;
    const float2 a = t < T ? qp[t] : make_float2(kFar, kFar);
    const float2 b = t + 1 < T ? qp[t + 1] : make_float2(kFar, kFar);
    QX[i] = pk2(a.x, b.x);
    QY[i] = pk2(a.y, b.y);
  }
}

__device__ __forceinline__ float group_sum16(float v, unsigned gmask) {
  v += __shfl_xor_sync(gmask, v, 1);
  v += __shfl_xor_sync(gmask, v, 2);
  v += __shfl_xor_sync(gmask, v, 4);
  v += __shfl_xor_sync(gmask, v, 8);
  return v;
}

// Squared distances of this lane's query points to database point (ax, ay), folded
// into the row minima (rmin) and returned as the lane's minimum (column minimum).
template <int PL>
__device__ __forceinline__ void fold_point4(const f2* QX, const f2* QY, const float2* c, float* rmin, float* m) {
  f2 CX[4], CY[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    CX[u] = pk2(c[u].x, c[u].x);
    CY[u] = pk2(c[u].y, c[u].y);
  }
#pragma unroll
  for (int i = 0; i < PL / 2; ++i) {
    float2 e[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const f2 dx = sub2(QX[i], CX[u]), dy = sub2(QY[i], CY[u]);
      e[u] = up2(fma2(dy, dy, mul2(dx, dx)));
      m[u] = min3(m[u], e[u].x, e[u].y);
    }
    rmin[2 * i] = min3(min3(rmin[2 * i], e[0].x, e[1].x), e[2].x, e[3].x);
    rmin[2 * i + 1] = min3(min3(rmin[2 * i + 1], e[0].y, e[1].y), e[2].y, e[3].y);
  }
}

// Minimum of four per-lane values over the 16-lane group, transposed: after the
// exchange the lane holds the minimum of value v = 2 * (gl >> 3) + ((gl >> 2) & 1)
// (five shuffles for four values instead of sixteen).
__device__ __forceinline__ float group_min4(const float* m, int gl, unsigned gmask) {
  const bool hi = gl & 8, b4 = gl & 4;
  const float k0 = hi ? m[2] : m[0], k1 = hi ? m[3] : m[1];
  const float s0 = hi ? m[0] : m[2], s1 = hi ? m[1] : m[3];
  const float a0 = fminf(k0, __shfl_xor_sync(gmask, s0, 8));
  const float a1 = fminf(k1, __shfl_xor_sync(gmask, s1, 8));
  float v = fminf(b4 ? a1 : a0, __shfl_xor_sync(gmask, b4 ? a0 : a1, 4));
  v = fminf(v, __shfl_xor_sync(gmask, v, 2));
  return fminf(v, __shfl_xor_sync(gmask, v, 1));
}

// Row-term lower bound: mean over query points of max(0, min_g |p - z_g| - rho),
// computed by the 16-lane group (all lanes return the same value).
template <int PL>
__device__ __forceinline__ float row_bound(const f2* QX, const f2* QY, const float2* cz, int G, float rho, int T,
                                           int gl, unsigned gmask, float invT) {
  float rmin[PL];
#pragma unroll
  for (int i = 0; i < PL; ++i) rmin[i] = INFINITY;
  for (int g = 0; g < G; g += 4) {
    float2 c[4];
    float m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c[u] = cz[g + u < G ? g + u : g];  // repeats change no minimum
      m[u] = INFINITY;
    }
    fold_point4<PL>(QX, QY, c, rmin, m);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PL; ++i)
    if (gl * PL + i < T) s += fmaxf(fmaf(sqrtf(rmin[i]), kLbShrink, -rho), 0.f);
  return group_sum16(s, gmask) * invT;
}

// Exact CD of the query (this lane's PL points, packed) and database curve cp,
// computed by the lane's 16-lane group (all lanes return the same value).  Returns
// +inf as soon as the partial column sum alone exceeds thr: the full value can only
// be larger (the sums only add non-negative terms), so such a curve cannot enter.
template <int PL>
__device__ __forceinline__ float chamfer_exact(const f2* QX, const f2* QY, const float2* cp, int T, int gl,
                                               unsigned gmask, float invT, float thr) {
  float rmin[PL];
#pragma unroll
  for (int i = 0; i < PL; ++i) rmin[i] = INFINITY;
  const int v = 2 * (gl >> 3) + ((gl >> 2) & 1);  // the database point this lane sums
  float csum = 0.f;                               // over the points j + v
  for (int j = 0; j < T; j += 4) {
    float2 c[4];
    float m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c[u] = cp[j + u < T ? j + u : j];  // repeats change no row minimum
      m[u] = INFINITY;
    }
    fold_point4<PL>(QX, QY, c, rmin, m);
    const float mv = group_min4(m, gl, gmask);
    if (j + v < T) csum += sqrtf(mv);
    if ((j & 15) == 12) {  // every 16 points: stop once the column sum alone passes thr
      float cs = csum + __shfl_xor_sync(gmask, csum, 4);
      cs += __shfl_xor_sync(gmask, cs, 8);
      if (cs * invT > thr) return INFINITY;  // uniform in the group
    }
  }
  float cs = csum + __shfl_xor_sync(gmask, csum, 4);
  cs += __shfl_xor_sync(gmask, cs, 8);
  float rsum = 0.f;
#pragma unroll
  for (int i = 0; i < PL; ++i)
    if (gl * PL + i < T) rsum += sqrtf(rmin[i]);
  rsum = group_sum16(rsum, gmask);
  return (rsum + cs) * invT;
}

// W queries per CTA (one warp each, which keeps the query's top-k), one chunk of the
// database per CTA column, staged kStage curves at a time.  Per stage, with pruning:
//   A. lane s of warp w bounds the column term of (query w, curve s) with the
//      query's distance table; pairs whose bound exceeds the pruning distance drop;
//   B. the CTA's 16-lane groups share out the remaining pairs and add the row-term
//      bound; pairs over the pruning distance drop again;
//   C. the groups share out the rest and compute exact CDs (stopping early once the
//      partial column sum passes the pruning distance), and each warp inserts its
//      query's results into its top-k.
// Without pruning every pair goes to C.  The pruning distance of a query is the
// smaller of its warp's current k-th distance and the query's shared one, the
// smallest k-th distance any chunk has published: either is the k-th smallest CD of
// some k database curves, so a curve whose CD is larger cannot be among the k
// nearest, and the result is the exhaustive one; only the work depends on timing.
// Both bounds carry a relative rounding error below 2e-5 (sums of at most 256
// terms), as does the exact CD; the comparison margin covers both.  Sharing the
// pairs of a stage among all groups keeps the warps' work equal between barriers.
//
// FIRST instead runs the paper's retrieval (Sec. "A Case Study of Mechanism
// Retrieval"): the database is read in the scan order fa.order (position r holds
// curve order[r]; M is then the number of positions), each query keeps the first k
// positions whose CD is below the fixed threshold fa.thr, and the pruning distance
// is that threshold.  A position at or past the k-th hit a query already has, in
// this chunk or in any chunk that published one (fa.gpos), cannot be among its first
// k, so it is skipped; a CTA stops once all its queries have their k hits before
// the stage it would read next.  A pair whose FP32 CD lies within the rounding band
// of the threshold is decided by the FP64 distance.
struct FirstArgs {
  const int32_t* order = nullptr;  // [M] database curve of each scan position
  int64_t n_db = 0;                // database curves (bound of the order entries)
  double thr = 0.0;                // hits are CD < thr
  int32_t* gpos = nullptr;         // [Q] smallest k-th hit position published
  int32_t* err = nullptr;          // device error word (bit 2: an order entry out of range)
};

template <int PL, int W, bool FIRST>
__global__ void __launch_bounds__(W * 32) chamfer_kernel(int Q, int64_t M, int T, const float2* __restrict__ qs,
                                                         const float2* __restrict__ db, int k, int64_t chunk,
                                                         float* __restrict__ part_d, int32_t* __restrict__ part_i,
                                                         const __half* __restrict__ grids,
                                                         const float4* __restrict__ gparam, float* gthr,
                                                         FirstArgs fa) {
  static_assert(PL % 2 == 0, "query points are processed in pairs");
  constexpr int kGroups = W * 2;
  extern __shared__ __align__(16) float2 dyn[];
  float2* stage = dyn;                     // [kStage][T] database curves
  float2* cen = stage + kStage * T;        // [kStage][kMaxG] run centres (pruning)
  __half* sgrid = reinterpret_cast<__half*>(cen + kStage * kMaxG);  // [W][kNG^2] (pruning)
  __shared__ unsigned rho_s[kStage];       // run radius per staged curve (float bits)
  __shared__ float thr_w[W];
  __shared__ uint16_t listA[W * kStage], listB[W * kStage];
  __shared__ float lbA[W * kStage];
  __shared__ int nA, nB, nres[W];
  __shared__ float res_d[W][kStage];
  __shared__ uint8_t res_s[W][kStage];
  __shared__ int32_t ord_s[kStage];        // FIRST: curve of each staged position (-1: bad entry)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 4, gl = lane & 15, gid = warp * 2 + g;
  const unsigned gmask = 0xffffu << (g * 16);
  const int qbase = blockIdx.x * W, q = qbase + warp;
  const int64_t c0 = (int64_t)blockIdx.y * chunk;
  const int64_t c1 = min(M, c0 + chunk);
  const bool prune = grids != nullptr;
  const int G = (T + kRun - 1) / kRun;
  const float invT = 1.0f / (float)T;
  const float margin = 4e-5f;
  __half* mygrid = sgrid + warp * kNG * kNG;
  float4 gp = make_float4(0.f, 0.f, 0.f, 0.f);
  if (prune && q < Q) {
    const uint4* src = reinterpret_cast<const uint4*>(grids + (int64_t)q * kNG * kNG);
    uint4* dst = reinterpret_cast<uint4*>(mygrid);
    for (int x = lane; x < kNG * kNG / 8; x += 32) dst[x] = src[x];
    gp = gparam[q];
  }
  float kd = INFINITY;
  int ki = INT32_MAX;
  float thr_pub = INFINITY;  // last k-th distance published (lane k-1)
  int pos_pub = INT32_MAX;   // FIRST: last k-th position published
  const float fthr = (float)fa.thr;
  const float fband = fthr < INFINITY ? margin * fthr + 1e-6f : 0.f;
  int cut = INT32_MAX;       // FIRST: positions from here on cannot be among the query's first k
  for (int64_t base = c0; base < c1; base += kStage) {
    const int nst = c1 - base < kStage ? (int)(c1 - base) : kStage;
    if constexpr (FIRST) {
      cut = __shfl_sync(kFull, ki, k - 1);
      if (q < Q) cut = min(cut, __ldcg(fa.gpos + q));
      if (!__syncthreads_or(q < Q && base < cut)) break;  // every query has its k hits
      if (threadIdx.x < nst) {
        const int64_t i = fa.order[base + threadIdx.x];
        const bool ok = i >= 0 && i < fa.n_db;
        if (!ok) atomicOr(fa.err, 2);
        ord_s[threadIdx.x] = ok ? (int32_t)i : -1;
      }
      __syncthreads();
      for (int x = threadIdx.x; x < nst * T; x += blockDim.x) {
        const int s = x / T, i = ord_s[s];
        stage[x] = i >= 0 ? db[(int64_t)i * T + (x - s * T)] : make_float2(0.f, 0.f);
      }
    } else {
      __syncthreads();
      for (int x = threadIdx.x; x < nst * T; x += blockDim.x) stage[x] = db[base * T + x];
    }
    if (threadIdx.x < kStage) rho_s[threadIdx.x] = 0u;
    if (threadIdx.x < W) nres[threadIdx.x] = 0;
    if (threadIdx.x == 0) nA = nB = 0;
    __syncthreads();
    if (prune) {  // run centres and radii of the staged curves
      for (int x = threadIdx.x; x < nst * G; x += blockDim.x) {
        const int s = x / G, r = x % G;
        const float2* cp = stage + s * T + r * kRun;
        const int cnt = min(kRun, T - r * kRun);
        float zx = 0.f, zy = 0.f;
        for (int i = 0; i < cnt; ++i) {
          zx += cp[i].x;
          zy += cp[i].y;
        }
        zx /= (float)cnt;
        zy /= (float)cnt;
        float r2 = 0.f;
        for (int i = 0; i < cnt; ++i) {
          const float dx = cp[i].x - zx, dy = cp[i].y - zy;
          r2 = fmaxf(r2, fmaf(dy, dy, dx * dx));
        }
        cen[s * kMaxG + r] = make_float2(zx, zy);
        atomicMax(&rho_s[s], __float_as_uint(fmaf(sqrtf(r2), kLbGrow, 1e-30f)));  // radii are >= 0
      }
    }
    // A: this warp's query against the staged curves
    if (q < Q) {
      float thr;
      if constexpr (FIRST) {
        thr = fthr;
      } else {
        thr = __shfl_sync(kFull, kd, k - 1);
        if (prune) thr = fminf(thr, __ldcg(gthr + q));
      }
      if (lane == 0) thr_w[warp] = thr;
      bool keep = lane < nst;
      if constexpr (FIRST) keep = keep && base + lane < cut && ord_s[lane] >= 0;
      const bool bounded = prune && thr < INFINITY;
      float lb = 0.f;
      if (bounded && keep) {
        // the walk starts at point s mod T so that the lanes' reads spread over banks
        const float2* cp = stage + lane * T;
        int t = lane % T;
        for (int n = 0; n < T; ++n) {
          const float2 c = cp[t];
          t = t + 1 == T ? 0 : t + 1;
          const float rx = fminf(fmaxf((c.x - gp.x) * gp.w, 0.f), (float)(kNG - 1)) + kRound;
          const float ry = fminf(fmaxf((c.y - gp.y) * gp.w, 0.f), (float)(kNG - 1)) + kRound;
          const int ix = __float_as_int(rx) - __float_as_int(kRound);
          const int iy = __float_as_int(ry) - __float_as_int(kRound);
          const float dx = c.x - fmaf(rx - kRound, gp.z, gp.x), dy = c.y - fmaf(ry - kRound, gp.z, gp.y);
          const float dt = __half2float(mygrid[iy * kNG + ix]);
          const float d2 = fmaf(dy, dy, dx * dx);
          lb += fmaxf(fmaf(-d2 * rsqrt_approx(d2), kLbGrow, dt), 0.f);
        }
        lb *= invT;
        keep = !(lb > thr + (margin * thr + 1e-6f));
      }
      const unsigned m = __ballot_sync(kFull, keep);
      if (m) {
        int at = 0;
        if (lane == 0) at = atomicAdd(bounded ? &nA : &nB, __popc(m));
        at = __shfl_sync(kFull, at, 0) + __popc(m & ((1u << lane) - 1u));
        if (keep) {
          if (bounded) {
            listA[at] = (uint16_t)(warp * kStage + lane);
            lbA[at] = lb;
          } else {
            listB[at] = (uint16_t)(warp * kStage + lane);
          }
        }
      }
    }
    __syncthreads();
    f2 QX[PL / 2], QY[PL / 2];
    if (prune) {  // B: row-term bound on the survivors of A
      const int n = nA;
      for (int e = gid; e < n; e += kGroups) {
        const int w = listA[e] / kStage, s = listA[e] % kStage;
        load_query<PL>(qs + (int64_t)(qbase + w) * T, T, gl, QX, QY);
        const float lb = lbA[e] + row_bound<PL>(QX, QY, cen + s * kMaxG, G, __uint_as_float(rho_s[s]), T, gl,
                                                gmask, invT);
        const float thr = thr_w[w];
        if (gl == 0 && !(lb > thr + (margin * thr + 1e-6f))) listB[atomicAdd(&nB, 1)] = listA[e];
      }
      __syncthreads();
    }
    {  // C: exact CDs
      const int n = nB;
      for (int e = gid; e < n; e += kGroups) {
        const int w = listB[e] / kStage, s = listB[e] % kStage;
        load_query<PL>(qs + (int64_t)(qbase + w) * T, T, gl, QX, QY);
        const float thr = thr_w[w];
        if constexpr (FIRST) {
          const float d = chamfer_exact<PL>(QX, QY, stage + s * T, T, gl, gmask, invT,
                                            prune ? fthr + fband : INFINITY);
          bool hit = d < fthr - fband;
          float dd = d;
          if (!hit && !(d > fthr + fband)) {  // within the rounding band (uniform in the group)
            const double d64 = chamfer_f64(qs + (int64_t)(qbase + w) * T, stage + s * T, T, gl, gmask);
            hit = d64 < fa.thr;
            dd = (float)d64;
          }
          if (gl == 0 && hit) {
            const int at = atomicAdd(&nres[w], 1);
            res_d[w][at] = dd;
            res_s[w][at] = (uint8_t)s;
          }
        } else {
          const float d = chamfer_exact<PL>(QX, QY, stage + s * T, T, gl, gmask, invT, prune ? thr : INFINITY);
          if (gl == 0 && d <= thr) {
            const int at = atomicAdd(&nres[w], 1);
            res_d[w][at] = d;
            res_s[w][at] = (uint8_t)s;
          }
        }
      }
    }
    __syncthreads();
    if (q < Q) {
      const int n = nres[warp];
      if constexpr (FIRST) {
        for (int r = 0; r < n; ++r) first_insert(kd, ki, k, res_d[warp][r], (int)(base + res_s[warp][r]));
        if (lane == k - 1 && ki < pos_pub) {  // publish this chunk's k-th position
          atomicMin(fa.gpos + q, ki);
          pos_pub = ki;
        }
      } else {
        for (int r = 0; r < n; ++r) topk_insert(kd, ki, k, res_d[warp][r], (int)(base + res_s[warp][r]));
      }
      if (!FIRST && prune && lane == k - 1 && kd < thr_pub) {  // publish this chunk's k-th distance
        atomicMin(reinterpret_cast<unsigned*>(gthr + q), __float_as_uint(kd));  // CDs are >= 0
        thr_pub = kd;
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

// One warp per query: the first k hits in scan order from the chunks' lists (chunks
// cover increasing positions, and each list is ascending with its empty entries
// last), mapped back to database curves.
__global__ void first_merge_kernel(int Q, int nchunk, int k, const float* __restrict__ part_d,
                                   const int32_t* __restrict__ part_i, const int32_t* __restrict__ order,
                                   int32_t* __restrict__ idx, float* __restrict__ dist) {
  const int lane = threadIdx.x & 31;
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= Q) return;
  int found = 0;
  for (int c = 0; c < nchunk && found < k; ++c) {
    const int64_t o = ((int64_t)q * nchunk + c) * k + lane;
    const int pos = lane < k ? part_i[o] : INT32_MAX;
    const bool hit = pos != INT32_MAX;
    if (hit && found + lane < k) {
      idx[(int64_t)q * k + found + lane] = order[pos];
      dist[(int64_t)q * k + found + lane] = part_d[o];
    }
    found += __popc(__ballot_sync(kFull, hit));
  }
  if (lane >= found && lane < k) {
    idx[(int64_t)q * k + lane] = -1;
    dist[(int64_t)q * k + lane] = INFINITY;
  }
}

__global__ void fill_i32_kernel(int n, int32_t v, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = v;
}

template <int PL, int W, bool FIRST>
int launch_chamfer(links_ctx ctx, int Q, int64_t M, int T, const float2* qs, const float2* db, int k,
                   int32_t* idx, float* dist, int prune, FirstArgs fa) {
  const int qtiles = (Q + W - 1) / W;
  if (M == 0) {  // nothing to rank: idx = -1, dist = +inf
    KernelScope ks(ctx, "topk_merge");
    topk_merge_kernel<<<(Q * 32 + 255) / 256, 256, 0, ctx->stream>>>(Q, 0, k, nullptr, nullptr, idx, dist);
    LINKS_CUDA(cudaGetLastError());
    return LINKS_OK;
  }
  // database chunks: one CTA per SM at a time; at least four waves (sixteen for the
  // scan, whose later chunks end early once the earlier ones have found the hits),
  // the CTA count a multiple of the SM count where the chunk count allows
  const int64_t max_chunks = (M + kStage - 1) / kStage;
  const int64_t sms = ctx->num_sms;
  const int64_t waves = FIRST ? 16 : 4;
  int64_t nchunk = std::max<int64_t>(1, (waves * sms + qtiles - 1) / qtiles);
  for (int64_t c = nchunk; c <= 2 * nchunk; ++c)
    if ((c * qtiles) % sms == 0) {
      nchunk = c;
      break;
    }
  nchunk = std::min<int64_t>(std::min<int64_t>(nchunk, max_chunks), 65535);
  int64_t chunk = (M + nchunk - 1) / nchunk;
  chunk = (chunk + kStage - 1) / kStage * kStage;
  nchunk = (M + chunk - 1) / chunk;
  const size_t part_bytes = (size_t)Q * nchunk * k * (sizeof(float) + sizeof(int32_t));
  const size_t grid_off = (part_bytes + 255) / 256 * 256;
  const size_t grid_bytes = prune ? (size_t)Q * kNG * kNG * sizeof(__half) : 0;
  const size_t param_off = grid_off + grid_bytes;
  const size_t thr_off = param_off + (prune ? (size_t)Q * sizeof(float4) : 0);
  const size_t pos_off = (thr_off + (prune ? (size_t)Q * sizeof(float) : 0) + 15) / 16 * 16;
  const size_t need = pos_off + (FIRST ? (size_t)Q * sizeof(int32_t) : 0);
  int st = ensure_workspace(ctx, need);
  if (st) return st;
  char* ws = reinterpret_cast<char*>(ctx->ws);
  float* part_d = reinterpret_cast<float*>(ws);
  int32_t* part_i = reinterpret_cast<int32_t*>(part_d + (size_t)Q * nchunk * k);
  __half* grids = prune ? reinterpret_cast<__half*>(ws + grid_off) : nullptr;
  float4* gparam = prune ? reinterpret_cast<float4*>(ws + param_off) : nullptr;
  float* gthr = prune ? reinterpret_cast<float*>(ws + thr_off) : nullptr;
  if (FIRST) {
    fa.gpos = reinterpret_cast<int32_t*>(ws + pos_off);
    fa.err = ctx->d_err;
    KernelScope ks(ctx, "first_init");
    fill_i32_kernel<<<(Q + 255) / 256, 256, 0, ctx->stream>>>(Q, INT32_MAX, fa.gpos);
    LINKS_CUDA(cudaGetLastError());
  }
  if (prune) {
    KernelScope ks(ctx, "dt_grid");
    dt_grid_kernel<<<Q, 256, 0, ctx->stream>>>(Q, T, qs, grids, gparam, gthr);
    LINKS_CUDA(cudaGetLastError());
  }
  const size_t smem = (size_t)kStage * T * sizeof(float2) +
                      (prune ? (size_t)kStage * kMaxG * sizeof(float2) + (size_t)W * kNG * kNG * sizeof(__half) : 0);
  LINKS_CUDA(cudaFuncSetAttribute(chamfer_kernel<PL, W, FIRST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  {
    KernelScope ks(ctx, FIRST ? "chamfer_first" : "chamfer");
    chamfer_kernel<PL, W, FIRST><<<dim3(qtiles, (unsigned)nchunk), W * 32, smem, ctx->stream>>>(
        Q, M, T, qs, db, k, chunk, part_d, part_i, grids, gparam, gthr, fa);
  }
  LINKS_CUDA(cudaGetLastError());
  if (FIRST) {
    KernelScope ks(ctx, "first_merge");
    first_merge_kernel<<<(Q * 32 + 255) / 256, 256, 0, ctx->stream>>>(Q, (int)nchunk, k, part_d, part_i,
                                                                       fa.order, idx, dist);
  } else {
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

template <int PL>
static int launch_maxline(links_ctx ctx, int64_t M, int T, const float2* in, float2* out, int32_t* pair,
                          float* circ_var) {
  int per_sm = 0;  // resident blocks per SM: the grid is one full wave
  LINKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, maxline_kernel<PL>, 256, 0));
  const unsigned grid = (unsigned)std::min<int64_t>((M + 7) / 8, (int64_t)ctx->num_sms * std::max(per_sm, 1));
  KernelScope ks(ctx, "normalize_maxline");
  maxline_kernel<PL><<<grid, 256, 0, ctx->stream>>>(M, T, in, out, pair, circ_var);
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

int normalize_maxline(links_ctx ctx, int64_t M, int T, const float* in, float* out, int32_t* pair,
                      float* circ_var) {
  if (M == 0) return LINKS_OK;
  const float2* i2 = reinterpret_cast<const float2*>(in);
  float2* o2 = reinterpret_cast<float2*>(out);
  if (T <= 64) return launch_maxline<2>(ctx, M, T, i2, o2, pair, circ_var);
  return launch_maxline<8>(ctx, M, T, i2, o2, pair, circ_var);
}

int normalize_paths(links_ctx ctx, int64_t M, int T, const float* in, float* out) {
  return normalize_launch(ctx, M, nullptr, T, in, out);
}

int normalize_paths_count(links_ctx ctx, const int32_t* M_dev, int64_t M_cap, int T, const float* in, float* out) {
  return normalize_launch(ctx, M_cap, M_dev, T, in, out);
}

int chamfer_topk(links_ctx ctx, int Q, int64_t M, int T, const float* q, const float* db, int k, int32_t* idx,
                 float* dist, int prune) {
  if (Q == 0) return LINKS_OK;
  const float2* q2 = reinterpret_cast<const float2*>(q);
  const float2* d2 = reinterpret_cast<const float2*>(db);
  const int pl = (T + 15) / 16;  // query points per lane of a 16-lane group
  const FirstArgs fa{};
  if (pl <= 2) return launch_chamfer<2, 16, false>(ctx, Q, M, T, q2, d2, k, idx, dist, prune, fa);
  if (pl <= 4) return launch_chamfer<4, 16, false>(ctx, Q, M, T, q2, d2, k, idx, dist, prune, fa);
  if (pl <= 8) return launch_chamfer<8, 16, false>(ctx, Q, M, T, q2, d2, k, idx, dist, prune, fa);
  if (pl <= 14) return launch_chamfer<14, 16, false>(ctx, Q, M, T, q2, d2, k, idx, dist, prune, fa);
  return launch_chamfer<16, 16, false>(ctx, Q, M, T, q2, d2, k, idx, dist, prune, fa);
}

int chamfer_first_under(links_ctx ctx, int Q, int64_t M, int T, const float* q, const float* db, int64_t L,
                        const int32_t* order, double thr, int k, int32_t* idx, float* dist, int prune) {
  if (Q == 0) return LINKS_OK;
  const float2* q2 = reinterpret_cast<const float2*>(q);
  const float2* d2 = reinterpret_cast<const float2*>(db);
  FirstArgs fa;
  fa.order = order;
  fa.n_db = M;
  fa.thr = thr;
  const int pl = (T + 15) / 16;
  if (pl <= 2) return launch_chamfer<2, 16, true>(ctx, Q, L, T, q2, d2, k, idx, dist, prune, fa);
  if (pl <= 4) return launch_chamfer<4, 16, true>(ctx, Q, L, T, q2, d2, k, idx, dist, prune, fa);
  if (pl <= 8) return launch_chamfer<8, 16, true>(ctx, Q, L, T, q2, d2, k, idx, dist, prune, fa);
  if (pl <= 14) return launch_chamfer<14, 16, true>(ctx, Q, L, T, q2, d2, k, idx, dist, prune, fa);
  return launch_chamfer<16, 16, true>(ctx, Q, L, T, q2, d2, k, idx, dist, prune, fa);
}

int curate_paths(links_ctx ctx, int64_t R, int n_max, int T, const float* traj, const int32_t* row_index,
                 int64_t B, const int32_t* n_joints, const uint8_t* adj, const int8_t* type, double circle_var,
                 double keep_rate, uint64_t seed, uint8_t* flags, float* circ_var, int32_t* pair,
                 int32_t* kept_index, float* kept_paths, int64_t kept_capacity, int32_t* n_kept) {
  const int64_t total = R * n_max;
  const size_t pair_bytes = pair ? 0 : ((size_t)total * 2 * sizeof(int32_t) + 255) / 256 * 256;
  const size_t need = pair_bytes + (size_t)compact_sums_count(total) * sizeof(int32_t) + 256;
  int st = ensure_workspace(ctx, need);
  if (st) return st;
  char* ws = reinterpret_cast<char*>(ctx->ws);
  CurateArgs ca;
  ca.R = R;
  ca.n_max = n_max;
  ca.T = T;
  ca.traj = reinterpret_cast<const float2*>(traj);
  ca.row_index = row_index;
  ca.B = B;
  ca.err = ctx->d_err;
  ca.n_joints = n_joints;
  ca.adj = adj;
  ca.type = type;
  ca.circle_var = circle_var;
  ca.keep_rate = keep_rate;
  ca.seed = seed;
  ca.flags = flags;
  ca.circ_var = circ_var;
  ca.pair = pair ? pair : reinterpret_cast<int32_t*>(ws);
  int32_t* sums = reinterpret_cast<int32_t*>(ws + pair_bytes);
  if (T <= 64) return launch_curate<2>(ctx, ca, kept_index, kept_paths, kept_capacity, n_kept, sums);
  return launch_curate<8>(ctx, ca, kept_index, kept_paths, kept_capacity, n_kept, sums);
}

}  // namespace links
