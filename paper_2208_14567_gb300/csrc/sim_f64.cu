// sim_f64.cu -- plain FP64 simulation (LINKS_PLAIN_F64) and the kernels shared by both
// precisions (flags of unsimulated mechanisms, compaction of valid rows).
//
// The plain kernel is the straightforward GPU form of the method: one thread per
// mechanism, absolute FP64 coordinates, steps in order, stop at the first lock.
// Per step t the crank is rotated by 2*pi*t/T about its pivot; each dyad (Sec.
// "Graphical Simulator") with d^2 = |p_j - p_i|^2, e = d^2 + r1^2 - r2^2 and
// D = 4 d^2 r1^2 - e^2 places p_k = p_i + (e (p_j - p_i) + sqrt(D) (p_j - p_i)^perp) / (2 d^2)
// on the branch of the initial configuration (the plan orders each dyad's parents
// so that this is the "+" branch); D <= 0 is a lock (Sec. "Finding Valid Initial
// Positions", Infeasibility rule).
#include <algorithm>

#include "links_internal.cuh"

namespace links {
namespace {

constexpr int kBlock = 128;

__device__ __forceinline__ double2 nan2() {
  double n = __longlong_as_double(0x7ff8000000000000ll);
  return make_double2(n, n);
}

// mode 0: flags (+ FULL traj/path rows = mechanism index) for all B mechanisms
// mode 1: flags only
// mode 2: rows of valid mechanisms (out_index), traj/path only
// mode 2 with row_off: packed rows, row r's joints at traj rows row_off[r] + j (the
// row is left out when it does not fit in traj_cap joint rows), no padding joints
__global__ void __launch_bounds__(kBlock) f64_kernel(PlanDev p, int64_t B, int T, const double2* __restrict__ cs,
                                                     int mode, double* __restrict__ traj, double* __restrict__ path,
                                                     uint8_t* __restrict__ valid, int16_t* __restrict__ lock_step,
                                                     float* __restrict__ min_disc,
                                                     const int32_t* __restrict__ out_index, int64_t out_capacity,
                                                     int32_t* err, const int64_t* __restrict__ row_off,
                                                     int64_t traj_cap) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = mode == 2 ? min((int64_t)p.ctrs[kNValid], out_capacity) : B;
  if (r >= rows) return;
  const int64_t b = mode == 2 ? (int64_t)out_index[r] : r;
  if (b < 0 || b >= B) {
    atomicOr(err, kErrBadIndex);
    return;
  }
  const int ns = p.n_max;
  const MechHdr h = p.hdr[b];
  const bool write = mode != 1 && (traj || path);
  double2* trow = nullptr;
  if (traj) {
    if (!row_off) trow = reinterpret_cast<double2*>(traj) + r * ns * T;
    else if (row_off[r] >= 0 && row_off[r] + h.n <= traj_cap) trow = reinterpret_cast<double2*>(traj) + row_off[r] * T;
  }
  double2* prow = path ? reinterpret_cast<double2*>(path) + r * T : nullptr;
  if (h.status != LINKS_MECH_OK) {  // only reached in mode 0
    if (write) {
      for (int64_t x = 0; trow && x < (int64_t)ns * T; ++x) trow[x] = nan2();
      for (int t = 0; prow && t < T; ++t) prow[t] = nan2();
    }
    return;
  }
  const int n = h.n, nf = h.nf, nd = h.nd;
  const uint8_t* sj = p.slot_joint + b * kMaxJ;
  const double2* p0 = p.pos64 + b * ns;
  const DyadRec* dy = p.dyad + b * p.max_dyads;
  double2 pos[kMaxJ];
  double r1s[kMaxJ], r2s[kMaxJ];
  int si[kMaxJ], sjx[kMaxJ];
  for (int s = 0; s < n; ++s) pos[s] = p0[s];
  for (int d = 0; d < nd; ++d) {
    uint32_t sl = __float_as_uint(__ldg(&dy[d].r2.w));
    si[d] = sl & 0xff;
    sjx[d] = (sl >> 8) & 0xff;
    const int k = nf + 1 + d;
    double ax = p0[k].x - p0[si[d]].x, ay = p0[k].y - p0[si[d]].y;
    double bx = p0[k].x - p0[sjx[d]].x, by = p0[k].y - p0[sjx[d]].y;
    r1s[d] = ax * ax + ay * ay;
    r2s[d] = bx * bx + by * by;
  }
  const double2 pv = p0[h.pad0];
  const double ux = p0[nf].x - pv.x, uy = p0[nf].y - pv.y;
  if (write && trow && !row_off)
    for (int j = n; j < ns; ++j)
      for (int t = 0; t < T; ++t) trow[(int64_t)j * T + t] = nan2();
  int lock = -1;
  double qmin = INFINITY;
  for (int t = 0; t < T; ++t) {
    const double2 c = cs[t];
    pos[nf] = make_double2(pv.x + (c.x * ux - c.y * uy), pv.y + (c.y * ux + c.x * uy));
    double qstep = INFINITY;
    bool locked = false;
    for (int d = 0; d < nd; ++d) {
      const double2 pi = pos[si[d]], pj = pos[sjx[d]];
      const double dx = pj.x - pi.x, dy_ = pj.y - pi.y;
      const double d2 = dx * dx + dy_ * dy_;
      const double e = d2 + r1s[d] - r2s[d];
      const double D = 4.0 * d2 * r1s[d] - e * e;
      const double q = D / (4.0 * r1s[d] * r2s[d]);
      if (!(q > 0.0)) { locked = true; break; }
      qstep = fmin(qstep, q);
      const double sq = sqrt(D);
      const double inv = 1.0 / (2.0 * d2);
      pos[nf + 1 + d] = make_double2(pi.x + (e * dx - sq * dy_) * inv, pi.y + (e * dy_ + sq * dx) * inv);
    }
    if (locked) {
      lock = t;
      break;
    }
    qmin = fmin(qmin, qstep);
    if (write) {
      if (trow)
        for (int s = 0; s < n; ++s) trow[(int64_t)sj[s] * T + t] = pos[s];
      if (prow) prow[t] = pos[h.coupler_slot];
    }
  }
  if (write && lock >= 0) {
    if (mode == 2) atomicOr(err, kErrEmitLock);
    for (int t = lock; t < T; ++t) {
      if (trow)
        for (int s = 0; s < n; ++s) trow[(int64_t)sj[s] * T + t] = nan2();
      if (prow) prow[t] = nan2();
    }
  }
  if (mode != 2) {
    valid[b] = lock < 0;
    lock_step[b] = (int16_t)lock;
    min_disc[b] = (float)qmin;
  }
}

__global__ void fill_kernel(PlanDev p, int64_t B, uint8_t* valid, int16_t* lock_step, float* min_disc) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || p.hdr[b].status == LINKS_MECH_OK) return;
  valid[b] = 0;
  lock_step[b] = -2;
  min_disc[b] = __int_as_float(0x7fc00000);
}

// Valid-row compaction: exclusive scan of valid[] in three passes over blocks of 1024.
constexpr int kScanBlock = 1024;

__device__ int block_excl_scan(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  int excl = x - v + (w ? ws[w - 1] : 0);
  if (total) *total = ws[31];
  __syncthreads();
  return excl;
}

__global__ void __launch_bounds__(kScanBlock) scan_count(int64_t B, const uint8_t* valid, int32_t* sums) {
  int64_t b = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int v = (b < B && valid[b]) ? 1 : 0;
  int tot;
  block_excl_scan(v, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) scan_top(int nblk, int32_t* sums, int32_t* ctrs, int32_t* n_out) {
  // sums[0..nblk) -> exclusive offsets, in rounds of 1024
  int carry = 0;
  for (int base = 0; base < nblk; base += kScanBlock) {
    int i = base + threadIdx.x;
    int v = i < nblk ? sums[i] : 0;
    int tot;
    int ex = block_excl_scan(v, &tot);
    if (i < nblk) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    ctrs[kNValid] = carry;
    if (n_out) *n_out = carry;
  }
}

__global__ void __launch_bounds__(kScanBlock) scan_write(int64_t B, const uint8_t* valid, const int32_t* sums,
                                                         int32_t* out_index, int64_t cap) {
  int64_t b = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int v = (b < B && valid[b]) ? 1 : 0;
  int ex = block_excl_scan(v, nullptr) + sums[blockIdx.x];
  if (v && ex < cap && out_index) out_index[ex] = (int32_t)b;
}

// Packed rows: the exclusive prefix of the rows' joint counts, in the same three passes
// over blocks of 1024 rows (rows = min(valid count, capacity), known on the device).
__device__ __forceinline__ int row_joints(const PlanDev& p, int64_t B, const int32_t* out_index, int64_t r,
                                          int64_t rows) {
  if (r >= rows) return 0;
  const int64_t b = out_index[r];
  return b >= 0 && b < B ? (int)p.hdr[b].n : 0;
}

__global__ void __launch_bounds__(kScanBlock) pack_count(PlanDev p, int64_t B, const int32_t* out_index,
                                                         int64_t cap, int64_t* sums) {
  const int64_t rows = min((int64_t)p.ctrs[kNValid], cap);
  const int v = row_joints(p, B, out_index, (int64_t)blockIdx.x * kScanBlock + threadIdx.x, rows);
  int tot;
  block_excl_scan(v, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) pack_top(PlanDev p, int nblk, int64_t cap, int64_t* sums,
                                                       int64_t* row_offset) {
  int64_t carry = 0;
  for (int base = 0; base < nblk; base += kScanBlock) {  // a round sums <= 1024 * 32 * 1024 joints
    const int i = base + threadIdx.x;
    const int v = i < nblk ? (int)sums[i] : 0;
    int tot;
    const int ex = block_excl_scan(v, &tot);
    if (i < nblk) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) row_offset[min((int64_t)p.ctrs[kNValid], cap)] = carry;
}

__global__ void __launch_bounds__(kScanBlock) pack_write(PlanDev p, int64_t B, const int32_t* out_index,
                                                         int64_t cap, const int64_t* sums, int64_t* row_offset) {
  const int64_t rows = min((int64_t)p.ctrs[kNValid], cap);
  const int64_t r = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const int v = row_joints(p, B, out_index, r, rows);
  const int ex = block_excl_scan(v, nullptr);
  if (r < rows) row_offset[r] = sums[blockIdx.x] + ex;
}

}  // namespace

int fill_unsimulated(links_ctx ctx, links_plan plan, uint8_t* valid, int16_t* lock_step, float* min_disc) {
  const int64_t B = plan->B;
  if (B == 0) return LINKS_OK;
  KernelScope ks(ctx, "fill_unsimulated");
  fill_kernel<<<(unsigned)((B + 255) / 256), 256, 0, ctx->stream>>>(plan->d, B, valid, lock_step, min_disc);
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

int compact_valid(links_ctx ctx, links_plan plan, const uint8_t* valid, int32_t* out_index,
                  int64_t out_capacity, int32_t* n_out) {
  const int64_t B = plan->B;
  const int nblk = (int)((B + kScanBlock - 1) / kScanBlock);
  if (nblk > 0) {
    KernelScope ks(ctx, "scan_count");
    scan_count<<<nblk, kScanBlock, 0, ctx->stream>>>(B, valid, plan->d.scan);
  }
  LINKS_CUDA(cudaGetLastError());
  {
    KernelScope ks(ctx, "scan_top");
    scan_top<<<1, kScanBlock, 0, ctx->stream>>>(nblk, plan->d.scan, plan->d.ctrs, n_out);
  }
  LINKS_CUDA(cudaGetLastError());
  if (nblk > 0) {
    KernelScope ks(ctx, "scan_write");
    scan_write<<<nblk, kScanBlock, 0, ctx->stream>>>(B, valid, plan->d.scan, out_index, out_capacity);
  }
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

int pack_offsets(links_ctx ctx, links_plan plan, const int32_t* out_index, int64_t out_capacity,
                 int64_t* row_offset) {
  const int64_t B = plan->B;
  const int64_t rmax = std::min<int64_t>(B, out_capacity);
  const int nblk = (int)((rmax + kScanBlock - 1) / kScanBlock);
  if (nblk > 0) {
    KernelScope ks(ctx, "pack_count");
    pack_count<<<nblk, kScanBlock, 0, ctx->stream>>>(plan->d, B, out_index, out_capacity, plan->d.scan64);
  }
  LINKS_CUDA(cudaGetLastError());
  {
    KernelScope ks(ctx, "pack_top");
    pack_top<<<1, kScanBlock, 0, ctx->stream>>>(plan->d, nblk, out_capacity, plan->d.scan64, row_offset);
  }
  LINKS_CUDA(cudaGetLastError());
  if (nblk > 0) {
    KernelScope ks(ctx, "pack_write");
    pack_write<<<nblk, kScanBlock, 0, ctx->stream>>>(plan->d, B, out_index, out_capacity, plan->d.scan64,
                                                     row_offset);
  }
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

int simulate_f64(links_ctx ctx, links_plan plan, const TTable* tab, int out_mode, double* traj,
                 double* path, uint8_t* valid, int16_t* lock_step, float* min_disc,
                 int32_t* out_index, int64_t out_capacity, int32_t* n_out, int64_t* row_offset,
                 int64_t traj_capacity) {
  const int64_t B = plan->B;
  const int T = tab->T;
  const bool full = out_mode == LINKS_OUT_FULL;
  int st0 = fill_unsimulated(ctx, plan, valid, lock_step, min_disc);
  if (st0) return st0;
  if (B > 0) {
    KernelScope ks(ctx, "f64_sim");
    f64_kernel<<<(unsigned)((B + kBlock - 1) / kBlock), kBlock, 0, ctx->stream>>>(
        plan->d, B, T, tab->cs64, full ? 0 : 1, traj, path, valid, lock_step, min_disc, nullptr, 0, ctx->d_err,
        nullptr, 0);
    LINKS_CUDA(cudaGetLastError());
  }
  if (!full) {
    int st = compact_valid(ctx, plan, valid, out_index, out_capacity, n_out);
    if (st) return st;
    if (row_offset) {
      st = pack_offsets(ctx, plan, out_index, out_capacity, row_offset);
      if (st) return st;
    }
    if ((traj || path) && out_capacity > 0) {
      int64_t rows = std::min<int64_t>(B, out_capacity);
      if (rows > 0) {
        KernelScope ks(ctx, "f64_emit");
        f64_kernel<<<(unsigned)((rows + kBlock - 1) / kBlock), kBlock, 0, ctx->stream>>>(
            plan->d, B, T, tab->cs64, 2, traj, path, valid, lock_step, min_disc, out_index, out_capacity,
            ctx->d_err, row_offset, traj_capacity);
        LINKS_CUDA(cudaGetLastError());
      }
    }
  }
  return LINKS_OK;
}

}  // namespace links
