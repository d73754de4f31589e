// plan.cu -- solve-order builder (graphical solver of Baecher et al. as adopted by LINKS,
// Sec. "Graphical Simulator", Fig. "solver").
//
// For each mechanism: start from the known joints (fixed + actuated), repeatedly take
// the lowest-index unknown joint with at least two known neighbours and record the
// dyad (joint, two parents); the path is found once and reused for every actuator
// position (Sec. "Graphical Simulator", last paragraph; Sec. "Computational Cost of
// Simulations").  The 1-DOF check counts links per Eq. 1 with the J-operator argument
// (Sec. "1-DOF Operator"): apart from ground-ground links and the crank, every simple
// joint owns exactly two links.
//
// The builder runs on host threads (build_one) and in CUDA kernels: the warp-flat
// builder (a lane per mechanism for the search, a lane per dyad for the geometry) and,
// for n_max <= 8 on request, a thread per mechanism (build_one).  All produce
// bit-identical plans.
#include <algorithm>
#include <thread>
#include <vector>

#include "plan_core.cuh"

namespace links {
namespace {

// Per-mechanism scratch of the builder: neighbour masks, the joint of each slot's
// dyad record (joint k, parents i, j), the slot of each joint and the position bound
// of each slot.  For n_max <= 8 it is packed into bit fields and a float array read
// by unrolled selects, so that the device thread keeps it in registers; larger
// mechanisms use plain arrays.  Only the storage differs, not the arithmetic.
template <int NJ>
struct Scratch {
  uint32_t nbv[NJ];
  int slotv[NJ], dkv[NJ], div_[NJ], djv[NJ];
  float bnd[NJ];
  LINKS_HD uint32_t nb(int a) const { return nbv[a]; }
  LINKS_HD void set_nb(int a, uint32_t m) { nbv[a] = m; }
  LINKS_HD int slot(int a) const { return slotv[a]; }
  LINKS_HD void set_slot(int a, int s) { slotv[a] = s; }
  LINKS_HD void set_dyad(int d, int k, int i, int j) {
    dkv[d] = k;
    div_[d] = i;
    djv[d] = j;
  }
  LINKS_HD int dk(int d) const { return dkv[d]; }
  LINKS_HD int di(int d) const { return div_[d]; }
  LINKS_HD int dj(int d) const { return djv[d]; }
  LINKS_HD float bound(int s) const { return bnd[s]; }
  LINKS_HD void set_bound(int s, float v) { bnd[s] = v; }
};

template <>
struct Scratch<8> {
  uint64_t nbw = 0;    // 8 bits per joint
  uint32_t slotw = 0;  // 4 bits per joint
  uint64_t dyw = 0;    // 9 bits per dyad (k, i, j: 3 bits each; at most 6 dyads)
  float bnd[8];
  LINKS_HD uint32_t nb(int a) const { return (uint32_t)(nbw >> (8 * a)) & 0xffu; }
  LINKS_HD void set_nb(int a, uint32_t m) { nbw |= (uint64_t)(m & 0xffu) << (8 * a); }
  LINKS_HD int slot(int a) const { return (int)((slotw >> (4 * a)) & 0xfu); }
  LINKS_HD void set_slot(int a, int s) { slotw |= (uint32_t)s << (4 * a); }  // set once per joint
  LINKS_HD void set_dyad(int d, int k, int i, int j) {
    dyw |= (uint64_t)(k | (i << 3) | (j << 6)) << (9 * d);
  }
  LINKS_HD int dk(int d) const { return (int)(dyw >> (9 * d)) & 7; }
  LINKS_HD int di(int d) const { return (int)(dyw >> (9 * d + 3)) & 7; }
  LINKS_HD int dj(int d) const { return (int)(dyw >> (9 * d + 6)) & 7; }
  LINKS_HD float bound(int s) const {
    float r = 0.0f;
#pragma unroll
    for (int t = 0; t < 8; ++t) r = t == s ? bnd[t] : r;
    return r;
  }
  LINKS_HD void set_bound(int s, float v) {
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (t == s) bnd[t] = v;
  }
};
template <typename PT, int NJ>
LINKS_HD int build_one(int n, int n_max, const uint8_t* adj, const int8_t* type, const PT* pos,
                       BuildOut o, int* nd_out = nullptr) {
  MechHdr h{};
  h.n = (uint8_t)(n > 0 && n <= 255 ? n : 0);
  int status = LINKS_MECH_OK;
  Scratch<NJ> S;
  uint32_t fixm = 0, simm = 0, motm = 0;
  int motor = -1, pivot = -1, nd = 0;

  if (n < 2 || n > n_max || n_max > NJ) {
    status = LINKS_MECH_BAD_SIZE;
  } else {
    for (int a = 0; a < n && status == LINKS_MECH_OK; ++a) {
      int t = type[a];
      if (t == 0) fixm |= 1u << a;
      else if (t == 1) simm |= 1u << a;
      else if (t == 2) motm |= 1u << a;
      else status = LINKS_MECH_BAD_TYPE;
    }
  }
  if (status == LINKS_MECH_OK) {
    for (int a = 0; a < n; ++a) {
      uint32_t m = 0;
      const uint8_t* row = adj + (size_t)a * n_max;
      for (int c = 0; c < n; ++c) m |= (row[c] != 0 ? 1u : 0u) << c;
      S.set_nb(a, m);
    }
    for (int a = 0; a < n && status == LINKS_MECH_OK; ++a) {
      if (S.nb(a) & (1u << a)) status = LINKS_MECH_BAD_ADJ;
      for (uint32_t m = S.nb(a); m && status == LINKS_MECH_OK; m &= m - 1)
        if (!((S.nb(ffs32(m)) >> a) & 1u)) status = LINKS_MECH_BAD_ADJ;
    }
  }
  if (status == LINKS_MECH_OK && popc32(motm) != 1) status = LINKS_MECH_NO_MOTOR;
  if (status == LINKS_MECH_OK) {
    motor = ffs32(motm);
    uint32_t pm = S.nb(motor) & fixm;
    if (!pm) status = LINKS_MECH_NO_PIVOT;
    else pivot = ffs32(pm);
  }
  if (status == LINKS_MECH_OK) {
    uint32_t known = fixm | motm, unknown = simm;
    while (unknown && status == LINKS_MECH_OK) {
      int pick = -1, cnt = 0;
      for (uint32_t u = unknown; u; u &= u - 1) {
        int a = ffs32(u);
        int c = popc32(S.nb(a) & known);
        if (c >= 2) { pick = a; cnt = c; break; }
      }
      if (pick < 0) { status = LINKS_MECH_NOT_DYAD_SOLVABLE; break; }
      if (cnt > 2) { status = LINKS_MECH_OVERCONSTRAINED; break; }
      uint32_t par = S.nb(pick) & known;
      S.set_dyad(nd, pick, ffs32(par), ffs32(par & (par - 1)));
      ++nd;
      known |= 1u << pick;
      unknown &= ~(1u << pick);
    }
  }
  if (status == LINKS_MECH_OK) {
    int e2 = 0, ff2 = 0;
    for (int a = 0; a < n; ++a) {
      e2 += popc32(S.nb(a));
      if ((fixm >> a) & 1u) ff2 += popc32(S.nb(a) & fixm);
    }
    int links_ = (e2 - ff2) / 2 - 1;  // minus the crank
    if (links_ != 2 * popc32(simm)) status = LINKS_MECH_OVERCONSTRAINED;
  }
  h.status = status;
  if (status != LINKS_MECH_OK) {
    h.nd = 0;
    *o.hdr = h;
    return status;
  }

  // Slots: fixed joints by index, then the actuated joint, then dyads in solve order.
  int nf = 0;
  for (uint32_t m = fixm; m; m &= m - 1) {
    int a = ffs32(m);
    S.set_slot(a, nf);
    o.slot_joint[nf] = (uint8_t)a;
    ++nf;
  }
  S.set_slot(motor, nf);
  o.slot_joint[nf] = (uint8_t)motor;
  for (int d = 0; d < nd; ++d) {
    S.set_slot(S.dk(d), nf + 1 + d);
    o.slot_joint[nf + 1 + d] = (uint8_t)S.dk(d);
  }
  for (int a = 0; a < n; ++a)  // every joint has a slot (fixed, actuated or dyad)
    o.pos64[S.slot(a)] = make_double2((double)pos[2 * a], (double)pos[2 * a + 1]);

  float bmax = 0.0f;
  {
    int s = 0;
    for (uint32_t m = fixm; m; m &= m - 1, ++s) {
      int a = ffs32(m);
      dw2 r = rel(pos, a, pivot);
      o.fixpos[s] = make_float4(r.x.h, r.x.l, r.y.h, r.y.l);
      const float bs = hyp_up(r.x.h, r.y.h);
      S.set_bound(s, bs);
      bmax = fmaxf(bmax, bs);
    }
  }
  dw2 u = rel(pos, motor, pivot);
  float crank = hyp_up(u.x.h, u.y.h);
  S.set_bound(nf, crank);
  bmax = fmaxf(bmax, crank);

  for (int d = 0; d < nd; ++d) {
    const int k = S.dk(d);
    const DyadGeo g = dyad_geo(pos, k, S.di(d), S.dj(d));
    const int si = S.slot(g.i), sj = S.slot(g.j), sk = nf + 1 + d;
    const float bk = dyad_bound(S.bound(si), S.bound(sj), g.r1.h, g.r2.h);
    S.set_bound(sk, bk);
    bmax = fmaxf(bmax, bk);
    o.dyad[d] = dyad_record(g, si, sj, k, sk);
  }

  h.nd = (uint8_t)nd;
  if (nd_out) *nd_out = nd;
  h.nf = (uint8_t)nf;
  h.motor_joint = (uint8_t)motor;
  h.pivot_joint = (uint8_t)pivot;
  h.pad0 = (uint8_t)S.slot(pivot);  // pivot slot
  h.coupler_slot = (uint8_t)(nd > 0 ? nf + nd : nf);
  h.ux_h = u.x.h; h.ux_l = u.x.l; h.uy_h = u.y.h; h.uy_l = u.y.l;
  dw px = abs_dw(pos, 2 * pivot), py = abs_dw(pos, 2 * pivot + 1);
  h.px_h = px.h; h.px_l = px.l; h.py_h = py.h; h.py_l = py.l;
  h.bmax = bmax;
  {  // bounding-box diagonal of the n initial positions
    float lo_x = (float)pos[0], hi_x = lo_x, lo_y = (float)pos[1], hi_y = lo_y;
    for (int a = 1; a < n; ++a) {
      float x = (float)pos[2 * a], y = (float)pos[2 * a + 1];
      lo_x = fminf(lo_x, x);
      hi_x = fmaxf(hi_x, x);
      lo_y = fminf(lo_y, y);
      hi_y = fmaxf(hi_y, y);
    }
    h.lbox = hyp_up(fsub(hi_x, lo_x), fsub(hi_y, lo_y));
  }
  h.e_motor = fmul(4.0f * kU, crank);
  h.e_fixed = fmul(kU, bmax);
  *o.hdr = h;
  return status;
}

// Inputs of the block's 256 mechanisms (n_max <= 8) staged in shared memory with
// coalesced loads: each mechanism's adjacency, type and position rows padded to an odd
// number of words, so that the threads' reads of their own rows fall in distinct banks.
constexpr int kStageRow = 17;  // words per staged adjacency / position row (<= 16 used)
constexpr int kTypeRow = 3;    // words per staged type row (<= 2 used)

template <typename PT, int NJ>
__global__ void __launch_bounds__(256) build_kernel(int64_t B, const int32_t* __restrict__ n_joints,
                                                    const uint8_t* __restrict__ adj,
                                                    const int8_t* __restrict__ type,
                                                    const PT* __restrict__ pos, PlanDev p,
                                                    int32_t* __restrict__ status_out) {
  constexpr bool kStaged = NJ <= 8;
  constexpr bool kStagedPos = kStaged && sizeof(PT) == 4;  // FP64 rows would pass 48 KB
  __shared__ int hist[32];
  __shared__ uint32_t s_adj[kStaged ? 256 * kStageRow : 1];
  __shared__ PT s_pos[kStagedPos ? 256 * kStageRow : 1];
  __shared__ uint32_t s_type[kStaged ? 256 * kTypeRow : 1];
  if (threadIdx.x < 32) hist[threadIdx.x] = 0;
  const int nm = p.n_max;
  const int64_t b0 = (int64_t)blockIdx.x * blockDim.x;
  const int t = threadIdx.x;
  const int64_t b = b0 + t;
  const uint8_t* my_adj = adj + b * nm * nm;
  const int8_t* my_type = type + b * nm;
  const PT* my_pos = pos + b * nm * 2;
  if (kStaged) {
    const int nb = B - b0 < 256 ? (int)(B - b0) : 256;
    const int nn = nm * nm;
    if ((nn & 3) == 0) {  // whole words per row, rows word-aligned
      const int wpm = nn >> 2;
      const uint32_t* src = reinterpret_cast<const uint32_t*>(adj + b0 * nn);
      for (int x = t; x < nb * wpm; x += 256) s_adj[(x / wpm) * kStageRow + x % wpm] = __ldg(src + x);
    } else {
      const uint8_t* src = adj + b0 * nn;
      uint8_t* dst = reinterpret_cast<uint8_t*>(s_adj);
      for (int x = t; x < nb * nn; x += 256) dst[(x / nn) * (4 * kStageRow) + x % nn] = __ldg(src + x);
    }
    if (kStagedPos) {
      const PT* psrc = pos + b0 * 2 * nm;
      for (int x = t; x < nb * 2 * nm; x += 256) s_pos[(x / (2 * nm)) * kStageRow + x % (2 * nm)] = __ldg(psrc + x);
      my_pos = s_pos + t * kStageRow;
    }
    const int8_t* tsrc = type + b0 * nm;
    int8_t* tdst = reinterpret_cast<int8_t*>(s_type);
    for (int x = t; x < nb * nm; x += 256) tdst[(x / nm) * (4 * kTypeRow) + x % nm] = __ldg(tsrc + x);
    my_adj = reinterpret_cast<const uint8_t*>(s_adj + t * kStageRow);
    my_type = reinterpret_cast<const int8_t*>(s_type + t * kTypeRow);
  }
  __syncthreads();
  if (b < B) {
    int n = n_joints[b];
    int nd = 0;
    int st = build_one<PT, NJ>(n, nm, my_adj, my_type, my_pos, out_of(p, b), &nd);
    if (status_out) status_out[b] = st;
    if (st == LINKS_MECH_OK) atomicAdd(&hist[nd], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32 && hist[threadIdx.x]) atomicAdd(&p.ctrs[kHist + threadIdx.x], hist[threadIdx.x]);
}

// Warp-flat builder kernel: each warp builds the 32 mechanisms from b0 = 32 x its global
// warp index (build_flat_warp in plan_core.cuh).
template <typename PT, bool STAGE>
__global__ void __launch_bounds__(32 * kFlatWarps, 8) build_flat_kernel(int64_t B, const int32_t* __restrict__ n_joints,
                                                                      const uint8_t* __restrict__ adj,
                                                                      const uint32_t* __restrict__ nbr,
                                                                      const int8_t* __restrict__ type,
                                                                      const PT* __restrict__ pos, PlanDev p,
                                                                      int32_t* __restrict__ status_out, int flags) {
  extern __shared__ __align__(16) char flat_smem[];
  __shared__ int hist[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < 32) hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t b0 = ((int64_t)blockIdx.x * kFlatWarps + warp) * 32;
  const FlatResult r = build_flat_warp<PT, true, STAGE>(
      B, b0, n_joints, adj, nbr, type, pos, p, flags, flat_smem + warp * FlatSmem<PT>::bytes(p.n_max, p.max_dyads, STAGE),
      lane);
  if (r.status >= 0) {
    if (status_out) status_out[b0 + lane] = r.status;
    if (r.status == LINKS_MECH_OK) atomicAdd(&hist[r.nd], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32 && hist[threadIdx.x]) atomicAdd(&p.ctrs[kHist + threadIdx.x], hist[threadIdx.x]);
}

// Counting sort of the OK mechanisms by dyad count (a processing order only: warps then
// meet mechanisms of equal length together).
__global__ void __launch_bounds__(256) scatter_kernel(int64_t B, PlanDev p) {
  __shared__ int off[32], cnt[32], base[32];
  if (threadIdx.x < 32) {
    int v = p.ctrs[kHist + threadIdx.x];
    int incl = v;
    for (int s = 1; s < 32; s <<= 1) {
      int o = __shfl_up_sync(0xffffffffu, incl, s);
      if ((int)threadIdx.x >= s) incl += o;
    }
    off[threadIdx.x] = incl - v;
    cnt[threadIdx.x] = 0;
  }
  __syncthreads();
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int nd = -1, rank = 0;
  if (b < B && p.hdr[b].status == LINKS_MECH_OK) {
    nd = p.hdr[b].nd;
    rank = atomicAdd(&cnt[nd], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32 && cnt[threadIdx.x]) base[threadIdx.x] = atomicAdd(&p.ctrs[kCursor + threadIdx.x], cnt[threadIdx.x]);
  __syncthreads();
  if (nd >= 0) p.order[off[nd] + base[nd] + rank] = (int32_t)b;
}

// The warp-flat builder with its positions staged in shared memory unless staging them
// would lower the resident blocks per SM (then they are read through the cache).
template <typename PT>
int launch_flat(links_ctx ctx, unsigned fgrid, int64_t B, const int32_t* n_joints, const uint8_t* adj,
                const uint32_t* nbr, const int8_t* type, const PT* ps, const PlanDev& p, int32_t* status_out,
                int flags) {
  const size_t sm1 = kFlatWarps * FlatSmem<PT>::bytes(p.n_max, p.max_dyads, true);
  const size_t sm0 = kFlatWarps * FlatSmem<PT>::bytes(p.n_max, p.max_dyads, false);
  LINKS_CUDA(cudaFuncSetAttribute(build_flat_kernel<PT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
  LINKS_CUDA(cudaFuncSetAttribute(build_flat_kernel<PT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0));
  int occ1 = 0, occ0 = 0;
  LINKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, build_flat_kernel<PT, true>, 32 * kFlatWarps, sm1));
  LINKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, build_flat_kernel<PT, false>, 32 * kFlatWarps, sm0));
  if (occ1 >= occ0)
    build_flat_kernel<PT, true><<<fgrid, 32 * kFlatWarps, sm1, ctx->stream>>>(B, n_joints, adj, nbr, type, ps, p,
                                                                             status_out, flags);
  else
    build_flat_kernel<PT, false><<<fgrid, 32 * kFlatWarps, sm0, ctx->stream>>>(B, n_joints, adj, nbr, type, ps, p,
                                                                              status_out, flags);
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

}  // namespace

int plan_one_host(int n, int n_max, const uint8_t* adj, const int8_t* type, const double* pos, MechHdr* hdr,
                  DyadRec* dyad) {
  std::vector<uint8_t> sj(kMaxJ);
  std::vector<float4> fix(std::max(n_max, 1));
  std::vector<double2> p64(std::max(n_max, 1));
  BuildOut o{hdr, sj.data(), fix.data(), p64.data(), dyad};
  return build_one<double, kMaxJ>(n, n_max, adj, type, pos, o);
}

int plan_build_device(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                      const uint8_t* adj, const int8_t* type, const void* pos0, int pos_dtype,
                      int32_t* status_out, const uint32_t* nbr) {
  PlanDev& p = plan->d;
  LINKS_CUDA(cudaMemsetAsync(p.ctrs, 0, kCtrs * sizeof(int32_t), ctx->stream));
  plan->B = B;
  if (B == 0) return LINKS_OK;
  unsigned grid = (unsigned)((B + 255) / 256);
  {
    KernelScope ks(ctx, "plan_build");
    // the warp-flat builder (a lane per mechanism for the search, a lane per dyad for the
    // geometry; measured faster at every n_max), or on request for n_max <= 8 a thread
    // per mechanism with its scratch in registers
    const int builder = tuning_of(ctx, p.n_max).builder;
    const bool small = p.n_max <= 8 && builder == 1 && !nbr;
    const bool vec = ((uintptr_t)pos0 & 15u) == 0 && ((uintptr_t)type & 15u) == 0 &&
                     (pos_dtype == LINKS_F64 || p.n_max % 2 == 0);
    const int flags = ((p.n_max % 4 == 0 && ((uintptr_t)adj & 3u) == 0) ? 1 : 0) | (vec ? 2 : 0);
    const unsigned fgrid = (unsigned)((B + 32 * kFlatWarps - 1) / (32 * kFlatWarps));
    if (pos_dtype == LINKS_F32) {
      const float* ps = (const float*)pos0;
      if (small) {
        build_kernel<float, 8><<<grid, 256, 0, ctx->stream>>>(B, n_joints, adj, type, ps, p, status_out);
      } else {
        int st = launch_flat<float>(ctx, fgrid, B, n_joints, adj, nbr, type, ps, p, status_out, flags);
        if (st) return st;
      }
    } else {
      const double* ps = (const double*)pos0;
      if (small) {
        build_kernel<double, 8><<<grid, 256, 0, ctx->stream>>>(B, n_joints, adj, type, ps, p, status_out);
      } else {
        int st = launch_flat<double>(ctx, fgrid, B, n_joints, adj, nbr, type, ps, p, status_out, flags);
        if (st) return st;
      }
    }
  }
  LINKS_CUDA(cudaGetLastError());
  {
    KernelScope ks(ctx, "plan_sort");
    scatter_kernel<<<grid, 256, 0, ctx->stream>>>(B, p);
  }
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

int plan_build_host(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                    const uint8_t* adj, const int8_t* type, const void* pos0, int pos_dtype,
                    int32_t* status_out) {
  PlanDev& p = plan->d;
  const int nm = p.n_max;
  std::vector<MechHdr> hdr(B);
  std::vector<uint8_t> sj((size_t)B * kMaxJ, 0);
  std::vector<float4> fix((size_t)B * nm, make_float4(0, 0, 0, 0));
  std::vector<double2> p64((size_t)B * nm, make_double2(0, 0));
  std::vector<DyadRec> dy((size_t)B * p.max_dyads, DyadRec{});
  unsigned nth = std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
  std::vector<std::thread> pool;
  auto work = [&](int64_t lo, int64_t hi) {
    for (int64_t b = lo; b < hi; ++b) {
      BuildOut o{&hdr[b], &sj[b * kMaxJ], &fix[b * nm], &p64[b * nm], &dy[b * p.max_dyads]};
      const int n = n_joints[b];
      const uint8_t* a = adj + b * nm * nm;
      const int8_t* t = type + b * nm;
      int st;
      if (pos_dtype == LINKS_F32) {
        const float* ps = (const float*)pos0 + b * nm * 2;
        st = nm <= 8 ? build_one<float, 8>(n, nm, a, t, ps, o) : build_one<float, kMaxJ>(n, nm, a, t, ps, o);
      } else {
        const double* ps = (const double*)pos0 + b * nm * 2;
        st = nm <= 8 ? build_one<double, 8>(n, nm, a, t, ps, o) : build_one<double, kMaxJ>(n, nm, a, t, ps, o);
      }
      if (status_out) status_out[b] = st;
    }
  };
  int64_t chunk = (B + nth - 1) / nth;
  for (unsigned t = 0; t < nth; ++t) {
    int64_t lo = t * chunk, hi = std::min<int64_t>(B, lo + chunk);
    if (lo < hi) pool.emplace_back(work, lo, hi);
  }
  for (auto& th : pool) th.join();
  // Counting sort by dyad count (same property as the device scatter).
  std::vector<int32_t> ctrs(kCtrs, 0), order;
  for (int64_t b = 0; b < B; ++b)
    if (hdr[b].status == LINKS_MECH_OK) ctrs[kHist + hdr[b].nd]++;
  std::vector<int32_t> off(33, 0);
  for (int i = 0; i < 32; ++i) off[i + 1] = off[i] + ctrs[kHist + i];
  order.resize(off[32]);
  std::vector<int32_t> cur(off.begin(), off.begin() + 32);
  for (int64_t b = 0; b < B; ++b)
    if (hdr[b].status == LINKS_MECH_OK) order[cur[hdr[b].nd]++] = (int32_t)b;
  for (int i = 0; i < 32; ++i) ctrs[kCursor + i] = ctrs[kHist + i];
  cudaStream_t s = ctx->stream;
  plan->B = B;
  if (B > 0) {
    LINKS_CUDA(cudaMemcpyAsync(p.hdr, hdr.data(), B * sizeof(MechHdr), cudaMemcpyHostToDevice, s));
    LINKS_CUDA(cudaMemcpyAsync(p.slot_joint, sj.data(), sj.size(), cudaMemcpyHostToDevice, s));
    LINKS_CUDA(cudaMemcpyAsync(p.fixpos, fix.data(), fix.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    LINKS_CUDA(cudaMemcpyAsync(p.pos64, p64.data(), p64.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    LINKS_CUDA(cudaMemcpyAsync(p.dyad, dy.data(), dy.size() * sizeof(DyadRec), cudaMemcpyHostToDevice, s));
    if (!order.empty())
      LINKS_CUDA(cudaMemcpyAsync(p.order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  }
  LINKS_CUDA(cudaMemcpyAsync(p.ctrs, ctrs.data(), kCtrs * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  LINKS_CUDA(cudaStreamSynchronize(s));
  return LINKS_OK;
}

}  // namespace links
