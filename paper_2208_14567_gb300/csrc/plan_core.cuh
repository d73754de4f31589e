// plan_core.cuh -- the device parts of the solve-order builder (graphical solver of
// Baecher et al. as adopted by LINKS, Sec. "Graphical Simulator", Fig. "solver"): the
// per-dyad geometry shared by every builder, and the warp-flat builder's body that
// plan.cu's kernel and the serving loop's persistent kernel run.  Each including
// translation unit gets its own copy.
#pragma once

#include "links_internal.cuh"

namespace links {
namespace {


struct BuildOut {
  MechHdr* hdr;
  uint8_t* slot_joint;
  float4* fixpos;
  double2* pos64;
  DyadRec* dyad;
};

struct dw2 {
  dw x, y;
};

LINKS_HD int popc32(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __popc(v);
#else
  return __builtin_popcount(v);
#endif
}
LINKS_HD int ffs32(uint32_t v) {  // index of the lowest set bit, v != 0
#if defined(__CUDA_ARCH__)
  return __ffs(v) - 1;
#else
  return __builtin_ctz(v);
#endif
}

// p_a - p_b as a double-word pair: exact for float inputs, ~2^-48 relative for double.
LINKS_HD dw2 rel(const float* pos, int a, int b) {
  return {two_sum(pos[2 * a], -pos[2 * b]), two_sum(pos[2 * a + 1], -pos[2 * b + 1])};
}
LINKS_HD dw2 rel(const double* pos, int a, int b) {
  return {dw_from_double(pos[2 * a] - pos[2 * b]), dw_from_double(pos[2 * a + 1] - pos[2 * b + 1])};
}
LINKS_HD dw abs_dw(const float* pos, int c) { return dw_make(pos[c]); }
LINKS_HD dw abs_dw(const double* pos, int c) { return dw_from_double(pos[c]); }
LINKS_HD dw norm2(dw2 v) { return dw_add(dw_sqr(v.x), dw_sqr(v.y)); }

LINKS_HD float u2f(uint32_t u) {
  union { uint32_t u; float f; } cv;
  cv.u = u;
  return cv.f;
}
// |(x, y)| rounded up a little (a bound, identical on host and device).
LINKS_HD float hyp_up(float x, float y) {
  return fmul(fsqrt_rn(fadd(fmul(x, x), fmul(y, y))), 1.0f + 4.0f * kU);
}

// Geometry of dyad (k; i, j) from the initial positions: the parents ordered so that the
// initial branch is the "+" one, (p_j - p_i) x (p_k - p_i) >= 0, and the double-word
// link lengths.  Every builder computes a dyad through these helpers, so their plans
// agree to the bit.
struct DyadGeo {
  int i, j;
  dw r1sq, r1, r2, R12, Rm, c;
};

template <typename PT>
LINKS_HD DyadGeo dyad_geo(const PT* pos, int k, int i, int j) {
  dw2 a = rel(pos, j, i), vi = rel(pos, k, i), vj = rel(pos, k, j);
  dw cross = dw_sub(dw_mul(a.x, vi.y), dw_mul(a.y, vi.x));
  if (dw_sign(cross) < 0.0f) {  // keep the initial branch as the "+" one
    int t = i; i = j; j = t;
    dw2 tv = vi; vi = vj; vj = tv;
  }
  DyadGeo g;
  g.i = i;
  g.j = j;
  g.r1sq = norm2(vi);
  const dw r2sq = norm2(vj);
  g.r1 = dw_sqrt_exact(g.r1sq);
  g.r2 = dw_sqrt_exact(r2sq);
  g.R12 = dw_add(g.r1, g.r2);
  dw Rm = dw_sub(g.r1, g.r2);
  if (dw_sign(Rm) < 0.0f) Rm = dw_neg(Rm);
  g.Rm = Rm;
  g.c = dw_sub(g.r1sq, r2sq);
  return g;
}

// The dyad's record for slots si, sj (parents), sk (the joint k solved).  Byte offsets
// into a lane's slot arrays of the screen: positions 256 B per slot, bounds 128 B.
LINKS_HD DyadRec dyad_record(const DyadGeo& g, int si, int sj, int k, int sk) {
  const uint32_t slots = (uint32_t)si | ((uint32_t)sj << 8) | ((uint32_t)k << 16) | ((uint32_t)sk << 24);
  const uint32_t offPij = ((uint32_t)si * 256u) | (((uint32_t)sj * 256u) << 16);
  const uint32_t offK = ((uint32_t)sk * 256u) | (((uint32_t)sk * 128u) << 16);
  const uint32_t offEij = ((uint32_t)si * 128u) | (((uint32_t)sj * 128u) << 16);
  DyadRec rec;
  rec.r0 = make_float4(u2f(offPij), g.R12.h, g.Rm.h, g.c.h);
  rec.r1 = make_float4(fmul(fadd(g.r1.h, g.r1.h), g.r2.h), fmul(kAmpErr * kU, g.R12.h), u2f(offK), u2f(offEij));
  rec.r2 = make_float4(g.r1sq.h, g.r1sq.l, g.c.l, u2f(slots));
  return rec;
}

// Bound of |p_k - pivot| during the turn from the parents' bounds and the link lengths.
LINKS_HD float dyad_bound(float bi, float bj, float r1h, float r2h) {
  return fmul(fminf(fadd(bi, r1h), fadd(bj, r2h)), 1.0f + 4.0f * kU);
}

LINKS_HD BuildOut out_of(const PlanDev& p, int64_t b) {
  BuildOut o;
  o.hdr = p.hdr + b;
  o.slot_joint = p.slot_joint + b * kMaxJ;
  o.fixpos = p.fixpos + b * p.n_max;
  o.pos64 = p.pos64 + b * p.n_max;
  o.dyad = p.dyad + b * p.max_dyads;
  return o;
}


// ---------------------------------------------------------------------------------------
// Warp-flat builder: each warp builds 32 mechanisms.  The lanes first stage the warp's
// neighbour masks (given as masks, or a lane per adjacency row, word loads issued in
// batches), joint types
// and (with STAGE) initial positions (vector loads) in shared memory; without STAGE the
// positions are sent to L2 and the later phases read them through the cache, which
// halves the warp's shared memory where staged positions would limit the resident warps
// (n_max 20: 11 KB per warp, 20 warps per SM, against 32 unstaged); then lane m runs mechanism m's
// checks, solve-order search and slot assignment (the decisions of build_one, on bit
// masks); then the warp computes the geometry of all its mechanisms' dyads as one flat
// list, a dyad per lane, so that mechanisms of different sizes keep every lane busy;
// finally lane m runs its mechanism's bound chain and writes the header and the FP64
// positions.  Each value is the same expression on the same operands as in build_one.
// ---------------------------------------------------------------------------------------
constexpr int kFlatWarps = 4;  // warps per block

// One warp's shared memory, per-mechanism arrays column-major ([e * 32 + m]) unless noted.
template <typename PT>
struct FlatSmem {
  PT* pos;        // [32][2 NM + 1]  initial positions, odd row stride (row-major; with staging)
  uint32_t* nb;   // [NM]            neighbour masks; after the search, the slot bounds (float)
  int* pfx;       // [33]            exclusive prefix of the dyad counts
  uint8_t* type;  // [32][NM]        joint types as stored in global memory (row-major)
  uint8_t* slot;  // [NM]            slot of each joint
  uint8_t* dk;    // [MD]            dyad d: the joint solved ...
  uint8_t* di;    // [MD]            ... and its parents; after the geometry pass, the
  uint8_t* dj;    // [MD]                parents' slots in branch order
  uint8_t* nfv;   // [32]            fixed joints of each mechanism
  __host__ __device__ static size_t pos_bytes(int NM) {
    return (sizeof(PT) * 32 * (2 * NM + 1) + 15) & ~size_t(15);
  }
  __host__ __device__ static size_t type_bytes(int NM) { return (32 * (size_t)NM + 15) & ~size_t(15); }
  __host__ __device__ static size_t bytes(int NM, int MD, bool stage) {
    const size_t b = (stage ? pos_bytes(NM) : 0) + type_bytes(NM) + 4 * 32 * NM + 4 * 36 + 32 * NM + 3 * 32 * MD + 32;
    return (b + 15) & ~size_t(15);
  }
  __device__ FlatSmem(char* base, int NM, int MD, bool stage) {
    size_t o = 0;
    pos = stage ? reinterpret_cast<PT*>(base) : nullptr;
    o += stage ? pos_bytes(NM) : 0;
    type = reinterpret_cast<uint8_t*>(base + o);
    o += type_bytes(NM);
    nb = reinterpret_cast<uint32_t*>(base + o);
    o += 4 * 32 * NM;
    pfx = reinterpret_cast<int*>(base + o);
    o += 4 * 36;
    slot = reinterpret_cast<uint8_t*>(base + o);
    o += 32 * NM;
    dk = reinterpret_cast<uint8_t*>(base + o);
    o += 32 * MD;
    di = reinterpret_cast<uint8_t*>(base + o);
    o += 32 * MD;
    dj = reinterpret_cast<uint8_t*>(base + o);
    o += 32 * MD;
    nfv = reinterpret_cast<uint8_t*>(base + o);
  }
};

template <typename PT>
struct Vec16;  // 16-byte vector of positions
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int kN = 4;
  __device__ static void put(float* d, const float4& v) { d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w; }
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int kN = 2;
  __device__ static void put(double* d, const double2& v) { d[0] = v.x; d[1] = v.y; }
};

// flags: bit 0 the adjacency rows are 4-byte aligned whole words (n_max % 4 == 0 and an
// aligned base); bit 1 positions and types are read as 16-byte vectors (aligned bases, and
// position rows of whole vectors).
// The per-lane outcome of build_flat_warp: the mechanism's status (-1 when the lane has
// no mechanism) and its dyad count.
struct FlatResult {
  int status, nd;
};

template <typename PT, bool NC = true, bool STAGE = true>
__device__ __forceinline__ FlatResult build_flat_warp(int64_t B, int64_t b0, const int32_t* __restrict__ n_joints,
                                                      const uint8_t* __restrict__ adj,
                                                      const uint32_t* __restrict__ nbr,
                                                      const int8_t* __restrict__ type, const PT* __restrict__ pos,
                                                      const PlanDev& p, int flags, char* wsmem, int lane) {
  const int NM = p.n_max, MD = p.max_dyads;
  FlatSmem<PT> S(wsmem, NM, MD, STAGE);
  const int mc = b0 < B ? (int)min((int64_t)32, B - b0) : 0;
  const int prow = 2 * NM + 1;
  const int m = lane;
  const int64_t b = b0 + m;
  const int n = m < mc ? ldro<NC>(n_joints + b) : 0;
  // coordinate x of mechanism mm's initial positions
  const auto posv = [&](int mm, int x) -> PT {
    if constexpr (STAGE) return S.pos[mm * prow + x];
    else return ldro<NC>(pos + (b0 + mm) * 2 * NM + x);
  };

  // 1. staging
  const int nrows = mc * NM;
  if (nbr) {  // neighbour masks given: one coalesced word per (mechanism, joint)
    const uint32_t* src = nbr + b0 * NM;
    for (int r = lane; r < nrows; r += 32) {
      const int mm = r / NM;
      S.nb[(r - mm * NM) * 32 + mm] = ldro<NC>(src + r);
    }
  } else if (flags & 1) {  // neighbour masks from whole words, two rows per lane in flight
    const int W = NM >> 2;
    const uint8_t* blk = adj + b0 * NM * NM;
    for (int r0 = 0; r0 < nrows; r0 += 64) {
      uint32_t wv[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = r0 + h * 32 + lane;
        const uint32_t* w = reinterpret_cast<const uint32_t*>(blk + (int64_t)r * NM);
#pragma unroll
        for (int q = 0; q < 8; ++q) wv[h][q] = (r < nrows && q < W) ? ldro<NC>(w + q) : 0u;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = r0 + h * 32 + lane;
        if (r < nrows) {
          uint32_t mask = 0;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            // one bit per nonzero byte: the four bits land on bits 21..24 of the product
            const uint32_t v = __vcmpne4(wv[h][q], 0u) & 0x01010101u;
            mask |= ((v * 0x00204081u) >> 21 & 0xfu) << (4 * q);
          }
          const int mm = r / NM;
          S.nb[(r - mm * NM) * 32 + mm] = mask;
        }
      }
    }
  } else {
    for (int r = lane; r < nrows; r += 32) {
      const uint8_t* row = adj + (b0 * NM + r) * NM;
      uint32_t mask = 0;
      for (int c = 0; c < NM; ++c) mask |= (ldro<NC>(row + c) != 0 ? 1u : 0u) << c;
      const int mm = r / NM;
      S.nb[(r - mm * NM) * 32 + mm] = mask;
    }
  }
  if constexpr (!STAGE) {  // the warp's positions on their way to L2
    const char* pb = reinterpret_cast<const char*>(pos + b0 * 2 * NM);
    const int nbytes = mc * 2 * NM * (int)sizeof(PT);
    for (int o = lane * 128; o < nbytes; o += 32 * 128) prefetch_l2(pb + o);
  }
  {
    const int per = 2 * NM, ne = mc * per;
    const PT* src = pos + b0 * per;
    if constexpr (STAGE) {
      if (flags & 2) {  // positions as 16-byte vectors, eight per lane in flight
        using V = typename Vec16<PT>::T;
        constexpr int kN = Vec16<PT>::kN;
        const V* vs = reinterpret_cast<const V*>(src);
        const int nv = ne / kN;
        for (int x0 = 0; x0 < nv; x0 += 256) {
          V v[8];
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            const int x = x0 + h * 32 + lane;
            if (x < nv) v[h] = ldro<NC>(vs + x);
          }
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            const int x = x0 + h * 32 + lane;
            if (x < nv) {
              const int e = x * kN, mm = e / per;
              Vec16<PT>::put(S.pos + mm * prow + (e - mm * per), v[h]);
            }
          }
        }
      } else {
        for (int x = lane; x < ne; x += 32) {
          const int mm = x / per;
          S.pos[mm * prow + (x - mm * per)] = ldro<NC>(src + x);
        }
      }
    }
    const int nt = mc * NM;  // types: 16-byte vectors over whole chunks, then bytes
    const int8_t* ts = type + b0 * NM;
    int done = 0;
    if (flags & 2) {
      const int n16 = nt >> 4;
      for (int x = lane; x < n16; x += 32)
        reinterpret_cast<uint4*>(S.type)[x] = ldro<NC>(reinterpret_cast<const uint4*>(ts) + x);
      done = n16 << 4;
    }
    for (int x = done + lane; x < nt; x += 32) S.type[x] = (uint8_t)ldro<NC>(ts + x);
  }
  __syncwarp();

  // 2. lane m: checks, solve order and slots of mechanism m (build_one's decisions)
  int status = LINKS_MECH_OK, nd = 0, nf = 0, motor = -1, pivot = -1;
  uint32_t fixm = 0, simm = 0, motm = 0;
  if (m < mc) {
    if (n < 2 || n > NM) status = LINKS_MECH_BAD_SIZE;
    const int8_t* ty = reinterpret_cast<const int8_t*>(S.type) + m * NM;
    for (int a = 0; a < n && status == LINKS_MECH_OK; ++a) {
      const int t = ty[a];
      if (t == 0) fixm |= 1u << a;
      else if (t == 1) simm |= 1u << a;
      else if (t == 2) motm |= 1u << a;
      else status = LINKS_MECH_BAD_TYPE;
    }
  } else {
    status = -1;  // no mechanism
  }
  const uint32_t live = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
  auto nbm = [&](int a) { return S.nb[a * 32 + m] & live; };
  // One pass over the masks: no self-loop and every link listed both ways; the link
  // count (e2 / 2, less the ground-ground links, ff2 / 2) for the mobility check below;
  // and the running counts of known neighbours (has1 / has2 / has3, see the search) from
  // the fixed and actuated joints.
  const uint32_t known0 = fixm | motm;
  uint32_t has1 = 0, has2 = 0, has3 = 0;
  int e2 = 0, ff2 = 0;
  if (status == LINKS_MECH_OK) {
    uint32_t asym = 0;
    for (int a = 0; a < n; ++a) {
      const uint32_t na = nbm(a);
      asym |= na & (1u << a);
      for (uint32_t q = na; q; q &= q - 1) asym |= ~nbm(ffs32(q)) & (1u << a);
      e2 += popc32(na);
      if ((fixm >> a) & 1u) ff2 += popc32(na & fixm);
      if ((known0 >> a) & 1u) {
        has3 |= has2 & na;
        has2 |= has1 & na;
        has1 |= na;
      }
    }
    if (asym) status = LINKS_MECH_BAD_ADJ;
  }
  if (status == LINKS_MECH_OK && popc32(motm) != 1) status = LINKS_MECH_NO_MOTOR;
  if (status == LINKS_MECH_OK) {
    motor = ffs32(motm);
    const uint32_t pm = nbm(motor) & fixm;
    if (!pm) status = LINKS_MECH_NO_PIVOT;
    else pivot = ffs32(pm);
  }
  if (status == LINKS_MECH_OK) {
    // The search of build_one (the lowest-index unknown joint with >= 2 known neighbours;
    // > 2 is over-constraint) on running counts: has1 / has2 / has3 mark the joints with
    // at least 1 / 2 / 3 known neighbours, updated from each newly known joint's mask.
    uint32_t known = known0, unknown = simm;
    while (unknown) {
      const uint32_t ready = has2 & unknown;
      if (!ready) { status = LINKS_MECH_NOT_DYAD_SOLVABLE; break; }
      const int pick = ffs32(ready);
      if ((has3 >> pick) & 1u) { status = LINKS_MECH_OVERCONSTRAINED; break; }
      const uint32_t nbp = nbm(pick);
      const uint32_t par = nbp & known;
      S.dk[nd * 32 + m] = (uint8_t)pick;
      S.di[nd * 32 + m] = (uint8_t)ffs32(par);
      S.dj[nd * 32 + m] = (uint8_t)ffs32(par & (par - 1));
      ++nd;
      known |= 1u << pick;
      unknown &= ~(1u << pick);
      has3 |= has2 & nbp;
      has2 |= has1 & nbp;
      has1 |= nbp;
    }
  }
  if (status == LINKS_MECH_OK && (e2 - ff2) / 2 - 1 != 2 * popc32(simm)) status = LINKS_MECH_OVERCONSTRAINED;
  // every lane reads only its own column of the masks, whose words now hold slot bounds
  float* const bnd = reinterpret_cast<float*>(S.nb);
  const BuildOut o = out_of(p, b);
  float bmax = 0.0f, crank = 0.0f;
  dw2 u{};
  if (status == LINKS_MECH_OK) {
    // slots: fixed joints by index, then the actuated joint, then dyads in solve order
    for (uint32_t q = fixm; q; q &= q - 1) {
      const int a = ffs32(q);
      S.slot[a * 32 + m] = (uint8_t)nf;
      o.slot_joint[nf] = (uint8_t)a;
      const PT pa[4] = {posv(m, 2 * a), posv(m, 2 * a + 1), posv(m, 2 * pivot), posv(m, 2 * pivot + 1)};
      const dw2 r = rel(pa, 0, 1);
      o.fixpos[nf] = make_float4(r.x.h, r.x.l, r.y.h, r.y.l);
      const float bs = hyp_up(r.x.h, r.y.h);
      bnd[nf * 32 + m] = bs;
      bmax = fmaxf(bmax, bs);
      ++nf;
    }
    S.slot[motor * 32 + m] = (uint8_t)nf;
    o.slot_joint[nf] = (uint8_t)motor;
    for (int d = 0; d < nd; ++d) {
      const int k = S.dk[d * 32 + m];
      S.slot[k * 32 + m] = (uint8_t)(nf + 1 + d);
      o.slot_joint[nf + 1 + d] = (uint8_t)k;
    }
    const PT pm[4] = {posv(m, 2 * motor), posv(m, 2 * motor + 1), posv(m, 2 * pivot), posv(m, 2 * pivot + 1)};
    u = rel(pm, 0, 1);
    crank = hyp_up(u.x.h, u.y.h);
    bnd[nf * 32 + m] = crank;
    bmax = fmaxf(bmax, crank);
  } else if (status > 0) {
    MechHdr h{};
    h.n = (uint8_t)(n > 0 && n <= 255 ? n : 0);
    h.status = status;
    *o.hdr = h;
    nd = 0;
  } else {
    nd = 0;
  }
  S.nfv[m] = (uint8_t)nf;
  // exclusive prefix of the dyad counts
  int incl = nd;
#pragma unroll
  for (int q = 1; q < 32; q <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, q);
    if (lane >= q) incl += y;
  }
  S.pfx[m] = incl - nd;
  if (lane == 31) S.pfx[32] = incl;
  __syncwarp();

  // 3. the warp's dyads as one flat list, a dyad per lane.  Each dyad's link lengths
  // (r1, r2 high words) go to its joint's FP64 position slot, which lane m reads back
  // for the bound chain and then overwrites with the position.
  const int total = S.pfx[32];
  for (int f = lane; f < total; f += 32) {
    int lo = 0, hi = 31;  // the mechanism mm with pfx[mm] <= f < pfx[mm + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (S.pfx[mid] <= f) lo = mid;
      else hi = mid - 1;
    }
    const int mm = lo, d = f - S.pfx[mm];
    const int k = S.dk[d * 32 + mm], sk = S.nfv[mm] + 1 + d;
    const int ji = S.di[d * 32 + mm], jj = S.dj[d * 32 + mm];
    const PT q[6] = {posv(mm, 2 * ji), posv(mm, 2 * ji + 1), posv(mm, 2 * jj), posv(mm, 2 * jj + 1),
                     posv(mm, 2 * k), posv(mm, 2 * k + 1)};
    DyadGeo g = dyad_geo(q, 2, 0, 1);  // the parents as local joints 0 and 1, k as 2
    g.i = g.i == 0 ? ji : jj;
    g.j = g.j == 0 ? ji : jj;
    const int si = S.slot[g.i * 32 + mm], sj = S.slot[g.j * 32 + mm];
    p.dyad[(b0 + mm) * MD + d] = dyad_record(g, si, sj, k, sk);
    S.di[d * 32 + mm] = (uint8_t)si;
    S.dj[d * 32 + mm] = (uint8_t)sj;
    *reinterpret_cast<float2*>(p.pos64 + (b0 + mm) * NM + sk) = make_float2(g.r1.h, g.r2.h);
  }
  __syncwarp();  // also orders the lanes' global writes above before the reads below

  // 4. lane m: the bound chain in solve order, the FP64 positions, the header
  if (status == LINKS_MECH_OK) {
    // the link lengths four dyads at a time, their loads issued before the chain uses them
    for (int d0 = 0; d0 < nd; d0 += 4) {
      float2 rr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (d0 + u < nd) rr[u] = *reinterpret_cast<const float2*>(o.pos64 + nf + 1 + d0 + u);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int d = d0 + u;
        if (d < nd) {
          const float bk = dyad_bound(bnd[S.di[d * 32 + m] * 32 + m], bnd[S.dj[d * 32 + m] * 32 + m], rr[u].x,
                                      rr[u].y);
          bnd[(nf + 1 + d) * 32 + m] = bk;
          bmax = fmaxf(bmax, bk);
        }
      }
    }
    // the FP64 positions by slot and, from the same loads, the bounding box
    float lo_x = INFINITY, hi_x = -INFINITY, lo_y = INFINITY, hi_y = -INFINITY;
    for (int a = 0; a < n; ++a) {
      const PT px = posv(m, 2 * a), py = posv(m, 2 * a + 1);
      o.pos64[S.slot[a * 32 + m]] = make_double2((double)px, (double)py);
      const float x = (float)px, y = (float)py;
      lo_x = fminf(lo_x, x);
      hi_x = fmaxf(hi_x, x);
      lo_y = fminf(lo_y, y);
      hi_y = fmaxf(hi_y, y);
    }
    MechHdr h{};
    h.n = (uint8_t)n;
    h.status = status;
    h.nd = (uint8_t)nd;
    h.nf = (uint8_t)nf;
    h.motor_joint = (uint8_t)motor;
    h.pivot_joint = (uint8_t)pivot;
    h.pad0 = S.slot[pivot * 32 + m];  // pivot slot
    h.coupler_slot = (uint8_t)(nd > 0 ? nf + nd : nf);
    h.ux_h = u.x.h; h.ux_l = u.x.l; h.uy_h = u.y.h; h.uy_l = u.y.l;
    const PT pv[2] = {posv(m, 2 * pivot), posv(m, 2 * pivot + 1)};
    const dw px = abs_dw(pv, 0), py = abs_dw(pv, 1);
    h.px_h = px.h; h.px_l = px.l; h.py_h = py.h; h.py_l = py.l;
    h.bmax = bmax;
    h.lbox = hyp_up(fsub(hi_x, lo_x), fsub(hi_y, lo_y));
    h.e_motor = fmul(4.0f * kU, crank);
    h.e_fixed = fmul(kU, bmax);
    *o.hdr = h;
  }
  return {status, nd};
}

}  // namespace
}  // namespace links
