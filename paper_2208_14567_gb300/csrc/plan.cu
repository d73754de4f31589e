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
// The builder runs on host threads and in CUDA kernels: one thread per mechanism
// (build_one) for n_max <= 8, a group of 16 or 32 lanes per mechanism (build_group)
// for larger mechanisms.  All produce bit-identical plans.
#include <algorithm>
#include <thread>
#include <vector>

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
LINKS_HD float u2f(uint32_t u) {
  union { uint32_t u; float f; } cv;
  cv.u = u;
  return cv.f;
}
// |(x, y)| rounded up a little (a bound, identical on host and device).
LINKS_HD float hyp_up(float x, float y) {
  return fmul(fsqrt_rn(fadd(fmul(x, x), fmul(y, y))), 1.0f + 4.0f * kU);
}

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
    int k = S.dk(d), i = S.di(d), j = S.dj(d);
    dw2 a = rel(pos, j, i), vi = rel(pos, k, i), vj = rel(pos, k, j);
    dw cross = dw_sub(dw_mul(a.x, vi.y), dw_mul(a.y, vi.x));
    if (dw_sign(cross) < 0.0f) {  // keep the initial branch as the "+" one
      int t = i; i = j; j = t;
      dw2 tv = vi; vi = vj; vj = tv;
    }
    dw r1sq = norm2(vi), r2sq = norm2(vj);
    dw r1 = dw_sqrt_exact(r1sq), r2 = dw_sqrt_exact(r2sq);
    dw R12 = dw_add(r1, r2);
    dw Rm = dw_sub(r1, r2);
    if (dw_sign(Rm) < 0.0f) Rm = dw_neg(Rm);
    dw c = dw_sub(r1sq, r2sq);
    int si = S.slot(i), sj = S.slot(j), sk = nf + 1 + d;
    float bi = S.bound(si), bj = S.bound(sj);
    const float bk = fmul(fminf(fadd(bi, r1.h), fadd(bj, r2.h)), 1.0f + 4.0f * kU);
    S.set_bound(sk, bk);
    bmax = fmaxf(bmax, bk);
    float locc = fmul(kAmpErr * kU, R12.h);
    const uint32_t slots = (uint32_t)si | ((uint32_t)sj << 8) | ((uint32_t)k << 16) | ((uint32_t)sk << 24);
    // byte offsets into a lane's slot arrays: positions 256 B per slot, bounds 128 B
    const uint32_t offPij = ((uint32_t)si * 256u) | (((uint32_t)sj * 256u) << 16);
    const uint32_t offK = ((uint32_t)sk * 256u) | (((uint32_t)sk * 128u) << 16);
    const uint32_t offEij = ((uint32_t)si * 128u) | (((uint32_t)sj * 128u) << 16);
    DyadRec rec;
    rec.r0 = make_float4(u2f(offPij), R12.h, Rm.h, c.h);
    rec.r1 = make_float4(fmul(fadd(r1.h, r1.h), r2.h), locc, u2f(offK), u2f(offEij));
    rec.r2 = make_float4(r1sq.h, r1sq.l, c.l, u2f(slots));
    o.dyad[d] = rec;
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

LINKS_HD BuildOut out_of(const PlanDev& p, int64_t b) {
  BuildOut o;
  o.hdr = p.hdr + b;
  o.slot_joint = p.slot_joint + b * kMaxJ;
  o.fixpos = p.fixpos + b * p.n_max;
  o.pos64 = p.pos64 + b * p.n_max;
  o.dyad = p.dyad + b * p.max_dyads;
  return o;
}

// The same builder on a group of G lanes per mechanism (G >= n_max): lane a holds
// joint a's neighbour mask and slot, lane s the bound of slot s, lane d the dyad d
// found d-th.  The checks and the solve-order search are group votes, the dyads'
// geometry is computed by their lanes in parallel, and the bound chain (each dyad's
// bound from its parents') runs over the dyads in solve order through shuffles.  Each
// value is the same expression on the same operands as in build_one, and the maxima
// and minima do not depend on the order they are taken in, so the plan is the same
// to the bit.
constexpr unsigned kFull = 0xffffffffu;

template <int G>
struct Group {
  unsigned mask;
  int base;
  __device__ unsigned ballot(bool v) const { return (__ballot_sync(mask, v) & mask) >> base; }
  __device__ bool any(bool v) const { return ballot(v) != 0; }
  template <class V>
  __device__ V bc(V v, int src) const { return __shfl_sync(mask, v, src, G); }
  __device__ int sum(int v) const {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
  }
  __device__ float max(float v) const {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, G));
    return v;
  }
  __device__ float min(float v) const {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v = fminf(v, __shfl_xor_sync(mask, v, o, G));
    return v;
  }
};

template <typename PT, int G>
__device__ int build_group(int n, int n_max, const uint8_t* __restrict__ adj, const int8_t* __restrict__ type,
                           const PT* __restrict__ pos, BuildOut o, int gl, const Group<G>& grp, int* nd_out) {
  MechHdr h{};
  h.n = (uint8_t)(n > 0 && n <= 255 ? n : 0);
  int status = LINKS_MECH_OK;
  if (n < 2 || n > n_max || n_max > G) status = LINKS_MECH_BAD_SIZE;
  const bool joint = status == LINKS_MECH_OK && gl < n;
  const int t = joint ? type[gl] : -1;
  const uint32_t fixm = grp.ballot(joint && t == 0), simm = grp.ballot(joint && t == 1);
  const uint32_t motm = grp.ballot(joint && t == 2);
  if (grp.any(joint && (t < 0 || t > 2))) status = LINKS_MECH_BAD_TYPE;
  uint32_t nb = 0;  // lane a: neighbours of joint a
  if (status == LINKS_MECH_OK) {
    if (gl < n) {
      const uint8_t* row = adj + (size_t)gl * n_max;
      for (int c = 0; c < n; ++c) nb |= (row[c] != 0 ? 1u : 0u) << c;
    }
    bool bad = gl < n && ((nb >> gl) & 1u);
    for (int c = 0; c < n; ++c) {
      const uint32_t nbc = grp.bc(nb, c);
      if (gl < n && ((nb >> c) & 1u) && !((nbc >> gl) & 1u)) bad = true;
    }
    if (grp.any(bad)) status = LINKS_MECH_BAD_ADJ;
  }
  if (status == LINKS_MECH_OK && popc32(motm) != 1) status = LINKS_MECH_NO_MOTOR;
  int motor = -1, pivot = -1, nd = 0;
  if (status == LINKS_MECH_OK) {
    motor = ffs32(motm);
    const uint32_t pm = grp.bc(nb, motor) & fixm;
    if (!pm) status = LINKS_MECH_NO_PIVOT;
    else pivot = ffs32(pm);
  }
  int dk = 0, di = 0, dj = 0, my_d = -1;  // lane d: dyad d; lane a: the dyad solving joint a
  if (status == LINKS_MECH_OK) {
    uint32_t known = fixm | motm, unknown = simm;
    while (unknown) {
      const int c = popc32(nb & known);
      const uint32_t cand = grp.ballot(gl < n && ((unknown >> gl) & 1u) && c >= 2);
      if (!cand) {
        status = LINKS_MECH_NOT_DYAD_SOLVABLE;
        break;
      }
      const int pick = ffs32(cand);
      if (grp.bc(c, pick) > 2) {
        status = LINKS_MECH_OVERCONSTRAINED;
        break;
      }
      const uint32_t par = grp.bc(nb, pick) & known;
      if (gl == nd) {
        dk = pick;
        di = ffs32(par);
        dj = ffs32(par & (par - 1));
      }
      if (gl == pick) my_d = nd;
      ++nd;
      known |= 1u << pick;
      unknown &= ~(1u << pick);
    }
  }
  if (status == LINKS_MECH_OK) {
    const int e2 = grp.sum(gl < n ? popc32(nb) : 0);
    const int ff2 = grp.sum(gl < n && ((fixm >> gl) & 1u) ? popc32(nb & fixm) : 0);
    if ((e2 - ff2) / 2 - 1 != 2 * popc32(simm)) status = LINKS_MECH_OVERCONSTRAINED;
  }
  h.status = status;
  if (status != LINKS_MECH_OK) {
    h.nd = 0;
    if (gl == 0) *o.hdr = h;
    return status;
  }

  // Slots: fixed joints by index, then the actuated joint, then dyads in solve order.
  const int nf = popc32(fixm);
  int slot = 0;  // lane a: slot of joint a
  if ((fixm >> gl) & 1u) slot = popc32(fixm & ((1u << gl) - 1u));
  else if (gl == motor) slot = nf;
  else if (my_d >= 0) slot = nf + 1 + my_d;
  if (gl < n) {
    o.slot_joint[slot] = (uint8_t)gl;
    o.pos64[slot] = make_double2((double)pos[2 * gl], (double)pos[2 * gl + 1]);
  }
  float bound = 0.0f, bmax = 0.0f;  // lane s: bound of slot s
  if (gl < nf) {
    uint32_t m = fixm;
    for (int q = 0; q < gl; ++q) m &= m - 1;
    const dw2 r = rel(pos, ffs32(m), pivot);
    o.fixpos[gl] = make_float4(r.x.h, r.x.l, r.y.h, r.y.l);
    bound = hyp_up(r.x.h, r.y.h);
    bmax = bound;
  }
  const dw2 u = rel(pos, motor, pivot);
  const float crank = hyp_up(u.x.h, u.y.h);
  if (gl == nf) bound = crank;
  bmax = fmaxf(bmax, crank);

  int i = di, j = dj;
  float r1h = 0.0f, r2h = 0.0f;
  DyadRec rec;
  if (gl < nd) {
    const int k = dk;
    dw2 a = rel(pos, j, i), vi = rel(pos, k, i), vj = rel(pos, k, j);
    dw cross = dw_sub(dw_mul(a.x, vi.y), dw_mul(a.y, vi.x));
    if (dw_sign(cross) < 0.0f) {  // keep the initial branch as the "+" one
      int tt = i; i = j; j = tt;
      dw2 tv = vi; vi = vj; vj = tv;
    }
    dw r1sq = norm2(vi), r2sq = norm2(vj);
    dw r1 = dw_sqrt_exact(r1sq), r2 = dw_sqrt_exact(r2sq);
    dw R12 = dw_add(r1, r2);
    dw Rm = dw_sub(r1, r2);
    if (dw_sign(Rm) < 0.0f) Rm = dw_neg(Rm);
    dw c = dw_sub(r1sq, r2sq);
    r1h = r1.h;
    r2h = r2.h;
    rec.r0 = make_float4(0.0f, R12.h, Rm.h, c.h);
    rec.r1 = make_float4(fmul(fadd(r1.h, r1.h), r2.h), fmul(kAmpErr * kU, R12.h), 0.0f, 0.0f);
    rec.r2 = make_float4(r1sq.h, r1sq.l, c.l, 0.0f);
  }
  const int si = grp.bc(slot, i), sj = grp.bc(slot, j);  // slots of the lane's dyad's parents
  if (gl < nd) {
    const int sk = nf + 1 + gl;
    const uint32_t slots = (uint32_t)si | ((uint32_t)sj << 8) | ((uint32_t)dk << 16) | ((uint32_t)sk << 24);
    const uint32_t offPij = ((uint32_t)si * 256u) | (((uint32_t)sj * 256u) << 16);
    const uint32_t offK = ((uint32_t)sk * 256u) | (((uint32_t)sk * 128u) << 16);
    const uint32_t offEij = ((uint32_t)si * 128u) | (((uint32_t)sj * 128u) << 16);
    rec.r0.x = u2f(offPij);
    rec.r1.z = u2f(offK);
    rec.r1.w = u2f(offEij);
    rec.r2.w = u2f(slots);
    o.dyad[gl] = rec;
  }
  for (int d = 0; d < nd; ++d) {  // the bound chain, in solve order
    const float bi = grp.bc(bound, grp.bc(si, d)), bj = grp.bc(bound, grp.bc(sj, d));
    const float bk = fmul(fminf(fadd(bi, grp.bc(r1h, d)), fadd(bj, grp.bc(r2h, d))), 1.0f + 4.0f * kU);
    if (gl == nf + 1 + d) bound = bk;
    bmax = fmaxf(bmax, bk);
  }
  bmax = grp.max(bmax);
  const float x = gl < n ? (float)pos[2 * gl] : INFINITY, y = gl < n ? (float)pos[2 * gl + 1] : INFINITY;
  const float lo_x = grp.min(x), lo_y = grp.min(y);
  const float hi_x = grp.max(gl < n ? x : -INFINITY), hi_y = grp.max(gl < n ? y : -INFINITY);
  const int pivot_slot = grp.bc(slot, pivot);
  if (gl == 0) {
    h.nd = (uint8_t)nd;
    h.nf = (uint8_t)nf;
    h.motor_joint = (uint8_t)motor;
    h.pivot_joint = (uint8_t)pivot;
    h.pad0 = (uint8_t)pivot_slot;
    h.coupler_slot = (uint8_t)(nd > 0 ? nf + nd : nf);
    h.ux_h = u.x.h; h.ux_l = u.x.l; h.uy_h = u.y.h; h.uy_l = u.y.l;
    dw px = abs_dw(pos, 2 * pivot), py = abs_dw(pos, 2 * pivot + 1);
    h.px_h = px.h; h.px_l = px.l; h.py_h = py.h; h.py_l = py.l;
    h.bmax = bmax;
    h.lbox = hyp_up(fsub(hi_x, lo_x), fsub(hi_y, lo_y));
    h.e_motor = fmul(4.0f * kU, crank);
    h.e_fixed = fmul(kU, bmax);
    *o.hdr = h;
  }
  if (nd_out) *nd_out = nd;
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

// G lanes per mechanism (build_group); 256 / G mechanisms per block.
template <typename PT, int G>
__global__ void __launch_bounds__(256) build_group_kernel(int64_t B, const int32_t* __restrict__ n_joints,
                                                          const uint8_t* __restrict__ adj,
                                                          const int8_t* __restrict__ type,
                                                          const PT* __restrict__ pos, PlanDev p,
                                                          int32_t* __restrict__ status_out) {
  __shared__ int hist[32];
  if (threadIdx.x < 32) hist[threadIdx.x] = 0;
  __syncthreads();
  const int nm = p.n_max;
  const int lane = threadIdx.x & 31, gl = lane % G;
  Group<G> grp;
  grp.base = lane - gl;
  grp.mask = G == 32 ? kFull : (((1u << G) - 1u) << grp.base);
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  if (b < B) {  // uniform in the group
    int nd = 0;
    const int st = build_group<PT, G>(n_joints[b], nm, adj + b * nm * nm, type + b * nm, pos + b * nm * 2,
                                      out_of(p, b), gl, grp, &nd);
    if (gl == 0) {
      if (status_out) status_out[b] = st;
      if (st == LINKS_MECH_OK) atomicAdd(&hist[nd], 1);
    }
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
                      int32_t* status_out) {
  PlanDev& p = plan->d;
  LINKS_CUDA(cudaMemsetAsync(p.ctrs, 0, kCtrs * sizeof(int32_t), ctx->stream));
  plan->B = B;
  if (B == 0) return LINKS_OK;
  unsigned grid = (unsigned)((B + 255) / 256);
  {
    KernelScope ks(ctx, "plan_build");
    // n_max <= 8: a thread per mechanism, scratch in registers (measured faster than a
    // lane group at this size); larger: a group of 16 or 32 lanes per mechanism
    const int G = p.n_max <= 16 ? 16 : 32;
    const unsigned ggrid = (unsigned)((B * G + 255) / 256);
    const bool small = p.n_max <= 8;
    if (pos_dtype == LINKS_F32) {
      const float* ps = (const float*)pos0;
      if (small) build_kernel<float, 8><<<grid, 256, 0, ctx->stream>>>(B, n_joints, adj, type, ps, p, status_out);
      else if (G == 16) build_group_kernel<float, 16><<<ggrid, 256, 0, ctx->stream>>>(B, n_joints, adj, type, ps, p, status_out);
      else build_group_kernel<float, 32><<<ggrid, 256, 0, ctx->stream>>>(B, n_joints, adj, type, ps, p, status_out);
    } else {
      const double* ps = (const double*)pos0;
      if (small) build_kernel<double, 8><<<grid, 256, 0, ctx->stream>>>(B, n_joints, adj, type, ps, p, status_out);
      else if (G == 16) build_group_kernel<double, 16><<<ggrid, 256, 0, ctx->stream>>>(B, n_joints, adj, type, ps, p, status_out);
      else build_group_kernel<double, 32><<<ggrid, 256, 0, ctx->stream>>>(B, n_joints, adj, type, ps, p, status_out);
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
