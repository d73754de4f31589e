// sim_core.cuh -- the bodies of the mixed-precision screen and emit (what sim_mixed.cu's
// kernels run, and what the serving loop runs inside its persistent kernel), and the
// FP32 dyad helpers they share.  Device code only; each including translation unit gets
// its own copy.
#pragma once

#include "links_internal.cuh"
#include "step.cuh"

namespace links {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kBatch = 16;  // work items taken per atomic by a warp of the main screen
constexpr int kEmitSlotBytes = 400;
constexpr int kEmitSlotBytesDW = 656;
constexpr int kEmitSharedDWMaxSlots = 12;

// Shared memory of one emit warp: the slot arrays and the row's dyad records (48 B per
// dyad).
__host__ __device__ constexpr size_t emit_warp_bytes(int n_max, int max_dyads, bool dws) {
  return (size_t)n_max * (dws ? kEmitSlotBytesDW : kEmitSlotBytes) + (size_t)max_dyads * 48;
}
// Shared memory of one screen warp: the slot arrays (384 B per slot and step of a lane)
// and the dyad records of its groups.
__host__ __device__ constexpr size_t screen_warp_bytes(int n_max, int max_dyads, int G, int S) {
  return (size_t)n_max * 384 * S + (size_t)(32 / G) * (2 * max_dyads + 1) * 16;
}
// Two steps per lane save record loads but double the slot arrays in shared memory;
// they pay for small mechanisms only (4 CTAs per SM still fit).
constexpr int kScreenTwoStepMaxSlots = 9;

// Adds a per-lane count to a 64-bit counter (one atomic per warp).
__device__ __forceinline__ void add_stat(int32_t* ctrs, int slot, unsigned v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v)
    atomicAdd(reinterpret_cast<unsigned long long*>(ctrs + slot), (unsigned long long)v);
}

struct LocShared {  // the lane's columns of shared slot arrays (x, y: 256 B per slot)
  static constexpr bool kFixInLoc = false;  // fixed slots stay in fix
  char* xb;
  char* yb;
  __device__ dwp get(int s) const {
    const float2 x = *reinterpret_cast<const float2*>(xb + s * 256);
    const float2 y = *reinterpret_cast<const float2*>(yb + s * 256);
    return {{x.x, x.y}, {y.x, y.y}};
  }
  __device__ void set(int s, const dwp& v) const {
    *reinterpret_cast<float2*>(xb + s * 256) = make_float2(v.x.h, v.x.l);
    *reinterpret_cast<float2*>(yb + s * 256) = make_float2(v.y.h, v.y.l);
  }
};
// One FP32 dyad of the screen for this lane.  Pb / Eb point at the lane's column of
// the warp's slot arrays (positions, error bounds); the record holds byte offsets.
// lockw = min over dyads of slack + bound (< 0: certainly locked), zmin = min of
// slack - bound (>= 0 everywhere: certainly free; NaN propagates), isgmax = max
// 1/sin(gamma).
template <bool EMAX = false>
__device__ __forceinline__ void fp32_dyad_rec(const float4& r0, const float4& r1, char* Pb, char* Eb, float& lockw,
                                              float& zmin, float& isgmax, float* emax = nullptr) {
  const uint32_t oij = __float_as_uint(r0.x), oe = __float_as_uint(r1.w), ok = __float_as_uint(r1.z);
  const float2 pi = *reinterpret_cast<const float2*>(Pb + (oij & 0xffffu));
  const float2 pj = *reinterpret_cast<const float2*>(Pb + (oij >> 16));
  const float ei = *reinterpret_cast<const float*>(Eb + (oe & 0xffffu));
  const float ej = *reinterpret_cast<const float*>(Eb + (oe >> 16));
  float kx, ky, ek;
  fp32_dyad_core(pi.x, pi.y, pj.x, pj.y, ei, ej, r0, r1, lockw, zmin, isgmax, kx, ky, ek);
  *reinterpret_cast<float2*>(Pb + (ok & 0xffffu)) = make_float2(kx, ky);
  *reinterpret_cast<float*>(Eb + (ok >> 16)) = ek;
  if (EMAX) *emax = fmaxf(*emax, ek);
}

// The same dyad for two steps of one lane (the two-step slot layout: per slot and lane
// a float4 (x of both steps, y of both steps) at P2 + 2 * (position offset), the two
// bounds at E2 + 2 * (bound offset)), one record load serving both.  The arithmetic is
// the scalar core twice: packed f32x2 arithmetic was measured to give other values at
// near-singular steps (and so another minimum discriminant) for a 3% gain.
__device__ __forceinline__ void fp32_dyad2(const float4& r0, const float4& r1, char* P2, char* E2, float* lockw,
                                           float* zmin, float* isgmax) {
  const uint32_t oij = __float_as_uint(r0.x), oe = __float_as_uint(r1.w), ok = __float_as_uint(r1.z);
  const float4 pi = *reinterpret_cast<const float4*>(P2 + 2 * (oij & 0xffffu));
  const float4 pj = *reinterpret_cast<const float4*>(P2 + 2 * (oij >> 16));
  const float2 ei = *reinterpret_cast<const float2*>(E2 + 2 * (oe & 0xffffu));
  const float2 ej = *reinterpret_cast<const float2*>(E2 + 2 * (oe >> 16));
  float kx0, ky0, ek0, kx1, ky1, ek1;
  fp32_dyad_core(pi.x, pi.z, pj.x, pj.z, ei.x, ej.x, r0, r1, lockw[0], zmin[0], isgmax[0], kx0, ky0, ek0);
  fp32_dyad_core(pi.y, pi.w, pj.y, pj.w, ei.y, ej.y, r0, r1, lockw[1], zmin[1], isgmax[1], kx1, ky1, ek1);
  *reinterpret_cast<float4*>(P2 + 2 * (ok & 0xffffu)) = make_float4(kx0, kx1, ky0, ky1);
  *reinterpret_cast<float2*>(E2 + 2 * (ok >> 16)) = make_float2(ek0, ek1);
}

template <bool EMAX = false>
__device__ __forceinline__ void fp32_dyad(const DyadRec* __restrict__ rec, char* Pb, char* Eb, float& lockw,
                                          float& zmin, float& isgmax, float* emax = nullptr) {
  const float4 r0 = rec->r0, r1 = rec->r1;  // records in global or shared memory
  fp32_dyad_rec<EMAX>(r0, r1, Pb, Eb, lockw, zmin, isgmax, emax);
}

// Groups of G lanes screen one mechanism; each lane takes S steps of a chunk of G * S
// consecutive steps (step chunk * G * S + u * G + lane-in-group, u < S), so that one
// load of a dyad record serves S steps.  The slot arrays hold S columns per lane.
// The work list is order[0, n) with n = *n_list, or p.order and the number of OK
// mechanisms when n_list is null; a warp takes `batch` (1 to 32) items of it per atomic.
// With RESCUE a step that the FP32 bounds leave uncertain is recomputed at once in
// double-word arithmetic by its lane (the others of the warp wait).  Without it, a
// mechanism whose first uncertain step of a chunk comes before the chunk's first
// certain lock (the only case where the uncertain step can decide anything) is put on
// the rescue list p.rescue and left; a second launch with RESCUE screens that list.
// Every other mechanism gets the same outputs either way.
template <int G, int S, bool RESCUE, bool NC = true>
__device__ __forceinline__ void screen_body(const PlanDev& p, int T, const float4* __restrict__ cs,
                                            uint8_t* __restrict__ valid, int16_t* __restrict__ lock_step,
                                            float* __restrict__ min_disc, const int32_t* __restrict__ order,
                                            const int32_t* __restrict__ n_list, char* smem, int warp, int lane,
                                            int batch = kBatch) {
  const int ns = p.n_max;
  const int g = lane / G, gl = lane % G;
  const int rstride = 2 * p.max_dyads + 1;  // float4 per group: (r0, r1) per dyad, padded
  char* const region = smem + (size_t)warp * screen_warp_bytes(ns, p.max_dyads, G, S);
  // one step per lane: positions (float2) at Pb + 256 * slot, bounds (float) at
  // Eb + 128 * slot; two steps per lane: both steps' positions (float4) at P2 + 512 *
  // slot, their bounds (float2) at E2 + 256 * slot
  char* const Pb = region + lane * 8;
  char* const Eb = region + ns * 256 + lane * 4;
  char* const P2 = region + lane * 16;
  char* const E2 = region + ns * 512 + lane * 8;
  // the group's mechanism: the FP32 parts of its dyad records
  float4* const Rg = reinterpret_cast<float4*>(region + S * ns * 384) + g * rstride;
  const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << (g * G));
  constexpr int CH = G * S;  // steps per chunk

  // The work list: n_list items of order, or p.order, the OK mechanisms sorted by dyad
  // count (bucket d of p.ctrs[kHist + d] entries from the exclusive prefix hpre of lane d),
  // taken from its end: the mechanisms with the most dyads first, so that the last work
  // of the launch is the lightest.
  int n_ok = 0, hpre = 0;
  if (n_list) {
    n_ok = *n_list;
  } else {
    const int h = p.ctrs[kHist + lane];
    int incl = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    hpre = incl - h;
    n_ok = __shfl_sync(kFull, incl, 31);
  }

  int qhead = 0, qend = 0, qbase = 0;
  int32_t qb = 0;  // lane i < batch: the mechanism of the batch's item i (item qbase + i)
  int qw = 0;      // ... and its header's counts word (n, nd, nf, motor joint)
  bool exhausted = false;
  int item = -1, chunk = 0;
  int32_t b = 0;
  int nd = 0, nf = 0;
  float ux = 0.f, uy = 0.f, e_motor = 0.f;
  float qacc = INFINITY;

  while (true) {
    // Give every idle group the next mechanism of the work list.
    unsigned need = __ballot_sync(kFull, gl == 0 && item < 0);
    bool fresh = false;
    while (need) {
      if (qhead >= qend) {
        if (exhausted) break;
        int base = 0;
        if (lane == 0) base = atomicAdd(&p.ctrs[kWork], batch);
        base = __shfl_sync(kFull, base, 0);
        if (base >= n_ok) { exhausted = true; break; }
        qhead = qbase = base;
        qend = min(base + batch, n_ok);
        // the batch's mechanisms, a lane each, with their header's counts word in a register
        // (a group that takes an item starts its record loads without waiting on the
        // header), their dyad records and fixed joints on their way to L2.  On the sorted
        // list an item's dyad count is its bucket: the last lane whose prefix does not
        // exceed the item's position.
        int ndq = p.max_dyads;
        if (!n_list) {
          const int q = n_ok - 1 - (qbase + lane);
          int lo = 0;
#pragma unroll
          for (int step = 16; step; step >>= 1) {
            const int v = __shfl_sync(kFull, hpre, lo + step);
            if (v <= q) lo += step;
          }
          ndq = lo;
        }
        if (lane < qend - qbase) {
          qb = ldro<NC>(order + (n_list ? qbase + lane : n_ok - 1 - (qbase + lane)));
          qw = ldro<NC>(reinterpret_cast<const int*>(p.hdr + qb) + 1);
          prefetch_l2(p.hdr + qb);
          const char* r0 = reinterpret_cast<const char*>(p.dyad + (int64_t)qb * p.max_dyads);
          for (int o = 0; o < ndq * (int)sizeof(DyadRec); o += 128) prefetch_l2(r0 + o);
          prefetch_l2(p.fixpos + (int64_t)qb * ns);
        }
      }
      int leader = __ffs(need) - 1;
      need &= need - 1;
      const int32_t bsel = __shfl_sync(kFull, qb, qhead - qbase);
      const int wsel = __shfl_sync(kFull, qw, qhead - qbase);
      if (g == leader / G) {
        item = qhead;
        b = bsel;
        fresh = true;
        nd = (wsel >> 8) & 0xff;
        nf = (wsel >> 16) & 0xff;
      }
      ++qhead;
    }
    if (__ballot_sync(kFull, item >= 0) == 0) break;
    __syncwarp();  // the previous mechanism's records are no longer read

    if (fresh) {
      const DyadRec* const rec = p.dyad + (int64_t)b * p.max_dyads;
      chunk = 0;
      qacc = INFINITY;
      const MechHdr* hp = p.hdr + b;
      ux = ldro<NC>(&hp->ux_h);
      uy = ldro<NC>(&hp->uy_h);
      const float2 eb = ldro<NC>(reinterpret_cast<const float2*>(&hp->e_motor));  // e_motor, e_fixed
      e_motor = eb.x;
      const float e_fixed = eb.y;
      for (int x = gl; x < 2 * nd; x += G) Rg[x] = ldro<NC>(x & 1 ? &rec[x >> 1].r1 : &rec[x >> 1].r0);
      const float4* fix = p.fixpos + (int64_t)b * ns;
      for (int s = 0; s < nf; ++s) {
        float4 f = ldro<NC>(fix + s);
        if (S == 2) {
          *reinterpret_cast<float4*>(P2 + s * 512) = make_float4(f.x, f.x, f.z, f.z);
          *reinterpret_cast<float2*>(E2 + s * 256) = make_float2(e_fixed, e_fixed);
        } else {
          *reinterpret_cast<float2*>(Pb + s * 256) = make_float2(f.x, f.z);
          *reinterpret_cast<float*>(Eb + s * 128) = e_fixed;
        }
      }
    }
    __syncwarp();  // a fresh group's records are in place
    const bool has = item >= 0;
    float lockw[S], zmin[S], isgmax[S];
    float2 mpos[S];
#pragma unroll
    for (int u = 0; u < S; ++u) {
      lockw[u] = INFINITY;
      zmin[u] = INFINITY;
      isgmax[u] = 0.0f;
      const int t = chunk * CH + u * G + gl;
      const float4 csv = __ldg(cs + min(t, T - 1));
      // rounded intrinsics: the topology-specialised screens compute the same values
      mpos[u] = make_float2(__fsub_rn(__fmul_rn(csv.x, ux), __fmul_rn(csv.z, uy)),
                            __fadd_rn(__fmul_rn(csv.z, ux), __fmul_rn(csv.x, uy)));
    }
    if (has) {
      if (S == 2) {
        *reinterpret_cast<float4*>(P2 + nf * 512) = make_float4(mpos[0].x, mpos[S - 1].x, mpos[0].y, mpos[S - 1].y);
        *reinterpret_cast<float2*>(E2 + nf * 256) = make_float2(e_motor, e_motor);
      } else {
        *reinterpret_cast<float2*>(Pb + nf * 256) = mpos[0];
        *reinterpret_cast<float*>(Eb + nf * 128) = e_motor;
      }
    }
    const int ndl = has ? nd : 0;
    const int ndw = __reduce_max_sync(kFull, (unsigned)ndl);
    for (int d = 0; d < ndw; ++d)
      if (d < ndl) {
        const float4 r0 = Rg[2 * d], r1 = Rg[2 * d + 1];
        if (S == 2) fp32_dyad2(r0, r1, P2, E2, lockw, zmin, isgmax);
        else fp32_dyad_rec(r0, r1, Pb, Eb, lockw[0], zmin[0], isgmax[0]);
      }
    // per step: certain lock, certain freedom, or a double-word rescue that decides
    int first = CH;      // first locking step of the chunk (group-uniform)
    int first_amb = CH;  // first uncertain step of the chunk (deferring launch)
    float qstep[S];
#pragma unroll
    for (int u = 0; u < S; ++u) {
      const int t = chunk * CH + u * G + gl;
      const bool act = has && t < T;
      const bool certain_lock = lockw[u] < 0.0f;
      const bool amb = act && !certain_lock && !(zmin[u] >= 0.0f);
      qstep[u] = __fdividef(1.0f, isgmax[u] * isgmax[u]);
      bool locked = act && certain_lock;
      if (RESCUE && amb) {
        dwp loc[kMaxJ];
        float qd;
        locked = dw_chain(p.hdr[b], p.fixpos + (int64_t)b * ns, p.dyad + (int64_t)b * p.max_dyads, __ldg(cs + t),
                          LocLocal{loc}, &qd);
        qstep[u] = qd;
      }
      const unsigned lb = __ballot_sync(kFull, locked) & gmask;
      if (lb && first == CH) first = u * G + (__ffs(lb) - 1 - g * G);
      if (!RESCUE) {
        const unsigned ab = __ballot_sync(kFull, amb) & gmask;
        if (ab && first_amb == CH) first_amb = u * G + (__ffs(ab) - 1 - g * G);
      }
    }
    // an uncertain step that decides (group-uniform): leave the mechanism to the rescue
    const bool defer = !RESCUE && has && first_amb < first;
    if (defer && gl == 0) p.rescue[atomicAdd(&p.ctrs[kNRescue], 1)] = b;
#pragma unroll
    for (int u = 0; u < S; ++u) {
      const int t = chunk * CH + u * G + gl;
      if (has && !defer && t < T && u * G + gl < first) qacc = fminf(qacc, qstep[u]);
    }
    const bool done = has && (defer || first < CH || (chunk + 1) * CH >= T);
    if (done) {
      if (!defer) {
        float qr = qacc;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) qr = fminf(qr, __shfl_xor_sync(gmask, qr, o));
        if (gl == 0) {
          valid[b] = first == CH;
          lock_step[b] = (int16_t)(first < CH ? chunk * CH + first : -1);
          min_disc[b] = qr;
        }
      }
      item = -1;
    } else {
      ++chunk;
    }
  }
}

// One warp per output row; 32 consecutive steps per pass.  Each step first runs the
// certified FP32 chain of the screen (shared-memory slot arrays); if every joint's
// forward error bound is within the tolerance (kEmitBudget of the bounding-box
// diagonal, less the output rounding) the FP32 positions are written, otherwise that
// lane recomputes the step in double-word arithmetic relative to the pivot, as the
// screen's rescue does (so a step the screen rescued gets the same operations on the
// same values, and the same lock decision), and writes those.  A row whose first 32
// steps all needed double-word computes the rest in double-word directly.
// Shared memory per warp and slot: FP32 positions (256 B), error bounds (128 B),
// double-word fixed joints (16 B, one per warp) and, with DWS, the double-word y of
// the lane's slot positions (256 B; x reuses the FP32 positions, the fixed slots stay
// in the warp's copy).  Larger mechanisms keep the double-word slots thread-local,
// which costs less occupancy.
// With CENSUS the kernel writes nothing and only counts what the emit does: steps
// computed, and steps (and dyad-steps) whose FP32 bound sends them to double-word
// (the same FP32 chain on the same inputs, so the same decisions).
template <bool CENSUS, bool DWS, bool NC = true>
__device__ __forceinline__ void emit_body(const PlanDev& p, int64_t B, int T, const float4* __restrict__ cs, int full,
                                          const int16_t* __restrict__ lock_step, const int32_t* __restrict__ out_index,
                                          int64_t out_capacity, float* __restrict__ traj, float* __restrict__ path,
                                          int32_t* err, char* smem, int* jofs, int warp, int lane, int64_t gw,
                                          int64_t nw, const int64_t* __restrict__ row_off = nullptr,
                                          int64_t traj_cap = 0, int32_t* work = nullptr) {
  const int ns = p.n_max;
  const int slot_bytes = DWS ? kEmitSlotBytesDW : kEmitSlotBytes;
  char* const region = smem + (size_t)warp * emit_warp_bytes(ns, p.max_dyads, DWS);
  float4* const Rw = reinterpret_cast<float4*>(region + ns * slot_bytes);  // the row's dyad records
  char* const Pb = region + lane * 8;
  char* const Eb = region + ns * 256 + lane * 4;
  float4* const Fb = reinterpret_cast<float4*>(region + ns * 384);  // double-word fixed joints (warp)
  char* const Yb = region + ns * 400 + lane * 8;                    // DWS: double-word y
  int64_t rows = full ? B : min((int64_t)p.ctrs[kNValid], out_capacity);
  const float nanf_ = __int_as_float(0x7fc00000);
  unsigned n_steps = 0, n_dw = 0, n_dw_dyads = 0;  // census counts of this lane
  // rows taken one at a time from the work counter (rows that go to double-word cost a few
  // times more, and a fixed assignment leaves the launch waiting on the unluckiest warp),
  // or, without one, every nw-th row
  const auto next_row = [&](int64_t r) -> int64_t {
    if (!work) return r + nw;
    int v = 0;
    if (lane == 0) v = atomicAdd(work, 1);
    return (int64_t)__shfl_sync(kFull, v, 0);
  };
  for (int64_t r = work ? next_row(0) : gw; r < rows; r = next_row(r)) {
    const int64_t b = full ? r : (int64_t)out_index[r];
    if (b < 0 || b >= B) {
      if (lane == 0) atomicOr(err, kErrBadIndex);
      continue;
    }
    const MechHdr h = p.hdr[b];
    const bool ok = h.status == LINKS_MECH_OK;
    const int n = ok ? h.n : 0;
    const int nf = h.nf, nd = ok ? h.nd : 0;
    int lock = T;
    if (full) lock = ok ? (lock_step[b] < 0 ? T : lock_step[b]) : 0;
    const uint8_t* sj = p.slot_joint + b * kMaxJ;
    const DyadRec* const rec = reinterpret_cast<const DyadRec*>(Rw);
    float2* trow = nullptr;  // packed rows (row_off): the row's own joints only
    if (traj) {
      if (!row_off) trow = reinterpret_cast<float2*>(traj) + r * ns * T;
      else if (row_off[r] >= 0 && row_off[r] + n <= traj_cap) trow = reinterpret_cast<float2*>(traj) + row_off[r] * T;
    }
    float2* prow = path ? reinterpret_cast<float2*>(path) + r * T : nullptr;
    // FP32 tolerance: the budget minus the rounding of the absolute output coordinates
    const float tol = fmaf(-2.0f * kU, fabsf(h.px_h) + fabsf(h.py_h) + h.bmax, kEmitBudget * h.lbox);
    const int nslot = nf + 1 + nd;
    __syncwarp();
    if (lane < nslot) jofs[lane] = (int)sj[lane] * T;
    for (int x = lane; x < 3 * nd; x += 32)
      Rw[x] = ldro<NC>(reinterpret_cast<const float4*>(p.dyad + b * p.max_dyads) + x);
    __syncwarp();
    // fixed joints relative to the pivot: FP32 (the lane's column) and double-word
    // (one copy per warp)
    if (ok) {
      const float4* fr = p.fixpos + b * ns;
      for (int s = 0; s < nf; ++s) {
        float4 f = ldro<NC>(fr + s);
        *reinterpret_cast<float2*>(Pb + s * 256) = make_float2(f.x, f.z);
        *reinterpret_cast<float*>(Eb + s * 128) = h.e_fixed;
        if (lane == s) Fb[s] = f;
      }
    }
    __syncwarp();
    bool dw_only = false;  // warp-uniform: the row goes straight to double-word
    for (int t0 = 0; t0 < T; t0 += 32) {
      const int t = t0 + lane;
      const bool act = t < T && t < lock;
      bool certified = false;
      if (act) {
        const float4 csv = __ldg(cs + t);
        if (!dw_only) {
          *reinterpret_cast<float2*>(Pb + nf * 256) =
              make_float2(__fsub_rn(__fmul_rn(csv.x, h.ux_h), __fmul_rn(csv.z, h.uy_h)),
                          __fadd_rn(__fmul_rn(csv.z, h.ux_h), __fmul_rn(csv.x, h.uy_h)));  // as the screen
          *reinterpret_cast<float*>(Eb + nf * 128) = h.e_motor;
          float lockw = INFINITY, zmin = INFINITY, isgmax = 0.0f, emax = 0.0f;
          for (int d = 0; d < nd; ++d) fp32_dyad<true>(rec + d, Pb, Eb, lockw, zmin, isgmax, &emax);
          certified = emax <= tol && zmin >= 0.0f;
          if (CENSUS) {
            ++n_steps;
            if (!certified) {
              ++n_dw;
              n_dw_dyads += nd;
            }
          } else if (certified) {
            for (int s = 0; s < nslot; ++s) {
              const float2 q = *reinterpret_cast<const float2*>(Pb + s * 256);
              const float2 v = make_float2(q.x + h.px_h, q.y + h.py_h);
              if (trow) trow[jofs[s] + t] = v;
              if (prow && s == h.coupler_slot) prow[t] = v;
            }
          }
        }
        if (!CENSUS && !certified) {
          dwp lbuf[DWS ? 1 : kMaxJ];
          const auto loc = [&] {
            if constexpr (DWS) return LocShared{Pb, Yb};
            else return LocLocal{lbuf};
          }();
          bool lk = dw_chain(h, Fb, rec, csv, loc, nullptr);  // no minimum q: the screen has it
          if (lk) atomicOr(err, kErrEmitLock);
          for (int s = 0; s < nslot; ++s) {
            const dwp ls = slot_pos(loc, Fb, nf, s);
            // the absolute coordinate as the FP32 path forms it, from the high parts
            // (the low parts are below the output rounding the tolerance reserves)
            const float2 v = lk ? make_float2(nanf_, nanf_) : make_float2(ls.x.h + h.px_h, ls.y.h + h.py_h);
            if (trow) trow[jofs[s] + t] = v;
            if (prow && s == h.coupler_slot) prow[t] = v;
          }
        }
      } else if (!CENSUS && t < T) {
        for (int s = 0; s < n; ++s)
          if (trow) trow[(int64_t)sj[s] * T + t] = make_float2(nanf_, nanf_);
        if (prow) prow[t] = make_float2(nanf_, nanf_);
      }
      if (!CENSUS && t < T && !row_off)
        for (int j = n; j < ns; ++j)
          if (trow) trow[(int64_t)j * T + t] = make_float2(nanf_, nanf_);
      if (!CENSUS && t0 == 0) {
        // A row whose first pass needed double-word on every step (at least half a pass)
        // skips the FP32 chain from then on: its bounds stay above the budget along the
        // turn, as the census shows for deep chains.
        const unsigned am = __ballot_sync(kFull, act), dm = __ballot_sync(kFull, act && !certified);
        dw_only = dm == am && __popc(am) >= 16;
      }
    }
  }
  if (CENSUS) {
    add_stat(p.ctrs, kStatEmitSteps, n_steps);
    add_stat(p.ctrs, kStatEmitDW, n_dw);
    add_stat(p.ctrs, kStatEmitDWDyads, n_dw_dyads);
  }
}

}  // namespace
}  // namespace links
