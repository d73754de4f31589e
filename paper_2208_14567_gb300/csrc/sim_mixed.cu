// sim_mixed.cu -- mixed-precision simulation of planned mechanisms (LINKS_MIXED).
//
// What is computed (Sec. "Graphical Simulator"; Sec. "Finding Valid Initial Positions",
// Infeasibility rule; Sec. "Dataset Features & Statistics", item Simulation Data): at step
// t the crank is turned by 2*pi*t/T about its pivot and each dyad joint k with parents i, j
// is placed at the intersection of the circles |p - p_i| = r1 and |p - p_j| = r2 on the
// branch of the initial configuration.  The step locks when a dyad has no
// intersection.  Steps are independent of each other (the branch is fixed by the
// initial positions), so lanes run different steps of the same mechanism.
//
// Two kernels:
//   screen  FP32 dyads in product form, D = (d + R12)(R12 - d)(d - Rm)(d + Rm), with a
//           per-joint forward error bound E (E_k = (E_i + E_j + local) / sin(gamma_k)).
//           A step is certainly locked if some dyad has slack = min(R12 - d, d - Rm)
//           < -(E_i + E_j + local), certainly free if every slack exceeds its bound; in
//           between the lane recomputes the step in double-word arithmetic (~48 bits),
//           which decides.  Groups of G lanes take consecutive steps of one mechanism,
//           a ballot finds the first locking step, and the group moves on to the next
//           mechanism of a work list sorted by dyad count.
//   emit    every requested trajectory step through the same certified FP32 chain; a
//           step whose bounds are all within the tolerance writes its FP32 positions,
//           any other is recomputed in double-word arithmetic (one warp per output row,
//           32 consecutive steps per store).
// The FP32 dyad and the double-word chain are in step.cuh, shared with the screens
// compiled per topology at run time (topo.cu).
#include "step.cuh"
#include "links_internal.cuh"

namespace links {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kBatch = 16;  // work items taken per atomic by a warp
constexpr int kEmitSlotBytes = 400;
constexpr int kEmitSlotBytesDW = 656;
constexpr int kEmitSharedDWMaxSlots = 12;
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
// mechanisms when n_list is null.
// With RESCUE a step that the FP32 bounds leave uncertain is recomputed at once in
// double-word arithmetic by its lane (the others of the warp wait).  Without it, a
// mechanism whose first uncertain step of a chunk comes before the chunk's first
// certain lock (the only case where the uncertain step can decide anything) is put on
// the rescue list p.rescue and left; a second launch with RESCUE screens that list.
// Every other mechanism gets the same outputs either way.
template <int G, int S, bool RESCUE>
__global__ void __launch_bounds__(kBlock, 4) screen_kernel(PlanDev p, int T, const float4* __restrict__ cs,
                                                        uint8_t* __restrict__ valid,
                                                        int16_t* __restrict__ lock_step,
                                                        float* __restrict__ min_disc,
                                                        const int32_t* __restrict__ order,
                                                        const int32_t* __restrict__ n_list) {
  extern __shared__ float4 smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ns = p.n_max;
  const int g = lane / G, gl = lane % G;
  const int rstride = 2 * p.max_dyads + 1;  // float4 per group: (r0, r1) per dyad, padded
  char* const region = reinterpret_cast<char*>(smem4) + (size_t)warp * (ns * 384 * S + (32 / G) * rstride * 16);
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

  int n_ok = 0;
  if (n_list) {
    n_ok = *n_list;
  } else {
    n_ok = p.ctrs[kHist + lane];
#pragma unroll
    for (int o = 16; o; o >>= 1) n_ok += __shfl_xor_sync(kFull, n_ok, o);
  }

  int qhead = 0, qend = 0;
  bool exhausted = false;
  int item = -1, chunk = 0;
  int64_t b = 0;
  int nd = 0, nf = 0;
  float ux = 0.f, uy = 0.f, e_motor = 0.f;
  const DyadRec* rec = p.dyad;
  float qacc = INFINITY;

  while (true) {
    // Give every idle group the next mechanism of the work list.
    unsigned need = __ballot_sync(kFull, gl == 0 && item < 0);
    bool fresh = false;
    while (need) {
      if (qhead >= qend) {
        if (exhausted) break;
        int base = 0;
        if (lane == 0) base = atomicAdd(&p.ctrs[kWork], kBatch);
        base = __shfl_sync(kFull, base, 0);
        if (base >= n_ok) { exhausted = true; break; }
        qhead = base;
        qend = min(base + kBatch, n_ok);
      }
      int leader = __ffs(need) - 1;
      need &= need - 1;
      if (g == leader / G) { item = qhead; fresh = true; }
      ++qhead;
    }
    if (__ballot_sync(kFull, item >= 0) == 0) break;
    __syncwarp();  // the previous mechanism's records are no longer read

    if (fresh) {
      b = order[item];
      const MechHdr* hp = p.hdr + b;
      const int4 w0 = __ldg(reinterpret_cast<const int4*>(hp));
      nd = (w0.y >> 8) & 0xff;
      nf = (w0.y >> 16) & 0xff;
      ux = __ldg(&hp->ux_h);
      uy = __ldg(&hp->uy_h);
      e_motor = __ldg(&hp->e_motor);
      const float e_fixed = __ldg(&hp->e_fixed);
      rec = p.dyad + b * p.max_dyads;
      chunk = 0;
      qacc = INFINITY;
      for (int x = gl; x < 2 * nd; x += G) Rg[x] = __ldg(x & 1 ? &rec[x >> 1].r1 : &rec[x >> 1].r0);
      const float4* fix = p.fixpos + b * ns;
      for (int s = 0; s < nf; ++s) {
        float4 f = __ldg(fix + s);
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
        locked = dw_chain<false>(p.hdr[b], p.fixpos + b * ns, rec, __ldg(cs + t), LocLocal{loc}, &qd);
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
    if (defer && gl == 0) p.rescue[atomicAdd(&p.ctrs[kNRescue], 1)] = (int32_t)b;
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
// lane recomputes the step in double-word arithmetic (absolute coordinates) and
// writes those.
// Shared memory per warp and slot: FP32 positions (256 B), error bounds (128 B),
// absolute fixed joints (16 B, one per warp) and, with DWS, the double-word y of the
// lane's slot positions (256 B; x reuses the FP32 positions, the fixed slots stay in
// the warp's copy).  Larger mechanisms keep the double-word slots thread-local, which
// costs less occupancy.
// With CENSUS the kernel writes nothing and only counts what the emit does: steps
// computed, and steps (and dyad-steps) whose FP32 bound sends them to double-word
// (the same FP32 chain on the same inputs, so the same decisions).
template <bool CENSUS, bool DWS>
__global__ void __launch_bounds__(kBlock) emit_kernel(PlanDev p, int64_t B, int T, const float4* __restrict__ cs,
                                                      int full, const int16_t* __restrict__ lock_step,
                                                      const int32_t* __restrict__ out_index,
                                                      int64_t out_capacity, float* __restrict__ traj,
                                                      float* __restrict__ path, int32_t* err) {
  extern __shared__ float4 smem4[];
  __shared__ int s_jofs[kWarps][kMaxJ];  // per warp: offset of each slot's joint row in the output row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ns = p.n_max;
  const int slot_bytes = DWS ? kEmitSlotBytesDW : kEmitSlotBytes;
  char* const region = reinterpret_cast<char*>(smem4) + (size_t)warp * (ns * slot_bytes + p.max_dyads * 48);
  float4* const Rw = reinterpret_cast<float4*>(region + ns * slot_bytes);  // the row's dyad records
  char* const Pb = region + lane * 8;
  char* const Eb = region + ns * 256 + lane * 4;
  float4* const Fb = reinterpret_cast<float4*>(region + ns * 384);  // absolute fixed joints (warp)
  char* const Yb = region + ns * 400 + lane * 8;                    // DWS: double-word y
  int* const jofs = s_jofs[warp];
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t rows = full ? B : min((int64_t)p.ctrs[kNValid], out_capacity);
  const float nanf_ = __int_as_float(0x7fc00000);
  unsigned n_steps = 0, n_dw = 0, n_dw_dyads = 0;  // census counts of this lane
  for (int64_t r = gw; r < rows; r += nw) {
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
    float2* trow = traj ? reinterpret_cast<float2*>(traj) + r * ns * T : nullptr;
    float2* prow = path ? reinterpret_cast<float2*>(path) + r * T : nullptr;
    // FP32 tolerance: the budget minus the rounding of the absolute output coordinates
    const float tol = fmaf(-2.0f * kU, fabsf(h.px_h) + fabsf(h.py_h) + h.bmax, kEmitBudget * h.lbox);
    const int nslot = nf + 1 + nd;
    __syncwarp();
    if (lane < nslot) jofs[lane] = (int)sj[lane] * T;
    for (int x = lane; x < 3 * nd; x += 32)
      Rw[x] = __ldg(reinterpret_cast<const float4*>(p.dyad + b * p.max_dyads) + x);
    __syncwarp();
    // fixed joints: FP32 relative (the lane's column) and double-word absolute (one
    // copy per warp)
    if (ok) {
      const dw px = {h.px_h, h.px_l}, py = {h.py_h, h.py_l};
      const float4* fr = p.fixpos + b * ns;
      for (int s = 0; s < nf; ++s) {
        float4 f = __ldg(fr + s);
        *reinterpret_cast<float2*>(Pb + s * 256) = make_float2(f.x, f.z);
        *reinterpret_cast<float*>(Eb + s * 128) = h.e_fixed;
        if (lane == s) {
          dw x = dw_add(px, dw{f.x, f.y}), y = dw_add(py, dw{f.z, f.w});
          Fb[s] = make_float4(x.h, x.l, y.h, y.l);
        }
      }
    }
    __syncwarp();
    for (int t0 = 0; t0 < T; t0 += 32) {
      const int t = t0 + lane;
      if (t >= T) continue;
      if (t < lock) {
        const float4 csv = __ldg(cs + t);
        *reinterpret_cast<float2*>(Pb + nf * 256) =
            make_float2(csv.x * h.ux_h - csv.z * h.uy_h, csv.z * h.ux_h + csv.x * h.uy_h);
        *reinterpret_cast<float*>(Eb + nf * 128) = h.e_motor;
        float lockw = INFINITY, zmin = INFINITY, isgmax = 0.0f, emax = 0.0f;
        for (int d = 0; d < nd; ++d) fp32_dyad<true>(rec + d, Pb, Eb, lockw, zmin, isgmax, &emax);
        if (CENSUS) {
          ++n_steps;
          if (!(emax <= tol && zmin >= 0.0f)) {
            ++n_dw;
            n_dw_dyads += nd;
          }
          continue;
        }
        if (emax <= tol && zmin >= 0.0f) {
          for (int s = 0; s < nslot; ++s) {
            const float2 q = *reinterpret_cast<const float2*>(Pb + s * 256);
            const float2 v = make_float2(q.x + h.px_h, q.y + h.py_h);
            if (trow) trow[jofs[s] + t] = v;
            if (prow && s == h.coupler_slot) prow[t] = v;
          }
        } else {
          dwp lbuf[DWS ? 1 : kMaxJ];
          const auto loc = [&] {
            if constexpr (DWS) return LocShared{Pb, Yb};
            else return LocLocal{lbuf};
          }();
          float qd;
          bool lk = dw_chain<true>(h, Fb, rec, csv, loc, &qd);
          if (lk) atomicOr(err, kErrEmitLock);
          for (int s = 0; s < nslot; ++s) {
            const dwp ls = slot_pos(loc, Fb, nf, s);
            float2 v = lk ? make_float2(nanf_, nanf_) : make_float2(ls.x.h, ls.y.h);
            if (trow) trow[jofs[s] + t] = v;
            if (prow && s == h.coupler_slot) prow[t] = v;
          }
        }
      } else if (!CENSUS) {
        for (int s = 0; s < n; ++s)
          if (trow) trow[(int64_t)sj[s] * T + t] = make_float2(nanf_, nanf_);
        if (prow) prow[t] = make_float2(nanf_, nanf_);
      }
      if (!CENSUS)
        for (int j = n; j < ns; ++j)
          if (trow) trow[(int64_t)j * T + t] = make_float2(nanf_, nanf_);
    }
  }
  if (CENSUS) {
    add_stat(p.ctrs, kStatEmitSteps, n_steps);
    add_stat(p.ctrs, kStatEmitDW, n_dw);
    add_stat(p.ctrs, kStatEmitDWDyads, n_dw_dyads);
  }
}

// Shapes of the screen: lanes per mechanism G, steps per lane S, CTAs per SM (0 = as many
// as fit).
struct ScreenShape {
  int G = 8, S = 1, ctas = 0;
  bool defer = false;
};

// The screen in two launches: the deferring screen over the work list, then the
// rescuing screen over the mechanisms it left (p.rescue, a list usually a few percent
// long; the persistent grid's idle CTAs exit at once).
template <int G, int S>
int launch_screen(links_ctx ctx, links_plan plan, int T, const TTable* tab, uint8_t* valid, int16_t* lock_step,
                  float* min_disc, const int32_t* order, const int32_t* n_list, int ctas, bool defer) {
  PlanDev& p = plan->d;
  size_t smem = (size_t)kWarps * (p.n_max * 384 * S + (32 / G) * (2 * p.max_dyads + 1) * 16);
  // a function attribute of the current device's context: set on every launch (a host
  // call, no stream work), so other devices and contexts get it too
  LINKS_CUDA(cudaFuncSetAttribute(screen_kernel<G, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  LINKS_CUDA(cudaFuncSetAttribute(screen_kernel<G, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  int per_sm = 0;
  LINKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, screen_kernel<G, S, false>, kBlock, smem));
  if (ctas > 0 && ctas < per_sm) per_sm = ctas;
  if (per_sm < 1) per_sm = 1;
  LINKS_CUDA(cudaMemsetAsync(p.ctrs + kWork, 0, sizeof(int32_t), ctx->stream));
  if (!defer) {
    KernelScope ks(ctx, "mixed_screen");
    screen_kernel<G, S, true><<<ctx->num_sms * per_sm, kBlock, smem, ctx->stream>>>(
        p, T, tab->cs, valid, lock_step, min_disc, order ? order : p.order, n_list);
    LINKS_CUDA(cudaGetLastError());
    return LINKS_OK;
  }
  LINKS_CUDA(cudaMemsetAsync(p.ctrs + kNRescue, 0, sizeof(int32_t), ctx->stream));
  {
    KernelScope ks(ctx, "mixed_screen");
    screen_kernel<G, S, false><<<ctx->num_sms * per_sm, kBlock, smem, ctx->stream>>>(
        p, T, tab->cs, valid, lock_step, min_disc, order ? order : p.order, n_list);
  }
  LINKS_CUDA(cudaGetLastError());
  LINKS_CUDA(cudaMemsetAsync(p.ctrs + kWork, 0, sizeof(int32_t), ctx->stream));
  {
    KernelScope ks(ctx, "mixed_screen_rescue");
    screen_kernel<G, S, true><<<ctx->num_sms * per_sm, kBlock, smem, ctx->stream>>>(
        p, T, tab->cs, valid, lock_step, min_disc, p.rescue, p.ctrs + kNRescue);
  }
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

// Two steps per lane need the doubled slot arrays in shared memory (at most 16 slots).
constexpr int kScreenTwoStepLimit = 16;

ScreenShape screen_shape(links_ctx ctx, int n_max) {
  const Tuning t = tuning_of(ctx, n_max);
  ScreenShape sh;
  sh.G = t.screen_lanes;
  sh.S = t.screen_steps ? t.screen_steps : (n_max <= kScreenTwoStepMaxSlots ? 2 : 1);
  if (n_max > kScreenTwoStepLimit) sh.S = 1;
  sh.ctas = t.screen_ctas;
  sh.defer = t.screen_defer != 0;
  return sh;
}

int launch_screen_shape(links_ctx ctx, links_plan plan, int T, const TTable* tab, uint8_t* valid,
                        int16_t* lock_step, float* min_disc, const ScreenShape& sh,
                        const int32_t* order = nullptr, const int32_t* n_list = nullptr) {
  const int c = sh.ctas;
  if (sh.S == 2) {
    if (sh.G == 32) return launch_screen<32, 2>(ctx, plan, T, tab, valid, lock_step, min_disc, order, n_list, c, sh.defer);
    if (sh.G == 16) return launch_screen<16, 2>(ctx, plan, T, tab, valid, lock_step, min_disc, order, n_list, c, sh.defer);
    return launch_screen<8, 2>(ctx, plan, T, tab, valid, lock_step, min_disc, order, n_list, c, sh.defer);
  }
  if (sh.G == 32) return launch_screen<32, 1>(ctx, plan, T, tab, valid, lock_step, min_disc, order, n_list, c, sh.defer);
  if (sh.G == 16) return launch_screen<16, 1>(ctx, plan, T, tab, valid, lock_step, min_disc, order, n_list, c, sh.defer);
  return launch_screen<8, 1>(ctx, plan, T, tab, valid, lock_step, min_disc, order, n_list, c, sh.defer);
}

int launch_screen_tuned(links_ctx ctx, links_plan plan, int T, const TTable* tab, uint8_t* valid,
                        int16_t* lock_step, float* min_disc, const int32_t* order = nullptr,
                        const int32_t* n_list = nullptr) {
  return launch_screen_shape(ctx, plan, T, tab, valid, lock_step, min_disc, screen_shape(ctx, plan->d.n_max), order,
                             n_list);
}

// After the low-fidelity pass: the mechanisms it found valid go, in work-list order
// within each block, to the confirmation list; the others keep their verdict, their
// lock step scaled to the fine grid (a locking step there: the coarse angles are fine
// grid angles).
__global__ void __launch_bounds__(256) confirm_list_kernel(PlanDev p, const uint8_t* __restrict__ valid,
                                                           int16_t* __restrict__ lock_step, int ratio) {
  __shared__ int base;
  int n_ok = 0;
  for (int i = 0; i < 32; ++i) n_ok += p.ctrs[kHist + i];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int b = -1;
  bool keep = false;
  if (i < n_ok) {
    b = p.order[i];
    keep = valid[b] != 0;
    if (!keep && lock_step[b] >= 0) lock_step[b] = (int16_t)(lock_step[b] * ratio);
  }
  // block-aggregated append: one atomic per block, positions in work-list order
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  __shared__ int wcount[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) wcount[warp] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < 8; ++w) {
      const int c = wcount[w];
      wcount[w] = tot;
      tot += c;
    }
    base = tot ? atomicAdd(&p.ctrs[kNConfirm], tot) : 0;
  }
  __syncthreads();
  if (keep) p.order2[base + wcount[warp] + __popc(m & ((1u << lane) - 1u))] = b;
}

}  // namespace

// Shapes of the emit: double-word slots in shared memory or thread-local, CTAs per SM.
struct EmitShape {
  bool dws = true;
  int ctas = 0;
};

EmitShape emit_shape(links_ctx ctx, int n_max) {
  const Tuning t = tuning_of(ctx, n_max);
  EmitShape e;
  e.dws = t.emit_dws < 0 ? n_max <= kEmitSharedDWMaxSlots : t.emit_dws != 0;
  e.ctas = t.emit_ctas;
  return e;
}

template <bool CENSUS>
int launch_emit(links_ctx ctx, links_plan plan, const TTable* tab, bool full, const int16_t* lock_step,
                const int32_t* out_index, int64_t out_capacity, float* traj, float* path, const char* name,
                const EmitShape* shape = nullptr) {
  const EmitShape sh = shape ? *shape : emit_shape(ctx, plan->d.n_max);
  const bool dws = sh.dws;
  auto kern = dws ? emit_kernel<CENSUS, true> : emit_kernel<CENSUS, false>;
  const size_t smem = (size_t)kWarps * (plan->d.n_max * (dws ? kEmitSlotBytesDW : kEmitSlotBytes) +
                                        plan->d.max_dyads * 48);
  if (smem > 48 * 1024)
    LINKS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LINKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem));
  if (sh.ctas > 0 && sh.ctas < per_sm) per_sm = sh.ctas;
  if (per_sm < 1) per_sm = 1;
  KernelScope ks(ctx, name);
  kern<<<ctx->num_sms * per_sm, kBlock, smem, ctx->stream>>>(plan->d, plan->B, tab->T, tab->cs, full ? 1 : 0,
                                                            lock_step, out_index, out_capacity, traj, path,
                                                            ctx->d_err);
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

// Autotuner: times the screen over its shapes (lanes per mechanism 8/16/32, one or two
// steps per lane, CTAs per SM) on the built plan, then the emit over its shapes
// (double-word slots in shared memory or thread-local, CTAs per SM) on up to
// kTuneRows valid rows of that screen's result, and keeps the fastest of each in the
// context's table for this n_max.  Each shape runs once to warm up and twice timed.
constexpr int64_t kTuneRows = 16384;

int autotune(links_ctx ctx, links_plan plan, const TTable* tab, int* lanes_out) {
  const int64_t B = std::max<int64_t>(plan->B, 1);
  const int n_max = plan->d.n_max, T = tab->T;
  uint8_t* v = nullptr;
  int16_t* l = nullptr;
  float *q = nullptr, *traj = nullptr, *path = nullptr;
  int32_t *idx = nullptr, *nout = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = LINKS_OK;
  cudaError_t e = cudaMalloc(&v, B);
  if (e == cudaSuccess) e = cudaMalloc(&l, 2 * B);
  if (e == cudaSuccess) e = cudaMalloc(&q, 4 * B);
  if (e == cudaSuccess) e = cudaMalloc(&idx, 4 * B);
  if (e == cudaSuccess) e = cudaMalloc(&nout, 4);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) st = cuda_status(e, "links_autotune");
  auto timed = [&](auto&& run) -> float {  // warm-up + 2 timed runs, ms (huge on failure)
    float total = 0.f;
    for (int rep = 0; rep < 3 && !st; ++rep) {
      cudaEventRecord(e0, ctx->stream);
      st = run();
      cudaEventRecord(e1, ctx->stream);
      if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = set_error(LINKS_ECUDA, "links_autotune: run failed");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) total += ms;
    }
    return st ? 1e30f : total;
  };
  Tuning best = tuning_of(ctx, n_max);
  float best_ms = 1e30f;
  ScreenShape best_sh = screen_shape(ctx, n_max);
  for (int S : {1, 2}) {
    if (S == 2 && n_max > kScreenTwoStepLimit) continue;
    for (int G : {8, 16, 32})
      for (int ctas : {0, 2, 1})
        for (int defer : {0, 1}) {
          if (st) break;
          ScreenShape sh{G, S, ctas, defer != 0};
          const float ms = timed([&] { return launch_screen_shape(ctx, plan, T, tab, v, l, q, sh); });
          if (ms < best_ms) {
            best_ms = ms;
            best_sh = sh;
          }
        }
  }
  if (!st) {
    best.screen_lanes = best_sh.G;
    best.screen_steps = best_sh.S;
    best.screen_ctas = best_sh.ctas;
    best.screen_defer = best_sh.defer ? 1 : 0;
    // the emit on up to kTuneRows valid rows of the chosen screen's result
    st = launch_screen_shape(ctx, plan, T, tab, v, l, q, best_sh);
    if (!st) st = compact_valid(ctx, plan, v, idx, B, nout);
    int32_t nv = 0;
    if (!st && cudaMemcpyAsync(&nv, nout, 4, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
      st = set_error(LINKS_ECUDA, "links_autotune: copy failed");
    if (!st && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
      st = set_error(LINKS_ECUDA, "links_autotune: screen failed");
    const int64_t R = std::min<int64_t>(nv, kTuneRows);
    if (!st && R > 0) {
      e = cudaMalloc(&traj, sizeof(float) * 2 * R * n_max * T);
      if (e == cudaSuccess) e = cudaMalloc(&path, sizeof(float) * 2 * R * T);
      if (e != cudaSuccess) st = cuda_status(e, "links_autotune");
      float emit_best = 1e30f;
      for (int dws : {1, 0})
        for (int ctas : {0, 2, 1}) {
          if (st) break;
          EmitShape es{dws != 0, ctas};
          const float ms = timed([&] {
            return launch_emit<false>(ctx, plan, tab, false, l, idx, R, traj, path, "mixed_emit", &es);
          });
          if (ms < emit_best) {
            emit_best = ms;
            best.emit_dws = dws;
            best.emit_ctas = ctas;
          }
        }
    }
  }
  if (!st) {
    ctx->tuning[n_max] = best;
    if (lanes_out) *lanes_out = best.screen_lanes;
  }
  cudaFree(v);
  cudaFree(l);
  cudaFree(q);
  cudaFree(idx);
  cudaFree(nout);
  cudaFree(traj);
  cudaFree(path);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

Tuning tuning_of(links_ctx ctx, int n_max) {
  auto it = ctx->tuning.find(n_max);
  return it == ctx->tuning.end() ? Tuning{} : it->second;
}

int simulate_mixed(links_ctx ctx, links_plan plan, const TTable* tab, int out_mode, float* traj,
                   float* path, uint8_t* valid, int16_t* lock_step, float* min_disc,
                   int32_t* out_index, int64_t out_capacity, int32_t* n_out) {
  const int T = tab->T;
  int st = fill_unsimulated(ctx, plan, valid, lock_step, min_disc);
  if (st) return st;
  st = launch_screen_tuned(ctx, plan, T, tab, valid, lock_step, min_disc);
  if (st) return st;
  const bool full = out_mode == LINKS_OUT_FULL;
  if (!full) {
    st = compact_valid(ctx, plan, valid, out_index, out_capacity, n_out);
    if (st) return st;
  }
  if (traj || path)
    return launch_emit<false>(ctx, plan, tab, full, lock_step, out_index, out_capacity, traj, path, "mixed_emit");
  return LINKS_OK;
}

// The mixed simulation with the screen done first by `prescreen`, which decides the OK
// mechanisms it can and lists the others in p.order2 (their count in
// p.ctrs[kNConfirm]); the generic screen takes that list, then compaction and emit.
int simulate_prescreened(links_ctx ctx, links_plan plan, const TTable* tab, int out_mode, float* traj,
                         float* path, uint8_t* valid, int16_t* lock_step, float* min_disc, int32_t* out_index,
                         int64_t out_capacity, int32_t* n_out, int32_t* n_escaped, const Prescreen& prescreen) {
  PlanDev& p = plan->d;
  int st = fill_unsimulated(ctx, plan, valid, lock_step, min_disc);
  if (st) return st;
  LINKS_CUDA(cudaMemsetAsync(p.ctrs + kNConfirm, 0, sizeof(int32_t), ctx->stream));
  st = prescreen(ctx, plan, tab, valid, lock_step, min_disc);
  if (st) return st;
  if (n_escaped)
    LINKS_CUDA(cudaMemcpyAsync(n_escaped, p.ctrs + kNConfirm, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                               ctx->stream));
  st = launch_screen_tuned(ctx, plan, tab->T, tab, valid, lock_step, min_disc, p.order2, p.ctrs + kNConfirm);
  if (st) return st;
  const bool full = out_mode == LINKS_OUT_FULL;
  if (!full) {
    st = compact_valid(ctx, plan, valid, out_index, out_capacity, n_out);
    if (st) return st;
  }
  if (traj || path)
    return launch_emit<false>(ctx, plan, tab, full, lock_step, out_index, out_capacity, traj, path, "mixed_emit");
  return LINKS_OK;
}

// Low-fidelity screen on the coarse grid (tab_lo), confirmation on the fine grid (tab)
// of the mechanisms valid on the coarse one, then valid-row compaction and emit.
int simulate_two_stage(links_ctx ctx, links_plan plan, const TTable* tab_lo, const TTable* tab, float* traj,
                       float* path, uint8_t* valid, int16_t* lock_step, float* min_disc, int32_t* out_index,
                       int64_t out_capacity, int32_t* n_out, int32_t* n_low_valid) {
  PlanDev& p = plan->d;
  int st = fill_unsimulated(ctx, plan, valid, lock_step, min_disc);
  if (st) return st;
  st = launch_screen_tuned(ctx, plan, tab_lo->T, tab_lo, valid, lock_step, min_disc);
  if (st) return st;
  LINKS_CUDA(cudaMemsetAsync(p.ctrs + kNConfirm, 0, sizeof(int32_t), ctx->stream));
  if (plan->B > 0) {
    KernelScope ks(ctx, "confirm_list");
    confirm_list_kernel<<<(unsigned)((plan->B + 255) / 256), 256, 0, ctx->stream>>>(p, valid, lock_step,
                                                                                   tab->T / tab_lo->T);
    LINKS_CUDA(cudaGetLastError());
  }
  if (n_low_valid)
    LINKS_CUDA(cudaMemcpyAsync(n_low_valid, p.ctrs + kNConfirm, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                               ctx->stream));
  st = launch_screen_tuned(ctx, plan, tab->T, tab, valid, lock_step, min_disc, p.order2, p.ctrs + kNConfirm);
  if (st) return st;
  st = compact_valid(ctx, plan, valid, out_index, out_capacity, n_out);
  if (st) return st;
  if (traj || path)
    return launch_emit<false>(ctx, plan, tab, false, lock_step, out_index, out_capacity, traj, path, "mixed_emit");
  return LINKS_OK;
}

int emit_census(links_ctx ctx, links_plan plan, const TTable* tab, int out_mode, const int16_t* lock_step,
                const int32_t* out_index, int64_t out_capacity, int64_t* out) {
  PlanDev& p = plan->d;
  LINKS_CUDA(cudaMemsetAsync(p.ctrs + kStatEmitSteps, 0, 6 * sizeof(int32_t), ctx->stream));
  int st = launch_emit<true>(ctx, plan, tab, out_mode == LINKS_OUT_FULL, lock_step, out_index, out_capacity,
                             nullptr, nullptr, "emit_census");
  if (st) return st;
  unsigned long long v[3];
  LINKS_CUDA(cudaMemcpyAsync(v, p.ctrs + kStatEmitSteps, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
  LINKS_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < 3; ++i) out[i] = (int64_t)v[i];
  return LINKS_OK;
}

}  // namespace links
