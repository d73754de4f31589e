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
#include "sim_core.cuh"

namespace links {
namespace {

// The kernels: one block's warps run the bodies of sim_core.cuh.
template <int G, int S, bool RESCUE>
__global__ void __launch_bounds__(kBlock, 4) screen_kernel(PlanDev p, int T, const float4* __restrict__ cs,
                                                        uint8_t* __restrict__ valid,
                                                        int16_t* __restrict__ lock_step,
                                                        float* __restrict__ min_disc,
                                                        const int32_t* __restrict__ order,
                                                        const int32_t* __restrict__ n_list, int batch) {
  extern __shared__ float4 smem4[];
  screen_body<G, S, RESCUE>(p, T, cs, valid, lock_step, min_disc, order, n_list, reinterpret_cast<char*>(smem4),
                            threadIdx.x >> 5, threadIdx.x & 31, batch);
}

template <bool CENSUS, bool DWS>
__global__ void __launch_bounds__(kBlock) emit_kernel(PlanDev p, int64_t B, int T, const float4* __restrict__ cs,
                                                      int full, const int16_t* __restrict__ lock_step,
                                                      const int32_t* __restrict__ out_index,
                                                      int64_t out_capacity, float* __restrict__ traj,
                                                      float* __restrict__ path, int32_t* err,
                                                      const int64_t* __restrict__ row_off, int64_t traj_cap) {
  extern __shared__ float4 smem4[];
  __shared__ int s_jofs[kWarps][kMaxJ];  // per warp: offset of each slot's joint row in the output row
  const int warp = threadIdx.x >> 5;
  emit_body<CENSUS, DWS>(p, B, T, cs, full, lock_step, out_index, out_capacity, traj, path, err,
                         reinterpret_cast<char*>(smem4), s_jofs[warp], warp, threadIdx.x & 31,
                         ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                         ((int64_t)gridDim.x * blockDim.x) >> 5, row_off, traj_cap, p.ctrs + kWork2);
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
  size_t smem = (size_t)kWarps * screen_warp_bytes(p.n_max, p.max_dyads, G, S);
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
        p, T, tab->cs, valid, lock_step, min_disc, order ? order : p.order, n_list, kBatch);
    LINKS_CUDA(cudaGetLastError());
    return LINKS_OK;
  }
  LINKS_CUDA(cudaMemsetAsync(p.ctrs + kNRescue, 0, sizeof(int32_t), ctx->stream));
  {
    KernelScope ks(ctx, "mixed_screen");
    screen_kernel<G, S, false><<<ctx->num_sms * per_sm, kBlock, smem, ctx->stream>>>(
        p, T, tab->cs, valid, lock_step, min_disc, order ? order : p.order, n_list, kBatch);
  }
  LINKS_CUDA(cudaGetLastError());
  LINKS_CUDA(cudaMemsetAsync(p.ctrs + kWork, 0, sizeof(int32_t), ctx->stream));
  {
    KernelScope ks(ctx, "mixed_screen_rescue");
    // The rescue list is short and unsorted: one item per atomic keeps the warps' tails even.
    screen_kernel<G, S, true><<<ctx->num_sms * per_sm, kBlock, smem, ctx->stream>>>(
        p, T, tab->cs, valid, lock_step, min_disc, p.rescue, p.ctrs + kNRescue, 1);
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
                const EmitShape* shape = nullptr, const int64_t* row_off = nullptr, int64_t traj_cap = 0) {
  const EmitShape sh = shape ? *shape : emit_shape(ctx, plan->d.n_max);
  const bool dws = sh.dws;
  auto kern = dws ? emit_kernel<CENSUS, true> : emit_kernel<CENSUS, false>;
  const size_t smem = (size_t)kWarps * emit_warp_bytes(plan->d.n_max, plan->d.max_dyads, dws);
  if (smem > 48 * 1024)
    LINKS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LINKS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem));
  if (sh.ctas > 0 && sh.ctas < per_sm) per_sm = sh.ctas;
  if (per_sm < 1) per_sm = 1;
  LINKS_CUDA(cudaMemsetAsync(plan->d.ctrs + kWork2, 0, sizeof(int32_t), ctx->stream));
  KernelScope ks(ctx, name);
  kern<<<ctx->num_sms * per_sm, kBlock, smem, ctx->stream>>>(plan->d, plan->B, tab->T, tab->cs, full ? 1 : 0,
                                                            lock_step, out_index, out_capacity, traj, path,
                                                            ctx->d_err, row_off, traj_cap);
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

// Autotuner: times the screen over its shapes (lanes per mechanism 8/16/32, one or two
// steps per lane, CTAs per SM, inline or deferred rescue) on the built plan, then the
// emit over its shapes (double-word slots in shared memory or thread-local, CTAs per
// SM) on up to kTuneRows packed valid rows of that screen's result, and keeps the
// fastest of each in the context's table for this n_max.  Each shape runs once to warm
// up and three times timed.
constexpr int64_t kTuneRows = 262144;

int autotune(links_ctx ctx, links_plan plan, const TTable* tab, int* lanes_out) {
  const int64_t B = std::max<int64_t>(plan->B, 1);
  const int n_max = plan->d.n_max, T = tab->T;
  uint8_t* v = nullptr;
  int16_t* l = nullptr;
  float *q = nullptr, *traj = nullptr, *path = nullptr;
  int32_t *idx = nullptr, *nout = nullptr;
  int64_t* row_off = nullptr;
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
  auto timed = [&](auto&& run) -> float {  // warm-up + 3 timed runs, ms (huge on failure)
    float total = 0.f;
    for (int rep = 0; rep < 4 && !st; ++rep) {
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
    if (!st && R > 0) {  // packed rows (their joints only), as links_simulate_packed writes them
      e = cudaMalloc(&row_off, sizeof(int64_t) * (R + 1));
      if (e != cudaSuccess) st = cuda_status(e, "links_autotune");
      if (!st) st = pack_offsets(ctx, plan, idx, R, row_off);
      int64_t J = 0;
      if (!st && cudaMemcpyAsync(&J, row_off + R, 8, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        st = set_error(LINKS_ECUDA, "links_autotune: copy failed");
      if (!st && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        st = set_error(LINKS_ECUDA, "links_autotune: offsets failed");
      if (!st) {
        e = cudaMalloc(&traj, sizeof(float) * 2 * std::max<int64_t>(J, 1) * T);
        if (e == cudaSuccess) e = cudaMalloc(&path, sizeof(float) * 2 * R * T);
        if (e != cudaSuccess) st = cuda_status(e, "links_autotune");
      }
      float emit_best = 1e30f;
      for (int dws : {1, 0})
        for (int ctas : {0, 2, 1}) {
          if (st) break;
          EmitShape es{dws != 0, ctas};
          const float ms = timed([&] {
            return launch_emit<false>(ctx, plan, tab, false, l, idx, R, traj, path, "mixed_emit", &es, row_off, J);
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
  cudaFree(row_off);
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
                   int32_t* out_index, int64_t out_capacity, int32_t* n_out, int64_t* row_offset,
                   int64_t traj_capacity) {
  const int T = tab->T;
  int st = fill_unsimulated(ctx, plan, valid, lock_step, min_disc);
  if (st) return st;
  st = launch_screen_tuned(ctx, plan, T, tab, valid, lock_step, min_disc);
  if (st) return st;
  const bool full = out_mode == LINKS_OUT_FULL;
  if (!full) {
    st = compact_valid(ctx, plan, valid, out_index, out_capacity, n_out);
    if (st) return st;
    if (row_offset) {
      st = pack_offsets(ctx, plan, out_index, out_capacity, row_offset);
      if (st) return st;
    }
  }
  if (traj || path)
    return launch_emit<false>(ctx, plan, tab, full, lock_step, out_index, out_capacity, traj, path, "mixed_emit",
                              nullptr, full ? nullptr : row_offset, traj_capacity);
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
