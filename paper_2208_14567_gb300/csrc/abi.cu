// abi.cu -- the extern "C" boundary declared in include/links.h: contexts, plans,
// actuator tables, simulation dispatch, graph capture and error reporting.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "links_internal.cuh"

namespace links {

namespace {
thread_local std::string g_last_error;

__global__ void table_kernel(int T, float4* cs, double2* cs64) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double s, c;
  sincospi(2.0 * (double)t / (double)T, &s, &c);  // angle 2*pi*t/T
  cs64[t] = make_double2(c, s);
  dw ch = dw_from_double(c), sh = dw_from_double(s);
  cs[t] = make_float4(ch.h, ch.l, sh.h, sh.l);
}
}  // namespace

int set_error(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_status(cudaError_t e, const char* what) {
  int st = (e == cudaErrorMemoryAllocation) ? LINKS_ENOMEM : LINKS_ECUDA;
  return set_error(st, std::string(what) + ": " + cudaGetErrorString(e));
}

static cudaEvent_t take_event(links_ctx ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

KernelScope::KernelScope(links_ctx c, const char* name) : ctx(c) {
  ++ctx->launches;
  if (!ctx->prof) return;
  cudaEvent_t a = take_event(ctx);
  b = take_event(ctx);
  if (!a || !b) {
    b = nullptr;
    return;
  }
  cudaEventRecord(a, ctx->stream);
  ctx->pending.push_back({name, a, b});
}

KernelScope::~KernelScope() {
  if (b) cudaEventRecord(b, ctx->stream);
}

int ensure_workspace(links_ctx ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return LINKS_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(ctx->stream, &cap);
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(LINKS_ESTATE, "workspace too small inside a graph capture: call links_workspace_reserve first");
  LINKS_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  LINKS_CUDA(cudaMalloc(&ctx->ws, bytes));
  ctx->ws_bytes = bytes;
  return LINKS_OK;
}

const TTable* get_table(links_ctx ctx, int T, int* status) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->tables.find(T);
  if (it != ctx->tables.end()) return &it->second;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(ctx->stream, &cap);
  if (cap != cudaStreamCaptureStatusNone) {
    *status = set_error(LINKS_ESTATE, "links_prepare(T) must run before capturing a new T");
    return nullptr;
  }
  TTable tab;
  tab.T = T;
  cudaError_t e = cudaMalloc(&tab.cs, sizeof(float4) * T);
  if (e == cudaSuccess) e = cudaMalloc(&tab.cs64, sizeof(double2) * T);
  if (e != cudaSuccess) {
    cudaFree(tab.cs);
    *status = cuda_status(e, "cudaMalloc(actuator table)");
    return nullptr;
  }
  {
    KernelScope ks(ctx, "actuator_table");
    table_kernel<<<(T + 255) / 256, 256, 0, ctx->stream>>>(T, tab.cs, tab.cs64);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    *status = cuda_status(e, "table_kernel");
    return nullptr;
  }
  auto res = ctx->tables.emplace(T, tab);
  return &res.first->second;
}

}  // namespace links

using namespace links;

extern "C" {

const char* links_last_error(void) { return g_last_error.c_str(); }

const char* links_strerror(int status) {
  switch (status) {
    case LINKS_OK: return "LINKS_OK";
    case LINKS_EINVAL: return "LINKS_EINVAL";
    case LINKS_ECUDA: return "LINKS_ECUDA";
    case LINKS_ENOMEM: return "LINKS_ENOMEM";
    case LINKS_ECAPACITY: return "LINKS_ECAPACITY";
    case LINKS_EBUSY: return "LINKS_EBUSY";
    case LINKS_ETIMEDOUT: return "LINKS_ETIMEDOUT";
    case LINKS_ESTATE: return "LINKS_ESTATE";
    case LINKS_EDEVICE: return "LINKS_EDEVICE";
    default: return "LINKS_UNKNOWN";
  }
}

int links_create(links_ctx* out, int device, void* cuda_stream) {
  if (!out) return set_error(LINKS_EINVAL, "links_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  LINKS_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_error(LINKS_EINVAL, "links_create: bad device index");
  LINKS_CUDA(cudaSetDevice(device));
  links_ctx c = new (std::nothrow) links_ctx_s();
  if (!c) return set_error(LINKS_ENOMEM, "links_create: host allocation");
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int32_t));
  if (e != cudaSuccess) {
    if (c->d_err) cudaFree(c->d_err);
    delete c;
    return cuda_status(e, "links_create");
  }
  *out = c;
  return LINKS_OK;
}

int links_destroy(links_ctx ctx) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_destroy: NULL ctx");
  if (ctx->serve) links_serve_stop(ctx);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->tables) {
    cudaFree(kv.second.cs);
    cudaFree(kv.second.cs64);
  }
  for (auto& r : ctx->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  if (ctx->ws) cudaFree(ctx->ws);
  cudaFree(ctx->d_err);
  delete ctx;
  return LINKS_OK;
}

int links_set_stream(links_ctx ctx, void* cuda_stream) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_set_stream: NULL ctx");
  ctx->stream = (cudaStream_t)cuda_stream;
  return LINKS_OK;
}

int links_sync(links_ctx ctx) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_sync: NULL ctx");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  LINKS_CUDA(cudaStreamSynchronize(ctx->stream));
  int32_t e = 0;
  LINKS_CUDA(cudaMemcpy(&e, ctx->d_err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e) {
    LINKS_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int32_t)));
    char buf[96];
    snprintf(buf, sizeof buf, "device error word 0x%x (1 = emit/screen disagreement, 2 = bad index)", e);
    return set_error(LINKS_EDEVICE, buf);
  }
  return LINKS_OK;
}

int links_prepare(links_ctx ctx, int T) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_prepare: NULL ctx");
  if (T < 1 || T > LINKS_MAX_T) return set_error(LINKS_EINVAL, "links_prepare: T out of [1, 32767]");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  int st = LINKS_OK;
  return get_table(ctx, T, &st) ? LINKS_OK : st;
}

int links_plan_create(links_ctx ctx, int64_t capacity, int n_max, links_plan* out) {
  if (!ctx || !out) return set_error(LINKS_EINVAL, "links_plan_create: NULL argument");
  *out = nullptr;
  if (capacity < 0 || capacity > (int64_t)INT32_MAX)
    return set_error(LINKS_EINVAL, "links_plan_create: capacity out of [0, 2^31)");
  if (n_max < 2 || n_max > LINKS_MAX_JOINTS)
    return set_error(LINKS_EINVAL, "links_plan_create: n_max out of [2, 32]");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  links_plan p = new (std::nothrow) links_plan_s();
  if (!p) return set_error(LINKS_ENOMEM, "links_plan_create: host allocation");
  p->ctx = ctx;
  PlanDev& d = p->d;
  d.n_max = n_max;
  d.max_dyads = std::max(1, n_max - 2);
  d.cap = capacity;
  const int64_t c = std::max<int64_t>(capacity, 1);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  alloc((void**)&d.hdr, sizeof(MechHdr) * c);
  alloc((void**)&d.slot_joint, (size_t)kMaxJ * c);
  alloc((void**)&d.fixpos, sizeof(float4) * n_max * c);
  alloc((void**)&d.pos64, sizeof(double2) * n_max * c);
  alloc((void**)&d.dyad, sizeof(DyadRec) * d.max_dyads * c);
  alloc((void**)&d.order, sizeof(int32_t) * c);
  alloc((void**)&d.order2, sizeof(int32_t) * c);
  alloc((void**)&d.rescue, sizeof(int32_t) * c);
  alloc((void**)&d.ctrs, sizeof(int32_t) * kCtrs);
  alloc((void**)&d.scan, sizeof(int32_t) * (c / 1024 + 2));
  alloc((void**)&d.scan64, sizeof(int64_t) * (c / 1024 + 2));
  if (e == cudaSuccess) e = cudaMemset(d.ctrs, 0, sizeof(int32_t) * kCtrs);
  if (e != cudaSuccess) {
    links_plan_free(p);
    return cuda_status(e, "links_plan_create");
  }
  *out = p;
  return LINKS_OK;
}

int links_plan_free(links_plan plan) {
  if (!plan) return set_error(LINKS_EINVAL, "links_plan_free: NULL plan");
  PlanDev& d = plan->d;
  cudaFree(d.hdr);
  cudaFree(d.slot_joint);
  cudaFree(d.fixpos);
  cudaFree(d.pos64);
  cudaFree(d.dyad);
  cudaFree(d.order);
  cudaFree(d.order2);
  cudaFree(d.rescue);
  cudaFree(d.ctrs);
  cudaFree(d.scan);
  cudaFree(d.scan64);
  delete plan;
  return LINKS_OK;
}

static int check_build(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints, const uint8_t* adj,
                       const int8_t* type, const void* pos0, int pos_dtype, const char* who) {
  if (!ctx || !plan) return set_error(LINKS_EINVAL, std::string(who) + ": NULL ctx or plan");
  if (plan->ctx != ctx) return set_error(LINKS_EINVAL, std::string(who) + ": plan belongs to another context");
  if (B < 0) return set_error(LINKS_EINVAL, std::string(who) + ": B < 0");
  if (B > plan->d.cap) return set_error(LINKS_ECAPACITY, std::string(who) + ": B exceeds the plan capacity");
  if (pos_dtype != LINKS_F32 && pos_dtype != LINKS_F64)
    return set_error(LINKS_EINVAL, std::string(who) + ": pos_dtype must be LINKS_F32 or LINKS_F64");
  if (B > 0 && (!n_joints || !adj || !type || !pos0))
    return set_error(LINKS_EINVAL, std::string(who) + ": NULL input");
  return LINKS_OK;
}

int links_plan_build(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints, const uint8_t* adj,
                     const int8_t* type, const void* pos0, int pos_dtype, int32_t* status_out) {
  int st = check_build(ctx, plan, B, n_joints, adj, type, pos0, pos_dtype, "links_plan_build");
  if (st) return st;
  LINKS_CUDA(cudaSetDevice(ctx->device));
  return plan_build_device(ctx, plan, B, n_joints, adj, type, pos0, pos_dtype, status_out);
}

int links_plan_build_masks(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                           const uint32_t* nbr, const int8_t* type, const void* pos0, int pos_dtype,
                           int32_t* status_out) {
  int st = check_build(ctx, plan, B, n_joints, reinterpret_cast<const uint8_t*>(nbr), type, pos0, pos_dtype,
                       "links_plan_build_masks");
  if (st) return st;
  LINKS_CUDA(cudaSetDevice(ctx->device));
  return plan_build_device(ctx, plan, B, n_joints, nullptr, type, pos0, pos_dtype, status_out, nbr);
}

int links_plan_build_host(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                          const uint8_t* adj, const int8_t* type, const void* pos0, int pos_dtype,
                          int32_t* status_out) {
  int st = check_build(ctx, plan, B, n_joints, adj, type, pos0, pos_dtype, "links_plan_build_host");
  if (st) return st;
  LINKS_CUDA(cudaSetDevice(ctx->device));
  return plan_build_host(ctx, plan, B, n_joints, adj, type, pos0, pos_dtype, status_out);
}

int links_plan_info(links_plan plan, int64_t* B, int* n_max, int64_t* capacity) {
  if (!plan) return set_error(LINKS_EINVAL, "links_plan_info: NULL plan");
  if (B) *B = plan->B;
  if (n_max) *n_max = plan->d.n_max;
  if (capacity) *capacity = plan->d.cap;
  return LINKS_OK;
}

int links_plan_export(links_plan plan, int64_t b0, int64_t count, int32_t* topo, double* lengths) {
  if (!plan || !topo) return set_error(LINKS_EINVAL, "links_plan_export: NULL argument");
  if (b0 < 0 || count < 0 || b0 + count > plan->B)
    return set_error(LINKS_EINVAL, "links_plan_export: range outside the last build");
  if (count == 0) return LINKS_OK;
  const PlanDev& d = plan->d;
  links_ctx ctx = plan->ctx;
  LINKS_CUDA(cudaSetDevice(ctx->device));
  LINKS_CUDA(cudaStreamSynchronize(ctx->stream));
  std::vector<MechHdr> hdr(count);
  std::vector<uint8_t> sj((size_t)count * kMaxJ);
  std::vector<DyadRec> dy((size_t)count * d.max_dyads);
  LINKS_CUDA(cudaMemcpy(hdr.data(), d.hdr + b0, count * sizeof(MechHdr), cudaMemcpyDeviceToHost));
  LINKS_CUDA(cudaMemcpy(sj.data(), d.slot_joint + b0 * kMaxJ, sj.size(), cudaMemcpyDeviceToHost));
  LINKS_CUDA(cudaMemcpy(dy.data(), d.dyad + b0 * d.max_dyads, dy.size() * sizeof(DyadRec), cudaMemcpyDeviceToHost));
  const int md = d.n_max - 2 > 0 ? d.n_max - 2 : 0;
  const int w = 6 + 3 * md;
  for (int64_t m = 0; m < count; ++m) {
    int32_t* o = topo + m * w;
    for (int x = 0; x < w; ++x) o[x] = -1;
    const MechHdr& h = hdr[m];
    o[0] = h.status;
    o[1] = h.n;
    double* L = lengths ? lengths + m * 2 * md : nullptr;
    if (L) for (int x = 0; x < 2 * md; ++x) L[x] = NAN;
    if (h.status != LINKS_MECH_OK) continue;
    const uint8_t* s2j = &sj[m * kMaxJ];
    o[2] = h.motor_joint;
    o[3] = h.pivot_joint;
    o[4] = s2j[h.coupler_slot];
    o[5] = h.nd;
    for (int q = 0; q < h.nd && q < md; ++q) {
      const DyadRec& r = dy[m * d.max_dyads + q];
      uint32_t sl;
      memcpy(&sl, &r.r2.w, 4);
      o[6 + 3 * q] = (sl >> 16) & 0xff;
      o[7 + 3 * q] = s2j[sl & 0xff];
      o[8 + 3 * q] = s2j[(sl >> 8) & 0xff];
      if (L) {
        double r1sq = (double)r.r2.x + (double)r.r2.y;
        double c = (double)r.r0.w + (double)r.r2.z;
        L[2 * q] = r1sq;
        L[2 * q + 1] = r1sq - c;
      }
    }
  }
  return LINKS_OK;
}

int links_simulate(links_ctx ctx, links_plan plan, int T, int precision, int out_mode, void* traj, void* path,
                   uint8_t* valid, int16_t* lock_step, float* min_disc, int32_t* out_index,
                   int64_t out_capacity, int32_t* n_out) {
  if (!ctx || !plan) return set_error(LINKS_EINVAL, "links_simulate: NULL ctx or plan");
  if (plan->ctx != ctx) return set_error(LINKS_EINVAL, "links_simulate: plan belongs to another context");
  if (T < 1 || T > LINKS_MAX_T) return set_error(LINKS_EINVAL, "links_simulate: T out of [1, 32767]");
  if (precision != LINKS_PLAIN_F64 && precision != LINKS_MIXED)
    return set_error(LINKS_EINVAL, "links_simulate: unknown precision");
  if (out_mode != LINKS_OUT_FULL && out_mode != LINKS_OUT_VALID_ONLY)
    return set_error(LINKS_EINVAL, "links_simulate: unknown out_mode");
  if (plan->B > 0 && (!valid || !lock_step || !min_disc))
    return set_error(LINKS_EINVAL, "links_simulate: valid, lock_step and min_disc are required");
  if (out_mode == LINKS_OUT_VALID_ONLY) {
    if (out_capacity < 0) return set_error(LINKS_EINVAL, "links_simulate: out_capacity < 0");
    if ((traj || path) && out_capacity > 0 && !out_index)
      return set_error(LINKS_EINVAL, "links_simulate: VALID_ONLY rows need out_index");
  }
  LINKS_CUDA(cudaSetDevice(ctx->device));
  int st = LINKS_OK;
  const TTable* tab = get_table(ctx, T, &st);
  if (!tab) return st;
  if (precision == LINKS_PLAIN_F64)
    return simulate_f64(ctx, plan, tab, out_mode, (double*)traj, (double*)path, valid, lock_step, min_disc,
                        out_index, out_capacity, n_out);
  return simulate_mixed(ctx, plan, tab, out_mode, (float*)traj, (float*)path, valid, lock_step, min_disc,
                        out_index, out_capacity, n_out);
}

int links_simulate_packed(links_ctx ctx, links_plan plan, int T, int precision, void* traj, int64_t traj_capacity,
                          void* path, uint8_t* valid, int16_t* lock_step, float* min_disc, int32_t* out_index,
                          int64_t* row_offset, int64_t out_capacity, int32_t* n_out) {
  if (!ctx || !plan) return set_error(LINKS_EINVAL, "links_simulate_packed: NULL ctx or plan");
  if (plan->ctx != ctx) return set_error(LINKS_EINVAL, "links_simulate_packed: plan belongs to another context");
  if (T < 1 || T > LINKS_MAX_T) return set_error(LINKS_EINVAL, "links_simulate_packed: T out of [1, 32767]");
  if (precision != LINKS_PLAIN_F64 && precision != LINKS_MIXED)
    return set_error(LINKS_EINVAL, "links_simulate_packed: unknown precision");
  if (plan->B > 0 && (!valid || !lock_step || !min_disc))
    return set_error(LINKS_EINVAL, "links_simulate_packed: valid, lock_step and min_disc are required");
  if (out_capacity < 0 || traj_capacity < 0)
    return set_error(LINKS_EINVAL, "links_simulate_packed: negative capacity");
  if (!row_offset) return set_error(LINKS_EINVAL, "links_simulate_packed: row_offset is required");
  if (out_capacity > 0 && !out_index) return set_error(LINKS_EINVAL, "links_simulate_packed: rows need out_index");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  int st = LINKS_OK;
  const TTable* tab = get_table(ctx, T, &st);
  if (!tab) return st;
  if (precision == LINKS_PLAIN_F64)
    return simulate_f64(ctx, plan, tab, LINKS_OUT_VALID_ONLY, (double*)traj, (double*)path, valid, lock_step,
                        min_disc, out_index, out_capacity, n_out, row_offset, traj_capacity);
  return simulate_mixed(ctx, plan, tab, LINKS_OUT_VALID_ONLY, (float*)traj, (float*)path, valid, lock_step,
                        min_disc, out_index, out_capacity, n_out, row_offset, traj_capacity);
}

int links_simulate_two_stage(links_ctx ctx, links_plan plan, int T, int T_low, float* traj, float* path,
                             uint8_t* valid, int16_t* lock_step, float* min_disc, int32_t* out_index,
                             int64_t out_capacity, int32_t* n_out, int32_t* n_low_valid) {
  if (!ctx || !plan) return set_error(LINKS_EINVAL, "links_simulate_two_stage: NULL ctx or plan");
  if (plan->ctx != ctx) return set_error(LINKS_EINVAL, "links_simulate_two_stage: plan belongs to another context");
  if (T < 1 || T > LINKS_MAX_T || T_low < 1 || T_low > T || T % T_low != 0)
    return set_error(LINKS_EINVAL, "links_simulate_two_stage: need 1 <= T_low <= T <= 32767 and T_low dividing T");
  if (plan->B > 0 && (!valid || !lock_step || !min_disc))
    return set_error(LINKS_EINVAL, "links_simulate_two_stage: valid, lock_step and min_disc are required");
  if (out_capacity < 0 || ((traj || path) && out_capacity > 0 && !out_index))
    return set_error(LINKS_EINVAL, "links_simulate_two_stage: rows need out_index and out_capacity >= 0");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  int st = LINKS_OK;
  const TTable* tab_lo = get_table(ctx, T_low, &st);
  if (!tab_lo) return st;
  const TTable* tab = get_table(ctx, T, &st);
  if (!tab) return st;
  return simulate_two_stage(ctx, plan, tab_lo, tab, traj, path, valid, lock_step, min_disc, out_index, out_capacity,
                            n_out, n_low_valid);
}

int links_emit_census(links_ctx ctx, links_plan plan, int T, int out_mode, const int16_t* lock_step,
                      const int32_t* out_index, int64_t out_capacity, int64_t* out) {
  if (!ctx || !plan || !out) return set_error(LINKS_EINVAL, "links_emit_census: NULL ctx, plan or out");
  if (plan->ctx != ctx) return set_error(LINKS_EINVAL, "links_emit_census: plan belongs to another context");
  if (T < 1 || T > LINKS_MAX_T) return set_error(LINKS_EINVAL, "links_emit_census: T out of [1, 32767]");
  if (out_mode != LINKS_OUT_FULL && out_mode != LINKS_OUT_VALID_ONLY)
    return set_error(LINKS_EINVAL, "links_emit_census: unknown out_mode");
  if (plan->B > 0 && out_mode == LINKS_OUT_FULL && !lock_step)
    return set_error(LINKS_EINVAL, "links_emit_census: FULL rows need lock_step");
  if (out_mode == LINKS_OUT_VALID_ONLY && (out_capacity < 0 || (out_capacity > 0 && !out_index)))
    return set_error(LINKS_EINVAL, "links_emit_census: VALID_ONLY rows need out_index and out_capacity >= 0");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  int st = LINKS_OK;
  const TTable* tab = get_table(ctx, T, &st);
  if (!tab) return st;
  out[0] = out[1] = out[2] = 0;
  if (plan->B == 0) return LINKS_OK;
  return emit_census(ctx, plan, tab, out_mode, lock_step, out_index, out_capacity, out);
}

int links_normalize(links_ctx ctx, int64_t M, int T, const float* curves, float* out) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_normalize: NULL ctx");
  if (M < 0 || T < 1 || T > 1024) return set_error(LINKS_EINVAL, "links_normalize: need M >= 0 and 1 <= T <= 1024");
  if (M > 0 && (!curves || !out)) return set_error(LINKS_EINVAL, "links_normalize: NULL pointer");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  return normalize_paths(ctx, M, T, curves, out);
}

int links_normalize_maxline(links_ctx ctx, int64_t M, int T, const float* curves, float* out, int32_t* pair,
                            float* circ_var) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_normalize_maxline: NULL ctx");
  if (M < 0 || T < 1 || T > 256) return set_error(LINKS_EINVAL, "links_normalize_maxline: need M >= 0 and 1 <= T <= 256");
  if (M > 0 && (!curves || !out)) return set_error(LINKS_EINVAL, "links_normalize_maxline: NULL pointer");
  if (M > 0 && curves == out) return set_error(LINKS_EINVAL, "links_normalize_maxline: out must not alias curves");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  return normalize_maxline(ctx, M, T, curves, out, pair, circ_var);
}

int links_workspace_reserve(links_ctx ctx, size_t bytes) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_workspace_reserve: NULL ctx");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  return ensure_workspace(ctx, bytes);
}

int links_chamfer_topk(links_ctx ctx, int Q, int64_t M, int T, const float* queries, const float* db, int k,
                       int32_t* idx, float* dist) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_chamfer_topk: NULL ctx");
  if (Q < 0 || M < 0 || M > INT32_MAX) return set_error(LINKS_EINVAL, "links_chamfer_topk: Q or M out of range");
  if (T < 1 || T > 256) return set_error(LINKS_EINVAL, "links_chamfer_topk: T must be in [1, 256]");
  if (k < 1 || k > 32) return set_error(LINKS_EINVAL, "links_chamfer_topk: k must be in [1, 32]");
  if (Q > 0 && (!queries || !idx || !dist || (M > 0 && !db)))
    return set_error(LINKS_EINVAL, "links_chamfer_topk: NULL pointer");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  return chamfer_topk(ctx, Q, M, T, queries, db, k, idx, dist, ctx->chamfer_prune);
}

int links_profile(links_ctx ctx, int enable) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_profile: NULL ctx");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  LINKS_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& r : ctx->pending) {
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->pending.clear();
  if (enable) ctx->acc.clear();
  ctx->prof = enable != 0;
  return LINKS_OK;
}

int links_profile_read(links_ctx ctx, int max, char* names, double* total_ms, int64_t* launches, int* count) {
  if (!ctx || !count || max < 0 || (max > 0 && (!names || !total_ms || !launches)))
    return set_error(LINKS_EINVAL, "links_profile_read: bad argument");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  LINKS_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& r : ctx->pending) {
    float ms = 0.0f;
    LINKS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    auto& slot = ctx->acc[r.name];
    slot.first += ms;
    slot.second += 1;
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->pending.clear();
  int n = 0;
  for (auto& kv : ctx->acc) {
    if (n >= max) break;
    snprintf(names + 32 * n, 32, "%s", kv.first.c_str());
    total_ms[n] = kv.second.first;
    launches[n] = kv.second.second;
    ++n;
  }
  *count = n;
  return LINKS_OK;
}

int links_launch_count(links_ctx ctx, int64_t* out) {
  if (!ctx || !out) return set_error(LINKS_EINVAL, "links_launch_count: NULL argument");
  *out = ctx->launches;
  return LINKS_OK;
}

int links_autotune(links_ctx ctx, links_plan plan, int T, int* lanes) {
  if (!ctx || !plan) return set_error(LINKS_EINVAL, "links_autotune: NULL ctx or plan");
  if (plan->ctx != ctx) return set_error(LINKS_EINVAL, "links_autotune: plan belongs to another context");
  if (T < 1 || T > LINKS_MAX_T) return set_error(LINKS_EINVAL, "links_autotune: T out of [1, 32767]");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  int st = LINKS_OK;
  const TTable* tab = get_table(ctx, T, &st);
  if (!tab) return st;
  return autotune(ctx, plan, tab, lanes);
}

int links_chamfer_first_under(links_ctx ctx, int Q, int64_t M, int T, const float* queries, const float* db,
                              int64_t L, const int32_t* order, double threshold, int k, int32_t* idx,
                              float* dist) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_chamfer_first_under: NULL ctx");
  if (Q < 0 || M < 0 || M > INT32_MAX || L < 0 || L >= INT32_MAX)
    return set_error(LINKS_EINVAL, "links_chamfer_first_under: Q, M or L out of range");
  if (T < 1 || T > 256) return set_error(LINKS_EINVAL, "links_chamfer_first_under: T must be in [1, 256]");
  if (k < 1 || k > 32) return set_error(LINKS_EINVAL, "links_chamfer_first_under: k must be in [1, 32]");
  if (threshold != threshold) return set_error(LINKS_EINVAL, "links_chamfer_first_under: threshold is NaN");
  if (Q > 0 && (!queries || !idx || !dist || (L > 0 && (!order || !db))))
    return set_error(LINKS_EINVAL, "links_chamfer_first_under: NULL pointer");
  return chamfer_first_under(ctx, Q, M, T, queries, db, L, order, threshold, k, idx, dist, ctx->chamfer_prune);
}

int links_curate_paths(links_ctx ctx, int64_t R, int n_max, int T, const float* traj, const int32_t* row_index,
                       int64_t B, const int32_t* n_joints, const uint8_t* adj, const int8_t* type,
                       double circle_var, double keep_rate, uint64_t seed, uint8_t* flags, float* circ_var,
                       int32_t* pair, int32_t* kept_index, float* kept_paths, int64_t kept_capacity,
                       int32_t* n_kept) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_curate_paths: NULL ctx");
  if (R < 0 || B < 0 || kept_capacity < 0) return set_error(LINKS_EINVAL, "links_curate_paths: negative size");
  if (n_max < 1 || n_max > 64) return set_error(LINKS_EINVAL, "links_curate_paths: n_max must be in [1, 64]");
  if (T < 1 || T > 256) return set_error(LINKS_EINVAL, "links_curate_paths: T must be in [1, 256]");
  if (R * n_max > INT32_MAX) return set_error(LINKS_EINVAL, "links_curate_paths: R x n_max exceeds 2^31 - 1");
  if (circle_var != circle_var || keep_rate != keep_rate)
    return set_error(LINKS_EINVAL, "links_curate_paths: NaN threshold or keep rate");
  if (!n_kept || (R > 0 && (!traj || !n_joints || !adj || !type || !flags)) || (kept_capacity > 0 && !kept_index))
    return set_error(LINKS_EINVAL, "links_curate_paths: NULL pointer");
  return curate_paths(ctx, R, n_max, T, traj, row_index, B, n_joints, adj, type, circle_var, keep_rate, seed, flags,
                      circ_var, pair, kept_index, kept_paths, kept_capacity, n_kept);
}

int links_set_chamfer_prune(links_ctx ctx, int on) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_set_chamfer_prune: NULL ctx");
  if (on != 0 && on != 1) return set_error(LINKS_EINVAL, "links_set_chamfer_prune: flag must be 0 or 1");
  ctx->chamfer_prune = on;
  return LINKS_OK;
}

int links_set_screen_lanes(links_ctx ctx, int n_max, int lanes) {
  return links_set_tuning(ctx, n_max, LINKS_TUNE_SCREEN_LANES, lanes);
}

static int* tuning_field(links::Tuning& t, int key) {
  switch (key) {
    case LINKS_TUNE_BUILDER: return &t.builder;
    case LINKS_TUNE_SCREEN_LANES: return &t.screen_lanes;
    case LINKS_TUNE_SCREEN_STEPS: return &t.screen_steps;
    case LINKS_TUNE_SCREEN_CTAS: return &t.screen_ctas;
    case LINKS_TUNE_EMIT_DWS: return &t.emit_dws;
    case LINKS_TUNE_EMIT_CTAS: return &t.emit_ctas;
    case LINKS_TUNE_SCREEN_DEFER: return &t.screen_defer;
    default: return nullptr;
  }
}

static bool tuning_value_ok(int n_max, int key, int v) {
  switch (key) {
    case LINKS_TUNE_BUILDER: return v == 0 || v == 2 || (v == 1 && n_max <= 8);
    case LINKS_TUNE_SCREEN_LANES: return v == 8 || v == 16 || v == 32;
    case LINKS_TUNE_SCREEN_STEPS: return v == 0 || v == 1 || (v == 2 && n_max <= 16);
    case LINKS_TUNE_SCREEN_CTAS: return v >= 0 && v <= 32;
    case LINKS_TUNE_EMIT_DWS: return v >= -1 && v <= 1;
    case LINKS_TUNE_EMIT_CTAS: return v >= 0 && v <= 32;
    case LINKS_TUNE_SCREEN_DEFER: return v == 0 || v == 1;
    default: return false;
  }
}

int links_set_tuning(links_ctx ctx, int n_max, int key, int value) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_set_tuning: NULL ctx");
  if (n_max < 2 || n_max > LINKS_MAX_JOINTS) return set_error(LINKS_EINVAL, "links_set_tuning: n_max out of [2, 32]");
  links::Tuning t = links::tuning_of(ctx, n_max);
  int* f = tuning_field(t, key);
  if (!f) return set_error(LINKS_EINVAL, "links_set_tuning: unknown key");
  if (!tuning_value_ok(n_max, key, value)) return set_error(LINKS_EINVAL, "links_set_tuning: value out of range for this key and n_max");
  *f = value;
  ctx->tuning[n_max] = t;
  return LINKS_OK;
}

int links_get_tuning(links_ctx ctx, int n_max, int key, int* value) {
  if (!ctx || !value) return set_error(LINKS_EINVAL, "links_get_tuning: NULL argument");
  links::Tuning t = links::tuning_of(ctx, n_max);
  int* f = tuning_field(t, key);
  if (!f) return set_error(LINKS_EINVAL, "links_get_tuning: unknown key");
  *value = *f;
  return LINKS_OK;
}

// Text file: a header naming the device, then one line per n_max with its seven keys.
int links_tuning_save(links_ctx ctx, const char* path) {
  if (!ctx || !path) return set_error(LINKS_EINVAL, "links_tuning_save: NULL argument");
  cudaDeviceProp prop;
  LINKS_CUDA(cudaGetDeviceProperties(&prop, ctx->device));
  FILE* f = fopen(path, "w");
  if (!f) return set_error(LINKS_EINVAL, std::string("links_tuning_save: cannot open ") + path);
  fprintf(f, "links-tuning 2 sms %d device %s\n", prop.multiProcessorCount, prop.name);
  for (const auto& kv : ctx->tuning) {
    const links::Tuning& t = kv.second;
    fprintf(f, "%d %d %d %d %d %d %d %d\n", kv.first, t.builder, t.screen_lanes, t.screen_steps, t.screen_ctas,
            t.emit_dws, t.emit_ctas, t.screen_defer);
  }
  const bool ok = fclose(f) == 0;
  return ok ? LINKS_OK : set_error(LINKS_EINVAL, std::string("links_tuning_save: write failed: ") + path);
}

int links_tuning_load(links_ctx ctx, const char* path) {
  if (!ctx || !path) return set_error(LINKS_EINVAL, "links_tuning_load: NULL argument");
  cudaDeviceProp prop;
  LINKS_CUDA(cudaGetDeviceProperties(&prop, ctx->device));
  FILE* f = fopen(path, "r");
  if (!f) return set_error(LINKS_EINVAL, std::string("links_tuning_load: cannot open ") + path);
  char name[256] = {0};
  int version = 0, sms = 0;
  if (fscanf(f, "links-tuning %d sms %d device %255[^\n]", &version, &sms, name) != 3 || version != 2) {
    fclose(f);
    return set_error(LINKS_EINVAL, "links_tuning_load: not a tuning file");
  }
  if (sms != prop.multiProcessorCount || std::string(name) != prop.name) {
    fclose(f);
    return set_error(LINKS_ESTATE, "links_tuning_load: the file was tuned on another device");
  }
  std::map<int, links::Tuning> table;
  int n, v[7];
  int st = LINKS_OK;
  while (fscanf(f, "%d %d %d %d %d %d %d %d", &n, &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6]) == 8) {
    links::Tuning t;
    const int keys[7] = {LINKS_TUNE_BUILDER, LINKS_TUNE_SCREEN_LANES, LINKS_TUNE_SCREEN_STEPS,
                         LINKS_TUNE_SCREEN_CTAS, LINKS_TUNE_EMIT_DWS, LINKS_TUNE_EMIT_CTAS,
                         LINKS_TUNE_SCREEN_DEFER};
    bool ok = n >= 2 && n <= LINKS_MAX_JOINTS;
    for (int k = 0; k < 7 && ok; ++k) {
      ok = tuning_value_ok(n, keys[k], v[k]);
      if (ok) *tuning_field(t, keys[k]) = v[k];
    }
    if (!ok) {
      st = set_error(LINKS_EINVAL, "links_tuning_load: an entry is out of range");
      break;
    }
    table[n] = t;
  }
  const bool at_end = feof(f) != 0;
  fclose(f);
  if (st) return st;
  if (!at_end) return set_error(LINKS_EINVAL, "links_tuning_load: malformed entry");
  for (const auto& kv : table) ctx->tuning[kv.first] = kv.second;
  return LINKS_OK;
}

int links_capture_begin(links_ctx ctx) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_capture_begin: NULL ctx");
  if (!ctx->stream) return set_error(LINKS_ESTATE, "links_capture_begin: the legacy default stream cannot be captured");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  LINKS_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  return LINKS_OK;
}

int links_capture_end(links_ctx ctx, links_graph* out) {
  if (!ctx || !out) return set_error(LINKS_EINVAL, "links_capture_end: NULL argument");
  *out = nullptr;
  cudaGraph_t g = nullptr;
  LINKS_CUDA(cudaStreamEndCapture(ctx->stream, &g));
  links_graph lg = new (std::nothrow) links_graph_s();
  if (!lg) {
    cudaGraphDestroy(g);
    return set_error(LINKS_ENOMEM, "links_capture_end: host allocation");
  }
  lg->graph = g;
  cudaError_t e = cudaGraphInstantiate(&lg->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    delete lg;
    return cuda_status(e, "cudaGraphInstantiate");
  }
  *out = lg;
  return LINKS_OK;
}

int links_graph_launch(links_ctx ctx, links_graph graph) {
  if (!ctx || !graph) return set_error(LINKS_EINVAL, "links_graph_launch: NULL argument");
  LINKS_CUDA(cudaGraphLaunch(graph->exec, ctx->stream));
  return LINKS_OK;
}

int links_graph_free(links_graph graph) {
  if (!graph) return set_error(LINKS_EINVAL, "links_graph_free: NULL graph");
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  delete graph;
  return LINKS_OK;
}

}  // extern "C"
