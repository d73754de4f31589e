// topo.cu -- screen kernels specialised to one topology, generated and compiled at run
// time (Sec. "Computational Cost of Simulations": the paper vectorises its solver for one
// topology once its solve path is known, and Sec. "Graphical Simulator": that path serves
// every position sample of the topology).
//
// For a topology the generator writes straight-line CUDA for its solve path: every
// joint's position and error bound live in registers of the lane that computes one
// step, the dyads' parent slots are compile-time names, and each mechanism's link data
// (R12, Rm, c, 2 r1 r2, the local error constant and which parent comes first) are
// loaded into registers once per mechanism.  The dyad is the library's own FP32 core
// and an uncertain step (neither certainly locked nor certainly free by the FP32
// bounds) is decided by the library's double-word chain (both in step.cuh, compiled
// into the same program), so every mechanism gets the generic screen's flags, lock
// step and minimum discriminant.  As in the generic screen, a group of G lanes takes
// one mechanism, G consecutive steps at a time; a warp advances its groups together
// and refills idle groups from batches of the work list.  A mechanism whose plan does
// not follow the compiled path is listed for the generic screen.
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include "embedded_headers.inc"  // dw_core.cuh and step.cuh as text (written by build.py)
#include "links_internal.cuh"

struct links_topo_s {
  links_ctx ctx = nullptr;
  int n = 0, nf = 0, nd = 0, G = 16;
  std::vector<int> sa, sb;  // parent slots of each dyad, in the reference plan's order
  cudaLibrary_t lib = nullptr;  // the compiled kernel, loaded through the runtime
  cudaKernel_t fn = nullptr;
  int per_sm = 1;
  double compile_ms = 0.0;
};

namespace links {
namespace {

// The per-step part of the generated kernel: the lane's step of its group's mechanism
// (slots in registers, the FP32 core per dyad, the double-word rescue of an uncertain
// step), then the group's decisions for the chunk.
std::string topo_source_step(int nf, int nd, const std::vector<int>& sa, const std::vector<int>& sb) {
  std::ostringstream o;
  for (int s2 = 0; s2 < nf; ++s2)
    o << "      const float x" << s2 << " = f" << s2 << ".x, y" << s2 << " = f" << s2 << ".z, e" << s2
      << " = h.e_fixed;\n";
  o << "      const float x" << nf << " = __fsub_rn(__fmul_rn(csv.x, h.ux_h), __fmul_rn(csv.z, h.uy_h)), y" << nf
    << " = __fadd_rn(__fmul_rn(csv.z, h.ux_h), __fmul_rn(csv.x, h.uy_h)), e" << nf << " = h.e_motor;\n";
  for (int d = 0; d < nd; ++d) {
    const int k = nf + 1 + d, A = sa[d], Bq = sb[d];
    const std::string D = std::to_string(d);
    o << "      float x" << k << ", y" << k << ", e" << k << ";\n"
      << "      links::fp32_dyad_core(sw" << D << " ? x" << Bq << " : x" << A << ", sw" << D << " ? y" << Bq
      << " : y" << A << ", sw" << D << " ? x" << A << " : x" << Bq << ", sw" << D << " ? y" << A << " : y" << Bq
      << ", sw" << D << " ? e" << Bq << " : e" << A << ", sw" << D << " ? e" << A << " : e" << Bq << ", ra" << D
      << ", rb" << D << ", lockw, zmin, isgmax, x" << k << ", y" << k << ", e" << k << ");\n";
  }
  o << "      (void)e" << nf + nd << ";  // the last slot's bound feeds no dyad\n"
       "      const bool certain_lock = lockw < 0.0f;\n"
       "      q = __fdividef(1.0f, isgmax * isgmax);\n"
       "      locked = act && certain_lock;\n"
       "      if (act && !certain_lock && !(zmin >= 0.0f)) {  // uncertain: double-word decides\n"
       "        links::dwp loc[" << nf + 1 + nd << "];\n"
       "        float qd;\n"
       "        locked = links::dw_chain(h, fixpos + (long long)b * n_max, dyad + (long long)b * max_dyads,\n"
       "                                        __ldg(cs + t), links::LocLocal{loc}, &qd);\n"
       "        q = qd;\n"
       "      }\n"
       "    }\n"
       "    const u32 lb = (__ballot_sync(full, locked) >> base) & (G == 32 ? full : ((1u << G) - 1u));\n"
       "    const int first = lb ? __ffs(lb) - 1 : G;\n"
       "    if (act && gl < first) qacc = fminf(qacc, q);\n"
       "    const bool done = has && (first < G || c0 + G >= T);\n"
       "    float qr = qacc;\n"
       "    for (int o = 1; o < G; o <<= 1) qr = fminf(qr, __shfl_xor_sync(full, qr, o));\n"
       "    if (done) {\n"
       "      if (gl == 0) {\n"
       "        valid[b] = first == G;\n"
       "        lock_step[b] = (short)(first < G ? c0 + first : -1);\n"
       "        min_disc[b] = qr;\n"
       "      }\n"
       "      item = -1;\n"
       "    } else if (has) {\n"
       "      c0 += G;\n"
       "    }\n"
       "  }\n"
       "}\n";
  return o.str();
}

// Paths of up to 6 dyads are compiled for 3 blocks per SM (80 registers: at 8 joints the screen
// ran 2.39 -> 2.18 ms per 1M samples); longer ones keep their registers (capped, 9 dyads spilled
// and ran 3.14 -> 3.24 ms).
std::string topo_source(int nf, int nd, const std::vector<int>& sa, const std::vector<int>& sb, int G) {
  std::ostringstream o;
  const int ns = nf + 1 + nd;
  o << "#include \"step.cuh\"\n"
       "typedef unsigned int u32;\n"
       "#define G " << G << "\n"
       "extern \"C\" __global__ void __launch_bounds__(256" << (nd <= 6 ? ", 3" : "") << ") topo_screen(\n"
       "    const links::MechHdr* __restrict__ hdr, const links::DyadRec* __restrict__ dyad, int max_dyads,\n"
       "    const float4* __restrict__ fixpos, int n_max, const int* __restrict__ order,\n"
       "    const int* __restrict__ hist, int* __restrict__ work, int T, const float4* __restrict__ cs,\n"
       "    unsigned char* __restrict__ valid, short* __restrict__ lock_step, float* __restrict__ min_disc,\n"
       "    int* __restrict__ esc, int* __restrict__ n_esc) {\n"
       "  const u32 full = 0xffffffffu;\n"
       "  const int lane = threadIdx.x & 31, gl = lane % G, g = lane / G, base = g * G;\n"
       "  int n_ok = hist[lane];\n"
       "  for (int o = 16; o; o >>= 1) n_ok += __shfl_xor_sync(full, n_ok, o);\n"
       "  int qhead = 0, qend = 0, item = -1, c0 = 0, b = 0;\n"
       "  bool exhausted = false;\n"
       "  float qacc = 0.0f;\n"
       "  links::MechHdr h = {};\n";
  for (int s2 = 0; s2 < nf; ++s2) o << "  float4 f" << s2 << " = {};\n";
  for (int d = 0; d < nd; ++d) o << "  float4 ra" << d << " = {}, rb" << d << " = {};\n  bool sw" << d << " = false;\n";
  // the warp advances all its groups one chunk per iteration (converged); idle groups
  // take the next mechanisms of a batch the warp claims from the shared work counter
  o << "  while (true) {\n"
       "    u32 need = __ballot_sync(full, gl == 0 && item < 0);\n"
       "    bool fresh = false;\n"
       "    while (need) {\n"
       "      if (qhead >= qend) {\n"
       "        if (exhausted) break;\n"
       "        int bs = 0;\n"
       "        if (lane == 0) bs = atomicAdd(work, 32);\n"
       "        bs = __shfl_sync(full, bs, 0);\n"
       "        if (bs >= n_ok) { exhausted = true; break; }\n"
       "        qhead = bs;\n"
       "        qend = min(bs + 32, n_ok);\n"
       "      }\n"
       "      const int leader = __ffs(need) - 1;\n"
       "      need &= need - 1;\n"
       "      if (g == leader / G) { item = qhead; fresh = true; }\n"
       "      ++qhead;\n"
       "    }\n"
       "    if (__ballot_sync(full, item >= 0) == 0) break;\n";
  o << "    if (fresh) {\n"
       "      b = order[item];\n"
       "      h = hdr[b];\n"
       "      bool match = h.nf == " << nf << " && h.nd == " << nd << ";\n";
  for (int s2 = 0; s2 < nf; ++s2)
    o << "      f" << s2 << " = __ldg(fixpos + (long long)b * n_max + " << s2 << ");\n";
  for (int d = 0; d < nd; ++d) {
    const unsigned direct = (unsigned)sa[d] * 256u | ((unsigned)sb[d] * 256u) << 16;
    const unsigned swapped = (unsigned)sb[d] * 256u | ((unsigned)sa[d] * 256u) << 16;
    o << "      ra" << d << " = __ldg(&dyad[(long long)b * max_dyads + " << d << "].r0);\n"
      << "      rb" << d << " = __ldg(&dyad[(long long)b * max_dyads + " << d << "].r1);\n"
      << "      sw" << d << " = __float_as_uint(ra" << d << ".x) == " << swapped << "u;\n"
      << "      match = match && (sw" << d << " || __float_as_uint(ra" << d << ".x) == " << direct << "u);\n";
  }
  o << "      c0 = 0;\n"
       "      qacc = __int_as_float(0x7f800000);\n"
       "      if (!match) {  // another solve path: the generic screen takes it\n"
       "        if (gl == 0) esc[atomicAdd(n_esc, 1)] = b;\n"
       "        item = -1;\n"
       "      }\n"
       "    }\n"
       "    const bool has = item >= 0;\n"
       "    const int t = c0 + gl;\n"
       "    const bool act = has && t < T;\n"
       "    bool locked = false;\n"
       "    float q = 0.0f;\n"
       "    if (has) {\n"
       "      const float4 csv = __ldg(cs + (t < T ? t : T - 1));\n"
       "      float lockw = __int_as_float(0x7f800000), zmin = lockw, isgmax = 0.0f;\n";
  (void)ns;
  return o.str() + topo_source_step(nf, nd, sa, sb);
}

// Plans the topology (positions on a spiral: the solve path does not depend on them)
// and reads the parent slots of its dyads.
int plan_topology(int n, int n_max, const uint8_t* adj, const int8_t* type, int* nf, int* nd,
                  std::vector<int>* sa, std::vector<int>* sb, const char* who) {
  if (n_max < 2 || n_max > kMaxJ || n < 2 || n > n_max) {
    std::string m = std::string(who) + ": need 2 <= n <= n_max <= 32";
    return set_error(LINKS_EINVAL, m.c_str());
  }
  if (!adj || !type) {
    std::string m = std::string(who) + ": NULL adj or type";
    return set_error(LINKS_EINVAL, m.c_str());
  }
  std::vector<double> pos(2 * n_max, 0.0);
  for (int a = 0; a < n; ++a) {
    const double r = 1.0 + 0.37 * a, th = 2.399963 * a;
    pos[2 * a] = r * std::cos(th);
    pos[2 * a + 1] = r * std::sin(th);
  }
  MechHdr h{};
  std::vector<DyadRec> rec(std::max(1, n_max - 2));
  const int st = plan_one_host(n, n_max, adj, type, pos.data(), &h, rec.data());
  if (st != LINKS_MECH_OK) {
    char buf[128];
    snprintf(buf, sizeof buf, "%s: the topology does not plan (mechanism status %d)", who, st);
    return set_error(LINKS_EINVAL, buf);
  }
  *nf = h.nf;
  *nd = h.nd;
  sa->clear();
  sb->clear();
  for (int d = 0; d < h.nd; ++d) {
    uint32_t slots;
    memcpy(&slots, &rec[d].r2.w, sizeof slots);
    sa->push_back((int)(slots & 0xffu));
    sb->push_back((int)((slots >> 8) & 0xffu));
  }
  return LINKS_OK;
}

}  // namespace
}  // namespace links

using namespace links;

extern "C" int links_topo_source(int n, int n_max, const uint8_t* adj, const int8_t* type, char* buf, size_t cap,
                                 size_t* len) {
  int nf = 0, nd = 0;
  std::vector<int> sa, sb;
  const int st = plan_topology(n, n_max, adj, type, &nf, &nd, &sa, &sb, "links_topo_source");
  if (st) return st;
  const std::string src = topo_source(nf, nd, sa, sb, nd <= 3 ? 8 : (nd <= 6 ? 16 : 32));  // the default lanes
  if (len) *len = src.size() + 1;
  if (buf && cap > 0) {
    const size_t m = std::min(cap - 1, src.size());
    memcpy(buf, src.data(), m);
    buf[m] = '\0';
  }
  return LINKS_OK;
}

extern "C" int links_topo_create(links_ctx ctx, int n, int n_max, const uint8_t* adj, const int8_t* type,
                                 int lanes, links_topo* out) {
  if (!ctx || !out) return set_error(LINKS_EINVAL, "links_topo_create: NULL ctx or out");
  *out = nullptr;
  if (lanes != 0 && lanes != 8 && lanes != 16 && lanes != 32)
    return set_error(LINKS_EINVAL, "links_topo_create: lanes must be 0, 8, 16 or 32");
  links_topo t = new links_topo_s();
  t->G = lanes;
  t->ctx = ctx;
  t->n = n;
  const int pst = plan_topology(n, n_max, adj, type, &t->nf, &t->nd, &t->sa, &t->sb, "links_topo_create");
  if (pst) {
    delete t;
    return pst;
  }
  // default group size by path length (measured on 1M samples of one topology, T = 200:
  // 3 dyads fastest at 8 lanes, 5 at 16, 9 at 32): longer paths keep more registers per
  // lane, and wider groups then keep enough steps in flight
  if (t->G == 0) t->G = t->nd <= 3 ? 8 : (t->nd <= 6 ? 16 : 32);
  const auto t0 = std::chrono::steady_clock::now();
  const std::string src = topo_source(t->nf, t->nd, t->sa, t->sb, t->G);
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "topo_screen.cu", kEmbeddedCount, kEmbeddedTexts, kEmbeddedNames) !=
      NVRTC_SUCCESS) {
    delete t;
    return set_error(LINKS_ECUDA, "links_topo_create: nvrtcCreateProgram failed");
  }
  const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo"};
  const nvrtcResult cr = nvrtcCompileProgram(prog, 3, opts);
  if (cr != NVRTC_SUCCESS) {
    size_t n_log = 0;
    nvrtcGetProgramLogSize(prog, &n_log);
    std::string log(n_log, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    delete t;
    std::string msg = "links_topo_create: NVRTC compile failed: " + log.substr(0, 400);
    return set_error(LINKS_ECUDA, msg.c_str());
  }
  size_t n_cubin = 0;
  nvrtcGetCUBINSize(prog, &n_cubin);
  std::vector<char> cubin(n_cubin);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  cudaError_t ce = cudaSetDevice(ctx->device);
  if (ce == cudaSuccess) ce = cudaFree(nullptr);  // the primary context is current
  if (ce != cudaSuccess) {
    delete t;
    return cuda_status(ce, "links_topo_create: cudaSetDevice");
  }
  ce = cudaLibraryLoadData(&t->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&t->fn, t->lib, "topo_screen");
  if (ce == cudaSuccess)
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t->per_sm, reinterpret_cast<const void*>(t->fn), 256, 0);
  if (ce != cudaSuccess) {
    if (t->lib) cudaLibraryUnload(t->lib);
    delete t;
    return cuda_status(ce, "links_topo_create: loading the compiled screen");
  }
  if (t->per_sm < 1) t->per_sm = 1;
  t->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = t;
  return LINKS_OK;
}

extern "C" int links_topo_info(links_topo topo, int* n_fixed, int* n_dyads, double* compile_ms) {
  if (!topo) return set_error(LINKS_EINVAL, "links_topo_info: NULL topo");
  if (n_fixed) *n_fixed = topo->nf;
  if (n_dyads) *n_dyads = topo->nd;
  if (compile_ms) *compile_ms = topo->compile_ms;
  return LINKS_OK;
}

extern "C" int links_topo_free(links_topo topo) {
  if (!topo) return LINKS_OK;
  if (topo->lib) cudaLibraryUnload(topo->lib);
  delete topo;
  return LINKS_OK;
}

extern "C" int links_simulate_topology(links_ctx ctx, links_plan plan, links_topo topo, int T, int out_mode,
                                       float* traj, float* path, uint8_t* valid, int16_t* lock_step,
                                       float* min_disc, int32_t* out_index, int64_t out_capacity, int32_t* n_out,
                                       int32_t* n_escaped) {
  if (!ctx || !plan || !topo) return set_error(LINKS_EINVAL, "links_simulate_topology: NULL ctx, plan or topo");
  if (plan->ctx != ctx || topo->ctx != ctx)
    return set_error(LINKS_EINVAL, "links_simulate_topology: plan or topo belongs to another context");
  if (T < 1 || T > LINKS_MAX_T) return set_error(LINKS_EINVAL, "links_simulate_topology: T out of [1, 32767]");
  if (topo->n > plan->d.n_max)  // the kernel reads the compiled path's rows of each mechanism's plan
    return set_error(LINKS_EINVAL, "links_simulate_topology: the topology has more joints than the plan's n_max");
  if (out_mode != LINKS_OUT_FULL && out_mode != LINKS_OUT_VALID_ONLY)
    return set_error(LINKS_EINVAL, "links_simulate_topology: unknown out_mode");
  if (plan->B > 0 && (!valid || !lock_step || !min_disc))
    return set_error(LINKS_EINVAL, "links_simulate_topology: valid, lock_step and min_disc are required");
  if (out_mode == LINKS_OUT_VALID_ONLY) {
    if (out_capacity < 0) return set_error(LINKS_EINVAL, "links_simulate_topology: out_capacity < 0");
    if ((traj || path) && out_capacity > 0 && !out_index)
      return set_error(LINKS_EINVAL, "links_simulate_topology: VALID_ONLY rows need out_index");
  }
  LINKS_CUDA(cudaSetDevice(ctx->device));
  int st = LINKS_OK;
  const TTable* tab = get_table(ctx, T, &st);
  if (!tab) return st;
  const Prescreen pre = [topo](links_ctx c, links_plan pl, const TTable* tb, uint8_t* v, int16_t* ls, float* md) {
    PlanDev& p = pl->d;
    if (pl->B == 0) return (int)LINKS_OK;
    const float4* dy = reinterpret_cast<const float4*>(p.dyad);
    const int32_t* hist = p.ctrs + kHist;
    int32_t* work = p.ctrs + kWork;
    int32_t* n_esc = p.ctrs + kNConfirm;
    int max_dyads = p.max_dyads, n_max = p.n_max, Tv = tb->T;
    LINKS_CUDA(cudaMemsetAsync(work, 0, sizeof(int32_t), c->stream));
    void* args[] = {&p.hdr, &dy, &max_dyads, &p.fixpos, &n_max, &p.order, &hist, &work, &Tv,
                    const_cast<float4**>(&tb->cs), &v, &ls, &md, &p.order2, &n_esc};
    KernelScope ks(c, "topo_screen");
    LINKS_CUDA(cudaLaunchKernel(reinterpret_cast<const void*>(topo->fn), dim3((unsigned)(c->num_sms * topo->per_sm)),
                                dim3(256), args, 0, c->stream));
    return (int)LINKS_OK;
  };
  return simulate_prescreened(ctx, plan, tab, out_mode, traj, path, valid, lock_step, min_disc, out_index,
                              out_capacity, n_out, n_escaped, pre);
}
