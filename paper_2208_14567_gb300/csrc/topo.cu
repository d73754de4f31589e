// topo.cu -- screen kernels specialised to one topology, generated and compiled at run
// time (the paper's "vectorised solver specific to a given topology", Sec. "Graphical
// Simulator": one solve path serves every position sample of a topology).
//
// For a topology the generator writes straight-line CUDA for its solve path: every
// joint's position and error bound live in registers of the lane that computes one
// step, the dyads' parent slots are compile-time names, and each mechanism's link data
// (R12, Rm, c, 2 r1 r2, the local error constant and which parent comes first) are
// loaded into registers once per mechanism.  The arithmetic is that of the generic
// screen's two-step form, operation for operation with round-to-nearest intrinsics (no
// contraction), so a decided mechanism gets the generic screen's flags, lock step and
// minimum discriminant.  A group of G lanes takes one mechanism, G consecutive steps at
// a time; a mechanism whose plan does not follow the compiled path, or that meets an
// uncertain step (neither certainly locked nor certainly free by the FP32 bounds)
// before its first certain lock, is listed for the generic screen, which decides it
// with its double-word rescue.
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include "links_internal.cuh"

struct links_topo_s {
  links_ctx ctx = nullptr;
  int nf = 0, nd = 0, G = 16;
  std::vector<int> sa, sb;  // parent slots of each dyad, in the reference plan's order
  cudaLibrary_t lib = nullptr;  // the compiled kernel, loaded through the runtime
  cudaKernel_t fn = nullptr;
  int per_sm = 1;
  double compile_ms = 0.0;
};

namespace links {
namespace {

std::string topo_source(int nf, int nd, const std::vector<int>& sa, const std::vector<int>& sb, int G) {
  std::ostringstream o;
  o << "typedef unsigned int u32;\n"
       "struct Hdr { int status; unsigned char n, nd, nf, motor; unsigned char cs, pj, p0, p1;\n"
       "  float ux_h, ux_l, uy_h, uy_l, px_h, px_l, py_h, py_l, bmax, e_motor, e_fixed, lbox; };\n"
       "__device__ __forceinline__ float min3(float a, float b, float c) {\n"
       "  float r; asm(\"min.f32 %0, %1, %2, %3;\" : \"=f\"(r) : \"f\"(a), \"f\"(b), \"f\"(c)); return r; }\n"
       "__device__ __forceinline__ float min3_nan(float a, float b, float c) {\n"
       "  float r; asm(\"min.NaN.f32 %0, %1, %2, %3;\" : \"=f\"(r) : \"f\"(a), \"f\"(b), \"f\"(c)); return r; }\n";
  o << "#define G " << G << "\n";
  o << "extern \"C\" __global__ void __launch_bounds__(256) topo_screen(\n"
       "    const Hdr* __restrict__ hdr, const float4* __restrict__ dyad, int max_dyads,\n"
       "    const float4* __restrict__ fixpos, int n_max, const int* __restrict__ order,\n"
       "    const int* __restrict__ hist, int T, const float4* __restrict__ cs,\n"
       "    unsigned char* __restrict__ valid, short* __restrict__ lock_step, float* __restrict__ min_disc,\n"
       "    int* __restrict__ esc, int* __restrict__ n_esc) {\n"
       "  const int lane = threadIdx.x & 31, gl = lane % G, base = lane - gl;\n"
       "  const u32 gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << base);\n"
       "  int n_ok = hist[lane];\n"
       "  for (int o = 16; o; o >>= 1) n_ok += __shfl_xor_sync(0xffffffffu, n_ok, o);\n"
       "  const int ngroups = (int)(gridDim.x * blockDim.x / G);\n"
       "  for (int item = (int)((blockIdx.x * blockDim.x + threadIdx.x) / G); item < n_ok; item += ngroups) {\n"
       "    const int b = order[item];\n"
       "    const Hdr h = hdr[b];\n"
       "    bool match = h.nf == " << nf << " && h.nd == " << nd << ";\n";
  for (int s = 0; s < nf; ++s)
    o << "    const float4 f" << s << " = __ldg(fixpos + (long long)b * n_max + " << s << ");\n";
  for (int d = 0; d < nd; ++d) {
    const unsigned direct = (unsigned)sa[d] * 256u | ((unsigned)sb[d] * 256u) << 16;
    const unsigned swapped = (unsigned)sb[d] * 256u | ((unsigned)sa[d] * 256u) << 16;
    o << "    const float4 ra" << d << " = __ldg(dyad + ((long long)b * max_dyads + " << d << ") * 3);\n"
      << "    const float4 rb" << d << " = __ldg(dyad + ((long long)b * max_dyads + " << d << ") * 3 + 1);\n"
      << "    const bool sw" << d << " = __float_as_uint(ra" << d << ".x) == " << swapped << "u;\n"
      << "    match = match && (sw" << d << " || __float_as_uint(ra" << d << ".x) == " << direct << "u);\n";
  }
  o << "    if (!match) {\n"
       "      if (gl == 0) esc[atomicAdd(n_esc, 1)] = b;\n"
       "      continue;\n"
       "    }\n"
       "    float qacc = __int_as_float(0x7f800000);\n"
       "    for (int c0 = 0; c0 < T; c0 += G) {\n"
       "      const int t = c0 + gl;\n"
       "      const bool act = t < T;\n"
       "      const float4 csv = __ldg(cs + (act ? t : T - 1));\n"
       "      float lockw = __int_as_float(0x7f800000), zmin = lockw, isgmax = 0.0f;\n";
  for (int s = 0; s < nf; ++s)
    o << "      const float x" << s << " = f" << s << ".x, y" << s << " = f" << s << ".z, e" << s
      << " = h.e_fixed;\n";
  o << "      const float x" << nf << " = csv.x * h.ux_h - csv.z * h.uy_h, y" << nf
    << " = csv.z * h.ux_h + csv.x * h.uy_h, e" << nf << " = h.e_motor;\n";
  for (int d = 0; d < nd; ++d) {
    const int k = nf + 1 + d, A = sa[d], Bq = sb[d];
    const std::string D = std::to_string(d);
    o << "      float x" << k << ", y" << k << ", e" << k << ";\n"
      << "      {\n"
      << "        const float pix = sw" << D << " ? x" << Bq << " : x" << A << ", piy = sw" << D << " ? y" << Bq
      << " : y" << A << ";\n"
      << "        const float pjx = sw" << D << " ? x" << A << " : x" << Bq << ", pjy = sw" << D << " ? y" << A
      << " : y" << Bq << ";\n"
      << "        const float ei = sw" << D << " ? e" << Bq << " : e" << A << ", ej = sw" << D << " ? e" << A
      << " : e" << Bq << ";\n"
      << "        const float R12 = ra" << D << ".y, Rm = ra" << D << ".z, C = ra" << D << ".w, W2 = rb" << D
      << ".x, LO = rb" << D << ".y;\n"
      << "        const float dx = __fsub_rn(pjx, pix), dy = __fsub_rn(pjy, piy);\n"
      << "        const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));\n"
      << "        const float rd = rsqrtf(d2);\n"
      << "        const float dd = __fmul_rn(d2, rd);\n"
      << "        const float s2 = __fsub_rn(R12, dd), s3 = __fsub_rn(dd, Rm);\n"
      << "        const float D = __fmul_rn(__fmul_rn(__fadd_rn(dd, R12), s2), __fmul_rn(s3, __fadd_rn(dd, Rm)));\n"
      << "        const float rD = rsqrtf(D);\n"
      << "        const float isg = __fmul_rn(W2, rD);\n"
      << "        const float del = __fadd_rn(__fadd_rn(ei, ej), LO);\n"
      << "        lockw = min3(lockw, __fadd_rn(s2, del), __fadd_rn(s3, del));\n"
      << "        zmin = min3_nan(zmin, __fsub_rn(s2, del), __fsub_rn(s3, del));\n"
      << "        isgmax = fmaxf(isgmax, isg);\n"
      << "        const float hinv = __fmul_rn(0.5f, __fmul_rn(rd, rd));\n"
      << "        const float a = __fmul_rn(__fadd_rn(d2, C), hinv), bq = __fmul_rn(__fmul_rn(D, rD), hinv);\n"
      << "        x" << k << " = __fmaf_rn(a, dx, __fmaf_rn(-bq, dy, pix));\n"
      << "        y" << k << " = __fmaf_rn(a, dy, __fmaf_rn(bq, dx, piy));\n"
      << "        e" << k << " = __fmaf_rn(del, isg, __fmul_rn(" << std::hexfloat << (kAddErr * kU)
      << std::defaultfloat << "f, __fadd_rn(R12, __fadd_rn(fabsf(x" << k << "), fabsf(y" << k << ")))));\n"
      << "      }\n";
  }
  // the last slot's bound is not read by any dyad: keep the compiler quiet about it
  o << "      (void)e" << nf + nd << ";\n";
  o << "      const bool certain_lock = lockw < 0.0f;\n"
       "      const bool amb = act && !certain_lock && !(zmin >= 0.0f);\n"
       "      const float q = __fdividef(1.0f, isgmax * isgmax);\n"
       "      const u32 lb = (__ballot_sync(gmask, act && certain_lock) & gmask) >> base;\n"
       "      const u32 ab = (__ballot_sync(gmask, amb) & gmask) >> base;\n"
       "      const int first = lb ? __ffs(lb) - 1 : G;\n"
       "      const u32 before = first >= 32 ? 0xffffffffu : ((1u << first) - 1u);\n"
       "      if (ab & before) {\n"
       "        if (gl == 0) esc[atomicAdd(n_esc, 1)] = b;\n"
       "        break;\n"
       "      }\n"
       "      if (act && gl < first) qacc = fminf(qacc, q);\n"
       "      if (first < G || c0 + G >= T) {\n"
       "        float qr = qacc;\n"
       "        for (int o = 1; o < G; o <<= 1) qr = fminf(qr, __shfl_xor_sync(gmask, qr, o));\n"
       "        if (gl == 0) {\n"
       "          valid[b] = first == G;\n"
       "          lock_step[b] = (short)(first < G ? c0 + first : -1);\n"
       "          min_disc[b] = qr;\n"
       "        }\n"
       "        break;\n"
       "      }\n"
       "    }\n"
       "  }\n"
       "}\n";
  return o.str();
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
  const std::string src = topo_source(nf, nd, sa, sb, 16);
  if (len) *len = src.size() + 1;
  if (buf && cap > 0) {
    const size_t m = std::min(cap - 1, src.size());
    memcpy(buf, src.data(), m);
    buf[m] = '\0';
  }
  return LINKS_OK;
}

extern "C" int links_topo_create(links_ctx ctx, int n, int n_max, const uint8_t* adj, const int8_t* type,
                                 links_topo* out) {
  if (!ctx || !out) return set_error(LINKS_EINVAL, "links_topo_create: NULL ctx or out");
  *out = nullptr;
  links_topo t = new links_topo_s();
  t->ctx = ctx;
  const int pst = plan_topology(n, n_max, adj, type, &t->nf, &t->nd, &t->sa, &t->sb, "links_topo_create");
  if (pst) {
    delete t;
    return pst;
  }
  const auto t0 = std::chrono::steady_clock::now();
  const std::string src = topo_source(t->nf, t->nd, t->sa, t->sb, t->G);
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "topo_screen.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
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
    int32_t* n_esc = p.ctrs + kNConfirm;
    int max_dyads = p.max_dyads, n_max = p.n_max, Tv = tb->T;
    void* args[] = {&p.hdr, &dy, &max_dyads, &p.fixpos, &n_max, &p.order, &hist, &Tv,
                    const_cast<float4**>(&tb->cs), &v, &ls, &md, &p.order2, &n_esc};
    KernelScope ks(c, "topo_screen");
    LINKS_CUDA(cudaLaunchKernel(reinterpret_cast<const void*>(topo->fn), dim3((unsigned)(c->num_sms * topo->per_sm)),
                                dim3(256), args, 0, c->stream));
    return (int)LINKS_OK;
  };
  return simulate_prescreened(ctx, plan, tab, out_mode, traj, path, valid, lock_step, min_disc, out_index,
                              out_capacity, n_out, n_escaped, pre);
}
