// links_internal.cuh -- plan layout, double-word arithmetic and context state shared by
// the library's translation units.  Not part of the public ABI (include/links.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/links.h"
#include "dw_core.cuh"

namespace links {

// Loads of data that a kernel only reads: through the non-coherent read-only path (NC,
// for data no one writes while the kernel runs), or L2-coherent (for a persistent
// kernel that reads what other blocks or copies wrote during its lifetime).
template <bool NC, class T>
__device__ __forceinline__ T ldro(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return __ldcg(p);
}

// Starts moving the 128-byte line holding p into L2 (no register result, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

constexpr int kMaxJ = LINKS_MAX_JOINTS;  // joints per mechanism (bit masks are uint32)
constexpr unsigned kFull = 0xffffffffu;  // every lane of a warp
constexpr float kEmitBudget = 9.5e-6f;

// ---------------------------------------------------------------------------------------
// Plan layout (device, one record per mechanism, padded to n_max joints).
//
// Slots number the joints in solve order: slots [0, nf) are the fixed joints in
// increasing joint index, slot nf is the actuated joint, slot nf+1+d is the joint
// solved by dyad d.  All positions used by the mixed path are relative to the crank
// pivot, kept as float pairs (hi, lo) whose sum carries ~48 bits.
// ---------------------------------------------------------------------------------------
struct PlanDev {
  MechHdr* hdr;          // [cap]
  uint8_t* slot_joint;   // [cap][kMaxJ]
  float4* fixpos;        // [cap][n_max]   fixed slots: (x_h, x_l, y_h, y_l) relative to pivot
  double2* pos64;        // [cap][n_max]   absolute initial positions by slot (FP64 path)
  DyadRec* dyad;         // [cap][n_max - 2]
  int32_t* order;        // [cap]          OK mechanisms sorted by dyad count
  int32_t* order2;       // [cap]          confirmation work list of the two-stage screen
  int32_t* rescue;       // [cap]          mechanisms the screen left to its double-word pass
  int32_t* ctrs;         // [kCtrs]        histogram / cursors / work counters
  int32_t* scan;         // [cap/1024 + 2] block sums of the valid-row scan
  int64_t* scan64;       // [cap/1024 + 2] block sums of the packed rows' joint offsets
  int32_t* row_of;       // [cap]          output row of each mechanism (VALID_ONLY), or -1
  int n_max;
  int max_dyads;
  int64_t cap;
};

// Counter block layout (int32 words inside PlanDev::ctrs).
constexpr int kHist = 0;          // [32] histogram of dyad counts (OK mechanisms)
constexpr int kCursor = 32;       // [32] scatter cursors
constexpr int kWork = 64;         // work counter of the screen / FP64 kernels
constexpr int kWork2 = 65;        // work counter of the emit kernel
constexpr int kNValid = 66;       // number of valid mechanisms (VALID_ONLY rows)
constexpr int kNConfirm = 67;     // length of the two-stage screen's confirmation list
// census counts of the emit (links_emit_census), 64-bit each (two slots)
constexpr int kStatEmitSteps = 68;     // steps the emit computes
constexpr int kStatEmitDW = 70;        // ... that its FP32 bound sends to double-word
constexpr int kStatEmitDWDyads = 72;   // ... in dyad-steps
constexpr int kNRescue = 74;      // length of the screen's rescue list
constexpr int kCtrs = 80;

struct TTable {
  int T = 0;
  float4* cs = nullptr;    // (cos_h, cos_l, sin_h, sin_l) of 2*pi*t/T
  double2* cs64 = nullptr; // (cos, sin) in FP64
};

struct ServeState;
void serve_free(ServeState* s);

// Kernel shapes for plans of one n_max (links_set_tuning; the autotuner's table).
struct Tuning {
  int builder = 0;       // 0 default (warp-flat), 1 thread per mechanism (n_max <= 8), 2 warp-flat
  int screen_lanes = 8;  // lanes per mechanism: 8, 16, 32
  int screen_steps = 0;  // steps per lane: 0 by size (2 when n_max <= 9), 1, 2
  int screen_ctas = 0;   // CTAs per SM of the persistent screen; 0 = as many as fit
  int screen_defer = 0;  // uncertain steps: 0 rescued inline, 1 deferred to a second launch
  int emit_dws = -1;     // double-word slots of the emit in shared memory: -1 by size, 0, 1
  int emit_ctas = 0;     // CTAs per SM of the emit; 0 = as many as fit
};
}  // namespace links

struct links_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  int32_t* d_err = nullptr;  // device error word
  int num_sms = 0;
  std::map<int, links::TTable> tables;
  std::mutex mu;
  // kernel timing (links_profile)
  bool prof = false;
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, std::pair<double, int64_t>> acc;
  int64_t launches = 0;
  // scratch of the retrieval kernels (grown outside graph capture)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  links::ServeState* serve = nullptr;
  std::map<int, links::Tuning> tuning;  // kernel shapes by n_max (set or autotuned)
  int chamfer_prune = 1;                // lower-bound pruning in links_chamfer_topk
};

struct links_plan_s {
  links_ctx ctx = nullptr;
  links::PlanDev d{};
  int64_t B = 0;  // mechanisms in the last build
};

struct links_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace links {

// Error plumbing (abi.cu).
int set_error(int status, const std::string& msg);
int cuda_status(cudaError_t e, const char* what);
#define LINKS_CUDA(call)                                         \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return ::links::cuda_status(_e, #call); \
  } while (0)

const TTable* get_table(links_ctx ctx, int T, int* status);
int ensure_workspace(links_ctx ctx, size_t bytes);
int normalize_paths(links_ctx ctx, int64_t M, int T, const float* in, float* out);
int normalize_maxline(links_ctx ctx, int64_t M, int T, const float* in, float* out, int32_t* pair,
                      float* circ_var);
// Same, for the first *M_dev of at most M_cap curves (count read on the device).
int normalize_paths_count(links_ctx ctx, const int32_t* M_dev, int64_t M_cap, int T, const float* in, float* out);
int chamfer_topk(links_ctx ctx, int Q, int64_t M, int T, const float* q, const float* db, int k, int32_t* idx,
                 float* dist, int prune);
// Indices of the n entries with flags[i] & mask != 0, in increasing order, into
// out_index (up to cap) and their count into *n_out (device); sums holds
// compact_sums_count(n) int32 of scratch.  Asynchronous on stream s.
int64_t compact_sums_count(int64_t n);
int compact_flags(cudaStream_t s, const uint8_t* flags, uint8_t mask, int64_t n, int32_t* sums, int32_t* out_index,
                  int64_t cap, int32_t* n_out);
int curate_paths(links_ctx ctx, int64_t R, int n_max, int T, const float* traj, const int32_t* row_index,
                 int64_t B, const int32_t* n_joints, const uint8_t* adj, const int8_t* type, double circle_var,
                 double keep_rate, uint64_t seed, uint8_t* flags, float* circ_var, int32_t* pair,
                 int32_t* kept_index, float* kept_paths, int64_t kept_capacity, int32_t* n_kept);
int chamfer_first_under(links_ctx ctx, int Q, int64_t M, int T, const float* q, const float* db, int64_t L,
                        const int32_t* order, double thr, int k, int32_t* idx, float* dist, int prune);

// Brackets one kernel launch: counts it and, while profiling, records events around it.
struct KernelScope {
  links_ctx ctx;
  cudaEvent_t b = nullptr;
  KernelScope(links_ctx c, const char* name);
  ~KernelScope();
};

// Device error bits.
constexpr int32_t kErrEmitLock = 1;   // emit found a lock in a mechanism the screen called valid
constexpr int32_t kErrBadIndex = 2;   // an index outside its buffer was skipped

// Entry points implemented per translation unit.
// nbr (device [B, n_max] neighbour masks, may be NULL) replaces adj when given.
int plan_build_device(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                      const uint8_t* adj, const int8_t* type, const void* pos0, int pos_dtype,
                      int32_t* status_out, const uint32_t* nbr = nullptr);
int plan_build_host(links_ctx ctx, links_plan plan, int64_t B, const int32_t* n_joints,
                    const uint8_t* adj, const int8_t* type, const void* pos0, int pos_dtype,
                    int32_t* status_out);
// row_offset (device [out_capacity + 1], VALID_ONLY only): packed rows, see
// links_simulate_packed; traj_capacity in joint rows of T points.
int simulate_f64(links_ctx ctx, links_plan plan, const TTable* tab, int out_mode, double* traj,
                 double* path, uint8_t* valid, int16_t* lock_step, float* min_disc,
                 int32_t* out_index, int64_t out_capacity, int32_t* n_out, int64_t* row_offset = nullptr,
                 int64_t traj_capacity = 0);
int simulate_two_stage(links_ctx ctx, links_plan plan, const TTable* tab_lo, const TTable* tab, float* traj,
                       float* path, uint8_t* valid, int16_t* lock_step, float* min_disc, int32_t* out_index,
                       int64_t out_capacity, int32_t* n_out, int32_t* n_low_valid);
int emit_census(links_ctx ctx, links_plan plan, const TTable* tab, int out_mode, const int16_t* lock_step,
                const int32_t* out_index, int64_t out_capacity, int64_t* out);
int simulate_mixed(links_ctx ctx, links_plan plan, const TTable* tab, int out_mode, float* traj,
                   float* path, uint8_t* valid, int16_t* lock_step, float* min_disc,
                   int32_t* out_index, int64_t out_capacity, int32_t* n_out, int64_t* row_offset = nullptr,
                   int64_t traj_capacity = 0);
// The kernel shapes for plans of n_max joints (defaults where none were set).
Tuning tuning_of(links_ctx ctx, int n_max);
// Times the screen's and the emit's shapes on the built plan and keeps the fastest for
// this n_max (allocates scratch; not inside a capture).
int autotune(links_ctx ctx, links_plan plan, const TTable* tab, int* lanes);
// Shared by both precisions: rows of the valid mechanisms in index order.
// A first screen of the OK mechanisms (see simulate_prescreened).
using Prescreen = std::function<int(links_ctx, links_plan, const TTable*, uint8_t*, int16_t*, float*)>;
int simulate_prescreened(links_ctx ctx, links_plan plan, const TTable* tab, int out_mode, float* traj,
                         float* path, uint8_t* valid, int16_t* lock_step, float* min_disc, int32_t* out_index,
                         int64_t out_capacity, int32_t* n_out, int32_t* n_escaped, const Prescreen& prescreen);
// The plan of one mechanism built on the host (status returned; hdr and dyad records
// [n_max - 2] written).
int plan_one_host(int n, int n_max, const uint8_t* adj, const int8_t* type, const double* pos, MechHdr* hdr,
                  DyadRec* dyad);
int compact_valid(links_ctx ctx, links_plan plan, const uint8_t* valid, int32_t* out_index,
                  int64_t out_capacity, int32_t* n_out);
// Joint offsets of the packed valid rows (after compact_valid): row_offset[r] = sum of
// the joint counts of rows < r, row_offset[rows] = the total.
int pack_offsets(links_ctx ctx, links_plan plan, const int32_t* out_index, int64_t out_capacity,
                 int64_t* row_offset);
int fill_unsimulated(links_ctx ctx, links_plan plan, uint8_t* valid, int16_t* lock_step,
                     float* min_disc);

}  // namespace links
