// serve.cu -- continuous-batching request loop on the device.
//
// Requests (batches of candidates of mixed joint counts) are submitted from any host
// thread.  A host feeder thread admits them into a device-resident arena when their
// candidates fit (memory-bounded admission), copies their inputs on a copy stream and
// then publishes a pass descriptor (the arena range of the requests admitted together)
// into a descriptor ring in device memory, with the ring's head written by the same
// copy stream after the inputs.  The request loop itself runs on the GPU: one
// persistent cooperative kernel takes the descriptors in order and runs each pass's
// phases -- plan build (warp-flat builder), ordering by dyad count, certified screen,
// ordered valid-row compaction, double-word emit of the coupler paths (and
// trajectories), normalisation -- separated by grid barriers, then reports the pass's
// valid count and completion to mapped host memory.  Requests that arrive while a pass
// runs are copied in meanwhile and published; the kernel takes them as soon as the
// pass ends, without any host launch.  The feeder copies the finished passes' flags
// and row indices, then each request's rows straight from the device into its
// buffers, and completes the tickets.
//
// Every wait is bounded: the kernel's poll for work ends after an idle limit (the
// kernel exits; the feeder relaunches it when work is published), each grid barrier
// gives up after a wall-clock limit and makes the kernel return with an error word
// the feeder reads (the pass's requests then fail with LINKS_EDEVICE), and
// links_serve_poll returns LINKS_ETIMEDOUT after its timeout.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "path_core.cuh"
#include "plan_core.cuh"
#include "sim_core.cuh"

namespace links {
namespace {

constexpr int kSlots = 64;            // passes in flight (each owns a count slot)
constexpr int kRing = 128;            // descriptor ring entries (> kSlots)
constexpr int kAhead = 2;             // passes published and not finished (one runs, one waits)
constexpr int kLoopWarps = 8;         // warps per block of the serving kernel
constexpr int kLoopThreads = 32 * kLoopWarps;
constexpr int kLoopPL = 8;            // normalisation: points per lane (T <= 256)
constexpr int kServeMaxT = 32 * kLoopPL;
constexpr int32_t kLoopErrTimeout = 1;  // a grid barrier's wait ran out
constexpr int32_t kLoopErrEmit = 2;     // the emit found a lock in a mechanism screened valid
constexpr int32_t kLoopErrDesc = 4;     // a descriptor out of sequence or out of the arena
constexpr long long kIdleNs = 2000000;      // the kernel exits after 2 ms without work
constexpr long long kWaitNs = 2000000000;   // a grid barrier gives up after 2 s

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// A pass as the kernel sees it (written by the copy stream into the ring).
struct PassDesc {
  int64_t a, b;              // arena range [a, b)
  unsigned long long seq;    // 1, 2, ... in publication order
  int32_t slot;              // count slot of the mailbox
  int32_t stall;             // fault injection: extra blocks one barrier of the pass waits for
  long long wait_ns;         // the pass's barrier wait limit
};

// Device control block of the serving kernel.
struct LoopCtl {
  unsigned long long head;   // passes published (written by the copy stream)
  unsigned long long quit;   // nonzero: exit at once instead of waiting (copy stream)
  unsigned long long tail;   // passes taken (the kernel)
  unsigned bar_count, bar_gen;
  int64_t a, B;              // the pass being run (block 0 sets them, all read them)
  unsigned long long seq;
  long long wait_ns;
  int32_t slot, exit_flag, stall, emit_err;
};

// Mapped pinned host memory the kernel reports to.
struct Mailbox {
  unsigned long long done;   // passes finished (stored with release after their outputs)
  int32_t err;               // kLoopErr* bits
  int32_t pad;
  int32_t n_valid[kSlots];   // valid rows of each slot's pass
};

struct LoopArgs {
  PlanDev plan;  // over the whole arena
  const int32_t* nj;
  const uint8_t* adj;
  const int8_t* type;
  const float* pos;
  int32_t* status;
  uint8_t* valid;
  int16_t* lock;
  float* md;
  int32_t* idx;
  float* path;
  float* traj;
  int32_t* block_sums;  // [gridDim.x]
  const float4* cs;
  int T;
  LoopCtl* ctl;
  const PassDesc* ring;
  Mailbox* mb;  // device address of the mapped mailbox
  long long idle_ns, wait_ns;
};

__device__ __forceinline__ long long gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier of the serving kernel: every block's thread 0 arrives on a counter, the
// last one (of nb + extra) releases the others through a generation word; a block that
// waits longer than limit_ns records kLoopErrTimeout and returns false (so does every
// block then, and the kernel returns).  Ends with an acquire fence, so the block reads
// what the other blocks wrote before they arrived.
__device__ bool grid_wait(LoopCtl* c, unsigned nb, unsigned extra, long long limit_ns, Mailbox* mb) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire_gpu(&c->bar_gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    if (arrived == nb + extra) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      const long long t0 = gtimer();
      while (ld_acquire_gpu(&c->bar_gen) == gen) {
        if (gtimer() - t0 > limit_ns) {
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    if (!ok) {
      *reinterpret_cast<volatile int32_t*>(&mb->err) = kLoopErrTimeout;
      __threadfence_system();
    }
    s_ok = ok;
  }
  __syncthreads();
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return s_ok != 0;
}

// Exclusive block scan of v over the block's threads; *total = the block's sum.
__device__ int block_excl_scan(int v, int* total) {
  __shared__ int ws[kLoopWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  int base = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < kLoopWarps; ++i) {
    const int wi = ws[i];
    if (i < w) base += wi;
    tot += wi;
  }
  __syncthreads();
  *total = tot;
  return base + x - v;
}

// The plan rows of the arena range starting at mechanism a (the counters are shared).
__host__ __device__ PlanDev plan_view(const PlanDev& p, int64_t a) {
  PlanDev v = p;
  v.hdr += a;
  v.slot_joint += a * kMaxJ;
  v.fixpos += a * p.n_max;
  v.pos64 += a * p.n_max;
  v.dyad += a * p.max_dyads;
  v.order += a;
  v.rescue += a;
  return v;
}

size_t loop_smem_bytes(int nm, int md, int G, bool dws) {
  const size_t build = (size_t)kLoopWarps * FlatSmem<float>::bytes(nm, md, true);
  const size_t screen = (size_t)kLoopWarps * screen_warp_bytes(nm, md, G, 1);
  const size_t emit = (size_t)kLoopWarps * emit_warp_bytes(nm, md, dws);
  return std::max(build, std::max(screen, emit));
}

// The request loop: each iteration takes the next published pass and runs its phases.
template <int G, bool DWS>
__global__ void __launch_bounds__(kLoopThreads, 2) serve_loop_kernel(LoopArgs A) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int s_jofs[kLoopWarps][kMaxJ];
  __shared__ int s_off[32];
  __shared__ long long s_pass[5];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned nb = gridDim.x;
  const int64_t gw = (int64_t)blockIdx.x * kLoopWarps + warp, nw = (int64_t)nb * kLoopWarps;
  LoopCtl* const c = A.ctl;
  const int nm = A.plan.n_max, md = A.plan.max_dyads, T = A.T;
  for (;;) {
    // block 0 waits (bounded) for the next pass and sets it up
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const long long t0 = gtimer();
      int ex = 0;
      for (;;) {
        if (ld_acquire_sys(&c->head) != c->tail) break;
        if (ld_acquire_sys(&c->quit) != 0 || gtimer() - t0 > A.idle_ns) {
          ex = 1;
          break;
        }
        __nanosleep(1000);
      }
      if (!ex) {
        const PassDesc* d = A.ring + (c->tail % kRing);
        const int64_t a = __ldcv(&d->a);
        c->a = a;
        c->B = __ldcv(&d->b) - a;
        c->seq = __ldcv(&d->seq);
        c->slot = __ldcv(&d->slot);
        c->stall = __ldcv(&d->stall);
        c->wait_ns = __ldcv(&d->wait_ns);
        for (int i = 0; i < kCtrs; ++i) A.plan.ctrs[i] = 0;
        // a descriptor out of sequence (or a range outside the arena) is not run
        if (c->seq != c->tail + 1 || a < 0 || c->B < 1 || a + c->B > A.plan.cap || c->slot < 0 || c->slot >= kSlots) {
          *reinterpret_cast<volatile int32_t*>(&A.mb->err) = kLoopErrDesc;
          __threadfence_system();
          ex = 1;
        }
      }
      c->exit_flag = ex;
      __threadfence();
    }
    if (!grid_wait(c, nb, 0, A.idle_ns + A.wait_ns, A.mb)) return;
    if (threadIdx.x == 0) {
      s_pass[0] = __ldcg(&c->exit_flag);
      s_pass[1] = __ldcg(&c->a);
      s_pass[2] = __ldcg(&c->B);
      s_pass[3] = __ldcg(&c->stall);
      s_pass[4] = __ldcg(&c->wait_ns);
    }
    __syncthreads();
    if (s_pass[0]) return;
    const int64_t a = s_pass[1], B = s_pass[2];
    const unsigned stall = (unsigned)s_pass[3];
    const long long wait = s_pass[4];
    const PlanDev p = plan_view(A.plan, a);
    const int32_t* nj = A.nj + a;
    const uint8_t* adj = A.adj + a * nm * nm;
    const int8_t* type = A.type + a * nm;
    const float* pos = A.pos + a * nm * 2;
    uint8_t* valid = A.valid + a;
    int16_t* lock = A.lock + a;
    float* md_out = A.md + a;
    int32_t* idx = A.idx + a;
    float* path = A.path + a * T * 2;

    // 1. plan build: a warp per 32 mechanisms
    {
      const int flags = ((nm % 4 == 0 && ((uintptr_t)adj & 3u) == 0) ? 1 : 0) |
                        ((((uintptr_t)pos & 15u) == 0 && ((uintptr_t)type & 15u) == 0 && nm % 2 == 0) ? 2 : 0);
      char* wsm = smem + warp * FlatSmem<float>::bytes(nm, md, true);
      for (int64_t t = gw; t < (B + 31) / 32; t += nw) {
        const FlatResult r = build_flat_warp<float, false>(B, t * 32, nj, adj, nullptr, type, pos, p, flags, wsm, lane);
        if (r.status >= 0) {
          A.status[a + t * 32 + lane] = r.status;
          if (r.status == LINKS_MECH_OK) atomicAdd(&p.ctrs[kHist + r.nd], 1);
        }
      }
    }
    if (!grid_wait(c, nb, stall, wait, A.mb)) return;
    // 2. the OK mechanisms in order of dyad count; the others' flags
    if (warp == 0) {
      const int v = __ldcg(&p.ctrs[kHist + lane]);
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      s_off[lane] = x - v;
    }
    __syncthreads();
    for (int64_t b = (int64_t)blockIdx.x * kLoopThreads + threadIdx.x; b < B; b += (int64_t)nb * kLoopThreads) {
      const int4 w0 = __ldcg(reinterpret_cast<const int4*>(p.hdr + b));
      if (w0.x == LINKS_MECH_OK) {
        const int nd = (w0.y >> 8) & 0xff;
        p.order[s_off[nd] + atomicAdd(&p.ctrs[kCursor + nd], 1)] = (int32_t)b;
      } else {
        valid[b] = 0;
        lock[b] = -2;
        md_out[b] = __int_as_float(0x7fc00000);
      }
    }
    if (!grid_wait(c, nb, 0, wait, A.mb)) return;
    // 3. the certified screen (uncertain steps rescued at once)
    screen_body<G, 1, true, false>(p, T, A.cs, valid, lock, md_out, p.order, nullptr, smem, warp, lane);
    if (!grid_wait(c, nb, 0, wait, A.mb)) return;
    // 4. valid rows in increasing index: counts per block range, their scan, the rows
    const int64_t chunk = ((B + nb - 1) / nb + kLoopThreads - 1) / kLoopThreads * kLoopThreads;
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(B, lo + chunk);
    {
      int cnt = 0;
      for (int64_t i = lo + threadIdx.x; i < hi; i += kLoopThreads) cnt += __ldcg(valid + i) != 0;
      int tot;
      block_excl_scan(cnt, &tot);
      if (threadIdx.x == 0) A.block_sums[blockIdx.x] = tot;
    }
    if (!grid_wait(c, nb, 0, wait, A.mb)) return;
    if (blockIdx.x == 0) {
      int carry = 0;
      for (unsigned base = 0; base < nb; base += kLoopThreads) {
        const unsigned i = base + threadIdx.x;
        const int v = i < nb ? __ldcg(A.block_sums + i) : 0;
        int tot;
        const int ex = block_excl_scan(v, &tot);
        if (i < nb) A.block_sums[i] = carry + ex;
        carry += tot;
      }
      if (threadIdx.x == 0) p.ctrs[kNValid] = carry;
    }
    if (!grid_wait(c, nb, 0, wait, A.mb)) return;
    {
      int off = __ldcg(A.block_sums + blockIdx.x);
      for (int64_t i0 = lo; i0 < hi; i0 += kLoopThreads) {
        const int64_t i = i0 + threadIdx.x;
        const int v = (i < hi && __ldcg(valid + i) != 0) ? 1 : 0;
        int tot;
        const int ex = block_excl_scan(v, &tot);
        if (v) idx[off + ex] = (int32_t)i;
        off += tot;
      }
    }
    if (!grid_wait(c, nb, 0, wait, A.mb)) return;
    // 5. the coupler paths (and trajectories) of the valid rows
    emit_body<false, DWS, false>(p, B, T, A.cs, 0, lock, idx, B, A.traj ? A.traj + a * nm * T * 2 : nullptr, path,
                                 &c->emit_err, smem, s_jofs[warp], warp, lane, gw, nw, nullptr, 0,
                                 p.ctrs + kWork2);  // rows from a counter (the setup cleared it)
    if (!grid_wait(c, nb, 0, wait, A.mb)) return;
    // 6. their normalisation
    {
      const int64_t n = __ldcg(&p.ctrs[kNValid]);
      float2* path2 = reinterpret_cast<float2*>(path);
      for (int64_t m = gw; m < n; m += nw) normalize_warp<kLoopPL>(m, T, path2, path2, lane);
    }
    if (!grid_wait(c, nb, 0, wait, A.mb)) return;
    // 7. report the pass
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const int slot = __ldcg(&c->slot);
      A.mb->n_valid[slot] = __ldcg(&p.ctrs[kNValid]);
      if (__ldcg(&c->emit_err)) *reinterpret_cast<volatile int32_t*>(&A.mb->err) = kLoopErrEmit;
      __threadfence_system();
      st_release_sys(&A.mb->done, __ldcg(&c->seq));
      c->tail = c->tail + 1;
      __threadfence();
    }
  }
}

struct Req {
  uint64_t ticket;
  links_request r;
  int64_t off = -1;  // arena offset (mechanisms)
  int status = LINKS_OK;
  int64_t n_valid = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  bool done = false;
};

struct Pass {
  int64_t a = 0, b = 0;  // arena range
  std::vector<Req*> reqs;
  cudaEvent_t d2h_done = nullptr;
  unsigned long long seq = 0;
  int slot = 0;   // count slot
  int stage = 0;  // 1 published, 2 flags and row indices being copied, 3 rows being copied, 4 failed
  int32_t n_valid = 0;
};

using LoopFn = void (*)(LoopArgs);

}  // namespace

struct ServeState {
  links_ctx_s priv;  // private context: own stream, tables, error word
  cudaStream_t copy = nullptr;
  int n_max = 0, T = 0;
  int64_t cap = 0;  // arena capacity (mechanisms)
  bool want_traj = false;
  // device arena
  int32_t* nj = nullptr;
  uint8_t* adj = nullptr;
  int8_t* type = nullptr;
  float* pos = nullptr;
  int32_t* status = nullptr;
  uint8_t* valid = nullptr;
  int16_t* lock = nullptr;
  float* md = nullptr;
  int32_t* idx = nullptr;
  float* path = nullptr;
  float* traj = nullptr;
  int32_t* block_sums = nullptr;
  PlanDev plan{};
  // the device loop
  LoopCtl* ctl = nullptr;
  PassDesc* ring = nullptr;
  PassDesc* h_desc = nullptr;             // [kRing] pinned sources of the ring copies
  unsigned long long* h_head = nullptr;   // [kRing] pinned sources of the head copies
  unsigned long long* h_ctl = nullptr;    // pinned sources of the quit and reset copies
  Mailbox* mb = nullptr;                  // mapped pinned mailbox (host address)
  Mailbox* mb_dev = nullptr;              // its device address
  LoopFn loop_fn = nullptr;
  int loop_grid = 0;
  size_t loop_smem = 0;
  const float4* cs = nullptr;
  cudaEvent_t loop_done = nullptr;
  bool loop_running = false;
  unsigned long long published = 0;
  int stall_next = 0;          // fault injection: the next pass's barrier waits for a missing block
  long long stall_wait_ns = 0;
  int64_t loop_launches = 0;
  int32_t last_loop_err = 0;  // the kernel's error word when it last returned with one
  unsigned long long last_done = 0;
  int idle_launches = 0;       // launches since the finished-pass count last moved
  // pinned host staging of the row indices of a pass
  int32_t* h_idx = nullptr;
  // scheduling
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::map<uint64_t, Req*> tickets;
  std::deque<Pass*> inflight;
  int64_t head = 0, tail = 0, used = 0;  // ring over [0, cap)
  uint64_t next_ticket = 1;
  int max_pending = 0;
  bool stop = false;
  bool paused = false;
  std::thread worker;
  int worker_error = LINKS_OK;
  int next_slot = 0;
};

namespace {

size_t bytes_per_mech(int n_max, int T, bool traj) {
  size_t in = (size_t)n_max * n_max + n_max + 8 * n_max + 4;
  size_t plan = sizeof(MechHdr) + kMaxJ + 16 * n_max + 16 * n_max + sizeof(DyadRec) * std::max(1, n_max - 2) + 8;
  size_t out = 4 + 1 + 2 + 4 + 4 + (size_t)T * 8 + (traj ? (size_t)n_max * T * 8 : 0);
  return in + plan + out;
}

// Ring allocation of `n` contiguous mechanisms; returns the offset or -1.  Occupied:
// [tail, head) when head >= tail, else [tail, cap) and [0, head) (the end of the ring
// past the last allocation before a wrap is counted as used until it drains).  A
// wrapped ring never lets head reach tail, so head == tail means empty.
int64_t ring_alloc(ServeState* s, int64_t n) {
  if (n > s->cap) return -1;
  if (s->used == 0) s->head = s->tail = 0;
  if (s->head >= s->tail) {
    if (s->cap - s->head >= n) {
      int64_t o = s->head;
      s->head += n;
      s->used += n;
      return o;
    }
    if (s->tail > n) {
      s->used += s->cap - s->head + n;
      s->head = n;
      return 0;
    }
    return -1;
  }
  if (s->tail - s->head > n) {
    int64_t o = s->head;
    s->head += n;
    s->used += n;
    return o;
  }
  return -1;
}

// Frees the oldest allocation [off, off + n) (passes complete in admission order).
void ring_free(ServeState* s, int64_t off, int64_t n) {
  if (off != s->tail) {  // the wrap left [tail, cap) unused
    s->used -= s->cap - s->tail;
    s->tail = 0;
  }
  s->tail = off + n;
  s->used -= n;
  if (s->used <= 0) {
    s->used = 0;
    s->head = s->tail = 0;
  }
}

int launch_loop(ServeState* s) {
  LoopArgs A;
  A.plan = s->plan;
  A.nj = s->nj;
  A.adj = s->adj;
  A.type = s->type;
  A.pos = s->pos;
  A.status = s->status;
  A.valid = s->valid;
  A.lock = s->lock;
  A.md = s->md;
  A.idx = s->idx;
  A.path = s->path;
  A.traj = s->traj;
  A.block_sums = s->block_sums;
  A.cs = s->cs;
  A.T = s->T;
  A.ctl = s->ctl;
  A.ring = s->ring;
  A.mb = s->mb_dev;
  A.idle_ns = kIdleNs;
  A.wait_ns = kWaitNs;
  void* args[] = {&A};
  LINKS_CUDA(cudaLaunchCooperativeKernel((const void*)s->loop_fn, dim3(s->loop_grid), dim3(kLoopThreads), args,
                                         s->loop_smem, s->priv.stream));
  LINKS_CUDA(cudaEventRecord(s->loop_done, s->priv.stream));
  s->loop_running = true;
  ++s->loop_launches;
  return LINKS_OK;
}

// The pass's row indices are in host staging (increasing arena index): each request's
// valid rows are one contiguous range of them.  Its indices go to valid_index, and its
// paths (and trajectories) are copied from the device straight into its buffers.
void copy_rows(ServeState* s, Pass* p) {
  const int64_t n = std::min<int64_t>(p->n_valid, p->b - p->a);
  int64_t row = 0;
  for (Req* r : p->reqs) {
    const int64_t lo = r->off - p->a, hi = lo + r->r.count;
    const int64_t first = row;
    while (row < n && s->h_idx[row] < hi) ++row;
    r->n_valid = row - first;
    const int64_t k = std::min<int64_t>(r->n_valid, r->r.out_capacity);
    if (r->r.valid_index)
      for (int64_t q = 0; q < k; ++q) r->r.valid_index[q] = (int32_t)(s->h_idx[first + q] - lo);
    if (k > 0 && r->r.paths)
      cudaMemcpyAsync(r->r.paths, s->path + (p->a + first) * s->T * 2, k * s->T * 8, cudaMemcpyDeviceToHost, s->copy);
    if (k > 0 && r->r.traj && s->traj)
      cudaMemcpyAsync(r->r.traj, s->traj + (p->a + first) * s->n_max * s->T * 2, k * s->n_max * s->T * 8,
                      cudaMemcpyDeviceToHost, s->copy);
  }
}

void finish_pass(ServeState* s, Pass* p) {
  const double t = now_ms();
  std::lock_guard<std::mutex> lk(s->mu);
  for (Req* r : p->reqs) {
    if (p->stage == 4) r->n_valid = 0;
    r->t_done = t;
    r->done = true;
    ring_free(s, r->off, r->r.count);
  }
  s->cv.notify_all();
}

// After the loop kernel returned with an error: the published passes not finished fail,
// and the control block is reset so that a new launch starts from the next pass.
void loop_failed(ServeState* s, int32_t err) {
  s->last_loop_err = err;
  // LINKS_EDEVICE (not LINKS_ETIMEDOUT, which links_serve_poll returns for a ticket
  // still running): the kernel's error word says which wait ran out
  (void)err;
  const int st = LINKS_EDEVICE;
  const unsigned long long done = *reinterpret_cast<volatile unsigned long long*>(&s->mb->done);
  for (Pass* p : s->inflight)
    if (p->stage == 1 && p->seq > done) {
      p->stage = 4;
      for (Req* r : p->reqs) r->status = st;
    }
  // the copies of every published pass are complete before the control block changes
  cudaStreamSynchronize(s->copy);
  s->h_ctl[1] = s->published;  // the next launch starts after the last published pass
  cudaMemcpyAsync(&s->ctl->tail, &s->h_ctl[1], sizeof(unsigned long long), cudaMemcpyHostToDevice, s->priv.stream);
  cudaMemsetAsync(&s->ctl->bar_count, 0, sizeof(unsigned), s->priv.stream);
  cudaMemsetAsync(&s->ctl->emit_err, 0, sizeof(int32_t), s->priv.stream);
  cudaStreamSynchronize(s->priv.stream);
  *reinterpret_cast<volatile unsigned long long*>(&s->mb->done) = s->published;
  *reinterpret_cast<volatile int32_t*>(&s->mb->err) = 0;
}

void worker_main(ServeState* s) {
  cudaSetDevice(s->priv.device);
  while (true) {
    std::vector<Req*> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->pending.empty() && s->inflight.empty()) break;
      // Each pass owns one of kSlots count slots until it retires.  A request may open
      // a new pass (one per contiguous run of the ring), so it is admitted only while
      // the passes in flight plus those this admission step opens leave a slot for one more.
      int64_t run_end = -1;
      int runs = 0;
      // Continuous batching: at most kAhead passes wait for the kernel; requests that
      // arrive meanwhile gather into the next pass.
      const unsigned long long done_now = *reinterpret_cast<volatile unsigned long long*>(&s->mb->done);
      const bool room = s->published - done_now < (unsigned long long)kAhead;
      while (room && !s->pending.empty() && !s->paused) {
        Req* r = s->pending.front();
        if ((int)s->inflight.size() + runs + 1 > kSlots) break;
        int64_t off = ring_alloc(s, r->r.count);
        if (off < 0) break;
        if (off != run_end) ++runs;
        run_end = off + r->r.count;
        r->off = off;
        r->t_admit = now_ms();
        admitted.push_back(r);
        s->pending.pop_front();
      }
    }
    bool progressed = false;
    // One pass per contiguous run of admitted requests: inputs, then its descriptor and
    // the ring head, all on the copy stream (so the kernel sees the head only after the
    // inputs are in place).
    size_t i = 0;
    while (i < admitted.size()) {
      Pass* p = new Pass();
      p->a = admitted[i]->off;
      p->b = p->a;
      while (i < admitted.size() && admitted[i]->off == p->b) {
        p->reqs.push_back(admitted[i]);
        p->b += admitted[i]->r.count;
        ++i;
      }
      p->slot = s->next_slot;
      s->next_slot = (s->next_slot + 1) % kSlots;
      cudaEventCreateWithFlags(&p->d2h_done, cudaEventDisableTiming);
      const int nm = s->n_max;
      for (Req* r : p->reqs) {
        const int64_t o = r->off, m = r->r.count;
        cudaMemcpyAsync(s->nj + o, r->r.n_joints, m * 4, cudaMemcpyHostToDevice, s->copy);
        cudaMemcpyAsync(s->adj + o * nm * nm, r->r.adj, m * nm * nm, cudaMemcpyHostToDevice, s->copy);
        cudaMemcpyAsync(s->type + o * nm, r->r.type, m * nm, cudaMemcpyHostToDevice, s->copy);
        cudaMemcpyAsync(s->pos + o * nm * 2, r->r.pos0, m * nm * 8, cudaMemcpyHostToDevice, s->copy);
      }
      p->seq = ++s->published;
      const int e = (int)((p->seq - 1) % kRing);  // the kernel takes pass seq from entry (seq - 1) mod kRing
      PassDesc& d = s->h_desc[e];
      d.a = p->a;
      d.b = p->b;
      d.seq = p->seq;
      d.slot = p->slot;
      d.stall = s->stall_next;
      d.wait_ns = s->stall_next ? s->stall_wait_ns : kWaitNs;
      s->stall_next = 0;
      s->h_head[e] = p->seq;
      cudaMemcpyAsync(s->ring + e, &d, sizeof(PassDesc), cudaMemcpyHostToDevice, s->copy);
      cudaMemcpyAsync(&s->ctl->head, &s->h_head[e], sizeof(unsigned long long), cudaMemcpyHostToDevice, s->copy);
      p->stage = 1;
      s->inflight.push_back(p);
      progressed = true;
    }
    // Keep the device loop running while published passes are not finished.
    if (s->loop_running && cudaEventQuery(s->loop_done) == cudaSuccess) {
      s->loop_running = false;
      const int32_t err = *reinterpret_cast<volatile int32_t*>(&s->mb->err);
      if (err) loop_failed(s, err);
      progressed = true;
    }
    unsigned long long done = *reinterpret_cast<volatile unsigned long long*>(&s->mb->done);
    std::atomic_thread_fence(std::memory_order_acquire);
    if (done != s->last_done) {
      s->last_done = done;
      s->idle_launches = 0;
    }
    // a kernel that keeps exiting without taking the published pass: fail it rather than
    // relaunch forever
    if (!s->loop_running && done < s->published && s->idle_launches > 1000) {
      loop_failed(s, kLoopErrDesc);
      s->idle_launches = 0;
      done = *reinterpret_cast<volatile unsigned long long*>(&s->mb->done);
    }
    if (!s->loop_running && done < s->published) {
      ++s->idle_launches;
      const int st = launch_loop(s);
      if (st) {
        s->worker_error = st;
        for (Pass* p : s->inflight)
          if (p->stage == 1) {
            p->stage = 4;
            for (Req* r : p->reqs) r->status = st;
          }
      }
      progressed = true;
    }
    // Retire passes in order: flags and row indices, then the rows, then the tickets.
    while (!s->inflight.empty()) {
      Pass* p = s->inflight.front();
      if (p->stage == 1) {
        if (done < p->seq) break;
        p->n_valid = *reinterpret_cast<volatile int32_t*>(&s->mb->n_valid[p->slot]);
        const int64_t B = p->b - p->a, n = std::min<int64_t>(p->n_valid, B);
        for (Req* r : p->reqs) {  // flags straight into the callers' buffers
          const int64_t o = r->off, m = r->r.count;
          cudaMemcpyAsync(r->r.valid, s->valid + o, m, cudaMemcpyDeviceToHost, s->copy);
          cudaMemcpyAsync(r->r.lock_step, s->lock + o, m * 2, cudaMemcpyDeviceToHost, s->copy);
          if (r->r.min_disc) cudaMemcpyAsync(r->r.min_disc, s->md + o, m * 4, cudaMemcpyDeviceToHost, s->copy);
        }
        if (n > 0) cudaMemcpyAsync(s->h_idx, s->idx + p->a, n * 4, cudaMemcpyDeviceToHost, s->copy);
        cudaEventRecord(p->d2h_done, s->copy);
        p->stage = 2;
        progressed = true;
      }
      if (p->stage == 2) {
        if (cudaEventQuery(p->d2h_done) != cudaSuccess) break;
        copy_rows(s, p);
        cudaEventRecord(p->d2h_done, s->copy);
        p->stage = 3;
        progressed = true;
      }
      if (p->stage == 3 && cudaEventQuery(p->d2h_done) != cudaSuccess) break;
      finish_pass(s, p);  // stage 3 with its copies done, or 4 (failed)
      cudaEventDestroy(p->d2h_done);
      s->inflight.pop_front();
      delete p;
      progressed = true;
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(s->mu);
      if ((s->pending.empty() || s->paused) && !s->stop)
        s->cv.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 2000 : 20));
      else if (!s->inflight.empty())
        s->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
  // ask the loop to exit and wait for it (its poll and barriers are bounded)
  s->h_ctl[0] = 1;
  cudaMemcpyAsync(&s->ctl->quit, &s->h_ctl[0], sizeof(unsigned long long), cudaMemcpyHostToDevice, s->copy);
  cudaStreamSynchronize(s->copy);
  cudaStreamSynchronize(s->priv.stream);
}

}  // namespace

void serve_free(ServeState* s) {
  cudaFree(s->nj);
  cudaFree(s->adj);
  cudaFree(s->type);
  cudaFree(s->pos);
  cudaFree(s->status);
  cudaFree(s->valid);
  cudaFree(s->lock);
  cudaFree(s->md);
  cudaFree(s->idx);
  cudaFree(s->path);
  cudaFree(s->traj);
  cudaFree(s->block_sums);
  cudaFree(s->ctl);
  cudaFree(s->ring);
  PlanDev& d = s->plan;
  cudaFree(d.hdr);
  cudaFree(d.slot_joint);
  cudaFree(d.fixpos);
  cudaFree(d.pos64);
  cudaFree(d.dyad);
  cudaFree(d.order);
  cudaFree(d.rescue);
  cudaFree(d.ctrs);
  cudaFree(d.scan);
  cudaFreeHost(s->h_idx);
  cudaFreeHost(s->h_desc);
  cudaFreeHost(s->h_head);
  cudaFreeHost(s->h_ctl);
  cudaFreeHost(s->mb);
  if (s->loop_done) cudaEventDestroy(s->loop_done);
  if (s->copy) cudaStreamDestroy(s->copy);
  if (s->priv.stream) cudaStreamDestroy(s->priv.stream);
  for (auto& kv : s->priv.tables) {
    cudaFree(kv.second.cs);
    cudaFree(kv.second.cs64);
  }
  if (s->priv.d_err) cudaFree(s->priv.d_err);
  if (s->priv.ws) cudaFree(s->priv.ws);
  for (auto& kv : s->tickets) delete kv.second;
  delete s;
}

}  // namespace links

using namespace links;

extern "C" {

int links_serve_start(links_ctx ctx, size_t mem_budget_bytes, int max_pending, int n_max, int T, int with_traj) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_serve_start: NULL ctx");
  if (ctx->serve) return set_error(LINKS_ESTATE, "links_serve_start: already serving");
  if (n_max < 2 || n_max > LINKS_MAX_JOINTS || T < 1 || T > kServeMaxT || max_pending < 1)
    return set_error(LINKS_EINVAL, "links_serve_start: need 2 <= n_max <= 32, 1 <= T <= 256, max_pending >= 1");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  int coop = 0;
  LINKS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  if (!coop) return set_error(LINKS_ESTATE, "links_serve_start: the device has no cooperative launch");
  const size_t per = bytes_per_mech(n_max, T, with_traj != 0);
  const int64_t cap = (int64_t)(mem_budget_bytes / per);
  if (cap < 1) return set_error(LINKS_EINVAL, "links_serve_start: memory budget below one candidate");
  if (cap > INT32_MAX) return set_error(LINKS_EINVAL, "links_serve_start: memory budget above 2^31 candidates");
  ServeState* s = new (std::nothrow) ServeState();
  if (!s) return set_error(LINKS_ENOMEM, "links_serve_start: host allocation");
  s->priv.device = ctx->device;
  s->priv.num_sms = ctx->num_sms;
  s->n_max = n_max;
  s->T = T;
  s->cap = cap;
  s->max_pending = max_pending;
  s->want_traj = with_traj != 0;
  cudaError_t e = cudaStreamCreateWithFlags(&s->priv.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->loop_done, cudaEventDisableTiming);
  auto al = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  al((void**)&s->priv.d_err, 4);
  al((void**)&s->nj, cap * 4);
  al((void**)&s->adj, cap * n_max * n_max);
  al((void**)&s->type, cap * n_max);
  al((void**)&s->pos, cap * n_max * 8);
  al((void**)&s->status, cap * 4);
  al((void**)&s->valid, cap);
  al((void**)&s->lock, cap * 2);
  al((void**)&s->md, cap * 4);
  al((void**)&s->idx, cap * 4);
  al((void**)&s->path, cap * T * 8);
  if (with_traj) al((void**)&s->traj, cap * n_max * T * 8);
  al((void**)&s->ctl, sizeof(LoopCtl));
  al((void**)&s->ring, sizeof(PassDesc) * kRing);
  PlanDev& d = s->plan;
  d.n_max = n_max;
  d.max_dyads = std::max(1, n_max - 2);
  d.cap = cap;
  al((void**)&d.hdr, sizeof(MechHdr) * cap);
  al((void**)&d.slot_joint, (size_t)kMaxJ * cap);
  al((void**)&d.fixpos, sizeof(float4) * n_max * cap);
  al((void**)&d.pos64, sizeof(double2) * n_max * cap);
  al((void**)&d.dyad, sizeof(DyadRec) * d.max_dyads * cap);
  al((void**)&d.order, sizeof(int32_t) * cap);
  al((void**)&d.rescue, sizeof(int32_t) * cap);
  al((void**)&d.ctrs, sizeof(int32_t) * kCtrs);
  al((void**)&d.scan, sizeof(int32_t) * (cap / 1024 + 2));
  if (e == cudaSuccess) e = cudaMemset(s->priv.d_err, 0, 4);
  if (e == cudaSuccess) e = cudaMemset(s->ctl, 0, sizeof(LoopCtl));
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_idx, cap * 4, 0);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_desc, sizeof(PassDesc) * kRing, 0);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_head, sizeof(unsigned long long) * kRing, 0);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_ctl, 2 * sizeof(unsigned long long), 0);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->mb, sizeof(Mailbox), cudaHostAllocMapped);
  if (e == cudaSuccess) {
    memset(s->mb, 0, sizeof(Mailbox));
    e = cudaHostGetDevicePointer((void**)&s->mb_dev, s->mb, 0);
  }
  // the serving kernel: lanes per mechanism of the screen from the context's shape table
  const Tuning tun = tuning_of(ctx, n_max);
  const int G = tun.screen_lanes == 16 ? 16 : 8;
  const bool dws = tun.emit_dws < 0 ? n_max <= kEmitSharedDWMaxSlots : tun.emit_dws != 0;
  s->loop_fn = G == 16 ? (dws ? serve_loop_kernel<16, true> : serve_loop_kernel<16, false>)
                       : (dws ? serve_loop_kernel<8, true> : serve_loop_kernel<8, false>);
  s->loop_smem = loop_smem_bytes(n_max, d.max_dyads, G, dws);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)s->loop_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->loop_smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s->loop_fn, kLoopThreads, s->loop_smem);
  if (e == cudaSuccess) {
    if (per_sm < 1) e = cudaErrorInvalidConfiguration;
    s->loop_grid = s->priv.num_sms * per_sm;
    al((void**)&s->block_sums, sizeof(int32_t) * (size_t)s->loop_grid);
  }
  if (e != cudaSuccess) {
    serve_free(s);
    return cuda_status(e, "links_serve_start");
  }
  int ts = LINKS_OK;
  const TTable* tab = get_table(&s->priv, T, &ts);
  if (!tab) {
    serve_free(s);
    return ts;
  }
  s->cs = tab->cs;
  if (cudaStreamSynchronize(s->priv.stream) != cudaSuccess) {
    serve_free(s);
    return set_error(LINKS_ECUDA, "links_serve_start: table setup failed");
  }
  s->worker = std::thread(worker_main, s);
  ctx->serve = s;
  return LINKS_OK;
}

int links_serve_submit(links_ctx ctx, const links_request* req, uint64_t* ticket) {
  if (!ctx || !req || !ticket) return set_error(LINKS_EINVAL, "links_serve_submit: NULL argument");
  ServeState* s = ctx->serve;
  if (!s) return set_error(LINKS_ESTATE, "links_serve_submit: serving not started");
  if (req->count < 1 || !req->n_joints || !req->adj || !req->type || !req->pos0 || !req->valid || !req->lock_step)
    return set_error(LINKS_EINVAL, "links_serve_submit: empty request or NULL buffer");
  if (req->out_capacity < 0) return set_error(LINKS_EINVAL, "links_serve_submit: out_capacity < 0");
  if (req->count > s->cap) return set_error(LINKS_ECAPACITY, "links_serve_submit: request larger than the memory budget");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return set_error(LINKS_ESTATE, "links_serve_submit: serving is stopping");
  if ((int)s->pending.size() >= s->max_pending) return set_error(LINKS_EBUSY, "links_serve_submit: queue full");
  Req* r = new (std::nothrow) Req();
  if (!r) return set_error(LINKS_ENOMEM, "links_serve_submit: host allocation");
  r->ticket = s->next_ticket++;
  r->r = *req;
  r->t_submit = now_ms();
  s->pending.push_back(r);
  s->tickets[r->ticket] = r;
  *ticket = r->ticket;
  s->cv.notify_all();
  return LINKS_OK;
}

int links_serve_poll(links_ctx ctx, uint64_t ticket, int timeout_us, links_result* res) {
  if (!ctx || !res) return set_error(LINKS_EINVAL, "links_serve_poll: NULL argument");
  ServeState* s = ctx->serve;
  if (!s) return set_error(LINKS_ESTATE, "links_serve_poll: serving not started");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return set_error(LINKS_EINVAL, "links_serve_poll: unknown ticket");
  Req* r = it->second;
  if (!r->done) {
    s->cv.wait_for(lk, std::chrono::microseconds(std::max(timeout_us, 0)), [&] { return r->done; });
    if (!r->done) return set_error(LINKS_ETIMEDOUT, "links_serve_poll: not finished");
  }
  res->status = r->status;
  res->n_valid = r->n_valid;
  res->submit_ms = r->t_submit;
  res->admit_ms = r->t_admit;
  res->done_ms = r->t_done;
  s->tickets.erase(it);
  delete r;
  return res->status;
}

int links_serve_pause(links_ctx ctx, int paused) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_serve_pause: NULL ctx");
  ServeState* s = ctx->serve;
  if (!s) return set_error(LINKS_ESTATE, "links_serve_pause: serving not started");
  std::lock_guard<std::mutex> lk(s->mu);
  s->paused = paused != 0;
  s->cv.notify_all();
  return LINKS_OK;
}

int links_serve_inject_stall(links_ctx ctx, int wait_ms) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_serve_inject_stall: NULL ctx");
  ServeState* s = ctx->serve;
  if (!s) return set_error(LINKS_ESTATE, "links_serve_inject_stall: serving not started");
  if (wait_ms < 1 || wait_ms > 10000)
    return set_error(LINKS_EINVAL, "links_serve_inject_stall: wait_ms out of [1, 10000]");
  std::lock_guard<std::mutex> lk(s->mu);
  s->stall_next = 1;
  s->stall_wait_ns = (long long)wait_ms * 1000000LL;
  return LINKS_OK;
}

int links_serve_stats(links_ctx ctx, int64_t* out) {
  if (!ctx || !out) return set_error(LINKS_EINVAL, "links_serve_stats: NULL argument");
  ServeState* s = ctx->serve;
  if (!s) return set_error(LINKS_ESTATE, "links_serve_stats: serving not started");
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = (int64_t)s->published;
  out[1] = s->loop_launches;
  out[2] = s->loop_grid;
  out[3] = s->cap;
  out[4] = s->last_loop_err;
  out[5] = (int64_t)*reinterpret_cast<volatile unsigned long long*>(&s->mb->done);
  return LINKS_OK;
}

int links_serve_stop(links_ctx ctx) {
  if (!ctx) return set_error(LINKS_EINVAL, "links_serve_stop: NULL ctx");
  ServeState* s = ctx->serve;
  if (!s) return set_error(LINKS_ESTATE, "links_serve_stop: serving not started");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->paused = false;
    s->cv.notify_all();
  }
  s->worker.join();
  cudaStreamSynchronize(s->priv.stream);
  cudaStreamSynchronize(s->copy);
  int st = s->worker_error;
  ctx->serve = nullptr;
  serve_free(s);
  return st;
}

}  // extern "C"
