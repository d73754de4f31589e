// serve.cu -- continuous-batching request loop over the simulation path.
//
// Requests (batches of candidates of mixed joint counts) are submitted from any host
// thread.  A scheduler thread inside the library admits them into a device-resident
// arena when their candidates fit (memory-bounded admission), copies their inputs
// on a copy stream, and runs "passes" on a compute stream: each pass covers every
// request admitted since the previous pass and runs plan build, certified screen,
// valid-row compaction, double-word emission of coupler paths (and trajectories)
// and path normalisation over all of them at once.  Requests that arrive while a
// pass is on the GPU join the next pass; the copies of one pass overlap the compute
// of the next.  Results go back to the caller's host buffers and the ticket
// completes.  All waits are bounded: polling returns LINKS_ETIMEDOUT, and the
// scheduler never blocks on the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "links_internal.cuh"

namespace links {
namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
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
  cudaEvent_t compute_done = nullptr, d2h_done = nullptr;
  int slot = 0;  // n_out slot
  int stage = 0; // 1 = compute issued, 2 = rows copy issued
  int32_t n_valid = 0;
};

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
  int32_t* nout = nullptr;  // [kSlots]
  PlanDev plan{};
  // pinned host staging of the rows of a pass
  int32_t* h_nout = nullptr;
  int32_t* h_idx = nullptr;
  float* h_path = nullptr;
  float* h_traj = nullptr;
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
  static constexpr int kSlots = 64;
  int next_slot = 0;
};

namespace {

size_t bytes_per_mech(int n_max, int T, bool traj) {
  size_t in = (size_t)n_max * n_max + n_max + 8 * n_max + 4;
  size_t plan = sizeof(MechHdr) + kMaxJ + 16 * n_max + 16 * n_max + sizeof(DyadRec) * std::max(1, n_max - 2) + 4;
  size_t out = 4 + 1 + 2 + 4 + 4 + (size_t)T * 8 + (traj ? (size_t)n_max * T * 8 : 0);
  return in + plan + out;
}

PlanDev view(const PlanDev& p, int64_t a) {
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

int launch_pass(ServeState* s, Pass* p) {
  links_ctx c = &s->priv;
  const int64_t a = p->a, B = p->b - p->a;
  links_plan_s pl;
  pl.ctx = c;
  pl.d = view(s->plan, a);
  int st = plan_build_device(c, &pl, B, s->nj + a, s->adj + a * s->n_max * s->n_max, s->type + a * s->n_max,
                             s->pos + a * s->n_max * 2, LINKS_F32, s->status + a);
  if (st) return st;
  int ts = LINKS_OK;
  const TTable* tab = get_table(c, s->T, &ts);
  if (!tab) return ts;
  int32_t* nout = s->nout + p->slot;
  st = simulate_mixed(c, &pl, tab, LINKS_OUT_VALID_ONLY, s->traj ? s->traj + a * s->n_max * s->T * 2 : nullptr,
                      s->path + a * s->T * 2, s->valid + a, s->lock + a, s->md + a, s->idx + a, B, nout);
  if (st) return st;
  st = normalize_paths_count(c, nout, B, s->T, s->path + a * s->T * 2, s->path + a * s->T * 2);
  if (st) return st;
  LINKS_CUDA(cudaMemcpyAsync(s->h_nout + p->slot, nout, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  LINKS_CUDA(cudaEventRecord(p->compute_done, c->stream));
  return LINKS_OK;
}

void finish_pass(ServeState* s, Pass* p) {
  // rows [0, n) of the pass, in increasing arena index, split by request
  const int n = p->n_valid;
  int row = 0;
  for (Req* r : p->reqs) {
    const int64_t lo = r->off - p->a, hi = lo + r->r.count;
    int64_t k = 0;
    while (row < n && s->h_idx[row] < hi) {
      const int64_t i = s->h_idx[row] - lo;
      if (k < r->r.out_capacity) {
        if (r->r.valid_index) r->r.valid_index[k] = (int32_t)i;
        if (r->r.paths) memcpy(r->r.paths + k * s->T * 2, s->h_path + (int64_t)row * s->T * 2, sizeof(float) * s->T * 2);
        if (r->r.traj && s->h_traj)
          memcpy(r->r.traj + k * s->n_max * s->T * 2, s->h_traj + (int64_t)row * s->n_max * s->T * 2,
                 sizeof(float) * s->n_max * s->T * 2);
      }
      ++k;
      ++row;
    }
    r->n_valid = k;
    r->t_done = now_ms();
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (Req* r : p->reqs) {
    r->done = true;
    ring_free(s, r->off, r->r.count);
  }
  s->cv.notify_all();
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
      // the passes in flight plus those of this round leave a slot for one more.
      int64_t run_end = -1;
      int runs = 0;
      while (!s->pending.empty() && !s->paused) {
        Req* r = s->pending.front();
        if ((int)s->inflight.size() + runs + 1 > ServeState::kSlots) break;
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
    // One pass per contiguous run of admitted requests.
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
      s->next_slot = (s->next_slot + 1) % ServeState::kSlots;
      cudaEventCreateWithFlags(&p->compute_done, cudaEventDisableTiming);
      cudaEventCreateWithFlags(&p->d2h_done, cudaEventDisableTiming);
      // inputs on the copy stream, then the compute stream waits for them
      const int nm = s->n_max;
      for (Req* r : p->reqs) {
        const int64_t o = r->off, m = r->r.count;
        cudaMemcpyAsync(s->nj + o, r->r.n_joints, m * 4, cudaMemcpyHostToDevice, s->copy);
        cudaMemcpyAsync(s->adj + o * nm * nm, r->r.adj, m * nm * nm, cudaMemcpyHostToDevice, s->copy);
        cudaMemcpyAsync(s->type + o * nm, r->r.type, m * nm, cudaMemcpyHostToDevice, s->copy);
        cudaMemcpyAsync(s->pos + o * nm * 2, r->r.pos0, m * nm * 8, cudaMemcpyHostToDevice, s->copy);
      }
      cudaEvent_t in_done;
      cudaEventCreateWithFlags(&in_done, cudaEventDisableTiming);
      cudaEventRecord(in_done, s->copy);
      cudaStreamWaitEvent(s->priv.stream, in_done, 0);
      cudaEventDestroy(in_done);
      int st = launch_pass(s, p);
      if (st) {
        s->worker_error = st;
        for (Req* r : p->reqs) r->status = st;
      }
      p->stage = 1;
      s->inflight.push_back(p);
      progressed = true;
    }
    // Retire passes in order.
    while (!s->inflight.empty()) {
      Pass* p = s->inflight.front();
      if (p->stage == 1) {
        if (cudaEventQuery(p->compute_done) != cudaSuccess) break;
        p->n_valid = s->h_nout[p->slot];
        const int64_t B = p->b - p->a, n = std::min<int64_t>(p->n_valid, B);
        // flags straight into the callers' buffers, rows into pinned staging
        for (Req* r : p->reqs) {
          const int64_t o = r->off, m = r->r.count;
          cudaMemcpyAsync(r->r.valid, s->valid + o, m, cudaMemcpyDeviceToHost, s->copy);
          cudaMemcpyAsync(r->r.lock_step, s->lock + o, m * 2, cudaMemcpyDeviceToHost, s->copy);
          if (r->r.min_disc) cudaMemcpyAsync(r->r.min_disc, s->md + o, m * 4, cudaMemcpyDeviceToHost, s->copy);
        }
        if (n > 0) {
          cudaMemcpyAsync(s->h_idx, s->idx + p->a, n * 4, cudaMemcpyDeviceToHost, s->copy);
          cudaMemcpyAsync(s->h_path, s->path + p->a * s->T * 2, n * s->T * 8, cudaMemcpyDeviceToHost, s->copy);
          if (s->traj)
            cudaMemcpyAsync(s->h_traj, s->traj + p->a * s->n_max * s->T * 2, n * s->n_max * s->T * 8,
                            cudaMemcpyDeviceToHost, s->copy);
        }
        cudaEventRecord(p->d2h_done, s->copy);
        p->stage = 2;
        progressed = true;
      }
      if (p->stage == 2) {
        if (cudaEventQuery(p->d2h_done) != cudaSuccess) break;
        // device errors (e.g. from a kernel's error word) fail the pass's requests
        finish_pass(s, p);
        cudaEventDestroy(p->compute_done);
        cudaEventDestroy(p->d2h_done);
        s->inflight.pop_front();
        delete p;
        progressed = true;
      }
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(s->mu);
      if ((s->pending.empty() || s->paused) && !s->stop)
        s->cv.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 2000 : 20));
      else if (!s->inflight.empty())
        s->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
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
  cudaFree(s->nout);
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
  cudaFreeHost(s->h_nout);
  cudaFreeHost(s->h_idx);
  cudaFreeHost(s->h_path);
  cudaFreeHost(s->h_traj);
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
  if (n_max < 2 || n_max > LINKS_MAX_JOINTS || T < 1 || T > 1024 || max_pending < 1)
    return set_error(LINKS_EINVAL, "links_serve_start: need 2 <= n_max <= 32, 1 <= T <= 1024, max_pending >= 1");
  LINKS_CUDA(cudaSetDevice(ctx->device));
  const size_t per = bytes_per_mech(n_max, T, with_traj != 0);
  const int64_t cap = (int64_t)(mem_budget_bytes / per);
  if (cap < 1) return set_error(LINKS_EINVAL, "links_serve_start: memory budget below one candidate");
  if (with_traj && (size_t)cap * n_max * T * 8 > ((size_t)8 << 30))
    return set_error(LINKS_EINVAL, "links_serve_start: with_traj needs a budget whose trajectories fit 8 GiB of staging");
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
  al((void**)&s->nout, ServeState::kSlots * 4);
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
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_nout, ServeState::kSlots * 4, 0);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_idx, cap * 4, 0);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_path, cap * T * 8, 0);
  if (e == cudaSuccess && with_traj) e = cudaHostAlloc((void**)&s->h_traj, cap * n_max * T * 8, 0);
  if (e != cudaSuccess) {
    serve_free(s);
    return cuda_status(e, "links_serve_start");
  }
  int ts = LINKS_OK;
  if (!get_table(&s->priv, T, &ts)) {
    serve_free(s);
    return ts;
  }
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
