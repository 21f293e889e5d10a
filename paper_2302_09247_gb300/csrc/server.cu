// Served form of the C ABI: a request loop with continuous batching (see
// fastcod_server_* in fastcod.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fc_ctx.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int32_t kOverflowCtas = 64;
constexpr size_t kDefaultChunkReserve = (size_t)256 << 20;

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Chunk {
  const int32_t* xyz;
  int64_t nv;
  const int64_t* off;
  int64_t ns;
  bool host_xyz, host_off;
};

enum class RState { Waiting, Setup, Active, Finishing, Done };

struct Request {
  uint64_t id = 0;
  fastcod_subject head{};
  bool host_roi = false, host_lab = false;
  std::deque<Chunk> chunks;
  bool last_pushed = false;
  std::atomic<RState> state{RState::Waiting};  // written by the worker, read by callers
  std::atomic<bool> cancel{false};
  std::atomic<int> status{FASTCOD_OK};
  size_t reserve = 0;  // bytes counted against the budget
  // device
  char* mem = nullptr;  // volumes, accumulators, state
  fc::VolView v{};
  fc::Accum acc{};
  DevState* st = nullptr;
  DevState* host_state = nullptr;  // page-locked, from the server's pool while admitted
  cudaEvent_t done_ev = nullptr;
  int64_t streamlines = 0, chunks_done = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

// A device buffer that host chunks are copied into.  It is kept for the
// server's life and handed out again once `reusable` (recorded on the
// compute stream after the pass that read it) has completed.
struct StageBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaEvent_t reusable = nullptr;
  bool taken = false;
  bool keep = true;  // false: beyond the server's number of kept buffers, freed after its pass
};

// One chunk staged for the current iteration.
struct Staged {
  Request* r;
  fc::Tract t;
  StageBuf* buf;  // server-owned staging (nullptr: the chunk is device memory)
};

}  // namespace

struct fastcod_server {
  std::atomic<int64_t> kernel_launches{0};  // this library's kernels launched by the worker
  int device = 0;
  int num_sms = 0;
  int32_t max_slots = 1;
  int64_t budget = 0;
  int64_t reserved = 0;
  uint32_t mode = 0;
  int prefilter = 1;
  int ctas = 2;
  int tma = 1;
  int near_log2 = -1;
  Clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv;       // wakes the worker
  std::condition_variable done_cv;  // wakes waiters
  std::thread worker;
  bool stop = false;
  std::string err;

  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::deque<uint64_t> waiting;
  std::vector<Request*> active;
  uint64_t next_id = 1;

  cudaStream_t compute = nullptr, copy = nullptr;
  cudaEvent_t copied = nullptr;
  // stream-ordered allocations of the loop come from a pool of the server's
  // own that keeps its memory between iterations (release threshold at the
  // maximum) and never makes an allocation wait for another stream's free
  // (no internal dependencies: a chunk's copy must not queue behind the
  // compute stream); blocks whose free has completed are reused
  cudaMemPool_t pool = nullptr;
  // iteration buffers (stream-ordered allocations on the compute stream)
  DevState* gst = nullptr;
  int32_t* lists = nullptr;  // survivors | overflow
  size_t lists_cap = 0;      // entries per list
  fc::BatchTask* tasks = nullptr;
  size_t tasks_cap = 0;
  uint32_t* scratch = nullptr;
  int64_t scratch_words = 0;
  fc::BatchTable* tbl = nullptr;
  // page-locked host memory, so that no copy of the loop waits for the
  // compute stream: the task tables of the last two iterations (reused once
  // their copy event has passed) and one state block per slot
  fc::BatchTask* tasks_host[2] = {nullptr, nullptr};
  size_t tasks_host_cap[2] = {0, 0};
  cudaEvent_t tasks_ev[2] = {nullptr, nullptr};
  int tasks_turn = 0;
  DevState* state_pool = nullptr;
  std::vector<DevState*> free_states;
  // host-side failure injection (FASTCOD_FAULT, read at creation): the k-th
  // per-request device allocation, the k-th chunk copy, the k-th submitted
  // request (0: none)
  int64_t fault_alloc = 0, fault_h2d = 0, fault_cancel = 0;
  int64_t n_alloc = 0, n_h2d = 0, n_submit = 0;  // worker / submit counters
  // staging buffers of host chunks, reused: an allocation per chunk from the
  // pool could block the loop for milliseconds whenever the blocks freed by
  // the compute stream were not yet reusable and the pool mapped new memory
  std::list<StageBuf> stage_bufs;
  size_t stage_kept = 0;  // buffers with keep set: at most 2 * max_slots + 2
};

namespace {

double now_s(fastcod_server* S) { return std::chrono::duration<double>(Clock::now() - S->t0).count(); }

// Staging buffers grow in 64 MiB steps, so that chunks of nearby sizes share
// them.
constexpr size_t kStageStep = (size_t)64 << 20;

// A staging buffer of at least `bytes` whose last reader has finished: a kept
// one when there is one, else a new one (from the pool, on the copy stream).
cudaError_t stage_acquire(fastcod_server* S, size_t bytes, StageBuf** out) {
  StageBuf* best = nullptr;
  for (StageBuf& b : S->stage_bufs) {
    if (b.taken || b.bytes < bytes || (best && b.bytes >= best->bytes)) continue;
    const cudaError_t q = cudaEventQuery(b.reusable);
    if (q == cudaErrorNotReady) {
      (void)cudaGetLastError();
      continue;
    }
    if (q != cudaSuccess) return q;
    best = &b;
  }
  if (!best) {
    StageBuf b;
    b.bytes = (bytes + kStageStep - 1) / kStageStep * kStageStep;
    cudaError_t e = cudaMallocFromPoolAsync(&b.p, b.bytes, S->pool, S->copy);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&b.reusable, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaFreeAsync(b.p, S->copy);
      return e;
    }
    b.keep = S->stage_kept < 2 * (size_t)S->max_slots + 2;
    if (b.keep) ++S->stage_kept;
    S->stage_bufs.push_back(b);
    best = &S->stage_bufs.back();
  }
  best->taken = true;
  *out = best;
  return cudaSuccess;
}

// The buffer may be handed out again once `s` has passed this point (a buffer
// beyond the kept number is freed there instead).
void stage_release(fastcod_server* S, StageBuf* b, cudaStream_t s) {
  if (!b->keep) {
    cudaFreeAsync(b->p, s);
    cudaEventDestroy(b->reusable);
    for (auto it = S->stage_bufs.begin(); it != S->stage_bufs.end(); ++it)
      if (&*it == b) {
        S->stage_bufs.erase(it);
        break;
      }
    return;
  }
  cudaEventRecord(b->reusable, s);
  b->taken = false;
}

// FASTCOD_FAULT = comma-separated "alloc:k", "h2d:k", "cancel:k" (k >= 1).
void parse_faults(fastcod_server* S) {
  const char* env = getenv("FASTCOD_FAULT");
  if (!env) return;
  std::string s(env);
  size_t at = 0;
  while (at < s.size()) {
    size_t end = s.find(',', at);
    if (end == std::string::npos) end = s.size();
    const std::string item = s.substr(at, end - at);
    const size_t colon = item.find(':');
    if (colon != std::string::npos) {
      const long long k = atoll(item.c_str() + colon + 1);
      const std::string what = item.substr(0, colon);
      if (k > 0 && what == "alloc") S->fault_alloc = k;
      if (k > 0 && what == "h2d") S->fault_h2d = k;
      if (k > 0 && what == "cancel") S->fault_cancel = k;
    }
    at = end + 1;
  }
}

// Worker: whether this per-request allocation / chunk copy is the one to fail.
bool inject_alloc(fastcod_server* S) { return S->fault_alloc && ++S->n_alloc == S->fault_alloc; }
bool inject_h2d(fastcod_server* S) { return S->fault_h2d && ++S->n_h2d == S->fault_h2d; }

int64_t near_words(const int32_t d[3], int near_log2) {
  fc::VolView v{};
  v.dx = d[0];
  v.dy = d[1];
  v.dz = d[2];
  fc::set_near_dims(v, fc::resolve_near_log2(near_log2, d[0], d[1], d[2]));
  return fc::near_words(v);
}

// Device bytes a request holds while admitted (without chunk staging).
size_t resident_bytes(const fastcod_subject& h, int near_log2) {
  const int64_t nvox = (int64_t)h.dims[0] * h.dims[1] * h.dims[2];
  const int64_t nb = (int64_t)((h.dims[0] + 3) / 4) * ((h.dims[1] + 3) / 4) * ((h.dims[2] + 3) / 4);
  const size_t nm = (size_t)h.n_roi * (size_t)h.n_targets;
  return a256(nvox * 4) + a256(nvox * 2) + a256((nb + 15) / 16 * 4) + a256((size_t)near_words(h.dims, near_log2) * 4) +
         2 * a256(nm * 4) + a256(sizeof(DevState));
}

size_t chunk_bytes(const Chunk& k) { return a256((size_t)k.nv * 12 + 16) + a256((size_t)(k.ns + 1) * 8); }

// Worker: allocate and prepare an admitted request's volumes (compute stream).
cudaError_t setup_request(fastcod_server* S, Request* r, uint32_t** tmp, size_t* tmp_cap) {
  const fastcod_subject& h = r->head;
  const int64_t nvox = (int64_t)h.dims[0] * h.dims[1] * h.dims[2];
  const int64_t nb = (int64_t)((h.dims[0] + 3) / 4) * ((h.dims[1] + 3) / 4) * ((h.dims[2] + 3) / 4);
  const size_t nm = (size_t)h.n_roi * (size_t)h.n_targets;
  size_t bytes = resident_bytes(h, S->near_log2);
  const size_t in_bytes = (r->host_roi ? a256(nvox * 4) : 0) + (r->host_lab ? a256(nvox * 2) : 0);
  if (inject_alloc(S)) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMallocFromPoolAsync((void**)&r->mem, bytes + in_bytes, S->pool, S->compute);
  if (e != cudaSuccess) return e;
  char* p = r->mem;
  auto take = [&](size_t n) {
    char* q = p;
    p += a256(n);
    return q;
  };
  fc::VolView& v = r->v;
  v.code = reinterpret_cast<uint32_t*>(take(nvox * 4));
  v.lab = reinterpret_cast<uint16_t*>(take(nvox * 2));
  v.bricks = reinterpret_cast<uint32_t*>(take((nb + 15) / 16 * 4));
  v.near = reinterpret_cast<uint32_t*>(take((size_t)near_words(h.dims, S->near_log2) * 4));
  r->acc.C = reinterpret_cast<int32_t*>(take(nm * 4));
  r->acc.Cend = reinterpret_cast<int32_t*>(take(nm * 4));
  r->st = reinterpret_cast<DevState*>(take(sizeof(DevState)));
  const int32_t* roi = h.roi_index_map;
  const uint16_t* lab = h.target_labels;
  if (r->host_roi) {
    int32_t* d = reinterpret_cast<int32_t*>(take(nvox * 4));
    e = cudaMemcpyAsync(d, roi, nvox * 4, cudaMemcpyHostToDevice, S->compute);
    roi = d;
  }
  if (e == cudaSuccess && r->host_lab) {
    uint16_t* d = reinterpret_cast<uint16_t*>(take(nvox * 2));
    e = cudaMemcpyAsync(d, lab, nvox * 2, cudaMemcpyHostToDevice, S->compute);
    lab = d;
  }
  v.dx = h.dims[0];
  v.dy = h.dims[1];
  v.dz = h.dims[2];
  v.bx = (h.dims[0] + 3) / 4;
  v.by = (h.dims[1] + 3) / 4;
  v.bz = (h.dims[2] + 3) / 4;
  fc::set_near_dims(v, fc::resolve_near_log2(S->near_log2, h.dims[0], h.dims[1], h.dims[2]));
  v.n_roi = h.n_roi;
  v.n_lab = h.n_targets;
  if (e == cudaSuccess) e = cudaMemsetAsync(r->acc.C, 0, nm * 4, S->compute);
  if (e == cudaSuccess) e = cudaMemsetAsync(r->acc.Cend, 0, nm * 4, S->compute);
  if (e == cudaSuccess) e = cudaMemsetAsync(r->st, 0, sizeof(DevState), S->compute);
  if (e == cudaSuccess) e = cudaMemsetAsync(const_cast<uint32_t*>(v.bricks), 0, (nb + 15) / 16 * 4, S->compute);
  const size_t need = (size_t)fc::plane_words(h.dims[0], h.dims[1], h.dims[2]) * 4;
  if (e == cudaSuccess && need > *tmp_cap) {
    if (*tmp) e = cudaFreeAsync(*tmp, S->compute);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)tmp, need, S->pool, S->compute);
    if (e == cudaSuccess) *tmp_cap = need;
  }
  if (e == cudaSuccess)
    e = fc::launch_volume_prep(roi, lab, nvox, v, const_cast<uint32_t*>(v.code), const_cast<uint16_t*>(v.lab),
                               const_cast<uint32_t*>(v.bricks), *tmp, r->st, S->compute);
  if (e == cudaSuccess) e = fc::launch_near(v, *tmp, const_cast<uint32_t*>(v.near), S->compute);
  if (e == cudaSuccess) S->kernel_launches += 2;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
  return e;
}

cudaError_t grow_iteration_buffers(fastcod_server* S, size_t entries, size_t ntasks, int64_t words) {
  cudaError_t e = cudaSuccess;
  if (entries > S->lists_cap) {
    if (S->lists) e = cudaFreeAsync(S->lists, S->compute);
    const size_t cap = std::max(entries, S->lists_cap * 2);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&S->lists, cap * 8, S->pool, S->compute);
    if (e == cudaSuccess) S->lists_cap = cap;
  }
  if (e == cudaSuccess && ntasks > S->tasks_cap) {
    if (S->tasks) e = cudaFreeAsync(S->tasks, S->compute);
    const size_t cap = std::max(ntasks, S->tasks_cap * 2);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&S->tasks, cap * sizeof(fc::BatchTask), S->pool, S->compute);
    if (e == cudaSuccess) S->tasks_cap = cap;
  }
  if (e == cudaSuccess && words > S->scratch_words) {
    if (S->scratch) e = cudaFreeAsync(S->scratch, S->compute);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&S->scratch, (size_t)kOverflowCtas * words * 4, S->pool, S->compute);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->scratch, 0, (size_t)kOverflowCtas * words * 4, S->compute);
    if (e == cudaSuccess) S->scratch_words = words;
  }
  return e;
}

void fail_request(fastcod_server* S, Request* r, int status) {
  r->status = status;
  r->state = RState::Done;
  r->t_done = now_s(S);
}

// One pass of the loop: admit, set up, run one batched pass over the next
// chunk of every active request, complete finished requests.  Returns true
// when it did any work.
bool iterate(fastcod_server* S, uint32_t** tmp, size_t* tmp_cap) {
  fcapi::Range nvtx_range("fastcod_server pass");
  std::vector<Request*> setups, finishing;
  std::vector<std::pair<Request*, Chunk>> work;
  std::vector<std::pair<Request*, bool>> lasts;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    // cancellations of waiting requests
    for (auto it = S->waiting.begin(); it != S->waiting.end();) {
      Request* r = S->reqs[*it].get();
      if (r->cancel) {
        fail_request(S, r, FASTCOD_ECANCELED);
        it = S->waiting.erase(it);
        S->done_cv.notify_all();
      } else {
        ++it;
      }
    }
    // admission in arrival order
    while (!S->waiting.empty() && (int32_t)S->active.size() < S->max_slots) {
      Request* r = S->reqs[S->waiting.front()].get();
      size_t stage = kDefaultChunkReserve;
      if (!r->chunks.empty()) stage = chunk_bytes(r->chunks.front());
      const size_t need = resident_bytes(r->head, S->near_log2) + 2 * stage;
      if (S->reserved + (int64_t)need > S->budget && !S->active.empty()) break;
      S->reserved += (int64_t)need;
      r->reserve = need;
      r->host_state = S->free_states.back();  // active requests <= slots = pool size
      S->free_states.pop_back();
      r->state = RState::Setup;
      r->t_admit = now_s(S);
      S->active.push_back(r);
      S->waiting.pop_front();
      setups.push_back(r);
    }
    // survivor ids of one pass are int32: the chunks of a pass hold at most
    // 2^31 - 1 streamlines (a chunk that would pass that waits for the next
    // pass; every chunk alone is within it)
    int64_t pass_ns = 0;
    for (Request* r : S->active) {
      if (r->state == RState::Active && r->cancel) {
        r->state = RState::Finishing;
        r->status = FASTCOD_ECANCELED;
        finishing.push_back(r);
        continue;
      }
      if ((r->state == RState::Active || r->state == RState::Setup) && !r->chunks.empty()) {
        if (pass_ns + r->chunks.front().ns > 0x7fffffffLL) continue;
        pass_ns += r->chunks.front().ns;
        work.emplace_back(r, r->chunks.front());
        r->chunks.pop_front();
        lasts.emplace_back(r, r->last_pushed && r->chunks.empty());
      } else if (r->state == RState::Active && r->last_pushed && r->chunks.empty()) {
        // an empty last chunk: nothing more to run
        lasts.emplace_back(r, true);
      }
    }
  }
  bool did = !setups.empty() || !work.empty() || !finishing.empty();
  for (Request* r : setups) {
    const cudaError_t e = setup_request(S, r, tmp, tmp_cap);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      std::lock_guard<std::mutex> lk(S->mu);
      r->status = e == cudaErrorMemoryAllocation ? FASTCOD_ENOMEM : FASTCOD_ECUDA;
    }
    r->state = RState::Active;
  }
  // stage the chunks on the copy stream
  std::vector<Staged> staged;
  int64_t total_ns = 0;
  int64_t words = 1;
  size_t ntasks = 0;
  for (auto& w : work) {
    Request* r = w.first;
    const Chunk& k = w.second;
    Staged sg{r, fc::Tract{k.xyz, k.off, k.nv, k.ns}, nullptr};
    if (r->status != FASTCOD_OK) continue;
    if (k.host_xyz || k.host_off) {
      const size_t xb = a256((size_t)k.nv * 12 + 16);
      cudaError_t e = inject_alloc(S) ? cudaErrorMemoryAllocation
                                      : stage_acquire(S, xb + (size_t)(k.ns + 1) * 8, &sg.buf);
      if (e == cudaSuccess && inject_h2d(S)) e = cudaErrorInvalidValue;  // the copy "fails" before it is issued
      if (e == cudaSuccess && k.host_xyz && k.nv) {
        e = cudaMemcpyAsync(sg.buf->p, k.xyz, (size_t)k.nv * 12, cudaMemcpyDefault, S->copy);
        sg.t.xyz = static_cast<int32_t*>(sg.buf->p);
      }
      if (e == cudaSuccess && k.host_off) {
        int64_t* o = reinterpret_cast<int64_t*>(static_cast<char*>(sg.buf->p) + xb);
        e = cudaMemcpyAsync(o, k.off, (size_t)(k.ns + 1) * 8, cudaMemcpyHostToDevice, S->copy);
        sg.t.off = o;
      }
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        r->status = e == cudaErrorMemoryAllocation ? FASTCOD_ENOMEM : FASTCOD_ECUDA;
        if (sg.buf) stage_release(S, sg.buf, S->copy);  // nothing reads it: free once the copies issued are done
        continue;
      }
    }
    staged.push_back(sg);
    total_ns += k.ns;
    words = std::max(words, fc::overflow_scratch_words(r->head.n_roi, r->head.n_targets));
    ntasks += (size_t)std::max<int64_t>(1, (k.nv + 65535) / 65536);
  }
  if (!staged.empty() && total_ns > 0x7fffffffLL) {
    // cannot happen (the work list is limited above); fail the requests
    // rather than return partial results
    for (const Staged& sg : staged) {
      sg.r->status = FASTCOD_EINVAL;
      if (sg.buf) stage_release(S, sg.buf, S->compute);
    }
    staged.clear();
  }
  if (!staged.empty()) {
    cudaEventRecord(S->copied, S->copy);
    cudaStreamWaitEvent(S->compute, S->copied, 0);
    cudaError_t e = grow_iteration_buffers(S, (size_t)total_ns, ntasks, words);
    fc::BatchTable& tbl = *S->tbl;
    memset(&tbl, 0, sizeof tbl);
    std::vector<fc::BatchTask> tasks;
    int64_t sbase = 0;
    for (size_t i = 0; i < staged.size(); ++i) {
      const Staged& sg = staged[i];
      fc::BatchSubject& B = tbl.s[i];
      B.v = sg.r->v;
      B.t = sg.t;
      B.acc = sg.r->acc;
      B.st = sg.r->st;
      B.sbase = sbase;
      sbase += sg.t.ns;
      const int64_t k = std::max<int64_t>(1, (sg.t.nv + 65535) / 65536);
      for (int64_t j = 0; j < k; ++j) {
        fc::BatchTask t{(int32_t)i, 0, sg.t.ns * j / k, sg.t.ns * (j + 1) / k};
        tasks.push_back(t);
      }
    }
    tbl.n = (int32_t)staged.size();
    // the task table goes through one of two page-locked buffers
    const int turn = S->tasks_turn;
    S->tasks_turn ^= 1;
    if (e == cudaSuccess) e = cudaEventSynchronize(S->tasks_ev[turn]);  // its copy two iterations ago is done
    if (e == cudaSuccess && tasks.size() > S->tasks_host_cap[turn]) {
      if (S->tasks_host[turn]) cudaFreeHost(S->tasks_host[turn]);
      S->tasks_host[turn] = nullptr;
      S->tasks_host_cap[turn] = 0;
      const size_t cap = std::max(tasks.size(), (size_t)1024);
      e = cudaMallocHost((void**)&S->tasks_host[turn], cap * sizeof(fc::BatchTask));
      if (e == cudaSuccess) S->tasks_host_cap[turn] = cap;
    }
    if (e == cudaSuccess) {
      memcpy(S->tasks_host[turn], tasks.data(), tasks.size() * sizeof(fc::BatchTask));
      e = cudaMemcpyAsync(S->tasks, S->tasks_host[turn], tasks.size() * sizeof(fc::BatchTask), cudaMemcpyHostToDevice,
                          S->compute);
    }
    if (e == cudaSuccess) e = cudaEventRecord(S->tasks_ev[turn], S->compute);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->gst, 0, sizeof(DevState), S->compute);
    if (e == cudaSuccess)
      e = fc::launch_prefilter_batch(tbl, S->tasks, (int32_t)tasks.size(), S->prefilter != 0, S->tma != 0, S->ctas,
                                     S->lists, (int64_t)S->lists_cap, S->gst, S->num_sms, S->compute);
    if (e == cudaSuccess)
      e = fc::launch_walk_batch(tbl, S->lists, (int64_t)S->lists_cap, S->mode, S->lists + S->lists_cap, S->gst,
                                S->num_sms, S->compute);
    if (e == cudaSuccess)
      e = fc::launch_walk_overflow_batch(tbl, S->lists + S->lists_cap, S->mode, S->scratch, kOverflowCtas, S->scratch_words,
                                         S->gst, S->compute);
    if (e == cudaSuccess) S->kernel_launches += 3;
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      for (const Staged& sg : staged) sg.r->status = FASTCOD_ECUDA;
    }
    for (const Staged& sg : staged) {
      if (sg.buf) stage_release(S, sg.buf, S->compute);
      sg.r->streamlines += sg.t.ns;
      sg.r->chunks_done += 1;
    }
  }
  // requests whose last chunk has been enqueued: results out, completion event
  for (auto& l : lasts) {
    if (!l.second) continue;
    Request* r = l.first;
    r->state = RState::Finishing;
    finishing.push_back(r);
  }
  for (Request* r : finishing) {
    const size_t nm = (size_t)r->head.n_roi * (size_t)r->head.n_targets;
    if (r->status == FASTCOD_OK && r->mem) {
      cudaMemcpyAsync(r->head.C_out, r->acc.C, nm * 4, cudaMemcpyDefault, S->compute);
      cudaMemcpyAsync(r->head.Cend_out, r->acc.Cend, nm * 4, cudaMemcpyDefault, S->compute);
    }
    if (r->mem) cudaMemcpyAsync(r->host_state, r->st, sizeof(DevState), cudaMemcpyDeviceToHost, S->compute);
    if (r->done_ev) cudaEventRecord(r->done_ev, S->compute);
  }
  // completion
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto it = S->active.begin(); it != S->active.end();) {
      Request* r = *it;
      if (r->state != RState::Finishing) {
        ++it;
        continue;
      }
      const cudaError_t q = r->done_ev ? cudaEventQuery(r->done_ev) : cudaSuccess;
      if (q == cudaErrorNotReady) {
        ++it;
        continue;
      }
      (void)cudaGetLastError();
      if (r->status == FASTCOD_OK && r->mem && r->host_state->error != fc::kErrNone)
        r->status = r->host_state->error == fc::kErrTimeout   ? FASTCOD_ETIMEOUT
                    : r->host_state->error == fc::kErrChecked ? FASTCOD_ECUDA
                                                               : FASTCOD_EINVAL;
      S->free_states.push_back(r->host_state);
      r->host_state = nullptr;
      if (r->mem) cudaFreeAsync(r->mem, S->compute);
      r->mem = nullptr;
      if (r->done_ev) cudaEventDestroy(r->done_ev);
      r->done_ev = nullptr;
      S->reserved -= (int64_t)r->reserve;
      r->state = RState::Done;
      r->t_done = now_s(S);
      it = S->active.erase(it);
      did = true;
      S->done_cv.notify_all();
    }
  }
  return did;
}

void worker_main(fastcod_server* S) {
  cudaSetDevice(S->device);
  uint32_t* tmp = nullptr;
  size_t tmp_cap = 0;
  for (;;) {
    const bool did = iterate(S, &tmp, &tmp_cap);
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->stop && S->waiting.empty() && S->active.empty()) break;
    if (!did) S->cv.wait_for(lk, std::chrono::microseconds(200));
  }
  if (tmp) cudaFreeAsync(tmp, S->compute);
  cudaStreamSynchronize(S->compute);
}

int sfail(fastcod_server* S, int code, const char* msg) {
  S->err = msg;
  return code;
}

}  // namespace

extern "C" {

FASTCOD_API int fastcod_server_create(fastcod_ctx* c, int32_t max_slots, int64_t hbm_budget_bytes,
                                      fastcod_server** out) {
  if (!c || !out) return FASTCOD_EINVAL;
  *out = nullptr;
  if (max_slots < 1 || max_slots > fc::kMaxBatch) return fcapi::fail(c, FASTCOD_EINVAL, "max_slots must be in 1..%d", fc::kMaxBatch);
  if (hbm_budget_bytes < 0) return fcapi::fail(c, FASTCOD_EINVAL, "negative budget");
  CU(cudaSetDevice(c->device));
  fastcod_server* S = new (std::nothrow) fastcod_server;
  if (!S) return fcapi::fail(c, FASTCOD_ENOMEM, "host allocation failed");
  S->device = c->device;
  S->num_sms = c->num_sms;
  S->max_slots = max_slots;
  S->mode = c->mode;
  S->prefilter = c->prefilter;
  S->ctas = c->prefilter_ctas;
  S->tma = c->staging_tma;
  S->near_log2 = c->near_log2;
  S->t0 = Clock::now();
  parse_faults(S);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  S->budget = hbm_budget_bytes ? hbm_budget_bytes : (int64_t)(free_b / 10 * 9);
  S->tbl = new (std::nothrow) fc::BatchTable;
  cudaError_t e = S->tbl ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    e = cudaMemPoolCreate(&S->pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) {
    int no = 0;
    e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->compute, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->copied, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&S->gst, sizeof(DevState));
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&S->tasks_ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&S->state_pool, sizeof(DevState) * (size_t)max_slots);
  if (e == cudaSuccess) {
    memset(S->state_pool, 0, sizeof(DevState) * (size_t)max_slots);
    for (int32_t k = 0; k < max_slots; ++k) S->free_states.push_back(S->state_pool + k);
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (S->compute) cudaStreamDestroy(S->compute);
    if (S->copy) cudaStreamDestroy(S->copy);
    if (S->copied) cudaEventDestroy(S->copied);
    for (int k = 0; k < 2; ++k)
      if (S->tasks_ev[k]) cudaEventDestroy(S->tasks_ev[k]);
    if (S->state_pool) cudaFreeHost(S->state_pool);
    cudaFree(S->gst);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S->tbl;
    delete S;
    return fcapi::fail(c, FASTCOD_ECUDA, "server initialisation failed");
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_server_submit(fastcod_server* S, const fastcod_subject* h, uint64_t* id) {
  if (!S || !h || !id) return FASTCOD_EINVAL;
  if (h->dims[0] <= 0 || h->dims[1] <= 0 || h->dims[2] <= 0 ||
      (int64_t)h->dims[0] * h->dims[1] * h->dims[2] >= ((int64_t)1 << 31))
    return sfail(S, FASTCOD_EINVAL, "invalid grid dims");
  if (h->n_roi <= 0 || h->n_roi >= (1 << 30) || h->n_targets <= 0 || h->n_targets > 65535)
    return sfail(S, FASTCOD_EINVAL, "need 0 < n_roi < 2^30 and 0 < n_targets < 65536");
  if (!h->roi_index_map || !h->target_labels || !h->C_out || !h->Cend_out) return sfail(S, FASTCOD_EINVAL, "NULL pointer");
  cudaSetDevice(S->device);
  const int kr = fcapi::ptr_kind(h->roi_index_map, S->device), kl = fcapi::ptr_kind(h->target_labels, S->device);
  if (kr < 0 || kl < 0 || fcapi::ptr_kind(h->C_out, S->device) < 0 || fcapi::ptr_kind(h->Cend_out, S->device) < 0)
    return sfail(S, FASTCOD_EINVAL, "device memory of another device");
  auto r = std::make_unique<Request>();
  r->head = *h;
  r->host_roi = kr == 0;
  r->host_lab = kl == 0;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return sfail(S, FASTCOD_ESTATE, "server is stopping");
  r->id = S->next_id++;
  r->t_submit = now_s(S);
  if (S->fault_cancel && ++S->n_submit == S->fault_cancel) r->cancel = true;  // injected cancellation
  *id = r->id;
  S->waiting.push_back(r->id);
  S->reqs[r->id] = std::move(r);
  S->cv.notify_one();
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_server_push_chunk(fastcod_server* S, uint64_t id, const int32_t* xyz, int64_t nv,
                                          const int64_t* offsets, int64_t ns, int32_t last) {
  if (!S) return FASTCOD_EINVAL;
  if (ns < 0 || nv < 0 || nv > 0x7fffffffLL || (ns > 0 && !offsets) || (nv > 0 && !xyz))
    return sfail(S, FASTCOD_EINVAL, "invalid chunk");
  Chunk k{xyz, nv, offsets, ns, false, false};
  if (ns > 0) {
    const int kx = nv ? fcapi::ptr_kind(xyz, S->device) : 1, ko = fcapi::ptr_kind(offsets, S->device);
    if (kx < 0 || ko < 0) return sfail(S, FASTCOD_EINVAL, "device memory of another device");
    // staged on the copy stream: host xyz, and device xyz off a 16-byte
    // boundary (the prefilter's bulk copies need aligned sources)
    k.host_xyz = kx == 0 || (nv && ((uintptr_t)xyz & 15u));
    k.host_off = ko == 0;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return sfail(S, FASTCOD_EINVAL, "no such request");
  Request* r = it->second.get();
  if (r->last_pushed || r->state == RState::Done) return sfail(S, FASTCOD_ESTATE, "request already complete");
  if (ns > 0) r->chunks.push_back(k);
  if (last) r->last_pushed = true;
  S->cv.notify_one();
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_server_poll(fastcod_server* S, uint64_t id, int32_t* done) {
  if (!S || !done) return FASTCOD_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return sfail(S, FASTCOD_EINVAL, "no such request");
  *done = it->second->state == RState::Done ? 1 : 0;
  return *done ? it->second->status.load() : FASTCOD_OK;
}

FASTCOD_API int fastcod_server_wait(fastcod_server* S, uint64_t id, double timeout_s) {
  if (!S) return FASTCOD_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return sfail(S, FASTCOD_EINVAL, "no such request");
  Request* r = it->second.get();
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (r->state != RState::Done) {
    if (S->done_cv.wait_until(lk, until) == std::cv_status::timeout && r->state != RState::Done) return FASTCOD_ETIMEOUT;
  }
  return r->status;
}

FASTCOD_API int fastcod_server_cancel(fastcod_server* S, uint64_t id) {
  if (!S) return FASTCOD_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return sfail(S, FASTCOD_EINVAL, "no such request");
  it->second->cancel = true;
  S->cv.notify_one();
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_server_request_info(fastcod_server* S, uint64_t id, fastcod_request_info* out) {
  if (!S || !out) return FASTCOD_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return sfail(S, FASTCOD_EINVAL, "no such request");
  const Request* r = it->second.get();
  out->status = r->status;
  out->done = r->state == RState::Done ? 1 : 0;
  out->streamlines = r->streamlines;
  out->chunks = r->chunks_done;
  out->t_submit = r->t_submit;
  out->t_admit = r->t_admit;
  out->t_done = r->t_done;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_server_kernel_launches(fastcod_server* S, int64_t* out) {
  if (!S || !out) return FASTCOD_EINVAL;
  *out = S->kernel_launches.load();
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_server_destroy(fastcod_server* S) {
  if (!S) return FASTCOD_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    // requests that will never receive their last chunk cannot finish: cancel them
    for (auto& kv : S->reqs)
      if (kv.second->state != RState::Done && !kv.second->last_pushed) kv.second->cancel = true;
    S->cv.notify_one();
  }
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  cudaStreamSynchronize(S->compute);
  cudaStreamSynchronize(S->copy);
  for (auto& kv : S->reqs) {
    if (kv.second->mem) cudaFree(kv.second->mem);
    if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
  }
  for (StageBuf& b : S->stage_bufs) {
    cudaFree(b.p);
    cudaEventDestroy(b.reusable);
  }
  if (S->lists) cudaFree(S->lists);
  if (S->tasks) cudaFree(S->tasks);
  if (S->scratch) cudaFree(S->scratch);
  cudaFree(S->gst);
  cudaEventDestroy(S->copied);
  for (int k = 0; k < 2; ++k) {
    cudaEventDestroy(S->tasks_ev[k]);
    if (S->tasks_host[k]) cudaFreeHost(S->tasks_host[k]);
  }
  cudaFreeHost(S->state_pool);
  cudaStreamDestroy(S->compute);
  cudaStreamDestroy(S->copy);
  cudaMemPoolDestroy(S->pool);  // released once no allocation of it is outstanding
  delete S->tbl;
  delete S;
  return FASTCOD_OK;
}

}  // extern "C"
