// Serving runtime: many CB-GMRES solves on one GPU with continuous batching.
//
// The server reserves its HBM budget once (one cudaMalloc) and hands out solver workspaces from
// it with a first-fit allocator, so admitting and finishing requests never allocates, frees or
// synchronises the device. Each slot has its own stream and pinned control block; a solve's
// Arnoldi steps are enqueued on its slot's stream in turns of steps_per_turn steps, so the
// steps of different requests overlap on the device. The solve itself is the same code path as
// cbgmres_solve (solver.cu), which keeps each result independent of the rest of the mix.
//
// Flow control: a slot enqueues its next turn only when the turn before the previous one has
// run (two events per slot). The host therefore stays at most two turns ahead of the device
// for every slot and never blocks on a full launch queue.
#include <chrono>
#include <cstring>
#include <iterator>
#include <list>
#include <map>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

using namespace cbg;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, size), 256-byte granules, free neighbours coalesced.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) {
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t at = it->first + bytes, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    used_ -= bytes;
    size_t start = off, len = bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    if (next != free_.end() && off + bytes == next->first) {
      len += next->second;
      free_.erase(next);
    }
    free_[start] = len;
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  size_t size_;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
};

enum SlotState { kFree = 0, kValidate = 1, kRun = 2 };

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t turn_ev[2] = {nullptr, nullptr};
  bool turn_pending[2] = {false, false};
  int turn = 0;  // index of the event the next turn records
  void* pinned = nullptr;
  int state = kFree;
  cbg_ctx* ctx = nullptr;
  cbg_request req{};
  size_t off = 0, bytes = 0;
  double t_submit = 0.0, t_admit = 0.0;
};

struct Queued {
  cbg_request req;
  size_t bytes;
  double t_submit;
  int bypassed;
};

}  // namespace

struct cbg_server {
  void* dmem = nullptr;
  void* pinned = nullptr;
  Arena arena{0};
  int steps_per_turn = 1;
  int max_bypass = 0;
  std::vector<Slot> slots;
  std::list<Queued> queue;
  std::list<cbg_completion> done;
  std::chrono::steady_clock::time_point t0;
  int active = 0;
};

namespace {

double clock_of(const cbg_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

void push_completion(cbg_server* s, uint64_t tag, int status, const cbg_result* r, double t_submit, double t_admit) {
  cbg_completion c;
  std::memset(&c, 0, sizeof(c));
  c.tag = tag;
  c.status = status;
  if (r) c.result = *r;
  c.result.status = status;
  c.t_submit = t_submit;
  c.t_admit = t_admit;
  c.t_done = clock_of(s);
  s->done.push_back(c);
}

// Ends the slot's solve: the context is released (its stream is idle unless the solve failed
// mid-enqueue, in which case release waits for that stream alone) and its workspace returns to
// the arena.
void finish_slot(cbg_server* s, Slot& sl, int status, const cbg_result* r) {
  ctx_release(sl.ctx);
  sl.ctx = nullptr;
  for (int i = 0; i < 2; ++i) sl.turn_pending[i] = false;
  s->arena.release(sl.off, sl.bytes);
  push_completion(s, sl.req.tag, status, r, sl.t_submit, sl.t_admit);
  sl.state = kFree;
  --s->active;
}

// Whether the turn recorded two turns ago has run (0 yes, 1 not yet, < 0 CUDA error).
int turn_blocked(Slot& sl) {
  const int k = sl.turn;
  if (!sl.turn_pending[k]) return 0;
  cudaError_t q = cudaEventQuery(sl.turn_ev[k]);
  if (q == cudaErrorNotReady) return 1;
  if (q != cudaSuccess) return cuda_fail(q, "server turn event");
  sl.turn_pending[k] = false;
  return 0;
}

int record_turn(Slot& sl) {
  const int k = sl.turn;
  cudaError_t e = cudaEventRecord(sl.turn_ev[k], sl.stream);
  if (e != cudaSuccess) return cuda_fail(e, "server turn record");
  sl.turn_pending[k] = true;
  sl.turn ^= 1;
  return CBG_OK;
}

void progress(cbg_server* s, Slot& sl) {
  if (sl.state == kValidate) {
    const int v = ctx_validated(sl.ctx);
    if (v == 0) return;
    if (v < 0) {
      finish_slot(s, sl, v, nullptr);
      return;
    }
    int st = cbgmres_start(sl.ctx, sl.req.d_b, sl.req.d_x);
    if (st) {
      finish_slot(s, sl, st, nullptr);
      return;
    }
    sl.state = kRun;
    st = record_turn(sl);
    if (st) finish_slot(s, sl, st, nullptr);
    return;
  }
  const int b = turn_blocked(sl);
  if (b == 1) return;
  if (b < 0) {
    finish_slot(s, sl, b, nullptr);
    return;
  }
  int32_t fin = 0;
  int st = cbgmres_advance(sl.ctx, s->steps_per_turn, &fin);
  if (fin) {
    cbg_result r;
    std::memset(&r, 0, sizeof(r));
    const int fs = cbgmres_finish(sl.ctx, &r);
    finish_slot(s, sl, fs, &r);
    return;
  }
  if (st && st != CBG_ERR_NOT_CONVERGED) {
    finish_slot(s, sl, st, nullptr);
    return;
  }
  st = record_turn(sl);
  if (st) finish_slot(s, sl, st, nullptr);
}

// Admits queued requests in arrival order while a slot is free and the workspace fits. A request
// that does not fit is passed by later ones at most max_bypass times.
void admit(cbg_server* s) {
  std::vector<std::list<Queued>::iterator> passed;
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Slot* free_slot = nullptr;
    for (auto& sl : s->slots) {
      if (sl.state == kFree) {
        free_slot = &sl;
        break;
      }
    }
    if (!free_slot) return;
    size_t off = 0;
    if (!s->arena.alloc(it->bytes, &off)) {
      if (it->bypassed >= s->max_bypass) return;  // it goes next: admit nothing else before it
      passed.push_back(it);
      ++it;
      continue;
    }
    Slot& sl = *free_slot;
    const cbg_request& r = it->req;
    cbg_ctx* c = nullptr;
    const double t_admit = clock_of(s);
    int st = ctx_create_in(&c, r.n, r.nnz, r.d_row_ptr, r.d_col, r.d_vals, &r.opts, sl.stream,
                           static_cast<uint8_t*>(s->dmem) + off, it->bytes, sl.pinned);
    if (st) {
      s->arena.release(off, it->bytes);
      push_completion(s, r.tag, st, nullptr, it->t_submit, t_admit);
    } else {
      sl.ctx = c;
      sl.req = r;
      sl.off = off;
      sl.bytes = it->bytes;
      sl.t_submit = it->t_submit;
      sl.t_admit = t_admit;
      sl.state = kValidate;
      sl.turn = 0;
      ++s->active;
      for (auto& p : passed) ++p->bypassed;
    }
    it = s->queue.erase(it);
  }
}

void server_free(cbg_server* s) {
  for (auto& sl : s->slots) {
    if (sl.ctx) ctx_release(sl.ctx);
    for (int i = 0; i < 2; ++i)
      if (sl.turn_ev[i]) cudaEventDestroy(sl.turn_ev[i]);
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
  }
  if (s->dmem) cudaFree(s->dmem);
  if (s->pinned) cudaFreeHost(s->pinned);
  delete s;
}

}  // namespace

extern "C" {

int cbg_server_create(cbg_server** out, size_t hbm_budget, int32_t max_active, int32_t steps_per_turn,
                      int32_t max_bypass) {
  if (!out) {
    set_error("cbg_server_create: null output pointer");
    return CBG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (hbm_budget < kAlign || max_active < 1 || max_active > 256 || steps_per_turn < 1 || max_bypass < 0) {
    set_error("cbg_server_create: need hbm_budget >= 256, 1 <= max_active <= 256, steps_per_turn >= 1, "
              "max_bypass >= 0");
    return CBG_ERR_INVALID_ARG;
  }
  DeviceInfo di;
  int st = device_info(&di);
  if (st) return st;
  cbg_server* s = new (std::nothrow) cbg_server();
  if (!s) {
    set_error("cbg_server_create: host allocation failed");
    return CBG_ERR_OOM;
  }
  hbm_budget = hbm_budget / kAlign * kAlign;
  cudaError_t e = cudaMalloc(&s->dmem, hbm_budget);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->dmem = nullptr;
    server_free(s);
    set_error("cbg_server_create: cudaMalloc of the %zu-byte budget failed", hbm_budget);
    return CBG_ERR_OOM;
  }
  s->arena = Arena(hbm_budget);
  const size_t pb = ctx_pinned_bytes();
  e = cudaMallocHost(&s->pinned, pb * max_active);
  if (e != cudaSuccess) {
    s->pinned = nullptr;
    server_free(s);
    return cuda_fail(e, "cbg_server_create: pinned control blocks");
  }
  s->slots.resize(max_active);
  for (int i = 0; i < max_active; ++i) {
    Slot& sl = s->slots[i];
    sl.pinned = static_cast<uint8_t*>(s->pinned) + pb * i;
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.turn_ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.turn_ev[1], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cbg_server_create: streams and events");
      server_free(s);
      return st;
    }
  }
  s->steps_per_turn = steps_per_turn;
  s->max_bypass = max_bypass;
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return CBG_OK;
}

int cbg_server_submit(cbg_server* s, const cbg_request* r) {
  if (!s || !r) {
    set_error("cbg_server_submit: null argument");
    return CBG_ERR_INVALID_ARG;
  }
  const size_t bytes = ctx_device_bytes(r->n, &r->opts);
  if (bytes == 0) {
    set_error("cbg_server_submit: invalid n or options (1 <= restart <= min(n, 1024), tol > 0, l in {16,21,32})");
    return CBG_ERR_INVALID_ARG;
  }
  if (r->nnz < 0 || r->nnz > INT32_MAX || !r->d_row_ptr || (r->nnz > 0 && (!r->d_col || !r->d_vals)) || !r->d_b ||
      !r->d_x) {
    set_error("cbg_server_submit: invalid CSR, b or x arguments");
    return CBG_ERR_INVALID_ARG;
  }
  if (align_up(bytes) > s->arena.size()) {
    set_error("cbg_server_submit: the request's workspace (%zu bytes) exceeds the server's budget (%zu bytes)", bytes,
              s->arena.size());
    return CBG_ERR_OOM;
  }
  Queued q;
  q.req = *r;
  q.bytes = align_up(bytes);
  q.t_submit = clock_of(s);
  q.bypassed = 0;
  s->queue.push_back(q);
  return CBG_OK;
}

int cbg_server_poll(cbg_server* s, cbg_completion* out, int32_t cap, int32_t* n_out) {
  if (!s || !n_out || cap < 0 || (cap > 0 && !out)) {
    set_error("cbg_server_poll: null argument or negative cap");
    return CBG_ERR_INVALID_ARG;
  }
  *n_out = 0;
  for (auto& sl : s->slots)
    if (sl.state != kFree) progress(s, sl);
  admit(s);
  int k = 0;
  while (k < cap && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n_out = k;
  return CBG_OK;
}

int cbg_server_stats(const cbg_server* s, int32_t* active, int32_t* queued, int32_t* pending, size_t* bytes_in_use) {
  if (!s) {
    set_error("cbg_server_stats: null server");
    return CBG_ERR_INVALID_ARG;
  }
  if (active) *active = s->active;
  if (queued) *queued = static_cast<int32_t>(s->queue.size());
  if (pending) *pending = static_cast<int32_t>(s->done.size());
  if (bytes_in_use) *bytes_in_use = s->arena.used();
  return CBG_OK;
}

double cbg_server_clock(const cbg_server* s) { return s ? clock_of(s) : 0.0; }

int cbg_server_destroy(cbg_server* s) {
  if (s) server_free(s);
  return CBG_OK;
}

}  // extern "C"
