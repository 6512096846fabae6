// Continuous-batching encode/decode server (C ABI in include/adct.h).
//
// A scheduler thread owns one codec context, a device-memory arena of the
// configured budget and the on-device coefficient store.  Each pass it
//   1. moves newly submitted requests into its FIFO queue,
//   2. retires launched batches whose completion events have fired (frees
//      their temporary arena space, publishes completions),
//   3. admits queued requests while the arena can hold them, evicting the
//      oldest store entries that no queued or running decode references,
//   4. launches everything admitted in this pass as at most one encode launch
//      (host-to-device copies, then forward + quantise with q kept in the
//      store) and one decode launch (dequantise + inverse, then device-to-host
//      copies), on the next of its streams,
// so requests that arrive while others run are admitted as memory frees up
// and their work overlaps on the device.  Clients poll completions.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "adct.h"
#include "adct_internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kAlign = 256;

// First-fit allocator over one device allocation; adjacent free ranges merge.
class Arena {
 public:
  bool init(size_t bytes) {
    bytes_ = (bytes + kAlign - 1) / kAlign * kAlign;
    if (adct::device_alloc((void**)&base_, bytes_) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return false;
    }
    free_[0] = bytes_;
    free_bytes_ = bytes_;
    return true;
  }
  void release() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  // Returns the offset, or SIZE_MAX when no free range is large enough.
  size_t alloc(size_t n) {
    n = (n + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const size_t off = it->first, rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        free_bytes_ -= n;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void free(size_t off, size_t n) {
    n = (n + kAlign - 1) / kAlign * kAlign;
    free_bytes_ += n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint8_t* ptr(size_t off) const { return (uint8_t*)base_ + off; }
  size_t free_bytes() const { return free_bytes_; }
  size_t bytes() const { return bytes_; }

 private:
  void* base_ = nullptr;
  size_t bytes_ = 0, free_bytes_ = 0;
  std::map<size_t, size_t> free_;
};

enum { KIND_ENCODE = 0, KIND_DECODE = 1 };

struct Req {
  uint64_t id;
  int32_t kind;
  const uint8_t* hsrc;  // encode input (host)
  uint8_t* hdst;        // decode output (host)
  int32_t width, height;
  int64_t pitch;
  uint64_t handle;      // decode: store handle; encode: assigned handle
  double t_submit, t_admit;
  size_t tmp_off, tmp_bytes;  // arena space freed at completion
};

struct Entry {
  size_t off, bytes;  // coefficients in the arena
  int32_t width, height;
  int32_t refs;       // queued or running decodes
  uint64_t tick;      // insertion order (oldest evicted first)
  bool ready;         // encode finished
};

struct Batch {
  cudaEvent_t ev;
  std::vector<Req> reqs;
};

}  // namespace

struct adct_server {
  int device = 0;
  adct_context* ctx = nullptr;
  adct_quant quant{};
  int32_t cpb = 64;  // int16 coefficients stored per block (r for the packed zonal layout)
  int32_t max_batch = 256;
  Arena arena;
  std::vector<cudaStream_t> streams;
  size_t rr = 0;
  std::vector<cudaEvent_t> event_pool;

  std::mutex mu;  // guards incoming, store, lru and counters touched by submit
  std::deque<Req> incoming;
  std::unordered_map<uint64_t, Entry> store;
  std::map<uint64_t, uint64_t> lru;  // tick -> handle
  uint64_t next_id = 1, next_handle = 1, tick = 0;

  std::deque<Req> queue;        // scheduler thread only
  std::vector<Batch> inflight;  // scheduler thread only

  std::mutex done_mu;
  std::condition_variable done_cv;
  std::deque<adct_completion> done;

  std::thread thread;
  std::atomic<bool> stop{false};
  std::unordered_set<uint64_t> pending;    // submitted, not completed (under mu)
  std::unordered_set<uint64_t> cancelled;  // cancellation asked while in the scheduler's queue (under mu)
  std::atomic<int64_t> s_launches{0}, s_admitted{0}, s_evicted{0}, s_unknown{0}, s_oversized{0}, s_errors{0};
  std::atomic<int64_t> s_cancelled{0};
  std::atomic<int64_t> s_hist[32] = {};
  std::atomic<int32_t> s_max_overlap{0};
};

namespace {

int latency_bucket(double seconds) {
  const double us = seconds * 1e6;
  int b = 0;
  while (b < 31 && us >= (double)(2ull << b)) ++b;
  return b;
}

// Drops a finished request from the pending and cancelled sets (caller holds s->mu).
void forget(adct_server* s, const Req& r) {
  s->pending.erase(r.id);
  if (!s->cancelled.empty()) s->cancelled.erase(r.id);
}

// Reports a request's completion (the caller has already forgotten it).
void complete(adct_server* s, const Req& r, int32_t status, double t_done) {
  ++s->s_hist[latency_bucket(t_done - r.t_submit)];
  adct_completion c{};
  c.request_id = r.id;
  c.status = status;
  c.kind = r.kind;
  c.handle = r.handle;
  c.t_submit = r.t_submit;
  c.t_admit = r.t_admit;
  c.t_done = t_done;
  {
    std::lock_guard<std::mutex> lk(s->done_mu);
    s->done.push_back(c);
  }
  s->done_cv.notify_all();
}

cudaEvent_t get_event(adct_server* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

void retire(adct_server* s) {
  std::vector<Batch> still;
  for (Batch& b : s->inflight) {
    const cudaError_t q = cudaEventQuery(b.ev);
    if (q == cudaErrorNotReady) {
      still.push_back(std::move(b));
      continue;
    }
    const double t = now_s();
    const int32_t status = (q == cudaSuccess) ? ADCT_OK : ADCT_ERR_CUDA;
    if (q != cudaSuccess) {
      cudaGetLastError();
      ++s->s_errors;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (const Req& r : b.reqs) {
        s->arena.free(r.tmp_off, r.tmp_bytes);
        forget(s, r);
        auto it = s->store.find(r.handle);
        if (r.kind == KIND_ENCODE) {
          if (it != s->store.end()) it->second.ready = true;
        } else if (it != s->store.end()) {
          --it->second.refs;
        }
      }
    }
    for (const Req& r : b.reqs) complete(s, r, status, t);
    s->event_pool.push_back(b.ev);
  }
  s->inflight.swap(still);
}

// Evicts the oldest ready, unreferenced store entry; false when none is evictable.
bool evict_one(adct_server* s) {
  for (auto it = s->lru.begin(); it != s->lru.end(); ++it) {
    auto e = s->store.find(it->second);
    if (e == s->store.end()) continue;
    if (e->second.refs == 0 && e->second.ready) {
      s->arena.free(e->second.off, e->second.bytes);
      s->store.erase(e);
      s->lru.erase(it);
      ++s->s_evicted;
      return true;
    }
  }
  return false;
}

// Admits from the head of the queue while memory allows; fills enc/dec.
void admit(adct_server* s, std::vector<Req>& enc, std::vector<Req>& dec) {
  std::lock_guard<std::mutex> lk(s->mu);
  while (!s->incoming.empty()) {
    s->queue.push_back(s->incoming.front());
    s->incoming.pop_front();
  }
  if (!s->cancelled.empty()) {  // withdraw cancelled requests still in the queue
    std::deque<Req> keep;
    for (Req& r : s->queue) {
      if (!s->cancelled.count(r.id)) {
        keep.push_back(r);
        continue;
      }
      if (r.kind == KIND_DECODE) {
        auto it = s->store.find(r.handle);
        if (it != s->store.end()) --it->second.refs;
      }
      ++s->s_cancelled;
      forget(s, r);
      complete(s, r, ADCT_ERR_CANCELLED, now_s());
    }
    s->queue.swap(keep);
  }
  while (!s->queue.empty() && (int32_t)(enc.size() + dec.size()) < s->max_batch) {
    Req& r = s->queue.front();
    const size_t pix = (size_t)r.width * r.height;
    if (r.kind == KIND_DECODE) {
      auto it = s->store.find(r.handle);
      if (it == s->store.end()) {
        Req gone = r;
        s->queue.pop_front();
        ++s->s_unknown;
        forget(s, gone);
        complete(s, gone, ADCT_ERR_INVALID_ARG, now_s());
        continue;
      }
      if (!it->second.ready) break;  // its encode is still running: keep FIFO order
    }
    const size_t cbytes = std::max<size_t>(pix / 64 * (size_t)s->cpb * 2, 16);  // the stored coefficients
    const size_t need = (r.kind == KIND_ENCODE) ? pix + cbytes : pix;
    if (need + 2 * kAlign > s->arena.bytes()) {
      Req big = r;
      s->queue.pop_front();
      ++s->s_oversized;
      forget(s, big);
      complete(s, big, ADCT_ERR_OOM, now_s());
      continue;
    }
    size_t off_tmp = s->arena.alloc(pix), off_coef = SIZE_MAX;
    if (off_tmp != SIZE_MAX && r.kind == KIND_ENCODE) off_coef = s->arena.alloc(cbytes);
    while ((off_tmp == SIZE_MAX || (r.kind == KIND_ENCODE && off_coef == SIZE_MAX)) && evict_one(s)) {
      if (off_tmp == SIZE_MAX) off_tmp = s->arena.alloc(pix);
      if (off_tmp != SIZE_MAX && r.kind == KIND_ENCODE && off_coef == SIZE_MAX) off_coef = s->arena.alloc(cbytes);
    }
    if (off_tmp == SIZE_MAX || (r.kind == KIND_ENCODE && off_coef == SIZE_MAX)) {
      if (off_tmp != SIZE_MAX) s->arena.free(off_tmp, pix);
      break;  // wait for running batches to free memory
    }
    Req a = r;
    s->queue.pop_front();
    a.t_admit = now_s();
    a.tmp_off = off_tmp;
    a.tmp_bytes = pix;
    if (a.kind == KIND_ENCODE) {
      a.handle = s->next_handle++;
      Entry e{off_coef, cbytes, a.width, a.height, 0, s->tick, false};
      s->store[a.handle] = e;
      s->lru[s->tick++] = a.handle;
      enc.push_back(a);
    } else {
      dec.push_back(a);  // its reference was taken at submission
    }
  }
}

void launch(adct_server* s, std::vector<Req>& reqs, int kind) {
  if (reqs.empty()) return;
  cudaStream_t st = s->streams[s->rr++ % s->streams.size()];
  std::vector<adct_image> imgs(reqs.size());
  bool ok = true;
  for (size_t k = 0; k < reqs.size(); ++k) {
    Req& r = reqs[k];
    adct_image& im = imgs[k];
    std::memset(&im, 0, sizeof im);
    im.width = r.width;
    im.height = r.height;
    im.channels = 1;
    im.pitch = r.width;
    im.plane_stride = (int64_t)r.width * r.height;
    uint8_t* tmp = s->arena.ptr(r.tmp_off);
    uint8_t* coef;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      coef = s->arena.ptr(s->store[r.handle].off);
    }
    im.coef = (int16_t*)coef;
    if (kind == KIND_ENCODE) {
      im.src = tmp;
      if (cudaMemcpy2DAsync(tmp, r.width, r.hsrc, r.pitch, r.width, r.height, cudaMemcpyHostToDevice, st) != cudaSuccess)
        ok = false;
    } else {
      im.dst = tmp;
    }
  }
  adct_status status = ADCT_OK;
  if (ok) {
    if (kind == KIND_ENCODE) {
      status = adct_roundtrip(s->ctx, imgs.data(), (int32_t)imgs.size(), &s->quant, st);
    } else {
      status = adct_inverse(s->ctx, imgs.data(), (int32_t)imgs.size(), &s->quant, st);
      for (size_t k = 0; k < reqs.size() && status == ADCT_OK; ++k) {
        const Req& r = reqs[k];
        if (cudaMemcpy2DAsync(r.hdst, r.pitch, imgs[k].dst, r.width, r.width, r.height, cudaMemcpyDeviceToHost,
                              st) != cudaSuccess)
          status = ADCT_ERR_CUDA;
      }
    }
  }
  if (!ok) status = ADCT_ERR_CUDA;
  Batch b;
  b.ev = get_event(s);
  b.reqs = std::move(reqs);
  if (status == ADCT_OK && b.ev && cudaEventRecord(b.ev, st) == cudaSuccess) {
    ++s->s_launches;
    s->inflight.push_back(std::move(b));
    int32_t ov = (int32_t)s->inflight.size();
    if (ov > s->s_max_overlap) s->s_max_overlap = ov;
    return;
  }
  // failed before the batch reached the device: release and report
  cudaGetLastError();
  ++s->s_errors;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (const Req& r : b.reqs) {
      s->arena.free(r.tmp_off, r.tmp_bytes);
      forget(s, r);
      auto it = s->store.find(r.handle);
      if (it == s->store.end()) continue;
      if (r.kind == KIND_ENCODE) {
        s->arena.free(it->second.off, it->second.bytes);
        s->store.erase(it);
      } else {
        --it->second.refs;
      }
    }
  }
  const double t = now_s();
  for (const Req& r : b.reqs) complete(s, r, status == ADCT_OK ? ADCT_ERR_CUDA : status, t);
  if (b.ev) s->event_pool.push_back(b.ev);
}

void scheduler(adct_server* s) {
  cudaSetDevice(s->device);
  std::vector<Req> enc, dec;
  while (!s->stop.load()) {
    retire(s);
    enc.clear();
    dec.clear();
    admit(s, enc, dec);
    const bool work = !enc.empty() || !dec.empty();
    if (work) {
      s->s_admitted += (int64_t)(enc.size() + dec.size());
      launch(s, enc, KIND_ENCODE);
      launch(s, dec, KIND_DECODE);
      continue;
    }
    bool waiting;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      waiting = !s->incoming.empty() || !s->queue.empty();
    }
    if (s->inflight.empty() && !waiting) {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    } else {
      std::this_thread::yield();
    }
  }
  for (Batch& b : s->inflight) cudaEventSynchronize(b.ev);
  retire(s);
}

}  // namespace

extern "C" {

adct_status adct_server_create(adct_server** out, int32_t device, const adct_server_config* cfg) {
  if (!out || !cfg) return ADCT_ERR_INVALID_ARG;
  *out = nullptr;
  adct_server* s = new adct_server();
  s->device = device;
  s->quant = cfg->quant;
  if (s->quant.mode == ADCT_Q_ZONAL_ZZ && s->quant.r >= 0 && s->quant.r <= 64) s->cpb = s->quant.r;
  s->max_batch = cfg->max_batch > 0 ? cfg->max_batch : 256;
  const int64_t budget = cfg->budget_bytes > 0 ? cfg->budget_bytes : (4ll << 30);
  const int nstreams = cfg->streams > 0 ? cfg->streams : 4;
  adct_status st = adct_create(&s->ctx, device);
  if (st != ADCT_OK) {
    delete s;
    return st;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  if (!s->arena.init((size_t)budget)) {
    adct_destroy(s->ctx);
    cudaSetDevice(prev);
    delete s;
    return ADCT_ERR_OOM;
  }
  for (int k = 0; k < nstreams; ++k) {
    cudaStream_t strm = nullptr;
    if (cudaStreamCreateWithFlags(&strm, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
      s->arena.release();
      adct_destroy(s->ctx);
      cudaSetDevice(prev);
      delete s;
      return ADCT_ERR_CUDA;
    }
    s->streams.push_back(strm);
  }
  cudaSetDevice(prev);
  s->thread = std::thread(scheduler, s);
  *out = s;
  return ADCT_OK;
}

void adct_server_destroy(adct_server* s) {
  if (!s) return;
  s->stop.store(true);
  if (s->thread.joinable()) s->thread.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (cudaStream_t t : s->streams) {
    cudaStreamSynchronize(t);
    cudaStreamDestroy(t);
  }
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  s->arena.release();
  adct_destroy(s->ctx);
  cudaSetDevice(prev);
  delete s;
}

adct_status adct_server_encode(adct_server* s, const uint8_t* pixels, int32_t width, int32_t height, int64_t pitch,
                               double t_submit, uint64_t* request_id) {
  if (!s || !pixels || !request_id) return ADCT_ERR_INVALID_ARG;
  if (width <= 0 || height <= 0 || width % 8 || height % 8 || width > 65536 || height > 65536 || pitch < width)
    return ADCT_ERR_SHAPE;
  Req r{};
  r.kind = KIND_ENCODE;
  r.hsrc = pixels;
  r.width = width;
  r.height = height;
  r.pitch = pitch;
  r.t_submit = t_submit > 0 ? t_submit : now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r.id = s->next_id++;
    s->pending.insert(r.id);
    s->incoming.push_back(r);
  }
  *request_id = r.id;
  return ADCT_OK;
}

adct_status adct_server_decode(adct_server* s, uint64_t handle, uint8_t* out, int64_t pitch, double t_submit,
                               uint64_t* request_id, int32_t* width, int32_t* height) {
  if (!s || !out || !request_id) return ADCT_ERR_INVALID_ARG;
  Req r{};
  r.kind = KIND_DECODE;
  r.hdst = out;
  r.handle = handle;
  r.t_submit = t_submit > 0 ? t_submit : now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->store.find(handle);
    if (it == s->store.end()) return ADCT_ERR_INVALID_ARG;  // unknown or evicted handle
    if (pitch < it->second.width) return ADCT_ERR_SHAPE;
    ++it->second.refs;  // pinned until this decode completes
    r.width = it->second.width;
    r.height = it->second.height;
    r.pitch = pitch;
    r.id = s->next_id++;
    s->pending.insert(r.id);
    s->incoming.push_back(r);
  }
  if (width) *width = r.width;
  if (height) *height = r.height;
  *request_id = r.id;
  return ADCT_OK;
}

int32_t adct_server_poll(adct_server* s, adct_completion* out, int32_t max, int32_t wait_us) {
  if (!s || !out || max <= 0) return 0;
  std::unique_lock<std::mutex> lk(s->done_mu);
  if (s->done.empty() && wait_us > 0)
    s->done_cv.wait_for(lk, std::chrono::microseconds(wait_us), [s] { return !s->done.empty(); });
  int32_t n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  return n;
}

adct_status adct_server_stats(adct_server* s, adct_server_stats_t* st) {
  if (!s || !st) return ADCT_ERR_INVALID_ARG;
  st->launches = s->s_launches;
  st->admitted = s->s_admitted;
  st->evicted = s->s_evicted;
  st->unknown_handle = s->s_unknown;
  st->oversized = s->s_oversized;
  st->errors = s->s_errors;
  st->max_overlap = s->s_max_overlap;
  st->reserved = 0;
  st->cancelled = s->s_cancelled;
  for (int b = 0; b < 32; ++b) st->latency_hist[b] = s->s_hist[b];
  {
    std::lock_guard<std::mutex> lk(s->mu);
    st->store_entries = (int64_t)s->store.size();
    st->arena_free_bytes = (int64_t)s->arena.free_bytes();
  }
  return ADCT_OK;
}

adct_status adct_server_cancel(adct_server* s, uint64_t request_id) {
  if (!s) return ADCT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->pending.count(request_id)) return ADCT_ERR_INVALID_ARG;
  for (auto it = s->incoming.begin(); it != s->incoming.end(); ++it) {
    if (it->id != request_id) continue;
    const Req r = *it;  // not yet seen by the scheduler: withdraw it here
    s->incoming.erase(it);
    if (r.kind == KIND_DECODE) {
      auto e = s->store.find(r.handle);
      if (e != s->store.end()) --e->second.refs;
    }
    ++s->s_cancelled;
    forget(s, r);
    complete(s, r, ADCT_ERR_CANCELLED, now_s());
    return ADCT_OK;
  }
  s->cancelled.insert(request_id);  // in the scheduler's queue, or already admitted
  return ADCT_OK;
}

double adct_server_clock(void) { return now_s(); }

}  // extern "C"
