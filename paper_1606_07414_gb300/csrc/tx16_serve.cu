// Serving loop (tx16_serve_*): requests of different sizes, each with its own
// quantiser, coded by the fused batch kernels with continuous batching.
//
//  submit   validates the request, stamps its arrival time and queues it.
//           If the server is idle (nothing queued or in flight), it admits
//           the request and puts it on a slot itself: a lone request skips
//           the hand-off to the worker.
//  worker   (one host thread) repeatedly
//             - admits queued requests, in arrival order, while the device
//               arena has room for their input and output planes and a batch
//               slot is free ("admission by free HBM");
//             - hands each admitted group to its slot's issuer thread (or,
//               when nothing else is queued or being issued, issues it
//               itself), which puts it on the slot's streams: host->device
//               copies of the inputs, ONE tx16_codec_batch launch over the group,
//               device->host copies of the reconstructions and SSEs, then an
//               event -- the slots' issuers run in parallel, so the CUDA calls
//               of one group do not hold up the admission of the next.
//               A group of at most 16 requests with a plane larger than
//               band_mb goes in bands of whole block rows on three streams:
//               all copies in, one after another; each band's launch once its
//               copies are in; each band's copies out once it is coded -- so
//               that copies out overlap copies in (the two directions have
//               their own copy engines: 16.6 MB each way took 142 us
//               overlapped against 190 us one after the other);
//             - retires slots whose event has fired: PSNR, latency, frees the
//               requests' arena space, wakes their waiters.
//           While a group is in flight it polls (submissions, slot events),
//           so a finished group is retired at once; with nothing in flight it
//           polls for up to spin_us after its last progress, then blocks until
//           a submit or a slot's host callback wakes it.
//           Groups on different slots overlap on the GPU (copies of one with
//           the kernel of another), and requests that arrive while others are
//           in flight join the next group: the batch is never closed.
//  wait     polls for up to wait_spin_us -- retiring the request's group
//           itself if its event has fired, so completion needs no hand-off
//           either -- then blocks (bounded) until the request is done.
//
// All device memory (the arena, per-slot SSE arrays) is allocated once at
// creation; requests never allocate.  Host buffers are the caller's: the input
// must stay valid until the request is done (pinned memory gives direct DMA).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "tx16_internal.h"

using Clock = std::chrono::steady_clock;
using tx16::valid_image;

namespace {

// First-fit arena over one device allocation, 256-byte granules.
class Arena {
 public:
  bool init(size_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) return false;
    size_ = bytes;
    free_[0] = bytes;
    return true;
  }
  void release() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  size_t capacity() const { return size_; }
  char* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_[off] = bytes;
        return static_cast<char*>(base_) + off;
      }
    }
    return nullptr;
  }
  void free(char* p) {
    if (p == nullptr) return;
    const size_t off = size_t(p - static_cast<char*>(base_));
    auto u = used_.find(off);
    if (u == used_.end()) return;
    auto it = free_.emplace(off, u->second).first;
    used_.erase(u);
    auto nx = std::next(it);  // merge with the following free range
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {  // and with the preceding one
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
 private:
  void* base_ = nullptr;
  size_t size_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  std::map<size_t, size_t> used_;
};

struct Request {
  uint64_t ticket;
  const void* host_in;
  void* host_out;  // may be null
  int w, h, bits;
  tx16_qparams qp;
  size_t bytes;  // per plane
  int64_t blocks;
  Clock::time_point t_submit;
  char* d_in = nullptr;
  char* d_out = nullptr;
  std::atomic<bool> done{false};
  std::atomic<struct Slot*> slot{nullptr};  // the group's slot while in flight
  int nbands = 1;   // bands of its group's launch (set when launched)
  int sse_pos = 0;  // its index in each band's launch
  tx16_status status = TX16_OK;
  double psnr = 0.0;
  double latency_us = 0.0;
};

constexpr int kMaxBands = 8;
constexpr int kBandMaxGroup = 16;  // groups of more requests are not cut into bands

struct Slot {
  cudaStream_t stream = nullptr;      // a group in one band: everything; in bands: the launches
  cudaStream_t in_stream = nullptr;   // copies in of a group in bands
  cudaStream_t out_stream = nullptr;  // copies out of a group in bands
  cudaEvent_t event = nullptr;
  cudaEvent_t in_ev[kMaxBands] = {};    // band b copied in
  cudaEvent_t band_ev[kMaxBands] = {};  // band b coded
  uint64_t* d_sse = nullptr;  // [band][request], kMaxBands x max_batch
  uint64_t* h_sse = nullptr;  // pinned, the same
  std::vector<Request*> reqs;
  bool busy = false;            // a group is admitted (under the server's lock)
  bool issue_pending = false;   // the issuer has a group to launch (under the lock)
  std::atomic<bool> launched{false};  // the group's work and event are on the stream
  std::condition_variable cv_issue;
  std::thread issuer;
  struct tx16_server* server = nullptr;
};

}  // namespace

struct tx16_server {
  int device = 0;
  int max_batch = 256;
  size_t max_queue = 1 << 20;
  Arena arena;
  std::deque<Slot> slots;  // built once at creation (slots hold threads and atomics)
  std::mutex mu;
  std::condition_variable cv_work;  // worker: new requests / stop
  std::condition_variable cv_done;  // waiters
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> live;  // ticket -> request (until waited)
  uint64_t next_ticket = 1;
  bool stop = false;
  bool stop_issuers = false;  // set after the worker has drained everything
  bool paused = false;  // admission held (tx16_serve_pause)
  int issuing = 0;      // groups being put on their streams (under the lock)
  std::atomic<uint64_t> pokes{0};  // bumped by submit, pause, stop and slot callbacks
  double spin_us = 300;            // polling window of the worker
  double wait_spin_us = 2000;      // polling window of waiters (they retire finished groups themselves)
  size_t band_bytes = size_t(4) << 20;  // planes above this go in bands (0: never)
  std::thread worker;
  // statistics
  std::vector<double> lat;  // reservoir of latencies (us)
  size_t lat_seen = 0;
  uint64_t rng = 0x9E3779B97F4A7C15ull;
  double blocks_done = 0;
  Clock::time_point t_first{}, t_last{};
  bool any = false;
  std::string error;
};

namespace {

constexpr size_t kReservoir = 1 << 20;

double now_us(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}

// Parse a flat JSON object of numbers: {"key": 12.5, ...}.  Unknown keys are
// ignored; returns false on malformed input.
bool parse_cfg(const char* s, std::map<std::string, double>& out) {
  if (s == nullptr || *s == 0) return true;
  const char* p = s;
  auto ws = [&] { while (*p == ' ' || *p == '\n' || *p == '\t' || *p == '\r') ++p; };
  ws();
  if (*p != '{') return false;
  ++p;
  for (;;) {
    ws();
    if (*p == '}') return true;
    if (*p != '"') return false;
    const char* k0 = ++p;
    while (*p && *p != '"') ++p;
    if (*p != '"') return false;
    std::string key(k0, p - k0);
    ++p;
    ws();
    if (*p != ':') return false;
    ++p;
    ws();
    char* end = nullptr;
    const double v = std::strtod(p, &end);
    if (end == p) return false;
    out[key] = v;
    p = end;
    ws();
    if (*p == ',') {
      ++p;
      continue;
    }
    if (*p == '}') return true;
    return false;
  }
}

void record_latency(tx16_server* s, double us) {
  ++s->lat_seen;
  if (s->lat.size() < kReservoir) {
    s->lat.push_back(us);
  } else {  // reservoir sampling keeps a uniform sample of every latency seen
    s->rng ^= s->rng << 13;
    s->rng ^= s->rng >> 7;
    s->rng ^= s->rng << 17;
    const size_t j = size_t(s->rng % s->lat_seen);
    if (j < kReservoir) s->lat[j] = us;
  }
}

// Runs on the CUDA runtime's callback thread when a slot's stream has passed
// its last copy: wakes the worker (no CUDA calls are allowed here).  The
// worker learns that a group is done from the slot's event, so a callback of
// a group that the worker already retired is only a spurious wake-up.  Taking
// the lock orders the wake-up after any event query the worker made before it
// blocked.
void CUDART_CB slot_done(void* arg) {
  Slot* slot = static_cast<Slot*>(arg);
  tx16_server* s = slot->server;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->pokes.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_one();
}

// Put one admitted group on a slot: copies in, one batched launch, copies out
// -- in bands when a plane is larger than band_bytes.  A request of k bands is
// cut into k runs of whole block rows; band b's launch codes band b of every
// request that has one.  The requests are taken in decreasing band count, so
// that those of band b are a prefix of the group and keep their index
// (sse_pos) in every band's launch.
tx16_status launch_group(Slot& slot) {
  TX16_TRACE("tx16 serve: launch group");
  tx16_server* s = slot.server;
  const int n = int(slot.reqs.size());
  std::vector<Request*> order(slot.reqs);
  int nbmax = 1;
  // bands shorten a small group's latency; a large group (a busy server) is
  // throughput-bound and takes one launch
  const bool may_band = s->band_bytes > 0 && n <= kBandMaxGroup;
  for (Request* r : order) {
    const int brows = r->h / 16;
    int k = 1;
    if (may_band) k = int(std::min<size_t>(kMaxBands, (r->bytes + s->band_bytes - 1) / s->band_bytes));
    k = std::max(1, std::min(k, brows));
    const int rows = (brows + k - 1) / k * 16;  // rows per band
    r->nbands = (r->h + rows - 1) / rows;
    nbmax = std::max(nbmax, r->nbands);
  }
  std::stable_sort(order.begin(), order.end(), [](const Request* a, const Request* b) { return a->nbands > b->nbands; });
  for (int i = 0; i < n; ++i) order[i]->sse_pos = i;
  const bool banded = nbmax > 1;
  cudaStream_t s_in = banded ? slot.in_stream : slot.stream;
  cudaStream_t s_out = banded ? slot.out_stream : slot.stream;
  // rows [y0, y0 + hb) of request r in band b, as a byte range of its plane
  auto band = [](const Request* r, int b, size_t& off, size_t& len, int& hb) {
    const int64_t pitch = int64_t(r->w) * (r->bits == 8 ? 1 : 2);
    const int rows = (r->h / 16 + r->nbands - 1) / r->nbands * 16;
    const int y0 = b * rows;
    hb = std::min(rows, r->h - y0);
    off = size_t(y0) * size_t(pitch);
    len = size_t(hb) * size_t(pitch);
  };
  for (int b = 0; b < nbmax; ++b) {  // copies in
    for (int i = 0; i < n && order[i]->nbands > b; ++i) {
      Request* r = order[i];
      size_t off, len;
      int hb;
      band(r, b, off, len, hb);
      if (cudaMemcpyAsync(r->d_in + off, static_cast<const char*>(r->host_in) + off, len, cudaMemcpyHostToDevice,
                          s_in) != cudaSuccess)
        return TX16_ECUDA;
    }
    if (banded && cudaEventRecord(slot.in_ev[b], s_in) != cudaSuccess) return TX16_ECUDA;
  }
  std::vector<tx16_image> in(n), out(n);
  std::vector<tx16_qparams> qp(n);
  for (int b = 0; b < nbmax; ++b) {  // launches, copies out
    int m = 0;
    for (; m < n && order[m]->nbands > b; ++m) {
      Request* r = order[m];
      size_t off, len;
      int hb;
      band(r, b, off, len, hb);
      const int64_t pitch = int64_t(r->w) * (r->bits == 8 ? 1 : 2);
      in[m] = tx16_image{r->d_in + off, r->w, hb, pitch, r->bits};
      out[m] = tx16_image{r->d_out + off, r->w, hb, pitch, r->bits};
      qp[m] = r->qp;
    }
    if (banded && cudaStreamWaitEvent(slot.stream, slot.in_ev[b], 0) != cudaSuccess) return TX16_ECUDA;
    const tx16_status st = tx16_codec_batch(in.data(), out.data(), m, qp.data(), slot.d_sse + size_t(b) * s->max_batch,
                                            nullptr, slot.stream);
    if (st != TX16_OK) return st;
    if (banded && (cudaEventRecord(slot.band_ev[b], slot.stream) != cudaSuccess ||
                   cudaStreamWaitEvent(s_out, slot.band_ev[b], 0) != cudaSuccess))
      return TX16_ECUDA;
    for (int i = 0; i < m; ++i) {
      Request* r = order[i];
      if (r->host_out == nullptr) continue;
      size_t off, len;
      int hb;
      band(r, b, off, len, hb);
      if (cudaMemcpyAsync(static_cast<char*>(r->host_out) + off, r->d_out + off, len, cudaMemcpyDeviceToHost, s_out) !=
          cudaSuccess)
        return TX16_ECUDA;
    }
  }
  const size_t nsse = size_t(nbmax - 1) * size_t(s->max_batch) + size_t(n);
  if (cudaMemcpyAsync(slot.h_sse, slot.d_sse, sizeof(uint64_t) * nsse, cudaMemcpyDeviceToHost, s_out) != cudaSuccess ||
      cudaEventRecord(slot.event, s_out) != cudaSuccess || cudaLaunchHostFunc(s_out, slot_done, &slot) != cudaSuccess)
    return TX16_ECUDA;
  return TX16_OK;
}

void retire(tx16_server* s, Slot& slot, tx16_status st) {
  TX16_TRACE("tx16 serve: retire group");
  const Clock::time_point t = Clock::now();
  for (size_t i = 0; i < slot.reqs.size(); ++i) {
    Request* r = slot.reqs[i];
    r->status = st;
    if (st == TX16_OK) {
      tx16_image d{r->d_in, r->w, r->h, int64_t(r->w) * (r->bits == 8 ? 1 : 2), r->bits};
      uint64_t e = 0;
      for (int b = 0; b < r->nbands; ++b) e += slot.h_sse[size_t(b) * size_t(s->max_batch) + size_t(r->sse_pos)];
      tx16_psnr(&e, &d, 1, &r->psnr);
      s->blocks_done += double(r->blocks);
    }
    r->latency_us = now_us(r->t_submit, t);
    record_latency(s, r->latency_us);
    s->arena.free(r->d_in);
    s->arena.free(r->d_out);
    r->d_in = r->d_out = nullptr;
    r->slot.store(nullptr, std::memory_order_relaxed);
    r->done.store(true, std::memory_order_release);
  }
  s->t_last = t;
  slot.reqs.clear();
  slot.launched.store(false, std::memory_order_relaxed);
  slot.busy = false;
}

// Admit queued requests into a free slot, in arrival order, while the arena
// has room (the caller holds the lock).  Returns false if none fits.
bool admit(tx16_server* s, Slot& slot) {
  while (!s->queue.empty() && int(slot.reqs.size()) < s->max_batch) {
    Request* r = s->queue.front();
    r->d_in = s->arena.alloc(r->bytes);
    r->d_out = r->d_in ? s->arena.alloc(r->bytes) : nullptr;
    if (r->d_out == nullptr) {  // no room now: wait for a group to retire
      s->arena.free(r->d_in);
      r->d_in = nullptr;
      break;
    }
    s->queue.pop_front();
    slot.reqs.push_back(r);
  }
  if (slot.reqs.empty()) return false;
  slot.busy = true;
  slot.launched.store(false, std::memory_order_relaxed);
  for (Request* r : slot.reqs) r->slot.store(&slot, std::memory_order_release);
  return true;
}

// Put the admitted group of `slot` on its stream, without the lock (lk is
// held on entry and on return).  On an error the group is retired with it.
void issue(tx16_server* s, Slot& slot, std::unique_lock<std::mutex>& lk) {
  ++s->issuing;
  lk.unlock();
  const tx16_status st = launch_group(slot);
  if (st != TX16_OK) {
    cudaStreamSynchronize(slot.in_stream);
    cudaStreamSynchronize(slot.stream);
    cudaStreamSynchronize(slot.out_stream);
  }
  lk.lock();
  --s->issuing;
  if (st != TX16_OK) {
    retire(s, slot, st);
    s->cv_done.notify_all();
  } else {
    slot.launched.store(true, std::memory_order_release);
  }
  s->pokes.fetch_add(1, std::memory_order_release);
  s->cv_work.notify_one();
}

// A slot whose group is on the stream and whose event has fired (no lock
// needed for the query): the error of the group's work, if any, in *st.
bool slot_finished(Slot& slot, tx16_status* st) {
  if (!slot.launched.load(std::memory_order_acquire)) return false;
  const cudaError_t q = cudaEventQuery(slot.event);
  if (q == cudaErrorNotReady) return false;
  *st = q == cudaSuccess ? TX16_OK : TX16_ECUDA;
  return true;
}

// The issuer thread of one slot: launches the groups the worker admits to it.
void issuer_main(tx16_server* s, Slot* slot) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    slot->cv_issue.wait(lk, [&] { return slot->issue_pending || s->stop_issuers; });
    if (!slot->issue_pending) break;
    slot->issue_pending = false;
    issue(s, *slot, lk);
  }
}

// Poll, without the lock, until a submission or callback arrives, a slot in
// flight finishes, or the window ends.  Returns at once when the window is 0.
void poll_for_work(tx16_server* s, uint64_t seen, Clock::time_point until) {
  while (Clock::now() < until) {
    if (s->pokes.load(std::memory_order_acquire) != seen) return;
    tx16_status st;
    for (Slot& slot : s->slots)
      if (slot.busy && slot_finished(slot, &st)) return;
  }
}

void worker_main(tx16_server* s) {
  cudaSetDevice(s->device);
  const auto spin = std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double, std::micro>(s->spin_us));
  Clock::time_point last_progress = Clock::now();
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    const uint64_t seen = s->pokes.load(std::memory_order_acquire);
    // retire groups whose event has completed (an error of the group's work
    // is reported by the query)
    bool progressed = false;
    for (Slot& slot : s->slots) {
      tx16_status st;
      if (!slot.busy || !slot_finished(slot, &st)) continue;
      retire(s, slot, st);
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    // admit: one group per free slot, launched by the slot's issuer -- or
    // by the worker itself when nothing else is queued or being issued (light
    // load: no hand-off, whose wake-up can cost a sleeping core tens of us)
    for (Slot& slot : s->slots) {
      if (slot.busy || s->queue.empty() || s->paused) continue;
      if (!admit(s, slot)) break;
      progressed = true;
      const bool handing = std::any_of(s->slots.begin(), s->slots.end(), [](const Slot& x) { return x.issue_pending; });
      if (s->queue.empty() && s->issuing == 0 && !handing) {
        issue(s, slot, lk);
      } else {
        slot.issue_pending = true;
        slot.cv_issue.notify_one();
      }
    }
    const bool inflight = std::any_of(s->slots.begin(), s->slots.end(), [](const Slot& x) { return x.busy; });
    if (s->stop && s->queue.empty() && !inflight) break;
    const Clock::time_point now = Clock::now();
    if (progressed) {
      last_progress = now;
    } else if (inflight || now < last_progress + spin) {
      // poll while a group is in flight (its completion is then seen at once,
      // not through the callback thread) and for the window after progress
      lk.unlock();
      poll_for_work(s, seen, inflight ? now + spin : last_progress + spin);
      lk.lock();
    } else if (s->pokes.load(std::memory_order_acquire) == seen) {
      // sleep until a callback, a submit, a resume or stop (bounded: re-check)
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
}

}  // namespace

extern "C" {

tx16_status tx16_serve_create(const char* json_cfg, tx16_server** out) {
  if (out == nullptr) return TX16_EINVAL;
  *out = nullptr;
  std::map<std::string, double> cfg;
  if (!parse_cfg(json_cfg, cfg)) return TX16_EINVAL;
  tx16_server* s = new tx16_server();
  cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete s;
    return TX16_ECUDA;
  }
  const double pool_mb = cfg.count("device_pool_mb") ? cfg["device_pool_mb"]
                                                      : std::min(4096.0, double(free_b) / 4.0 / (1 << 20));
  const int nslots = cfg.count("streams") ? int(cfg["streams"]) : 6;
  s->max_batch = cfg.count("max_batch") ? int(cfg["max_batch"]) : 256;
  s->max_queue = cfg.count("max_queue") ? size_t(cfg["max_queue"]) : size_t(1) << 20;
  s->spin_us = cfg.count("spin_us") ? cfg["spin_us"] : 300.0;
  s->wait_spin_us = cfg.count("wait_spin_us") ? cfg["wait_spin_us"] : 2000.0;
  const double band_mb = cfg.count("band_mb") ? cfg["band_mb"] : 4.0;
  if (!(band_mb >= 0 && band_mb <= 65536)) {
    delete s;
    return TX16_EINVAL;
  }
  s->band_bytes = size_t(band_mb * (1 << 20));
  const size_t pool = size_t(pool_mb * (1 << 20));
  if (pool < 4096 || nslots < 1 || nslots > 16 || s->max_batch < 1 || s->max_batch > 4096 || s->max_queue < 1 ||
      !(s->spin_us >= 0 && s->spin_us <= 1e6) || !(s->wait_spin_us >= 0 && s->wait_spin_us <= 1e6)) {
    delete s;
    return TX16_EINVAL;
  }
  if (pool > free_b || !s->arena.init(pool)) {  // admission is bounded by free HBM
    delete s;
    return TX16_ENOMEM;
  }
  for (int i = 0; i < nslots; ++i) s->slots.emplace_back();
  for (Slot& slot : s->slots) {
    slot.server = s;
    bool ok = cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&slot.in_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&slot.out_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&slot.event, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&slot.d_sse, sizeof(uint64_t) * kMaxBands * size_t(s->max_batch)) == cudaSuccess &&
              cudaMallocHost(&slot.h_sse, sizeof(uint64_t) * kMaxBands * size_t(s->max_batch)) == cudaSuccess;
    for (int b = 0; ok && b < kMaxBands; ++b)
      ok = cudaEventCreateWithFlags(&slot.in_ev[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&slot.band_ev[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      tx16_serve_destroy(s);
      return TX16_ENOMEM;
    }
  }
  for (Slot& slot : s->slots) slot.issuer = std::thread(issuer_main, s, &slot);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return TX16_OK;
}

tx16_status tx16_serve_submit(tx16_server* s, const void* host_pixels, int32_t w, int32_t h, int32_t bits,
                              tx16_qparams qp, void* host_recon, uint64_t* ticket) {
  TX16_TRACE("tx16_serve_submit");
  if (s == nullptr || host_pixels == nullptr || ticket == nullptr) return TX16_EINVAL;
  tx16_image probe{const_cast<void*>(host_pixels), w, h, int64_t(w) * (bits == 8 ? 1 : 2), bits};
  if ((reinterpret_cast<uintptr_t>(host_pixels) & 15u) != 0) probe.data = reinterpret_cast<void*>(16);
  if (!valid_image(probe) || qp.r < 1 || qp.r > 256 || !std::isfinite(qp.q)) return TX16_EINVAL;
  const size_t bytes = size_t(w) * size_t(h) * (bits == 8 ? 1 : 2);
  if (2 * ((bytes + 255) & ~size_t(255)) > s->arena.capacity()) return TX16_ENOMEM;  // can never be admitted
  Request* r = new Request();
  r->host_in = host_pixels;
  r->host_out = host_recon;
  r->w = w;
  r->h = h;
  r->bits = bits;
  r->qp = qp;
  r->bytes = bytes;
  r->blocks = int64_t(w / 16) * (h / 16);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return TX16_EINVAL;
    }
    if (s->queue.size() >= s->max_queue) {
      delete r;
      return TX16_EBUSY;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    if (!s->any) {
      s->t_first = r->t_submit;
      s->any = true;
    }
    s->queue.push_back(r);
    s->live[r->ticket] = r;
    *ticket = r->ticket;
    s->pokes.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_one();
  // An idle server: admit and launch the request here, on the caller's
  // thread, instead of waking the worker for it.
  {
    std::unique_lock<std::mutex> lk(s->mu);
    const bool idle = !s->paused && !s->stop && s->queue.size() == 1 && s->queue.front() == r &&
                      std::none_of(s->slots.begin(), s->slots.end(), [](const Slot& x) { return x.busy; });
    if (idle && admit(s, s->slots.front())) issue(s, s->slots.front(), lk);
  }
  return TX16_OK;
}

tx16_status tx16_serve_wait(tx16_server* s, uint64_t ticket, int32_t timeout_ms, double* psnr, double* latency_us) {
  TX16_TRACE("tx16_serve_wait");
  if (s == nullptr) return TX16_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->live.find(ticket);
  if (it == s->live.end()) return TX16_EINVAL;
  Request* r = it->second;  // only its waiter frees it, so it outlives the unlocked poll
  const Clock::time_point t0 = Clock::now();
  const auto deadline = t0 + std::chrono::milliseconds(std::max(0, timeout_ms));
  if (!r->done.load(std::memory_order_acquire) && s->wait_spin_us > 0) {
    const auto until = std::min(deadline, t0 + std::chrono::duration_cast<Clock::duration>(
                                                   std::chrono::duration<double, std::micro>(s->wait_spin_us)));
    lk.unlock();
    while (!r->done.load(std::memory_order_acquire) && Clock::now() < until) {
      // retire the request's group here once its event has fired
      Slot* slot = r->slot.load(std::memory_order_acquire);
      tx16_status st;
      if (slot != nullptr && slot_finished(*slot, &st)) {
        lk.lock();
        if (!r->done.load(std::memory_order_acquire) && r->slot.load(std::memory_order_acquire) == slot &&
            slot->busy && slot_finished(*slot, &st)) {
          retire(s, *slot, st);
          s->cv_done.notify_all();
          s->pokes.fetch_add(1, std::memory_order_release);  // the worker may admit into the freed slot
          s->cv_work.notify_one();
        }
        lk.unlock();
      }
    }
    lk.lock();
  }
  while (!r->done.load(std::memory_order_acquire)) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done.load(std::memory_order_acquire))
      return TX16_ETIMEOUT;
  }
  if (psnr) *psnr = r->psnr;
  if (latency_us) *latency_us = r->latency_us;
  const tx16_status st = r->status;
  s->live.erase(it);
  delete r;
  return st;
}

tx16_status tx16_serve_stats(tx16_server* s, double* p50_us, double* p99_us, double* p999_us,
                             double* mblocks_per_s) {
  if (s == nullptr) return TX16_EINVAL;
  std::vector<double> v;
  double blocks = 0, span = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    v = s->lat;
    blocks = s->blocks_done;
    span = s->any ? now_us(s->t_first, s->t_last) : 0.0;
  }
  auto pct = [&](double f) {
    if (v.empty()) return 0.0;
    size_t k = std::min(v.size() - 1, size_t(f * double(v.size())));
    std::nth_element(v.begin(), v.begin() + long(k), v.end());
    return v[k];
  };
  if (p50_us) *p50_us = pct(0.50);
  if (p99_us) *p99_us = pct(0.99);
  if (p999_us) *p999_us = pct(0.999);
  if (mblocks_per_s) *mblocks_per_s = span > 0 ? blocks / span : 0.0;  // blocks per us = Mblocks/s
  return TX16_OK;
}

tx16_status tx16_serve_pause(tx16_server* s, int32_t paused) {
  if (s == nullptr) return TX16_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
    s->pokes.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_all();
  return TX16_OK;
}

tx16_status tx16_serve_reset_stats(tx16_server* s) {
  if (s == nullptr) return TX16_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat.clear();
  s->lat_seen = 0;
  s->blocks_done = 0;
  s->any = false;
  return TX16_OK;
}

void tx16_serve_destroy(tx16_server* s) {
  if (s == nullptr) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->paused = false;  // let queued work drain
    s->pokes.fetch_add(1, std::memory_order_release);
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_issuers = true;
  }
  for (Slot& slot : s->slots) {
    slot.cv_issue.notify_all();
    if (slot.issuer.joinable()) slot.issuer.join();
  }
  for (Slot& slot : s->slots) {
    if (slot.stream) cudaStreamSynchronize(slot.stream);
    if (slot.in_stream) cudaStreamSynchronize(slot.in_stream);
    if (slot.out_stream) cudaStreamSynchronize(slot.out_stream);
    if (slot.event) cudaEventDestroy(slot.event);
    for (int b = 0; b < kMaxBands; ++b) {
      if (slot.in_ev[b]) cudaEventDestroy(slot.in_ev[b]);
      if (slot.band_ev[b]) cudaEventDestroy(slot.band_ev[b]);
    }
    if (slot.stream) cudaStreamDestroy(slot.stream);
    if (slot.in_stream) cudaStreamDestroy(slot.in_stream);
    if (slot.out_stream) cudaStreamDestroy(slot.out_stream);
    if (slot.d_sse) cudaFree(slot.d_sse);
    if (slot.h_sse) cudaFreeHost(slot.h_sse);
  }
  for (auto& kv : s->live) delete kv.second;
  s->arena.release();
  delete s;
}

}  // extern "C"
