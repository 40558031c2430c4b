// server.cu -- the serving loop behind sv_submit / sv_poll / sv_cancel.
//
// Continuous batching: a worker thread keeps up to serve_slots launches in flight,
// each on its own stream with its own device workspace, so their kernels
// overlap on the GPU.  Whenever a slot frees up, everything queued is packed
// into the next launch: range requests are cut into chunks of at most
// kChunkLen integers (a long range never blocks short ones for long), point
// requests into batches; a launch is bounded in odd n, chunks and points, and
// is admitted only while the device memory of all launches in flight stays
// within the configured budget.  Chunks of one range may run in different
// launches; their aggregates merge exactly (sums of histograms, minima of
// first occurrences, union of lists), so a result never depends on what else
// was in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "ctx.h"

namespace sv {

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxSlots = 8;  // launch slots at most (sv_config.serve_slots)
constexpr uint64_t kChunkLen = 1ull << 30;        // integers per range chunk
constexpr uint64_t kMaxOddPerLaunch = 1ull << 32; // odd n per launch
constexpr uint64_t kMaxPointsPerLaunch = 1ull << 16;
constexpr size_t kMaxChunksPerLaunch = 4096;
constexpr size_t kMaxQueued = 1u << 20;

struct Request {
  uint64_t ticket = 0;
  sv_request r{};
  enum State { kQueued, kRunning, kDone, kCancelled } state = kQueued;
  uint64_t next_lo = 0;
  uint64_t next_point = 0;
  uint32_t outstanding = 0;
  bool issued_all = false;
  sv_status status = SV_OK;
  uint64_t hist[kMaxK] = {0};
  uint64_t first[kMaxK];
  uint64_t list_count = 0, fail_count = 0;
  std::vector<std::pair<uint64_t, uint8_t>> list;
  std::vector<uint64_t> fails;
  Clock::time_point t_submit;
};

struct Item {
  uint64_t ticket, lo, hi;
};
struct PItem {
  uint64_t ticket, first, count, off;
};

struct Slot {
  Workspace ws;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  uint64_t mem = 0;  // device bytes this launch was admitted with
  std::vector<Item> items;
  std::vector<RangeSpec> specs;
  std::vector<PItem> pitems;
  uint64_t npoints = 0;
  std::vector<sv_range_result> outs;
  std::vector<std::vector<uint64_t>> lbuf, fbuf;
  std::vector<std::vector<uint8_t>> kbuf;
};

uint64_t chunk_list_cap(uint64_t n_odd, uint32_t T, uint64_t caller_cap) {
  return list_cap_estimate(n_odd, T, caller_cap);
}

// Device bytes a launch of `items` range chunks with `tiles` tiles in all,
// `list` list entries and `points` point queries holds: tile buckets
// (bucket_cap entries per tile, 1024 before the first launch sized them),
// the per-tile list staging, lists, points, descriptors and result slots,
// and 1 MiB of headers and straggler queue.
uint64_t launch_mem(uint64_t tiles, uint64_t list, uint64_t points, uint64_t items, uint32_t bucket_cap) {
  return tiles * 4ull * (bucket_cap ? bucket_cap + 1 : 1024) + tiles * (9ull * kStageCap + 4) + list * 9 +
         points * 17 + (items + 1) * (sizeof(ReqDesc) + sizeof(ResultSlot)) + (1u << 20);
}

}  // namespace

class Server {
 public:
  explicit Server(sv_ctx *c) : c_(c), n_slots_((int)std::min<uint32_t>(std::max<uint32_t>(c->cfg.serve_slots, 1), kMaxSlots)) {}
  ~Server() { shutdown(); }

  sv_status init() {
    for (int i = 0; i < n_slots_; ++i) {
      Slot &s = slots_[i];
      if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess) return SV_ECUDA;
      if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) return SV_ECUDA;
      // staging for the points of one launch, sized once: fill() packs several
      // requests into it and must never see it reallocated
      if (s.ws.h_points.ensure(kMaxPointsPerLaunch) || s.ws.h_points_out.ensure(kMaxPointsPerLaunch))
        return SV_ENOMEM;
    }
    th_ = std::thread([this] { loop(); });
    return SV_OK;
  }

  void shutdown() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (stop_) return;
      stop_ = true;
    }
    cv_work_.notify_all();
    if (th_.joinable()) th_.join();
    std::lock_guard<std::mutex> lk(mu_);
    for (auto &kv : reqs_)
      if (kv.second.state == Request::kQueued || kv.second.state == Request::kRunning)
        kv.second.state = Request::kCancelled;
    cv_done_.notify_all();
    for (int i = 0; i < n_slots_; ++i) {
      Slot &s = slots_[i];
      if (s.st) cudaStreamSynchronize(s.st);
      s.ws.release_all();
      if (s.ev) cudaEventDestroy(s.ev);
      if (s.st) cudaStreamDestroy(s.st);
      s.ev = nullptr;
      s.st = nullptr;
    }
  }

  // Validates one request and estimates its smallest unit's device memory
  // (mu_ not needed).
  sv_status check(const sv_request *req, uint64_t *unit_mem) const {
    if (req->kind == SV_REQ_RANGE) {
      if (!req->result) return SV_EINVAL;
      if (req->hi > c_->max_hi || req->hi > (1ull << 62)) return SV_ERANGE;
      const uint64_t len = req->hi > req->lo ? req->hi - req->lo : 0;
      const uint64_t n = range_odd_count(req->lo, req->lo + (len < kChunkLen ? len : kChunkLen));
      const uint64_t tile_odd = 1ull << c_->cfg.tile_log2;
      *unit_mem = launch_mem((n + tile_odd - 1) / tile_odd + 1,
                             chunk_list_cap(n, c_->cfg.record_k_threshold, req->result->list_cap), 0, 1, 0);
    } else if (req->kind == SV_REQ_POINTS) {
      if (req->n_points && (!req->points || !req->out_k)) return SV_EINVAL;
      for (uint64_t i = 0; i < req->n_points; ++i)
        if (req->points[i] > c_->max_hi) return SV_ERANGE;
      *unit_mem = launch_mem(0, 0, std::min<uint64_t>(req->n_points, kMaxPointsPerLaunch), 0, 0);
    } else {
      return SV_EINVAL;
    }
    return SV_OK;
  }

  // Queues a checked request (mu_ held).
  sv_status enqueue_locked(const sv_request *req, uint64_t unit_mem, uint64_t *ticket) {
    if (stop_) return SV_ECANCELLED;
    if (queue_.size() >= kMaxQueued || unit_mem > c_->cfg.device_mem_budget) {
      ++refused_;
      return SV_ENOMEM;
    }
    const uint64_t t = next_ticket_++;
    Request &r = reqs_[t];
    r.ticket = t;
    r.r = *req;
    r.t_submit = Clock::now();
    r.next_lo = req->lo;
    for (int k = 0; k < kMaxK; ++k) r.first[k] = kNoN;
    ++submitted_;
    *ticket = t;
    const bool empty = (req->kind == SV_REQ_RANGE) ? (range_odd_count(req->lo, req->hi) == 0) : (req->n_points == 0);
    if (empty) {
      r.issued_all = true;
      complete(r);
    } else {
      queue_.push_back(t);
    }
    return SV_OK;
  }

  // Several requests under one lock; status[i] per request, tickets[i] valid
  // where status[i] is SV_OK.  Returns the first failing status (or SV_OK).
  sv_status submit_many(const sv_request *reqs, size_t count, uint64_t *tickets, sv_status *status) {
    std::vector<uint64_t> mem(count);
    sv_status first = SV_OK;
    for (size_t i = 0; i < count; ++i) {
      status[i] = check(&reqs[i], &mem[i]);
      if (status[i] && !first) first = status[i];
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      for (size_t i = 0; i < count; ++i) {
        if (status[i]) continue;
        status[i] = enqueue_locked(&reqs[i], mem[i], &tickets[i]);
        if (status[i] && !first) first = status[i];
      }
    }
    cv_work_.notify_one();
    return first;
  }

  sv_status submit(const sv_request *req, uint64_t *ticket) {
    sv_status st;
    return submit_many(req, 1, ticket, &st);
  }

  sv_status poll(uint64_t ticket, int64_t timeout_us) {
    std::unique_lock<std::mutex> lk(mu_);
    auto it = reqs_.find(ticket);
    if (it == reqs_.end()) return SV_ENOTFOUND;
    auto done = [&] {
      auto j = reqs_.find(ticket);
      return j == reqs_.end() || j->second.state == Request::kDone || j->second.state == Request::kCancelled;
    };
    if (timeout_us < 0)
      cv_done_.wait(lk, done);
    else if (timeout_us > 0)
      cv_done_.wait_for(lk, std::chrono::microseconds(timeout_us), done);
    it = reqs_.find(ticket);
    if (it == reqs_.end()) return SV_ENOTFOUND;
    if (it->second.state == Request::kDone) {
      const sv_status s = it->second.status;
      reqs_.erase(it);
      return s;
    }
    if (it->second.state == Request::kCancelled) {
      reqs_.erase(it);
      return SV_ECANCELLED;
    }
    return SV_EAGAIN;
  }

  sv_status cancel(uint64_t ticket) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = reqs_.find(ticket);
    if (it == reqs_.end()) return SV_ENOTFOUND;
    Request &r = it->second;
    if (r.state == Request::kCancelled) return SV_OK;
    if (r.state != Request::kQueued || r.outstanding || r.next_point || r.next_lo != r.r.lo) return SV_EAGAIN;
    r.state = Request::kCancelled;
    queue_.erase(std::remove(queue_.begin(), queue_.end(), ticket), queue_.end());
    ++cancelled_;
    cv_done_.notify_all();
    return SV_OK;
  }

  void reset_stats() {
    std::lock_guard<std::mutex> lk(mu_);
    submitted_ = completed_ = cancelled_ = refused_ = odd_done_ = launches_ = 0;
    peak_mem_ = 0;
    lat_us_.clear();
    t_reset_ = Clock::now();
    busy_us_ = 0.0;
  }

  sv_status stats(sv_server_stats *o) {
    std::lock_guard<std::mutex> lk(mu_);
    std::memset(o, 0, sizeof(*o));
    o->submitted = submitted_;
    o->completed = completed_;
    o->cancelled = cancelled_;
    o->refused = refused_;
    o->odd_n_done = odd_done_;
    o->launches = launches_;
    o->queued = queue_.size();
    uint64_t inflight = 0;
    for (auto &kv : reqs_)
      if (kv.second.state == Request::kRunning) ++inflight;
    o->in_flight = inflight;
    o->peak_mem_in_flight = peak_mem_;
    o->wall_us = std::chrono::duration<double, std::micro>(Clock::now() - t_reset_).count();
    o->loop_busy_us = busy_us_;
    if (!lat_us_.empty()) {
      std::vector<double> v = lat_us_;
      const size_t i50 = v.size() / 2, i99 = std::min(v.size() - 1, (v.size() * 99) / 100);
      std::nth_element(v.begin(), v.begin() + i50, v.end());
      o->p50_us = v[i50];
      std::nth_element(v.begin(), v.begin() + i99, v.end());
      o->p99_us = v[i99];
    }
    return SV_OK;
  }

 private:
  uint64_t mem_in_flight() const {
    uint64_t m = 0;
    for (int i = 0; i < n_slots_; ++i)
      if (slots_[i].busy) m += slots_[i].mem;
    return m;
  }

  // Packs queued work into slot s (mu_ held).  Returns false if nothing fits.
  bool fill(Slot &s) {
    s.items.clear();
    s.specs.clear();
    s.pitems.clear();
    s.npoints = 0;
    uint64_t odd = 0, tiles = 0, listb = 0;
    const uint64_t tile_odd = 1ull << c_->cfg.tile_log2;
    const uint32_t T = c_->cfg.record_k_threshold;
    const uint64_t budget = c_->cfg.device_mem_budget;
    const uint64_t in_flight = mem_in_flight();
    auto mem = [&](uint64_t t, uint64_t l, uint64_t np, uint64_t items) {
      return launch_mem(t, l, np, items, s.ws.bucket_cap);
    };
    // the budget holds for all launches in flight; the first unit of a
    // launch may exceed it only when nothing else is in flight (it fits the
    // budget alone: submit checked that)
    auto over = [&](uint64_t m) { return in_flight + m > budget && (!s.items.empty() || s.npoints || in_flight); };
    for (auto it = queue_.begin(); it != queue_.end();) {
      Request &r = reqs_[*it];
      if (r.r.kind == SV_REQ_RANGE) {
        while (r.next_lo < r.r.hi && odd < kMaxOddPerLaunch && s.items.size() < kMaxChunksPerLaunch) {
          const uint64_t clo = r.next_lo;
          const uint64_t chi = (r.r.hi - clo > kChunkLen) ? clo + kChunkLen : r.r.hi;
          const uint64_t n = range_odd_count(clo, chi);
          const uint64_t lc = chunk_list_cap(n, T, r.r.result->list_cap);
          const uint64_t t = (n + tile_odd - 1) / tile_odd + 1;
          if (over(mem(tiles + t, listb + lc, s.npoints, s.items.size() + 1))) break;
          RangeSpec sp;
          sp.lo = clo;
          sp.hi = chi;
          sp.list_cap = lc;
          sp.want_cap = r.r.result->list_cap;
          sp.fail_cap = 64;
          s.items.push_back({r.ticket, clo, chi});
          s.specs.push_back(sp);
          odd += n;
          tiles += t;
          listb += lc;
          r.next_lo = chi;
          r.outstanding++;
          r.state = Request::kRunning;
        }
        if (r.next_lo >= r.r.hi) {
          r.issued_all = true;
          it = queue_.erase(it);
          continue;
        }
        break;  // this launch is full
      } else {
        const uint64_t room = kMaxPointsPerLaunch - s.npoints;
        if (room == 0) break;
        const uint64_t cnt = std::min<uint64_t>(room, r.r.n_points - r.next_point);
        if (over(mem(tiles, listb, s.npoints + cnt, s.items.size()))) break;
        std::memcpy(s.ws.h_points.p + s.npoints, r.r.points + r.next_point, 8 * cnt);
        s.pitems.push_back({r.ticket, r.next_point, cnt, s.npoints});
        s.npoints += cnt;
        r.next_point += cnt;
        r.outstanding++;
        r.state = Request::kRunning;
        if (r.next_point >= r.r.n_points) {
          r.issued_all = true;
          it = queue_.erase(it);
          continue;
        }
        break;
      }
    }
    s.mem = mem(tiles, listb, s.npoints, s.items.size());
    const bool any = !s.items.empty() || s.npoints;
    if (any) peak_mem_ = std::max(peak_mem_, in_flight + s.mem);
    return any;
  }

  // Enqueues slot s's launch (mu_ not held).
  sv_status start(Slot &s) {
    sv_status st = SV_OK;
    if (!s.items.empty()) st = launch_ranges_async(c_, s.specs, s.ws, s.st);
    if (!st && s.npoints) st = launch_points_async(c_, s.npoints, s.ws, s.st);
    if (cudaEventRecord(s.ev, s.st) != cudaSuccess && !st) st = SV_ECUDA;
    return st;
  }

  // Collects slot s's results (mu_ not held); then merges them (mu_ taken).
  void finish(Slot &s, sv_status launch_status) {
    sv_status st = launch_status;
    const size_t n = s.items.size();
    s.outs.assign(n, sv_range_result{});
    s.lbuf.resize(n);
    s.kbuf.resize(n);
    s.fbuf.resize(n);
    std::vector<sv_range_result *> ptrs(n);
    for (size_t i = 0; i < n; ++i) {
      s.lbuf[i].resize(std::max<uint64_t>(s.specs[i].list_cap, 1));
      s.kbuf[i].resize(std::max<uint64_t>(s.specs[i].list_cap, 1));
      s.fbuf[i].resize(64);
      sv_range_result &o = s.outs[i];
      o.list = s.lbuf[i].data();
      o.list_k = s.kbuf[i].data();
      o.list_cap = s.specs[i].list_cap;
      o.failures = s.fbuf[i].data();
      o.fail_cap = 64;
      ptrs[i] = &o;
    }
    if (!st && n) {
      bool retry = false;
      st = collect_ranges(c_, s.specs, ptrs.data(), s.ws, s.st, &retry);
      if (!st && retry) {
        // an overflow: give the chunks full room and repeat them, blocking
        for (size_t i = 0; i < n; ++i) {
          const uint64_t full = s.outs[i].list_len > s.specs[i].list_cap ? s.outs[i].list_len : 0;
          if (full) {
            s.specs[i].list_cap = full;
            s.lbuf[i].resize(full);
            s.kbuf[i].resize(full);
            s.outs[i].list = s.lbuf[i].data();
            s.outs[i].list_k = s.kbuf[i].data();
            s.outs[i].list_cap = full;
          }
        }
        st = run_ranges(c_, s.specs, ptrs.data(), s.st, s.ws);
      }
    }
    if (!st && cudaStreamSynchronize(s.st) != cudaSuccess) st = SV_ECUDA;

    std::lock_guard<std::mutex> lk(mu_);
    ++launches_;
    for (size_t i = 0; i < n; ++i) {
      auto it = reqs_.find(s.items[i].ticket);
      if (it == reqs_.end()) continue;
      Request &r = it->second;
      if (st) r.status = st;
      const sv_range_result &o = s.outs[i];
      if (!st) {
        for (int k = 0; k < kMaxK; ++k) {
          r.hist[k] += o.hist[k];
          if (o.first_n[k] < r.first[k]) r.first[k] = o.first_n[k];
        }
        r.list_count += o.list_len;
        r.fail_count += o.fail_len;
        const uint64_t nl = std::min<uint64_t>(o.list_len, o.list_cap);
        for (uint64_t j = 0; j < nl; ++j) r.list.emplace_back(o.list[j], o.list_k[j]);
        const uint64_t nf = std::min<uint64_t>(o.fail_len, o.fail_cap);
        for (uint64_t j = 0; j < nf; ++j) r.fails.push_back(o.failures[j]);
      }
      if (--r.outstanding == 0 && r.issued_all) complete(r);
    }
    for (const PItem &p : s.pitems) {
      auto it = reqs_.find(p.ticket);
      if (it == reqs_.end()) continue;
      Request &r = it->second;
      if (st) r.status = st;
      else std::memcpy(r.r.out_k + p.first, s.ws.h_points_out.p + p.off, p.count);
      if (--r.outstanding == 0 && r.issued_all) complete(r);
    }
    s.busy = false;
    s.items.clear();
    s.pitems.clear();
    s.npoints = 0;
  }

  // Writes the merged result into the caller's buffers (mu_ held).
  void complete(Request &r) {
    if (r.r.kind == SV_REQ_RANGE && r.status == SV_OK) {
      sv_range_result *o = r.r.result;
      o->lo = r.r.lo;
      o->hi = r.r.hi;
      o->n_odd = range_odd_count(r.r.lo, r.r.hi);
      o->ksum = 0;
      o->kmax = 0;
      for (int k = 0; k < kMaxK; ++k) {
        o->hist[k] = r.hist[k];
        o->first_n[k] = r.first[k];
        if (k && r.hist[k]) {
          o->ksum += (uint64_t)k * r.hist[k];
          o->kmax = (uint64_t)k;
        }
      }
      std::sort(r.list.begin(), r.list.end());
      const uint64_t m = std::min<uint64_t>(r.list.size(), o->list_cap);
      for (uint64_t j = 0; j < m; ++j) {
        if (o->list) o->list[j] = r.list[j].first;
        if (o->list_k) o->list_k[j] = r.list[j].second;
      }
      o->list_len = r.list_count;
      o->list_overflow = r.list_count > o->list_cap ? 1 : 0;
      std::sort(r.fails.begin(), r.fails.end());
      const uint64_t mf = std::min<uint64_t>(r.fails.size(), o->fail_cap);
      if (o->failures)
        for (uint64_t j = 0; j < mf; ++j) o->failures[j] = r.fails[j];
      o->fail_len = r.fail_count;
      odd_done_ += o->n_odd;
    } else if (r.r.kind == SV_REQ_POINTS && r.status == SV_OK) {
      odd_done_ += r.r.n_points;
    }
    r.list.clear();
    r.list.shrink_to_fit();
    r.fails.clear();
    r.state = Request::kDone;
    ++completed_;
    lat_us_.push_back(std::chrono::duration<double, std::micro>(Clock::now() - r.t_submit).count());
    cv_done_.notify_all();
  }

  void loop() {
    cudaSetDevice(c_->device);
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      bool busy = false;
      for (int i = 0; i < n_slots_; ++i) {
        Slot &s = slots_[i];
        if (!s.busy) continue;
        if (cudaEventQuery(s.ev) != cudaErrorNotReady) {
          lk.unlock();
          const auto t0 = Clock::now();
          finish(s, SV_OK);
          const auto t1 = Clock::now();
          lk.lock();
          busy_us_ += std::chrono::duration<double, std::micro>(t1 - t0).count();
        } else {
          busy = true;
        }
      }
      if (!stop_) {
        for (int i = 0; i < n_slots_; ++i) {
          Slot &s = slots_[i];
          if (s.busy || queue_.empty()) continue;
          const auto t0 = Clock::now();
          if (!fill(s)) continue;
          s.busy = true;
          lk.unlock();
          const sv_status st = start(s);
          if (st) {
            finish(s, st);
            lk.lock();
            busy_us_ += std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
            continue;
          }
          const auto t1 = Clock::now();
          lk.lock();
          busy_us_ += std::chrono::duration<double, std::micro>(t1 - t0).count();
          busy = true;
        }
      }
      if (!busy) {
        if (stop_) break;
        if (queue_.empty()) {
          cv_work_.wait(lk);
          continue;
        }
      }
      cv_work_.wait_for(lk, std::chrono::microseconds(20));
    }
  }

  sv_ctx *c_;
  std::mutex mu_;
  std::condition_variable cv_work_, cv_done_;
  std::deque<uint64_t> queue_;
  std::unordered_map<uint64_t, Request> reqs_;
  uint64_t next_ticket_ = 1;
  bool stop_ = false;
  Slot slots_[kMaxSlots];
  int n_slots_ = 3;
  Clock::time_point t_reset_ = Clock::now();
  double busy_us_ = 0.0;  // the loop thread's time in fill / start / finish
  std::thread th_;
  uint64_t submitted_ = 0, completed_ = 0, cancelled_ = 0, refused_ = 0, odd_done_ = 0, launches_ = 0;
  uint64_t peak_mem_ = 0;  // largest device memory of the launches in flight at once (estimated)
  std::vector<double> lat_us_;
};

Server *server_create(sv_ctx *c) {
  Server *s = new (std::nothrow) Server(c);
  if (!s) return nullptr;
  if (s->init() != SV_OK) {
    delete s;
    return nullptr;
  }
  return s;
}

void server_destroy(Server *s) { delete s; }
sv_status server_submit(Server *s, const sv_request *req, uint64_t *ticket) { return s->submit(req, ticket); }
sv_status server_submit_many(Server *s, const sv_request *reqs, size_t count, uint64_t *tickets, sv_status *status) {
  return s->submit_many(reqs, count, tickets, status);
}
sv_status server_poll(Server *s, uint64_t ticket, int64_t timeout_us) { return s->poll(ticket, timeout_us); }
sv_status server_cancel(Server *s, uint64_t ticket) { return s->cancel(ticket); }
sv_status server_stats(Server *s, sv_server_stats *out) { return s->stats(out); }
void server_reset_stats(Server *s) { s->reset_stats(); }

}  // namespace sv
