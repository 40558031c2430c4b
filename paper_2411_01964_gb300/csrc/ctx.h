// ctx.h -- the host-side context behind the opaque sv_ctx (host runtime only).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <vector>

#include "sv.h"
#include "sv_internal.h"

namespace sv {

constexpr int kPiBlockLog2 = 12;  // block size of the host prime-count index

// Allocations still to fail on purpose (sv_inject_alloc_failures); takes one
// if any is left.
extern std::atomic<uint32_t> g_inject_alloc_failures;
inline bool take_injected_failure() {
  uint32_t n = g_inject_alloc_failures.load();
  while (n > 0 && !g_inject_alloc_failures.compare_exchange_weak(n, n - 1)) {
  }
  return n > 0;
}

// Growable device / pinned-host buffer (grows geometrically, never shrinks).
template <class T, bool PINNED>
struct Buf {
  T *p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    size_t c = cap ? cap : 1;
    while (c < n) c *= 2;
    release();
    if (take_injected_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = PINNED ? cudaMallocHost((void **)&p, c * sizeof(T)) : cudaMalloc((void **)&p, c * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      cap = 0;
      return e;
    }
    cap = c;
    return cudaSuccess;
  }
  void release() {
    if (p) {
      if (PINNED) cudaFreeHost(p);
      else cudaFree(p);
    }
    p = nullptr;
    cap = 0;
  }
};
template <class T> using DBuf = Buf<T, false>;
template <class T> using HBuf = Buf<T, true>;

// One range of a launch as the host plans it.
struct RangeSpec {
  uint64_t lo = 0, hi = 0;
  uint8_t *d_per_n = nullptr;   // device per-n output or null
  uint64_t list_cap = 0;        // device list entries reserved for it
  uint64_t want_cap = 0;        // entries the final consumer can hold (0: list_cap); an ordered
                                // list truncated below it is repeated with more room
  uint64_t fail_cap = 0;
  bool sieve_only = false;
  uint32_t *bitmap_out = nullptr;
  const uint32_t *bitmap_in = nullptr;  // scan pass of the plain path: windows from this bitmap
  int64_t bitmap_w0 = 0;                // absolute word held by bitmap_in[0]
};

// What a captured launch graph depends on (compared bytewise).
struct GraphKey {
  const void *p[16];
  Geometry g;
  uint32_t threads, ctas, mode, strag_cap;
  uint64_t req_copy;
  uint32_t n_table;
  uint32_t timed;  // 1: event-record nodes bracket the tile kernel
};

// Everything one launch needs on the device, reused across launches.
struct Workspace {
  DBuf<ReqDesc> reqs;
  HBuf<ReqDesc> h_reqs;
  DBuf<LaunchHeader> hdr;
  HBuf<LaunchHeader> h_hdr;
  DBuf<ResultSlot> slots;
  HBuf<ResultSlot> h_slots;
  DBuf<uint64_t> list_n;
  DBuf<uint8_t> list_k;
  HBuf<uint64_t> h_list_n;
  HBuf<uint8_t> h_list_k;
  DBuf<uint64_t> fail_n;
  HBuf<uint64_t> h_fail_n;
  DBuf<Straggler> strag;
  DBuf<uint32_t> bucket_count;
  DBuf<uint32_t> bucket_data;
  DBuf<uint8_t> per_n;
  DBuf<uint64_t> stage_n;    // ordered lists: per-tile staged entries (kStageCap per tile)
  DBuf<uint8_t> stage_k;
  DBuf<uint32_t> stage_cnt;
  DBuf<uint64_t> points;
  DBuf<uint8_t> points_out;
  HBuf<uint64_t> h_points;
  HBuf<uint8_t> h_points_out;
  // sizes of the launch currently described by the buffers
  uint32_t n_reqs = 0, total_tiles = 0, max_primes = 0;
  uint64_t list_total = 0, fail_total = 0;
  uint32_t strag_cap = 1u << 16;
  uint32_t bucket_cap = 0;
  bool any_per_n = false;
  bool ordered = false;        // the planned launch produces ordered lists (tile kernel mode 0)
  bool force_general = false;  // repeat with the unordered list path (a tile's staging overflowed)
  bool all_from_bitmap = false;  // every range reads its windows from a bitmap: no bucket fill
  int tile_kernel_id = 2;        // per-kernel timing id of this workspace's tile kernel launches
  uint64_t j_max = 0;  // largest odd-multiplier count of the launch (bucket fill by j)
  uint32_t inject_bulk_timeouts = 0;  // plain-path launches still to run with their bulk loads left out (test hook)
  uint64_t h2d_bytes = 0, d2h_bytes = 0;
  // the captured launch graph and what it was captured for; a timed graph
  // keeps its event-record nodes around the tile kernel (gnode), whose
  // events are swapped for fresh ones before each replay
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  GraphKey gkey{};
  cudaGraphNode_t gnode[2] = {nullptr, nullptr};
  cudaEvent_t gev[2] = {nullptr, nullptr};  // the events recorded at capture
  cudaEvent_t staged = nullptr;  // recorded after the launch's reads of the pinned staging
  void release_all();
};

class Server;  // serving loop (server.cu)

// Makes the context's device current for the length of an entry point and
// gives the calling thread its own device back afterwards, so that a call from
// a thread that has another GPU current still works on the context's GPU.
struct DevGuard {
  int prev = -1;
  bool switched = false, ok = true;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev) {
      switched = cudaSetDevice(dev) == cudaSuccess;
      ok = switched;
    }
  }
  ~DevGuard() {
    if (switched) cudaSetDevice(prev);
  }
  DevGuard(const DevGuard &) = delete;
  DevGuard &operator=(const DevGuard &) = delete;
};

}  // namespace sv

struct sv_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  sv_config cfg{};          // effective configuration
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::mutex mu;            // serialises the blocking / device-resident calls
  // prime table
  uint64_t max_hi = 0, pmax = 0;
  uint32_t *d_p = nullptr;
  uint64_t *d_mu = nullptr, *d_inv = nullptr, *d_lim = nullptr;
  uint32_t *d_pbits = nullptr;  // odd-prime bitmap of the table's range
  uint64_t pbits_words = 0;
  uint32_t n_primes = 0, n_div = 0;
  std::vector<uint32_t> h_p;
  std::vector<uint32_t> h_pi;  // h_pi[b] = number of h_p entries below b * 2^kPiBlockLog2
  std::vector<double> inv_sq_suffix;  // sum over j >= i of 1/p_j^2 (bucket sizing only)
  std::atomic<size_t> smem_set{0};  // dynamic smem the tile kernel was configured for
  sv::Workspace ws;
  // the plain (unfused) path: the sieve pass's workspace and the bitmap
  // between the two passes
  sv::Workspace ws_sieve;
  sv::DBuf<uint32_t> plain_bitmap;
  // device-resident pending launch
  bool pending = false;
  bool pending_graph = false;
  bool pending_plain = false;
  std::vector<sv::RangeSpec> pending_specs;
  std::vector<sv::RangeSpec> pending_sieve_specs;
  // per-kernel timing with events on the launching stream (sv_kernel_timing)
  uint32_t kprof = 0;  // kernel ids timed with events (bit i: id i)
  struct KEv {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<KEv> kev;
  std::vector<cudaEvent_t> ev_pool;
  double k_ms[8] = {0};
  uint64_t k_n[8] = {0};
  // counters
  std::atomic<uint64_t> launches{0};
  uint64_t last_h2d = 0, last_d2h = 0;
  sv::Server *server = nullptr;
};

namespace sv {
// Shared by api.cu and server.cu.
sv_status run_ranges(sv_ctx *c, std::vector<RangeSpec> &specs, sv_range_result **outs, cudaStream_t st,
                     Workspace &ws, bool graph = false);
sv_status run_points(sv_ctx *c, const uint64_t *points, size_t count, uint8_t *out_k, cudaStream_t st,
                     Workspace &ws);
// Asynchronous halves used by the serving loop: enqueue a launch of ranges on
// `st` (no wait), then later collect it (waits for `st`); *retry is set when
// the device reported an overflow and the launch must be repeated.
sv_status launch_ranges_async(sv_ctx *c, std::vector<RangeSpec> &specs, Workspace &ws, cudaStream_t st);
sv_status collect_ranges(sv_ctx *c, const std::vector<RangeSpec> &specs, sv_range_result **outs, Workspace &ws,
                         cudaStream_t st, bool *retry);
// Points already staged in ws.h_points: upload, test, download into
// ws.h_points_out (no wait).
sv_status launch_points_async(sv_ctx *c, uint64_t count, Workspace &ws, cudaStream_t st);
uint64_t range_odd_count(uint64_t lo, uint64_t hi);
// Device list entries to reserve for a range of n_odd odd n with threshold T
// (twice the heuristic expectation plus slack, at most cap); an overflow is
// detected on the device and the launch repeated with exact room.
uint64_t list_cap_estimate(uint64_t n_odd, uint32_t T, uint64_t cap);
Geometry geometry_for_span(const sv_ctx *c, uint64_t span_bits);
PrimeTab prime_table_of(const sv_ctx *c);
uint32_t primes_upto_of(const sv_ctx *c, uint64_t x);
sv_status tile_smem_ready(sv_ctx *c);
Server *server_create(sv_ctx *c);
void server_destroy(Server *s);
sv_status server_submit(Server *s, const sv_request *req, uint64_t *ticket);
sv_status server_submit_many(Server *s, const sv_request *reqs, size_t count, uint64_t *tickets, sv_status *status);
sv_status server_poll(Server *s, uint64_t ticket, int64_t timeout_us);
sv_status server_cancel(Server *s, uint64_t ticket);
sv_status server_stats(Server *s, sv_server_stats *out);
void server_reset_stats(Server *s);
}  // namespace sv
