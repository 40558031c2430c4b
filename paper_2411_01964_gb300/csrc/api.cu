// api.cu -- host runtime behind include/sv.h: context, prime table, launch
// planning (ranges -> tiles -> buckets), the fixed kernel sequence of one
// launch, result collection and the retry-on-overflow policy.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "ctx.h"

using namespace sv;

namespace sv {

std::atomic<uint32_t> g_inject_alloc_failures{0};

void Workspace::release_all() {
  if (gexec) cudaGraphExecDestroy(gexec);
  gexec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  graph = nullptr;
  for (cudaEvent_t &e : gev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  if (staged) cudaEventDestroy(staged);
  staged = nullptr;
  reqs.release();
  h_reqs.release();
  hdr.release();
  h_hdr.release();
  slots.release();
  h_slots.release();
  list_n.release();
  list_k.release();
  h_list_n.release();
  h_list_k.release();
  fail_n.release();
  h_fail_n.release();
  strag.release();
  bucket_count.release();
  bucket_data.release();
  per_n.release();
  stage_n.release();
  stage_k.release();
  stage_cnt.release();
  points.release();
  points_out.release();
  h_points.release();
  h_points_out.release();
}

uint64_t host_isqrt(uint64_t x) {
  // floor(sqrt(x)): a double-precision first guess (within a few units of
  // the root), then exact integer steps to r^2 <= x < (r+1)^2 (r < 2^32, so
  // the squares do not overflow)
  uint64_t r = (uint64_t)std::sqrt((double)x);
  if (r > 0xFFFFFFFFull) r = 0xFFFFFFFFull;
  while (r > 0 && r * r > x) --r;
  while (r < 0xFFFFFFFFull && (r + 1) * (r + 1) <= x) ++r;
  return r;
}

uint64_t range_odd_count(uint64_t lo, uint64_t hi) {
  const uint64_t nlo = (lo < 3 ? 3 : lo) | 1ull;
  return hi > nlo ? (hi - nlo + 1) / 2 : 0;
}

}  // namespace sv

namespace {

constexpr uint64_t kMaxHi = 1ull << 62;

sv_status cuda_status(cudaError_t e) { return e == cudaSuccess ? SV_OK : SV_ECUDA; }

#define SV_TRY_CUDA(expr)                       \
  do {                                          \
    cudaError_t e__ = (expr);                   \
    if (e__ != cudaSuccess) return SV_ECUDA;    \
  } while (0)

// The context's device is current until the end of the enclosing entry point.
#define SV_ON_DEVICE(c)                       \
  DevGuard dev_guard__((c)->device);          \
  if (!dev_guard__.ok) return SV_ECUDA

uint32_t ilog2_u32(uint32_t x) { return 31u - (uint32_t)__builtin_clz(x); }

// Number of table primes p with p <= x.
uint32_t primes_upto(const sv_ctx *c, uint64_t x) {
  if (x > 0xFFFFFFFFull) x = 0xFFFFFFFFull;
  // the index narrows the search to the primes of x's block of 2^kPiBlockLog2
  const uint64_t blk = x >> kPiBlockLog2;
  if (blk + 1 >= c->h_pi.size())
    return (uint32_t)(std::upper_bound(c->h_p.begin(), c->h_p.end(), (uint32_t)x) - c->h_p.begin());
  const auto b = c->h_p.begin();
  return (uint32_t)(std::upper_bound(b + c->h_pi[blk], b + c->h_pi[blk + 1], (uint32_t)x) - b);
}

// Defaults and validation of the tuning knobs.
sv_status normalise_config(sv_ctx *c, sv_config *k) {
  // defaults: the fastest shape measured on GB300 for 2^33-odd-n ranges
  if (k->tile_log2 == 0) k->tile_log2 = 19;
  if (k->margin_log2 == 0) k->margin_log2 = 13;
  if (k->threads == 0) k->threads = 512;
  if (k->record_k_threshold == 0) k->record_k_threshold = 6;
  if (k->ctas_per_sm == 0) k->ctas_per_sm = 2;
  if (k->stamp_primes == 0) k->stamp_primes = 4;
  if (k->stamp_primes > 8 || (k->stamp_primes & 1)) return SV_EINVAL;
  if (k->list_capacity == 0) k->list_capacity = 1ull << 16;
  if (k->device_mem_budget == 0) k->device_mem_budget = 8ull << 30;
  if (k->tile_log2 < 12 || k->tile_log2 > 20) return SV_EINVAL;
  if (k->margin_log2 < 6 || k->margin_log2 > k->tile_log2 + 1) return SV_EINVAL;
  if (k->threads < 128 || k->threads > 1024 || (k->threads & 31)) return SV_EINVAL;
  if (k->record_k_threshold > 63) return SV_EINVAL;
  if (k->ctas_per_sm > 4) return SV_EINVAL;
  const size_t tw = 1ull << (k->tile_log2 - 5), mw = 1ull << (k->margin_log2 - 6);
  const size_t smem = 4 * (tw + mw);
  if (c->smem_optin && smem + tile_static_smem() + 1024 > c->smem_optin) return SV_EINVAL;  // window + static
  if (k->large_prime_min == 0) k->large_prime_min = 1u << ((k->tile_log2 + 1) / 2);
  if (k->mult_prime_log2 == 0) k->mult_prime_log2 = kMultPrimeLog2;
  if (k->serve_slots == 0) k->serve_slots = 4;
  if (k->serve_slots > 8) return SV_EINVAL;
  if (k->mult_prime_log2 < 10 || k->mult_prime_log2 > 31) return SV_EINVAL;
  return SV_OK;
}

// Largest window span (bits) of any range of a launch.
uint64_t max_span_bits(const sv_ctx *c, const std::vector<RangeSpec> &specs) {
  uint64_t m = 0;
  for (const RangeSpec &s : specs)
    if (s.hi > s.lo) m = std::max<uint64_t>(m, (s.hi - s.lo) / 2 + (1ull << c->cfg.margin_log2) / 2 + 64);
  return m;
}

// span_bits > 0: primes are bucketed only if they hit any window of the launch
// at most ~64 times, so that the bucket fill stays balanced (one thread walks
// one prime's hits); smaller primes are struck per tile instead.  A launch of
// at most kFillReqChunk ranges has those hits cut into segments by the fill,
// so it buckets every prime from kSegmentedLargeMin up (measured best on
// single ranges of 2^34 and 2^36 integers: a sparse prime costs every tile
// some work, a bucketed one only the tiles it strikes).
Geometry make_geometry(const sv_ctx *c, uint64_t span_bits = 0, size_t n_ranges = 0) {
  const sv_config &k = c->cfg;
  Geometry g{};
  g.tw = 1u << (k.tile_log2 - 5);
  g.tw_log2 = ilog2_u32(g.tw);
  g.mw = 1u << (k.margin_log2 - 6);
  g.kwin = k.margin_log2;
  g.rec_t = k.record_k_threshold;
  g.i_med = k.stamp_primes;  // the stamped primes are the table's first entries
  // dense: at least kDenseMinHits strikes in a full window of 32*(tw+mw) bits
  const uint64_t dense_q = 32ull * ((uint64_t)g.tw + g.mw) / (uint64_t)kDenseMinHits;
  uint32_t i = g.i_med;
  while (i < c->n_primes && i < g.i_med + (uint32_t)kMaxDensePrimes && (uint64_t)c->h_p[i] * c->h_p[i] <= dense_q)
    ++i;
  g.i_dense = i;
  // head: at least one strike per thread and window (struck with a stride of
  // one thread block); the rest of the dense primes share a numbering
  const uint64_t head_q = 32ull * ((uint64_t)g.tw + g.mw) / (uint64_t)k.threads;
  uint32_t h = g.i_med;
  while (h < g.i_dense && (uint64_t)c->h_p[h] * c->h_p[h] <= head_q) ++h;
  g.n_head = h - g.i_med;
  uint64_t lp = k.large_prime_min;
  if (span_bits) {
    uint64_t lp_span = host_isqrt(span_bits / 64) + 1;
    if (n_ranges && n_ranges <= kFillReqChunk) lp_span = std::min(lp_span, kSegmentedLargeMin);
    lp = std::max<uint64_t>(lp, lp_span);
  }
  uint32_t il = primes_upto(c, lp - 1);
  if (il < g.i_dense) il = g.i_dense;
  if (il > g.i_dense + (uint32_t)kMaxSparsePrimes) il = g.i_dense + (uint32_t)kMaxSparsePrimes;
  g.i_large = il;
  // primes >= 2^mult_prime_log2 reach the buckets by enumerating their odd
  // multipliers (the multiplier items of bucket_fill_kernel)
  uint32_t ih = primes_upto(c, (1ull << k.mult_prime_log2) - 1);
  if (ih < il) ih = il;
  g.i_hyb = ih;
  g.p_hyb = ih < c->n_primes ? c->h_p[ih] : 0xFFFFFFFFu;
  // expected bucket hits per full window: 32*(tw+mw) * sum_{large p} 1/p^2
  // (only sizes a buffer; overflow is detected and the launch repeated)
  const double s = il < c->inv_sq_suffix.size() ? c->inv_sq_suffix[il] : 0.0;  // sum_{j >= il} 1/p_j^2
  const double lam = 32.0 * (double)(g.tw + g.mw) * s;
  uint32_t cap = (uint32_t)(lam + 8.0 * std::sqrt(lam) + 64.0);
  cap = (cap + 31u) & ~31u;
  g.bucket_auto = cap;
  if (k.bucket_capacity) cap = k.bucket_capacity;  // explicit override (grown on overflow)
  g.bucket_cap = cap;
  g.stage_cap = k.list_stage_capacity ? std::min<uint32_t>(k.list_stage_capacity, kStageCap) : kStageCap;
  return g;
}

// p_hyb^2: multiples j p^2 with p >= p_hyb are enumerated by j (0: none)
uint64_t p_hyb_sq(const Geometry &g) { return g.p_hyb == 0xFFFFFFFFu ? 0 : (uint64_t)g.p_hyb * g.p_hyb; }

PrimeTab prime_tab(const sv_ctx *c) {
  PrimeTab pt{};
  pt.p = c->d_p;
  pt.mu = c->d_mu;
  pt.inv = c->d_inv;
  pt.lim = c->d_lim;
  pt.bits = c->d_pbits;
  pt.bits_words = c->pbits_words;
  pt.n = c->n_primes;
  pt.n_div = c->n_div;
  return pt;
}

sv_status ensure_tile_smem(sv_ctx *c) {
  const size_t smem = 4ull * ((1ull << (c->cfg.tile_log2 - 5)) + (1ull << (c->cfg.margin_log2 - 6)));
  if (smem > c->smem_set.load()) {
    SV_TRY_CUDA(tile_kernel_setup(smem));
    c->smem_set.store(smem);
  }
  return SV_OK;
}

// Plans the descriptors of `specs` into ws.h_reqs / ws.h_hdr.
sv_status plan(sv_ctx *c, const std::vector<RangeSpec> &specs, const Geometry &g, Workspace &ws) {
  const uint32_t n = (uint32_t)specs.size();
  // the previous launch may still be copying from the pinned staging
  if (ws.staged && cudaEventSynchronize(ws.staged) != cudaSuccess) return SV_ECUDA;
  if (ws.h_reqs.ensure(n ? n : 1) != cudaSuccess) return SV_ENOMEM;
  if (ws.h_hdr.ensure(1) != cudaSuccess) return SV_ENOMEM;
  uint64_t tiles = 0, list_total = 0, fail_total = 0;
  uint32_t max_primes = 0;
  uint64_t jhi_max = 0;  // the largest odd multiplier floor((2 jhi - 1) / p_hyb^2) grows with jhi
  uint64_t span_max = 0;  // the longest range, in bits
  uint64_t hi_max = 0;   // and the largest prime count with hi
  const uint64_t ph2 = g.p_hyb == 0xFFFFFFFFu ? 0 : (uint64_t)g.p_hyb * g.p_hyb;
  bool any_per_n = false;
  bool all_from_bitmap = n > 0;
  for (uint32_t r = 0; r < n; ++r) {
    const RangeSpec &s = specs[r];
    ReqDesc d{};
    d.lo = s.lo;
    d.hi = s.hi;
    d.slot = r;
    if (s.sieve_only) {
      d.nlo = s.lo | 1ull;
      d.jlo = s.lo / 2;
    } else {
      d.nlo = (s.lo < 3 ? 3 : s.lo) | 1ull;
      d.jlo = (d.nlo - 1) / 2;
    }
    d.jhi = s.hi / 2;
    if (d.jhi < d.jlo) d.jhi = d.jlo;
    d.w0 = (int64_t)(d.jlo >> 5);
    d.wend = (int64_t)((d.jhi + 31) >> 5);
    const uint64_t nwords = (d.jhi > d.jlo) ? (uint64_t)(d.wend - d.w0) : 0;
    const uint64_t nt = (nwords + g.tw - 1) / g.tw;
    if (tiles + nt > 0xFFFFFFF0ull) return SV_ERANGE;
    d.n_tiles = (uint32_t)nt;
    d.tile_base = (uint32_t)tiles;
    tiles += nt;
    if (nt && s.hi > hi_max) hi_max = s.hi;
    if (n <= kHostPlanMax) {  // few ranges: planned here; many: by the init kernel, in parallel
      d.n_primes = s.hi > 1 ? primes_upto(c, host_isqrt(s.hi - 1)) : 0;
      const int64_t ws = d.w0 - (int64_t)g.mw;
      const uint64_t A = 32ull * (uint64_t)(ws < 0 ? 0 : ws);
      d.sq_lo = (uint32_t)host_isqrt(2 * A);
      d.sq_hi = d.jhi ? (uint32_t)host_isqrt(2 * d.jhi - 1) : 0u;
      d.j_max = (ph2 && d.jhi) ? (2 * d.jhi - 1) / ph2 : 0;
    } else {
      d.n_primes = kPlanOnDevice;
    }
    if (nt && d.jhi > jhi_max) jhi_max = d.jhi;
    if (nt && d.jhi - d.jlo > span_max) span_max = d.jhi - d.jlo;
    d.per_n_k = s.d_per_n;
    any_per_n |= (s.d_per_n != nullptr);
    d.list_off = list_total;
    d.list_cap = s.list_cap;
    list_total += s.list_cap;
    d.fail_off = fail_total;
    d.fail_cap = s.fail_cap;
    fail_total += s.fail_cap;
    d.sieve_only = s.sieve_only ? 1u : 0u;
    d.bitmap_out = s.bitmap_out;
    d.bitmap_in = s.bitmap_in;
    d.bitmap_w0 = s.bitmap_w0;
    all_from_bitmap &= (s.bitmap_in != nullptr);
    ws.h_reqs.p[r] = d;
  }
  if (hi_max > 1) max_primes = primes_upto(c, host_isqrt(hi_max - 1));
  LaunchHeader h{};
  h.j_max = (ph2 && jhi_max) ? (2 * jhi_max - 1) / ph2 : 0;
  h.fill_span = span_max;
  if (all_from_bitmap && ws.inject_bulk_timeouts) {  // the test hook of sv_inject_bulk_timeout
    --ws.inject_bulk_timeouts;
    h.skip_bulk_loads = 1;
    h.bulk_wait_cycles = 1u << 20;  // about half a millisecond
  }
  h.n_reqs = n;
  h.total_tiles = (uint32_t)tiles;
  h.max_primes = max_primes;
  *ws.h_hdr.p = h;
  ws.n_reqs = n;
  ws.total_tiles = (uint32_t)tiles;
  ws.max_primes = max_primes;
  ws.list_total = list_total;
  ws.fail_total = fail_total;
  ws.j_max = (ph2 && jhi_max) ? (2 * jhi_max - 1) / ph2 : 0;
  ws.any_per_n = any_per_n;
  ws.all_from_bitmap = all_from_bitmap;
  ws.ordered = !any_per_n && g.rec_t > 5 && !ws.force_general;
  return SV_OK;
}

// Tile kernel mode of the planned launch: 0 lean with ordered lists, 1
// general, 2 general with the per-n output.
int launch_mode(const Workspace &ws) { return ws.any_per_n ? 2 : (ws.ordered ? 0 : 1); }

// Ordered lists: one staging slot of kStageCap entries per tile.
bool ensure_stage(Workspace &ws) {
  const size_t t = ws.total_tiles ? ws.total_tiles : 1;
  return !(ws.stage_n.ensure(t * kStageCap) || ws.stage_k.ensure(t * kStageCap) || ws.stage_cnt.ensure(t));
}

// Blocks of the bucket fill: one full wave.
uint32_t fill_blocks(const sv_ctx *c) { return (uint32_t)c->num_sms * kFillBlocksPerSm; }

// Kernel ids of the per-kernel timing.
enum { kKInit = 0, kKBucket = 1, kKTiles = 2, kKStrag = 3, kKPoints = 4, kKCompact = 5, kKSievePass = 6,
       kKScanPass = 7 };

cudaEvent_t pool_event(sv_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with events when timing is enabled.
struct KTimer {
  sv_ctx *c;
  int id;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  KTimer(sv_ctx *c_, int id_, cudaStream_t st_) : c(c_), id(id_), st(st_) {
    if (((c->kprof >> id) & 1u) && st == c->stream) {  // the serving thread's streams are never timed
      a = pool_event(c);
      cudaEventRecord(a, st);
    }
  }
  void done() {
    if (a) {
      cudaEvent_t b = pool_event(c);
      cudaEventRecord(b, st);
      c->kev.push_back({id, a, b});
    }
  }
};

// Enqueues init -> bucket fill -> tiles -> stragglers for the planned launch.
sv_status enqueue(sv_ctx *c, const Geometry &g, Workspace &ws, cudaStream_t st) {
  const uint32_t n = ws.n_reqs;
  if (ws.reqs.ensure(n ? n : 1) || ws.hdr.ensure(1) || ws.slots.ensure(n ? n : 1) ||
      ws.h_slots.ensure(n ? n : 1) || ws.list_n.ensure(ws.list_total ? ws.list_total : 1) ||
      ws.list_k.ensure(ws.list_total ? ws.list_total : 1) || ws.fail_n.ensure(ws.fail_total ? ws.fail_total : 1) ||
      ws.strag.ensure(ws.strag_cap) || ws.bucket_count.ensure(ws.total_tiles ? ws.total_tiles : 1) ||
      ws.bucket_data.ensure((size_t)(ws.total_tiles ? ws.total_tiles : 1) * g.bucket_cap))
    return SV_ENOMEM;
  const int mode = launch_mode(ws);
  if (mode == 0 && !ensure_stage(ws)) return SV_ENOMEM;
  ws.bucket_cap = g.bucket_cap;
  SV_TRY_CUDA(cudaMemcpyAsync(ws.reqs.p, ws.h_reqs.p, sizeof(ReqDesc) * n, cudaMemcpyHostToDevice, st));
  SV_TRY_CUDA(cudaMemcpyAsync(ws.hdr.p, ws.h_hdr.p, sizeof(LaunchHeader), cudaMemcpyHostToDevice, st));
  ws.h2d_bytes = sizeof(ReqDesc) * n + sizeof(LaunchHeader);
  if (!ws.staged && cudaEventCreateWithFlags(&ws.staged, cudaEventDisableTiming) != cudaSuccess) return SV_ECUDA;
  SV_TRY_CUDA(cudaEventRecord(ws.staged, st));
  {
    KTimer kt(c, kKInit, st);
    SV_TRY_CUDA(launch_init(ws.hdr.p, ws.slots.p, n, ws.bucket_count.p, mode == 0 ? ws.stage_cnt.p : nullptr,
                            ws.total_tiles, ws.reqs.p, g.mw, c->d_p, c->n_primes, p_hyb_sq(g), st));
    kt.done();
  }
  c->launches++;
  const PrimeTab pt = prime_tab(c);
  if (ws.max_primes > g.i_large && ws.total_tiles && !ws.all_from_bitmap) {
    BucketArgs b{};
    b.pt = pt;
    b.g = g;
    b.reqs = ws.reqs.p;
    b.hdr = ws.hdr.p;
    b.bucket_count = ws.bucket_count.p;
    b.bucket_data = ws.bucket_data.p;
    KTimer kt(c, kKBucket, st);
    SV_TRY_CUDA(launch_bucket_fill(b, ws.max_primes - g.i_large, n, ws.j_max, fill_blocks(c), st));
    kt.done();
    c->launches++;
  }
  if (ws.total_tiles) {
    TileArgs t{};
    t.pt = pt;
    t.g = g;
    t.reqs = ws.reqs.p;
    t.hdr = ws.hdr.p;
    t.slots = ws.slots.p;
    t.list_n = ws.list_n.p;
    t.list_k = ws.list_k.p;
    t.fail_n = ws.fail_n.p;
    t.strag = ws.strag.p;
    t.strag_cap = ws.strag_cap;
    t.bucket_count = ws.bucket_count.p;
    t.bucket_data = ws.bucket_data.p;
    if (mode == 0) {
      t.stage_n = ws.stage_n.p;
      t.stage_k = ws.stage_k.p;
      t.stage_cnt = ws.stage_cnt.p;
    }
    const size_t smem = 4ull * (g.tw + g.mw);
    uint32_t grid = (uint32_t)c->num_sms * c->cfg.ctas_per_sm;
    if (grid > ws.total_tiles) grid = ws.total_tiles;
    {
      KTimer kt(c, ws.tile_kernel_id, st);
      SV_TRY_CUDA(launch_tiles(t, c->cfg.threads, grid, smem, mode, st));
      kt.done();
    }
    c->launches++;
    StragArgs s{};
    s.pt = pt;
    s.reqs = ws.reqs.p;
    s.hdr = ws.hdr.p;
    s.slots = ws.slots.p;
    s.list_n = ws.list_n.p;
    s.list_k = ws.list_k.p;
    s.fail_n = ws.fail_n.p;
    s.strag = ws.strag.p;
    s.strag_cap = ws.strag_cap;
    s.rec_t = g.rec_t;
    if (mode == 0) {
      s.stage_n = ws.stage_n.p;
      s.stage_k = ws.stage_k.p;
      s.stage_cnt = ws.stage_cnt.p;
      s.stage_cap = g.stage_cap;
      s.tw_log2 = g.tw_log2;
    }
    {
      KTimer kt(c, kKStrag, st);
      SV_TRY_CUDA(launch_stragglers(s, (uint32_t)c->num_sms * 2, st));
      kt.done();
    }
    c->launches++;
    if (mode == 0) {
      CompactArgs ca{};
      ca.reqs = ws.reqs.p;
      ca.hdr = ws.hdr.p;
      ca.slots = ws.slots.p;
      ca.list_n = ws.list_n.p;
      ca.list_k = ws.list_k.p;
      ca.stage_n = ws.stage_n.p;
      ca.stage_k = ws.stage_k.p;
      ca.stage_cnt = ws.stage_cnt.p;
      ca.stage_cap = g.stage_cap;
      KTimer kt(c, kKCompact, st);
      SV_TRY_CUDA(launch_compact(ca, std::min<uint32_t>((ws.total_tiles + 127) / 128, 4u * (uint32_t)c->num_sms), st));
      kt.done();
      c->launches++;
    }
  }
  return SV_OK;
}

// The same launch as a CUDA graph.  The grids are fixed and persistent (every
// kernel reads the launch's sizes from the device header), so one captured
// graph is replayed for every launch that fits the current buffers, geometry
// and kernel mode; it is re-captured when any of them changes.
sv_status enqueue_graph(sv_ctx *c, const Geometry &g, Workspace &ws, cudaStream_t st) {
  const uint32_t n = ws.n_reqs;
  if (ws.reqs.ensure(n ? n : 1) || ws.hdr.ensure(1) || ws.slots.ensure(n ? n : 1) ||
      ws.h_slots.ensure(n ? n : 1) || ws.list_n.ensure(ws.list_total ? ws.list_total : 1) ||
      ws.list_k.ensure(ws.list_total ? ws.list_total : 1) || ws.fail_n.ensure(ws.fail_total ? ws.fail_total : 1) ||
      ws.strag.ensure(ws.strag_cap) || ws.bucket_count.ensure(ws.total_tiles ? ws.total_tiles : 1) ||
      ws.bucket_data.ensure((size_t)(ws.total_tiles ? ws.total_tiles : 1) * g.bucket_cap))
    return SV_ENOMEM;
  const int mode = launch_mode(ws);
  if (mode == 0 && !ensure_stage(ws)) return SV_ENOMEM;
  ws.bucket_cap = g.bucket_cap;
  const size_t req_copy = std::min(ws.h_reqs.cap, ws.reqs.cap);
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  const void *ptrs[] = {ws.reqs.p,    ws.hdr.p,   ws.slots.p,        ws.list_n.p,       ws.list_k.p,
                        ws.fail_n.p,  ws.strag.p, ws.bucket_count.p, ws.bucket_data.p, ws.h_reqs.p,
                        ws.h_hdr.p,   c->d_p,     (const void *)st,  ws.stage_n.p,      ws.stage_k.p,
                        ws.stage_cnt.p};
  std::memcpy(key.p, ptrs, sizeof(ptrs));
  key.g = g;
  key.threads = c->cfg.threads;
  key.ctas = c->cfg.ctas_per_sm;
  key.mode = (uint32_t)mode;
  key.strag_cap = ws.strag_cap;
  key.req_copy = req_copy;
  key.n_table = c->n_primes;
  // per-kernel timing of the tile kernel: event-record nodes around it
  const bool timed = ((c->kprof >> ws.tile_kernel_id) & 1u) && st == c->stream;
  key.timed = timed ? 1u : 0u;
  if (!ws.gexec || std::memcmp(&key, &ws.gkey, sizeof(key)) != 0) {
    if (ws.gexec) cudaGraphExecDestroy(ws.gexec);
    ws.gexec = nullptr;
    if (ws.graph) cudaGraphDestroy(ws.graph);
    ws.graph = nullptr;
    ws.gnode[0] = ws.gnode[1] = nullptr;
    if (timed)
      for (cudaEvent_t &ev : ws.gev)
        if (!ev && cudaEventCreate(&ev) != cudaSuccess) return SV_ECUDA;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SV_ECUDA;
    const PrimeTab pt = prime_tab(c);
    cudaError_t e = cudaMemcpyAsync(ws.reqs.p, ws.h_reqs.p, sizeof(ReqDesc) * req_copy, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(ws.hdr.p, ws.h_hdr.p, sizeof(LaunchHeader), cudaMemcpyHostToDevice, st);
    // sized for the buffers (the kernel reads the launch's sizes from the header)
    if (!e) e = launch_init(ws.hdr.p, ws.slots.p, (uint32_t)std::min<size_t>(ws.slots.cap, 1u << 20), ws.bucket_count.p,
                            mode == 0 ? ws.stage_cnt.p : nullptr, (uint32_t)std::min<size_t>(ws.bucket_count.cap, 1u << 30),
                            ws.reqs.p, g.mw, c->d_p, c->n_primes, p_hyb_sq(g), st);
    if (!e && pt.n > g.i_large) {
      BucketArgs b{};
      b.pt = pt;
      b.g = g;
      b.reqs = ws.reqs.p;
      b.hdr = ws.hdr.p;
      b.bucket_count = ws.bucket_count.p;
      b.bucket_data = ws.bucket_data.p;
      e = launch_bucket_fill(b, pt.n - g.i_large, 1u << 20, 1ull << 23, fill_blocks(c), st);
    }
    if (!e) {
      TileArgs t{};
      t.pt = pt;
      t.g = g;
      t.reqs = ws.reqs.p;
      t.hdr = ws.hdr.p;
      t.slots = ws.slots.p;
      t.list_n = ws.list_n.p;
      t.list_k = ws.list_k.p;
      t.fail_n = ws.fail_n.p;
      t.strag = ws.strag.p;
      t.strag_cap = ws.strag_cap;
      t.bucket_count = ws.bucket_count.p;
      t.bucket_data = ws.bucket_data.p;
      if (mode == 0) {
        t.stage_n = ws.stage_n.p;
        t.stage_k = ws.stage_k.p;
        t.stage_cnt = ws.stage_cnt.p;
      }
      if (timed) e = cudaEventRecordWithFlags(ws.gev[0], st, cudaEventRecordExternal);
      if (!e) e = launch_tiles(t, c->cfg.threads, (uint32_t)c->num_sms * c->cfg.ctas_per_sm, 4ull * (g.tw + g.mw), mode, st);
      if (!e && timed) e = cudaEventRecordWithFlags(ws.gev[1], st, cudaEventRecordExternal);
    }
    if (!e) {
      StragArgs sa{};
      sa.pt = pt;
      sa.reqs = ws.reqs.p;
      sa.hdr = ws.hdr.p;
      sa.slots = ws.slots.p;
      sa.list_n = ws.list_n.p;
      sa.list_k = ws.list_k.p;
      sa.fail_n = ws.fail_n.p;
      sa.strag = ws.strag.p;
      sa.strag_cap = ws.strag_cap;
      sa.rec_t = g.rec_t;
      if (mode == 0) {
        sa.stage_n = ws.stage_n.p;
        sa.stage_k = ws.stage_k.p;
        sa.stage_cnt = ws.stage_cnt.p;
        sa.stage_cap = g.stage_cap;
        sa.tw_log2 = g.tw_log2;
      }
      e = launch_stragglers(sa, (uint32_t)c->num_sms * 2, st);
    }
    if (!e && mode == 0) {
      CompactArgs ca{};
      ca.reqs = ws.reqs.p;
      ca.hdr = ws.hdr.p;
      ca.slots = ws.slots.p;
      ca.list_n = ws.list_n.p;
      ca.list_k = ws.list_k.p;
      ca.stage_n = ws.stage_n.p;
      ca.stage_k = ws.stage_k.p;
      ca.stage_cnt = ws.stage_cnt.p;
      ca.stage_cap = g.stage_cap;
      e = launch_compact(ca, 4u * (uint32_t)c->num_sms, st);  // blocks of 128 tiles, grid-stride
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    if (e || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return SV_ECUDA;
    }
    if (timed) {  // the two event-record nodes, found by their events
      size_t nn = 0;
      std::vector<cudaGraphNode_t> nodes;
      cudaError_t e4 = cudaGraphGetNodes(graph, nullptr, &nn);
      if (!e4) {
        nodes.resize(nn);
        e4 = cudaGraphGetNodes(graph, nodes.data(), &nn);
      }
      for (size_t i = 0; !e4 && i < nn; ++i) {
        cudaGraphNodeType ty;
        if ((e4 = cudaGraphNodeGetType(nodes[i], &ty)) || ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        if ((e4 = cudaGraphEventRecordNodeGetEvent(nodes[i], &ev))) break;
        for (int k = 0; k < 2; ++k)
          if (ev == ws.gev[k]) ws.gnode[k] = nodes[i];
      }
      if (e4 || !ws.gnode[0] || !ws.gnode[1]) {
        cudaGraphDestroy(graph);
        return SV_ECUDA;
      }
    }
    const cudaError_t e3 = cudaGraphInstantiate(&ws.gexec, graph, 0);
    if (e3 != cudaSuccess) {
      cudaGraphDestroy(graph);
      ws.gexec = nullptr;
      return SV_ECUDA;
    }
    ws.graph = graph;  // kept: the exec's event nodes are addressed through it
    ws.gkey = key;
  }
  if (timed) {  // fresh events for this replay's tile kernel
    cudaEvent_t a = pool_event(c), b = pool_event(c);
    SV_TRY_CUDA(cudaGraphExecEventRecordNodeSetEvent(ws.gexec, ws.gnode[0], a));
    SV_TRY_CUDA(cudaGraphExecEventRecordNodeSetEvent(ws.gexec, ws.gnode[1], b));
    c->kev.push_back({ws.tile_kernel_id, a, b});
  }
  SV_TRY_CUDA(cudaGraphLaunch(ws.gexec, st));
  // the graph reads the staging when it runs: the next plan waits for it
  if (!ws.staged && cudaEventCreateWithFlags(&ws.staged, cudaEventDisableTiming) != cudaSuccess) return SV_ECUDA;
  SV_TRY_CUDA(cudaEventRecord(ws.staged, st));
  c->launches += mode == 0 ? 5 : 4;
  ws.h2d_bytes = sizeof(ReqDesc) * req_copy + sizeof(LaunchHeader);
  return SV_OK;
}

// (n, k) pairs of one range, ascending in n, into out.  The listed n are
// spread over [lo, hi), so a bucket pass on the position in the range (about
// one bucket per entry) followed by insertion sorts is linear in practice.
void sort_by_n(const uint64_t *ns, const uint8_t *ks, uint64_t cnt, uint64_t lo, uint64_t hi,
               std::vector<std::pair<uint64_t, uint8_t>> &out) {
  out.resize(cnt);
  if (cnt < 64 || hi <= lo) {
    for (uint64_t i = 0; i < cnt; ++i) out[i] = {ns[i], ks[i]};
    std::sort(out.begin(), out.end());
    return;
  }
  int lb = 0;
  while ((1ull << lb) < cnt) ++lb;
  const uint64_t span = hi - lo;
  const int sb = 64 - __builtin_clzll(span);
  const int shift = sb > lb ? sb - lb : 0;
  const uint64_t nb = ((span - 1) >> shift) + 1;
  std::vector<uint32_t> start(nb + 1, 0);
  for (uint64_t i = 0; i < cnt; ++i) ++start[((ns[i] - lo) >> shift) + 1];
  for (uint64_t b = 0; b < nb; ++b) start[b + 1] += start[b];
  std::vector<uint32_t> fill(start.begin(), start.end() - 1);
  for (uint64_t i = 0; i < cnt; ++i) out[fill[(ns[i] - lo) >> shift]++] = {ns[i], ks[i]};
  for (uint64_t b = 0; b < nb; ++b)
    for (uint32_t i = start[b] + 1; i < start[b + 1]; ++i)
      for (uint32_t x = i; x > start[b] && out[x - 1].first > out[x].first; --x) std::swap(out[x - 1], out[x]);
}

enum Collect { kDone, kRetryBucket, kRetryStrag, kRetryList, kRetryGeneral };
constexpr uint64_t kSpeculativeList = 1ull << 18;  // list entries copied without waiting for the count

// How many list entries the consumer of range r can take: its result buffer,
// the device region, or (a serving chunk) its request's buffer.
uint64_t list_want(const RangeSpec &sp, const sv_range_result *o) {
  return std::max(std::max(sp.list_cap, sp.want_cap), o ? o->list_cap : 0);
}
constexpr uint64_t kListRetryMax = 1ull << 26;  // larger lists are returned truncated, unordered

// Waits for the launch, checks the device status word and copies results out.
// Host memory the device can copy into directly (allocated or registered as
// page-locked); null counts as pinned (nothing to copy).
bool is_pinned(const void *p) {
  if (!p) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unregistered pointer is not an error to keep
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

sv_status collect(sv_ctx *c, const std::vector<RangeSpec> &specs, sv_range_result **outs, Workspace &ws,
                  cudaStream_t st, Collect *what) {
  const uint32_t n = ws.n_reqs;
  *what = kDone;
  SV_TRY_CUDA(cudaMemcpyAsync(ws.h_hdr.p, ws.hdr.p, sizeof(LaunchHeader), cudaMemcpyDeviceToHost, st));
  SV_TRY_CUDA(cudaMemcpyAsync(ws.h_slots.p, ws.slots.p, sizeof(ResultSlot) * n, cudaMemcpyDeviceToHost, st));
  // an ordered list region is copied with the header (one wait instead of
  // two) when it is small enough to copy whole
  uint64_t spec_end = 0;
  if (ws.ordered && outs) {
    for (uint32_t r = 0; r < n; ++r)
      if (outs[r] && (outs[r]->list || outs[r]->list_k))
        spec_end = std::max<uint64_t>(spec_end, ws.h_reqs.p[r].list_off + ws.h_reqs.p[r].list_cap);
    if (spec_end > kSpeculativeList) spec_end = 0;
  }
  // one range whose caller buffers are pinned host memory: its list region
  // goes straight into them (no staging copy, no host copy afterwards); the
  // entries past the list's length are left unspecified
  bool direct = false;
  uint64_t direct_m = 0;
  if (spec_end && n == 1 && outs[0] && is_pinned(outs[0]->list) && is_pinned(outs[0]->list_k)) {
    direct = true;
    direct_m = std::min<uint64_t>(ws.h_reqs.p[0].list_cap, outs[0]->list_cap);
    const uint64_t off = ws.h_reqs.p[0].list_off;
    if (direct_m && outs[0]->list)
      SV_TRY_CUDA(cudaMemcpyAsync(outs[0]->list, ws.list_n.p + off, 8 * direct_m, cudaMemcpyDeviceToHost, st));
    if (direct_m && outs[0]->list_k)
      SV_TRY_CUDA(cudaMemcpyAsync(outs[0]->list_k, ws.list_k.p + off, direct_m, cudaMemcpyDeviceToHost, st));
  } else if (spec_end) {
    if (ws.h_list_n.ensure(spec_end) || ws.h_list_k.ensure(spec_end)) return SV_ENOMEM;
    SV_TRY_CUDA(cudaMemcpyAsync(ws.h_list_n.p, ws.list_n.p, 8 * spec_end, cudaMemcpyDeviceToHost, st));
    SV_TRY_CUDA(cudaMemcpyAsync(ws.h_list_k.p, ws.list_k.p, spec_end, cudaMemcpyDeviceToHost, st));
  }
  SV_TRY_CUDA(cudaStreamSynchronize(st));
  uint64_t d2h = sizeof(LaunchHeader) + sizeof(ResultSlot) * n + (direct ? 9 * direct_m : 9 * spec_end);
  const uint32_t status = ws.h_hdr.p->status;
  if (status & kStBadTile) return SV_ECUDA;
  if (status & kStTimeout) return SV_ETIMEDOUT;
  if (status & kStBucketOverflow) {
    *what = kRetryBucket;
    return SV_OK;
  }
  if (status & kStStragOverflow) {
    *what = kRetryStrag;
    return SV_OK;
  }
  if (status & kStListStage) {
    *what = kRetryGeneral;
    return SV_OK;
  }
  // an unordered list that the device truncated is re-run with exact room,
  // so that the caller receives the smallest entries, deterministically; an
  // ordered list already holds the smallest ones and is re-run only when
  // the consumer can hold more than the device region did
  for (uint32_t r = 0; r < n; ++r) {
    const ResultSlot &s = ws.h_slots.p[r];
    if (!outs || !outs[r]) continue;
    const uint64_t limit = ws.ordered ? std::min<uint64_t>(list_want(specs[r], outs[r]), kListRetryMax) : kListRetryMax;
    if (outs[r]->list_cap && s.list_count > specs[r].list_cap && specs[r].list_cap < limit) {
      *what = kRetryList;
      return SV_OK;
    }
  }
  // one copy of the used parts of the list and failure arenas for all ranges
  uint64_t list_end = 0, fail_end = 0;
  for (uint32_t r = 0; r < n; ++r) {
    if (!outs || !outs[r]) continue;
    const ReqDesc &d = ws.h_reqs.p[r];
    const ResultSlot &s = ws.h_slots.p[r];
    const uint64_t nl = std::min<uint64_t>(s.list_count, d.list_cap);
    const uint64_t nf = std::min<uint64_t>(s.fail_count, d.fail_cap);
    if (nl && (outs[r]->list || outs[r]->list_k)) list_end = std::max<uint64_t>(list_end, d.list_off + nl);
    if (nf && outs[r]->failures) fail_end = std::max<uint64_t>(fail_end, d.fail_off + nf);
  }
  if (list_end <= spec_end) list_end = 0;  // already here
  if (list_end || fail_end) {
    if ((list_end && (ws.h_list_n.ensure(list_end) || ws.h_list_k.ensure(list_end))) ||
        ws.h_fail_n.ensure(fail_end ? fail_end : 1))
      return SV_ENOMEM;
    if (list_end) {
      SV_TRY_CUDA(cudaMemcpyAsync(ws.h_list_n.p, ws.list_n.p, 8 * list_end, cudaMemcpyDeviceToHost, st));
      SV_TRY_CUDA(cudaMemcpyAsync(ws.h_list_k.p, ws.list_k.p, list_end, cudaMemcpyDeviceToHost, st));
    }
    if (fail_end) SV_TRY_CUDA(cudaMemcpyAsync(ws.h_fail_n.p, ws.fail_n.p, 8 * fail_end, cudaMemcpyDeviceToHost, st));
    SV_TRY_CUDA(cudaStreamSynchronize(st));
    d2h += 9 * list_end + 8 * fail_end;
  }
  std::vector<std::pair<uint64_t, uint8_t>> v;
  for (uint32_t r = 0; r < n; ++r) {
    if (!outs || !outs[r]) continue;
    sv_range_result *o = outs[r];
    const ResultSlot &s = ws.h_slots.p[r];
    const RangeSpec &sp = specs[r];
    o->lo = sp.lo;
    o->hi = sp.hi;
    o->n_odd = range_odd_count(sp.lo, sp.hi);
    o->ksum = 0;
    o->kmax = 0;
    for (int k = 0; k < kMaxK; ++k) {
      o->hist[k] = s.hist[k];
      o->first_n[k] = s.first_n[k];
      if (k > 0) {
        o->ksum += (uint64_t)k * s.hist[k];
        if (s.hist[k]) o->kmax = (uint64_t)k;
      }
    }
    o->list_len = s.list_count;
    o->fail_len = s.fail_count;
    o->list_overflow = s.list_count > o->list_cap ? 1 : 0;
    const ReqDesc &d = ws.h_reqs.p[r];
    const uint64_t nl = std::min<uint64_t>(s.list_count, d.list_cap);
    if (nl && (o->list || o->list_k) && !direct) {
      const uint64_t m = std::min<uint64_t>(nl, o->list_cap);
      if (ws.ordered) {  // ascending already (list_compact_kernel)
        if (o->list) std::memcpy(o->list, ws.h_list_n.p + d.list_off, 8 * m);
        if (o->list_k) std::memcpy(o->list_k, ws.h_list_k.p + d.list_off, m);
      } else {
        sort_by_n(ws.h_list_n.p + d.list_off, ws.h_list_k.p + d.list_off, nl, sp.lo, sp.hi, v);
        for (uint64_t i = 0; i < m; ++i) {
          if (o->list) o->list[i] = v[i].first;
          if (o->list_k) o->list_k[i] = v[i].second;
        }
      }
    }
    const uint64_t nf = std::min<uint64_t>(s.fail_count, d.fail_cap);
    if (nf && o->failures) {
      uint64_t *f = ws.h_fail_n.p + d.fail_off;
      std::sort(f, f + nf);
      const uint64_t m = std::min<uint64_t>(nf, o->fail_cap);
      std::memcpy(o->failures, f, 8 * m);
    }
  }
  ws.d2h_bytes = d2h;
  return SV_OK;
}

sv_status check_ready(sv_ctx *c) {
  if (!c) return SV_EINVAL;
  if (!c->d_p) return SV_ENOPRIMES;
  return SV_OK;
}

sv_status check_range(const sv_ctx *c, uint64_t lo, uint64_t hi) {
  (void)lo;
  if (hi > kMaxHi) return SV_ERANGE;
  if (hi > c->max_hi) return SV_ERANGE;
  return SV_OK;
}

}  // namespace

namespace sv {

// 1 - c_l from Table 2 (Sec. 2): the heuristic probability that mink > l.
// Only sizes buffers; results never depend on it.
constexpr double kTail[8] = {1.0, 1.8943e-1, 2.4129e-2, 2.1482e-3, 1.3902e-4, 6.8527e-6, 2.6694e-7, 4.9973e-8};

uint64_t list_cap_estimate(uint64_t n_odd, uint32_t T, uint64_t cap) {
  if (cap == 0) return 0;
  const double p = T < 8 ? kTail[T ? T - 1 : 0] : kTail[7];
  const uint64_t est = (uint64_t)(2.0 * p * (double)n_odd) + 256;
  return std::min<uint64_t>(est, cap);
}

// Accessors for the no-allocation entry point (noalloc.cu); none allocates.
Geometry geometry_for_span(const sv_ctx *c, uint64_t span_bits) { return make_geometry(c, span_bits, 1); }
PrimeTab prime_table_of(const sv_ctx *c) { return prime_tab(c); }
uint32_t primes_upto_of(const sv_ctx *c, uint64_t x) { return primes_upto(c, x); }
sv_status tile_smem_ready(sv_ctx *c) { return ensure_tile_smem(c); }

// Runs a launch of ranges to completion, growing buffers and repeating the
// launch when the device reports an overflow.  Results never depend on the
// buffer sizes.
sv_status run_ranges(sv_ctx *c, std::vector<RangeSpec> &specs, sv_range_result **outs, cudaStream_t st,
                     Workspace &ws, bool graph) {
  sv_status s = ensure_tile_smem(c);
  if (s) return s;
  Geometry g = make_geometry(c, max_span_bits(c, specs), specs.size());
  if (ws.bucket_cap > g.bucket_cap) g.bucket_cap = ws.bucket_cap;
  for (int attempt = 0; attempt < 8; ++attempt) {
    if ((s = plan(c, specs, g, ws))) return s;
    if ((s = graph ? enqueue_graph(c, g, ws, st) : enqueue(c, g, ws, st))) return s;
    Collect what;
    if ((s = collect(c, specs, outs, ws, st, &what))) return s;
    if (what == kDone) {
      c->last_h2d = ws.h2d_bytes;
      c->last_d2h = ws.d2h_bytes;
      ws.force_general = false;
      return SV_OK;
    }
    if (what == kRetryGeneral) ws.force_general = true;
    if (what == kRetryBucket) {
      g.bucket_cap = std::max<uint32_t>(g.bucket_cap * 4, g.bucket_auto);
      ws.bucket_cap = g.bucket_cap;
    }
    if (what == kRetryStrag) ws.strag_cap *= 4;
    if (what == kRetryList) {
      for (uint32_t r = 0; r < specs.size(); ++r) {
        const uint64_t cnt = ws.h_slots.p[r].list_count;
        if (outs && outs[r] && cnt > specs[r].list_cap) {
          uint64_t cap = std::min<uint64_t>(cnt, kListRetryMax);
          if (ws.ordered) cap = std::min<uint64_t>(cap, list_want(specs[r], outs[r]));
          specs[r].list_cap = cap;
        }
      }
    }
  }
  return SV_EOVERFLOW;
}

// ---- the plain (unfused) path -------------------------------------------------
// Algorithm 1 writes the squarefree flags of the odd integers to a bitmap in
// device memory (the sieve pass: sieve_only tiles, one bulk store per tile),
// and Algorithm 2 reads them back (the scan pass: every tile's window comes
// from the bitmap by one bulk load).  The bitmap starts at the first window's
// start, max(w0 - mw, 0) words, so every window of the scan lies inside it.

// The two passes' ranges for [lo, hi); an empty range has no sieve pass.
sv_status plain_specs(sv_ctx *c, uint64_t lo, uint64_t hi, uint8_t *d_per_n, uint64_t list_cap, uint64_t fail_cap,
                      std::vector<RangeSpec> &sieve, std::vector<RangeSpec> &scan) {
  const int64_t mw = (int64_t)1 << (c->cfg.margin_log2 - 6);
  const uint64_t nlo = (lo < 3 ? 3 : lo) | 1ull, jlo = (nlo - 1) / 2;
  const uint64_t jhi = std::max<uint64_t>(hi / 2, jlo);
  scan.assign(1, RangeSpec{});
  scan[0].lo = lo;
  scan[0].hi = hi;
  scan[0].d_per_n = d_per_n;
  scan[0].list_cap = list_cap;
  scan[0].fail_cap = fail_cap;
  sieve.clear();
  if (jhi <= jlo) return SV_OK;
  const int64_t bw0 = std::max<int64_t>((int64_t)(jlo >> 5) - mw, 0);
  const uint64_t words = ((jhi + 31) >> 5) - (uint64_t)bw0;
  if (c->plain_bitmap.ensure(words + 4)) return SV_ENOMEM;  // room for a bulk load rounded up to 16 bytes
  RangeSpec sp;
  sp.lo = 64ull * (uint64_t)bw0;
  sp.hi = hi;
  sp.sieve_only = true;
  sp.bitmap_out = c->plain_bitmap.p;
  sieve.push_back(sp);
  scan[0].bitmap_in = c->plain_bitmap.p;
  scan[0].bitmap_w0 = bw0;
  return SV_OK;
}

// Enqueues the sieve pass (its own workspace) and the scan pass on st.
sv_status plain_enqueue(sv_ctx *c, std::vector<RangeSpec> &sieve, std::vector<RangeSpec> &scan, cudaStream_t st) {
  sv_status s = ensure_tile_smem(c);
  if (s) return s;
  Geometry g = make_geometry(c, max_span_bits(c, sieve.empty() ? scan : sieve), (sieve.empty() ? scan : sieve).size());
  if (c->ws_sieve.bucket_cap > g.bucket_cap) g.bucket_cap = c->ws_sieve.bucket_cap;
  if (!sieve.empty()) {
    c->ws_sieve.force_general = true;  // no lists in the sieve pass: no staging, no compaction
    c->ws_sieve.tile_kernel_id = kKSievePass;
    if ((s = plan(c, sieve, g, c->ws_sieve))) return s;
    if ((s = enqueue(c, g, c->ws_sieve, st))) return s;
  }
  c->ws.tile_kernel_id = sieve.empty() ? kKTiles : kKScanPass;
  if ((s = plan(c, scan, g, c->ws))) return s;
  s = enqueue(c, g, c->ws, st);
  c->ws.tile_kernel_id = kKTiles;
  return s;
}

// Waits for both passes and collects the scan's results into *out.  A retry
// the sieve pass needs is reported through *what with *sieve_retry set.
sv_status plain_collect(sv_ctx *c, const std::vector<RangeSpec> &sieve, const std::vector<RangeSpec> &scan,
                        sv_range_result *out, cudaStream_t st, Collect *what, bool *sieve_retry) {
  *sieve_retry = false;
  if (!sieve.empty()) {
    Collect w1;
    sv_status s = collect(c, sieve, nullptr, c->ws_sieve, st, &w1);
    if (s) return s;
    if (w1 != kDone) {
      *what = w1;
      *sieve_retry = true;
      return SV_OK;
    }
  }
  sv_range_result *outs[1] = {out};
  return collect(c, scan, outs, c->ws, st, what);
}

// Adjusts the buffers after an overflow either pass reported.
void plain_retry(sv_ctx *c, Collect what, bool sieve_retry, std::vector<RangeSpec> &sieve, std::vector<RangeSpec> &scan,
                 const sv_range_result *out) {
  if (sieve_retry) {
    if (what == kRetryBucket)
      c->ws_sieve.bucket_cap =
          std::max<uint32_t>(c->ws_sieve.bucket_cap, make_geometry(c, max_span_bits(c, sieve), sieve.size()).bucket_auto) * 4;
    return;
  }
  if (what == kRetryStrag) c->ws.strag_cap *= 4;
  if (what == kRetryGeneral) c->ws.force_general = true;
  if (what == kRetryList) {
    uint64_t cap = std::min<uint64_t>(c->ws.h_slots.p[0].list_count, kListRetryMax);
    if (c->ws.ordered) cap = std::min<uint64_t>(cap, list_want(scan[0], out));
    scan[0].list_cap = cap;
  }
}

// The plain path to completion (blocking), with the retry policy of run_ranges.
sv_status run_plain(sv_ctx *c, std::vector<RangeSpec> &sieve, std::vector<RangeSpec> &scan, sv_range_result *out,
                    cudaStream_t st) {
  for (int attempt = 0; attempt < 8; ++attempt) {
    sv_status s = plain_enqueue(c, sieve, scan, st);
    if (s) return s;
    Collect what;
    bool sr;
    if ((s = plain_collect(c, sieve, scan, out, st, &what, &sr))) return s;
    if (what == kDone) {
      c->last_h2d = c->ws.h2d_bytes + (sieve.empty() ? 0 : c->ws_sieve.h2d_bytes);
      c->last_d2h = c->ws.d2h_bytes + (sieve.empty() ? 0 : c->ws_sieve.d2h_bytes);
      c->ws.force_general = false;
      return SV_OK;
    }
    plain_retry(c, what, sr, sieve, scan, out);
  }
  return SV_EOVERFLOW;
}

sv_status launch_ranges_async(sv_ctx *c, std::vector<RangeSpec> &specs, Workspace &ws, cudaStream_t st) {
  sv_status s = ensure_tile_smem(c);
  if (s) return s;
  Geometry g = make_geometry(c, max_span_bits(c, specs), specs.size());
  if (ws.bucket_cap > g.bucket_cap) g.bucket_cap = ws.bucket_cap;
  if ((s = plan(c, specs, g, ws))) return s;
  return enqueue_graph(c, g, ws, st);
}

sv_status collect_ranges(sv_ctx *c, const std::vector<RangeSpec> &specs, sv_range_result **outs, Workspace &ws,
                         cudaStream_t st, bool *retry) {
  Collect what;
  sv_status s = collect(c, specs, outs, ws, st, &what);
  *retry = (what != kDone);
  if (what == kDone) ws.force_general = false;
  if (what == kRetryGeneral) ws.force_general = true;
  if (what == kRetryBucket)
    ws.bucket_cap = std::max<uint32_t>(ws.bucket_cap * 4, make_geometry(c, max_span_bits(c, specs), specs.size()).bucket_auto);
  if (what == kRetryStrag) ws.strag_cap *= 4;
  return s;
}

sv_status launch_points_async(sv_ctx *c, uint64_t count, Workspace &ws, cudaStream_t st) {
  if (count == 0) return SV_OK;
  if (ws.points.ensure(count) || ws.points_out.ensure(count)) return SV_ENOMEM;
  SV_TRY_CUDA(cudaMemcpyAsync(ws.points.p, ws.h_points.p, 8 * count, cudaMemcpyHostToDevice, st));
  uint64_t grid = (count * 32 + 255) / 256;
  const uint64_t gmax = (uint64_t)c->num_sms * 8;
  if (grid > gmax) grid = gmax;
  SV_TRY_CUDA(launch_points(prime_tab(c), ws.points.p, count, ws.points_out.p, (uint32_t)grid, st));
  c->launches++;
  SV_TRY_CUDA(cudaMemcpyAsync(ws.h_points_out.p, ws.points_out.p, count, cudaMemcpyDeviceToHost, st));
  return SV_OK;
}

sv_status run_points(sv_ctx *c, const uint64_t *points, size_t count, uint8_t *out_k, cudaStream_t st,
                     Workspace &ws) {
  if (count == 0) return SV_OK;
  for (size_t i = 0; i < count; ++i)
    if (points[i] > c->max_hi) return SV_ERANGE;
  if (ws.points.ensure(count) || ws.points_out.ensure(count) || ws.h_points.ensure(count) ||
      ws.h_points_out.ensure(count))
    return SV_ENOMEM;
  std::memcpy(ws.h_points.p, points, 8 * count);
  SV_TRY_CUDA(cudaMemcpyAsync(ws.points.p, ws.h_points.p, 8 * count, cudaMemcpyHostToDevice, st));
  uint64_t warps = count;
  uint64_t grid = (warps * 32 + 255) / 256;
  const uint64_t gmax = (uint64_t)c->num_sms * 8;
  if (grid > gmax) grid = gmax;
  {
    KTimer kt(c, kKPoints, st);
    SV_TRY_CUDA(launch_points(prime_tab(c), ws.points.p, count, ws.points_out.p, (uint32_t)grid, st));
    kt.done();
  }
  c->launches++;
  SV_TRY_CUDA(cudaMemcpyAsync(ws.h_points_out.p, ws.points_out.p, count, cudaMemcpyDeviceToHost, st));
  SV_TRY_CUDA(cudaStreamSynchronize(st));
  std::memcpy(out_k, ws.h_points_out.p, count);
  c->last_h2d = 8 * count;
  c->last_d2h = count;
  return SV_OK;
}

}  // namespace sv

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *sv_strerror(sv_status s) {
  switch (s) {
    case SV_OK: return "ok";
    case SV_EINVAL: return "invalid argument";
    case SV_ERANGE: return "out of range (hi beyond 2^62 or beyond the prime table)";
    case SV_ENOMEM: return "out of memory / admission refused";
    case SV_EAGAIN: return "not finished yet";
    case SV_ETIMEDOUT: return "timed out";
    case SV_ECANCELLED: return "cancelled";
    case SV_ECUDA: return "CUDA error";
    case SV_ENOPRIMES: return "prime table not initialised (sv_init_primes)";
    case SV_ENOTFOUND: return "unknown ticket";
    case SV_EOVERFLOW: return "device buffer overflow persisted after retries";
  }
  return "unknown status";
}

sv_status sv_create(sv_ctx **out, const sv_config *cfg) {
  if (!out) return SV_EINVAL;
  *out = nullptr;
  sv_ctx *c = new (std::nothrow) sv_ctx();
  if (!c) return SV_ENOMEM;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return SV_ECUDA;
  }
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess) {
    delete c;
    return SV_ECUDA;
  }
  c->smem_optin = (size_t)optin;
  if (cfg) c->cfg = *cfg;
  sv_status s = normalise_config(c, &c->cfg);
  if (s) {
    delete c;
    return s;
  }
  if (c->cfg.cuda_stream) {
    c->stream = (cudaStream_t)c->cfg.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return SV_ECUDA;
    }
    c->own_stream = true;
    c->cfg.cuda_stream = c->stream;
  }
  *out = c;
  return SV_OK;
}

void sv_destroy(sv_ctx *c) {
  if (!c) return;
  DevGuard dev_guard__(c->device);
  if (c->server) server_destroy(c->server);
  c->server = nullptr;
  cudaStreamSynchronize(c->stream);
  c->ws.release_all();
  c->ws_sieve.release_all();
  c->plain_bitmap.release();
  cudaFree(c->d_p);
  cudaFree(c->d_mu);
  cudaFree(c->d_inv);
  cudaFree(c->d_lim);
  cudaFree(c->d_pbits);
  for (auto &k : c->kev) {
    cudaEventDestroy(k.a);
    cudaEventDestroy(k.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

sv_status sv_get_config(const sv_ctx *c, sv_config *out) {
  if (!c || !out) return SV_EINVAL;
  *out = c->cfg;
  return SV_OK;
}

sv_status sv_init_primes(sv_ctx *c, uint64_t max_hi) {
  if (!c) return SV_EINVAL;
  if (max_hi > kMaxHi) return SV_ERANGE;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->d_p && max_hi <= c->max_hi) return SV_OK;
  const uint64_t pmax = host_isqrt(max_hi > 1 ? max_hi - 1 : 1);
  uint32_t *d_p = nullptr, *d_bits = nullptr;
  uint64_t *d_mu = nullptr, *d_inv = nullptr, *d_lim = nullptr;
  uint64_t bits_words = 0;
  uint32_t n = 0, n_div = 0;
  cudaError_t e = build_prime_table(pmax, &d_p, &d_mu, &d_inv, &d_lim, &d_bits, &bits_words, &n, &n_div, c->stream);
  if (e == cudaErrorMemoryAllocation) return SV_ENOMEM;
  if (e != cudaSuccess) return SV_ECUDA;
  std::vector<uint32_t> hp(n);
  if (n && cudaMemcpy(hp.data(), d_p, 4ull * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaFree(d_p);
    cudaFree(d_mu);
    cudaFree(d_inv);
    cudaFree(d_lim);
    cudaFree(d_bits);
    return SV_ECUDA;
  }
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_p);
  cudaFree(c->d_mu);
  cudaFree(c->d_inv);
  cudaFree(c->d_lim);
  cudaFree(c->d_pbits);
  c->d_p = d_p;
  c->d_mu = d_mu;
  c->d_inv = d_inv;
  c->d_lim = d_lim;
  c->d_pbits = d_bits;
  c->pbits_words = bits_words;
  c->n_primes = n;
  c->n_div = n_div;
  c->h_p.swap(hp);
  // h_pi[b]: the number of table primes below b * 2^kPiBlockLog2
  c->h_pi.assign((pmax >> kPiBlockLog2) + 2, 0u);
  for (size_t b = 0, j = 0; b < c->h_pi.size(); ++b) {
    while (j < c->h_p.size() && ((uint64_t)c->h_p[j] >> kPiBlockLog2) < b) ++j;
    c->h_pi[b] = (uint32_t)j;
  }
  // suffix sums of 1/p^2 (sizing of the tile buckets, host only)
  c->inv_sq_suffix.assign(c->h_p.size() + 1, 0.0);
  for (size_t j = c->h_p.size(); j-- > 0;)
    c->inv_sq_suffix[j] = c->inv_sq_suffix[j + 1] + 1.0 / ((double)c->h_p[j] * (double)c->h_p[j]);
  c->pmax = pmax;
  c->max_hi = max_hi;
  c->launches += 5;
  return SV_OK;
}

sv_status sv_prime_count(const sv_ctx *c, uint64_t *count, uint64_t *largest) {
  if (!c) return SV_EINVAL;
  if (count) *count = c->n_primes;
  if (largest) *largest = c->n_primes ? c->h_p.back() : 0;
  return SV_OK;
}

sv_status sv_prime_table_copy(sv_ctx *c, uint32_t *p, uint64_t *mu, uint64_t *inv, uint64_t *lim, uint64_t cap,
                              uint64_t *n_div) {
  sv_status s = check_ready(c);
  if (s) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  const uint64_t n = std::min<uint64_t>(cap, c->n_primes), nd = std::min<uint64_t>(cap, c->n_div);
  if (n_div) *n_div = c->n_div;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SV_ECUDA;
  if (p && n && cudaMemcpy(p, c->d_p, 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess) return SV_ECUDA;
  if (mu && n && cudaMemcpy(mu, c->d_mu, 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess) return SV_ECUDA;
  if (inv && nd && cudaMemcpy(inv, c->d_inv, 8 * nd, cudaMemcpyDeviceToHost) != cudaSuccess) return SV_ECUDA;
  if (lim && nd && cudaMemcpy(lim, c->d_lim, 8 * nd, cudaMemcpyDeviceToHost) != cudaSuccess) return SV_ECUDA;
  return SV_OK;
}

uint64_t sv_bitmap_words(uint64_t lo, uint64_t hi) {
  const uint64_t jlo = lo / 2, jhi = hi / 2;
  if (jhi <= jlo) return 0;
  return ((jhi + 31) >> 5) - (jlo >> 5);
}

sv_status sv_verify_range(sv_ctx *c, uint64_t lo, uint64_t hi, sv_range_result *out) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (!out) return SV_EINVAL;
  if ((s = check_range(c, lo, hi))) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<RangeSpec> specs(1);
  specs[0].lo = lo;
  specs[0].hi = hi;
  specs[0].list_cap = out->list_cap;
  specs[0].fail_cap = std::max<uint64_t>(out->fail_cap, 64);
  const uint64_t n_odd = range_odd_count(lo, hi);
  if (out->per_n_k && n_odd) {
    if (c->ws.per_n.ensure(n_odd)) return SV_ENOMEM;
    specs[0].d_per_n = c->ws.per_n.p;
  }
  sv_range_result *outs[1] = {out};
  // the launch as the captured graph (replayed while the sizes fit)
  s = run_ranges(c, specs, outs, c->stream, c->ws, true);
  if (s) return s;
  if (out->per_n_k && n_odd) {
    if (cudaMemcpyAsync(out->per_n_k, c->ws.per_n.p, n_odd, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return SV_ECUDA;
    c->last_d2h += n_odd;
  }
  return SV_OK;
}

sv_status sv_verify_batch(sv_ctx *c, const uint64_t *lo, const uint64_t *hi, size_t count, sv_range_result *out) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (count && (!lo || !hi || !out)) return SV_EINVAL;
  for (size_t i = 0; i < count; ++i)
    if ((s = check_range(c, lo[i], hi[i]))) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<RangeSpec> specs(count);
  std::vector<sv_range_result *> outs(count);
  for (size_t i = 0; i < count; ++i) {
    specs[i].lo = lo[i];
    specs[i].hi = hi[i];
    specs[i].list_cap = out[i].list_cap;
    specs[i].fail_cap = std::max<uint64_t>(out[i].fail_cap, 16);
    outs[i] = &out[i];
  }
  if (count == 0) return SV_OK;
  return run_ranges(c, specs, outs.data(), c->stream, c->ws, true);
}

sv_status sv_launch_batch(sv_ctx *c, const uint64_t *lo, const uint64_t *hi, size_t count) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (count == 0 || !lo || !hi) return SV_EINVAL;
  for (size_t i = 0; i < count; ++i)
    if ((s = check_range(c, lo[i], hi[i]))) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  if ((s = ensure_tile_smem(c))) return s;
  std::vector<RangeSpec> specs(count);
  for (size_t i = 0; i < count; ++i) {
    specs[i].lo = lo[i];
    specs[i].hi = hi[i];
    specs[i].list_cap = list_cap_estimate(range_odd_count(lo[i], hi[i]), c->cfg.record_k_threshold,
                                          c->cfg.list_capacity);
    specs[i].fail_cap = 16;
  }
  Geometry g = make_geometry(c, max_span_bits(c, specs), specs.size());
  if (c->ws.bucket_cap > g.bucket_cap) g.bucket_cap = c->ws.bucket_cap;
  if ((s = plan(c, specs, g, c->ws))) return s;
  if ((s = enqueue_graph(c, g, c->ws, c->stream))) return s;
  c->pending = true;
  c->pending_graph = true;
  c->pending_plain = false;
  c->pending_specs.swap(specs);
  return SV_OK;
}

sv_status sv_fetch_batch(sv_ctx *c, sv_range_result *out, size_t count) {
  if (!c || (count && !out)) return SV_EINVAL;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->pending || c->pending_plain || count != c->pending_specs.size()) return SV_EINVAL;
  c->pending = false;
  std::vector<sv_range_result *> outs(count);
  for (size_t i = 0; i < count; ++i) outs[i] = &out[i];
  Collect what;
  sv_status s = collect(c, c->pending_specs, outs.data(), c->ws, c->stream, &what);
  if (s) return s;
  if (what != kDone) {
    std::vector<RangeSpec> specs = c->pending_specs;
    if (what == kRetryBucket) c->ws.bucket_cap = make_geometry(c, max_span_bits(c, specs), specs.size()).bucket_cap * 4;
    if (what == kRetryStrag) c->ws.strag_cap *= 4;
    if (what == kRetryGeneral) c->ws.force_general = true;
    s = run_ranges(c, specs, outs.data(), c->stream, c->ws, true);
  }
  return s;
}

sv_status sv_min_k(sv_ctx *c, const uint64_t *points, size_t count, uint8_t *out_k) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (count && (!points || !out_k)) return SV_EINVAL;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  return run_points(c, points, count, out_k, c->stream, c->ws);
}

sv_status sv_min_k_device(sv_ctx *c, const uint64_t *d_points, size_t count, uint8_t *d_out_k) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (count && (!d_points || !d_out_k)) return SV_EINVAL;
  if (count == 0) return SV_OK;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  uint64_t grid = ((uint64_t)count * 32 + 255) / 256;
  const uint64_t gmax = (uint64_t)c->num_sms * 8;
  if (grid > gmax) grid = gmax;
  if (launch_points(prime_tab(c), d_points, count, d_out_k, (uint32_t)grid, c->stream) != cudaSuccess)
    return SV_ECUDA;
  c->launches++;
  return SV_OK;
}

sv_status sv_sieve_bitmap(sv_ctx *c, uint64_t lo, uint64_t hi, uint32_t *d_bitmap) {
  sv_status s = check_ready(c);
  if (s) return s;
  if ((s = check_range(c, lo, hi))) return s;
  if (sv_bitmap_words(lo, hi) == 0) return SV_OK;
  if (!d_bitmap) return SV_EINVAL;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<RangeSpec> specs(1);
  specs[0].lo = lo;
  specs[0].hi = hi;
  specs[0].sieve_only = true;
  specs[0].bitmap_out = d_bitmap;
  return run_ranges(c, specs, nullptr, c->stream, c->ws, false);
}

sv_status sv_launch_range(sv_ctx *c, uint64_t lo, uint64_t hi, uint8_t *d_per_n_k) {
  sv_status s = check_ready(c);
  if (s) return s;
  if ((s = check_range(c, lo, hi))) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  if ((s = ensure_tile_smem(c))) return s;
  std::vector<RangeSpec> specs(1);
  specs[0].lo = lo;
  specs[0].hi = hi;
  specs[0].d_per_n = d_per_n_k;
  specs[0].list_cap = c->cfg.list_capacity;
  specs[0].fail_cap = 1024;
  Geometry g = make_geometry(c, max_span_bits(c, specs), specs.size());
  if (c->ws.bucket_cap > g.bucket_cap) g.bucket_cap = c->ws.bucket_cap;
  if ((s = plan(c, specs, g, c->ws))) return s;
  // the captured graph (fewer launch gaps), unless a kernel other than the
  // tile kernel is being timed: a graph brackets only the tile kernel
  const bool graph = (c->kprof & ~(1u << c->ws.tile_kernel_id)) == 0;
  if ((s = graph ? enqueue_graph(c, g, c->ws, c->stream) : enqueue(c, g, c->ws, c->stream))) return s;
  c->pending = true;
  c->pending_plain = false;
  c->pending_specs = specs;
  return SV_OK;
}

sv_status sv_fetch_range(sv_ctx *c, sv_range_result *out) {
  if (!c || !out) return SV_EINVAL;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->pending || c->pending_specs.size() != 1) return SV_EINVAL;
  c->pending = false;
  if (c->pending_plain) {
    c->pending_plain = false;
    Collect what;
    bool sr;
    sv_status s = plain_collect(c, c->pending_sieve_specs, c->pending_specs, out, c->stream, &what, &sr);
    if (s) return s;
    if (what != kDone) {  // an overflow: repeat both passes with grown buffers, blocking
      plain_retry(c, what, sr, c->pending_sieve_specs, c->pending_specs, out);
      return run_plain(c, c->pending_sieve_specs, c->pending_specs, out, c->stream);
    }
    c->ws.force_general = false;
    c->last_h2d = c->ws.h2d_bytes + c->ws_sieve.h2d_bytes;
    c->last_d2h = c->ws.d2h_bytes + c->ws_sieve.d2h_bytes;
    return SV_OK;
  }
  sv_range_result *outs[1] = {out};
  Collect what;
  sv_status s = collect(c, c->pending_specs, outs, c->ws, c->stream, &what);
  if (s) return s;
  if (what != kDone) {
    // an overflow: repeat the range with grown buffers, blocking
    std::vector<RangeSpec> specs = c->pending_specs;
    if (what == kRetryBucket) c->ws.bucket_cap = make_geometry(c, max_span_bits(c, specs), specs.size()).bucket_cap * 4;
    if (what == kRetryStrag) c->ws.strag_cap *= 4;
    if (what == kRetryGeneral) c->ws.force_general = true;
    s = run_ranges(c, specs, outs, c->stream, c->ws, false);
    if (s) return s;
  }
  c->last_h2d = c->ws.h2d_bytes;
  c->last_d2h = c->ws.d2h_bytes;
  return SV_OK;
}

sv_status sv_verify_range_plain(sv_ctx *c, uint64_t lo, uint64_t hi, sv_range_result *out) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (!out) return SV_EINVAL;
  if ((s = check_range(c, lo, hi))) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  const uint64_t n_odd = range_odd_count(lo, hi);
  uint8_t *d_per_n = nullptr;
  if (out->per_n_k && n_odd) {
    if (c->ws.per_n.ensure(n_odd)) return SV_ENOMEM;
    d_per_n = c->ws.per_n.p;
  }
  std::vector<RangeSpec> sieve, scan;
  if ((s = plain_specs(c, lo, hi, d_per_n, out->list_cap, std::max<uint64_t>(out->fail_cap, 64), sieve, scan)))
    return s;
  if ((s = run_plain(c, sieve, scan, out, c->stream))) return s;
  if (d_per_n) {
    if (cudaMemcpyAsync(out->per_n_k, d_per_n, n_odd, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return SV_ECUDA;
    c->last_d2h += n_odd;
  }
  return SV_OK;
}

sv_status sv_launch_range_plain(sv_ctx *c, uint64_t lo, uint64_t hi, uint8_t *d_per_n_k) {
  sv_status s = check_ready(c);
  if (s) return s;
  if ((s = check_range(c, lo, hi))) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<RangeSpec> sieve, scan;
  if ((s = plain_specs(c, lo, hi, d_per_n_k, c->cfg.list_capacity, 1024, sieve, scan))) return s;
  if ((s = plain_enqueue(c, sieve, scan, c->stream))) return s;
  c->pending = true;
  c->pending_plain = true;
  c->pending_specs.swap(scan);
  c->pending_sieve_specs.swap(sieve);
  return SV_OK;
}

sv_status sv_synchronize(sv_ctx *c) {
  if (!c) return SV_EINVAL;
  SV_ON_DEVICE(c);
  return cuda_status(cudaStreamSynchronize(c->stream));
}

// Bytes the last blocking call moved host->device and device->host, and the
// number of kernels the library has launched so far.
sv_status sv_last_transfer(const sv_ctx *c, uint64_t *h2d, uint64_t *d2h) {
  if (!c) return SV_EINVAL;
  if (h2d) *h2d = c->last_h2d;
  if (d2h) *d2h = c->last_d2h;
  return SV_OK;
}

uint64_t sv_kernel_launches(const sv_ctx *c) { return c ? c->launches.load() : 0; }

sv_status sv_inject_bulk_timeout(sv_ctx *c, uint32_t count) {
  if (!c) return SV_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->ws.inject_bulk_timeouts = count;
  return SV_OK;
}

sv_status sv_inject_alloc_failures(sv_ctx *c, uint32_t count) {
  if (!c) return SV_EINVAL;
  g_inject_alloc_failures.store(count);
  return SV_OK;
}

sv_status sv_kernel_timing(sv_ctx *c, int enable) {
  if (!c) return SV_EINVAL;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SV_ECUDA;
  for (auto &k : c->kev) {
    c->ev_pool.push_back(k.a);
    c->ev_pool.push_back(k.b);
  }
  c->kev.clear();
  for (int i = 0; i < 8; ++i) {
    c->k_ms[i] = 0.0;
    c->k_n[i] = 0;
  }
  c->kprof = enable == -1 ? 0xFFFFFFFFu : (uint32_t)enable;
  return SV_OK;
}

sv_status sv_kernel_time(sv_ctx *c, int kernel, double *total_ms, uint64_t *launches) {
  if (!c || kernel < 0 || kernel >= 8) return SV_EINVAL;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SV_ECUDA;
  for (auto &k : c->kev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, k.a, k.b) != cudaSuccess) return SV_ECUDA;
    c->k_ms[k.id] += ms;
    c->k_n[k.id] += 1;
    c->ev_pool.push_back(k.a);
    c->ev_pool.push_back(k.b);
  }
  c->kev.clear();
  if (total_ms) *total_ms = c->k_ms[kernel];
  if (launches) *launches = c->k_n[kernel];
  return SV_OK;
}

sv_status sv_set_config(sv_ctx *c, const sv_config *cfg) {
  if (!c || !cfg) return SV_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  sv_config k = *cfg;
  k.cuda_stream = c->cfg.cuda_stream;
  sv_status s = normalise_config(c, &k);
  if (s) return s;
  c->cfg = k;
  c->ws.bucket_cap = 0;
  return SV_OK;
}

}  // extern "C"

namespace sv {

// ---- autotuner ---------------------------------------------------------------

// Device time of one launch of `specs` under the context's current
// configuration: a warm-up launch (it sizes the buffers and captures the
// graph), then the best of three, each bracketed by CUDA events on the
// context's stream around the descriptor upload and the kernels.
sv_status time_launch(sv_ctx *c, const std::vector<RangeSpec> &specs0, double *best_ms) {
  std::vector<RangeSpec> specs = specs0;
  sv_status s = run_ranges(c, specs, nullptr, c->stream, c->ws, true);
  if (s) return s;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return SV_ECUDA;
  }
  double best = 1e300;
  for (int rep = 0; rep < 3 && !s; ++rep) {
    Geometry g = make_geometry(c, max_span_bits(c, specs), specs.size());
    if (c->ws.bucket_cap > g.bucket_cap) g.bucket_cap = c->ws.bucket_cap;
    if ((s = plan(c, specs, g, c->ws))) break;
    if (cudaEventRecord(a, c->stream) != cudaSuccess) s = SV_ECUDA;
    if (!s) s = enqueue_graph(c, g, c->ws, c->stream);
    if (!s && cudaEventRecord(b, c->stream) != cudaSuccess) s = SV_ECUDA;
    Collect what = kDone;
    if (!s) s = collect(c, specs, nullptr, c->ws, c->stream, &what);
    if (s) break;
    if (what != kDone) {  // the warm-up grew everything: this launch reported an overflow anyway
      s = run_ranges(c, specs, nullptr, c->stream, c->ws, true);
      continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) s = SV_ECUDA;
    else if (ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *best_ms = best;
  return s;
}

// Coordinate descent over the knobs, two rounds; the context keeps the best.
sv_status tune(sv_ctx *c, const std::vector<RangeSpec> &specs, sv_config *chosen) {
  const sv_config base = c->cfg;
  sv_config best = base;
  double best_t = 1e300;
  // times candidate k (skipped when invalid or when its CTAs cannot be resident)
  auto eval = [&](sv_config k, double *t) -> sv_status {
    *t = 1e300;
    if (normalise_config(c, &k)) return SV_OK;
    const size_t smem = 4ull * ((1ull << (k.tile_log2 - 5)) + (1ull << (k.margin_log2 - 6)));
    if (k.ctas_per_sm * (smem + tile_static_smem() + 1024) > c->smem_optin + 1024 ||
        (size_t)k.ctas_per_sm * k.threads > 2048)
      return SV_OK;
    c->cfg = k;
    c->ws.bucket_cap = 0;
    c->ws_sieve.bucket_cap = 0;
    sv_status s = time_launch(c, specs, t);
    if (s == SV_ENOMEM || s == SV_EOVERFLOW) {  // this candidate does not fit: skip it
      *t = 1e300;
      return SV_OK;
    }
    return s;
  };
  auto consider = [&](const sv_config &k) -> sv_status {
    double t;
    sv_status s = eval(k, &t);
    if (!s && t < best_t) {
      best_t = t;
      best = c->cfg;
    }
    return s;
  };
  sv_status s = consider(base);
  struct Shape {
    uint32_t tile_log2, threads, ctas;
  };
  const Shape shapes[] = {{19, 512, 2}, {18, 512, 2}, {18, 256, 3}, {20, 1024, 1}, {19, 1024, 1}, {17, 256, 4}};
  const uint32_t stamps[] = {2, 4, 6, 8};
  const uint32_t margins[] = {12, 13, 14, 16};
  const uint32_t lpmins[] = {512, 1024, 2048, 4096, 8192, 16384};
  const uint32_t mults[] = {15, 16, 17, 18, 19, 20, 21};
  for (int round = 0; round < 2 && !s; ++round) {
    for (const Shape &sh : shapes) {
      if (s) break;
      sv_config k = best;
      k.tile_log2 = sh.tile_log2;
      k.threads = sh.threads;
      k.ctas_per_sm = sh.ctas;
      if (k.margin_log2 > k.tile_log2 + 1) k.margin_log2 = k.tile_log2 + 1;
      s = consider(k);
    }
    for (uint32_t v : stamps) {
      if (s) break;
      sv_config k = best;
      k.stamp_primes = v;
      s = consider(k);
    }
    for (uint32_t v : margins) {
      if (s) break;
      sv_config k = best;
      k.margin_log2 = v;
      s = consider(k);
    }
    for (uint32_t v : lpmins) {
      if (s) break;
      sv_config k = best;
      k.large_prime_min = v;
      s = consider(k);
    }
    for (uint32_t v : mults) {
      if (s) break;
      sv_config k = best;
      k.mult_prime_log2 = v;
      s = consider(k);
    }
    {  // bucket depth: the automatic estimate, or twice it
      c->cfg = best;
      const uint32_t cap_auto = make_geometry(c, max_span_bits(c, specs), specs.size()).bucket_auto;
      for (uint32_t v : {0u, 2u * cap_auto}) {
        if (s) break;
        sv_config k = best;
        k.bucket_capacity = v;
        s = consider(k);
      }
    }
  }
  c->cfg = s ? base : best;
  c->ws.bucket_cap = 0;
  c->ws_sieve.bucket_cap = 0;
  if (!s && chosen) *chosen = best;
  return s;
}

}  // namespace sv

extern "C" {

sv_status sv_autotune(sv_ctx *c, uint64_t lo, uint64_t hi, sv_config *chosen) {
  sv_status s = check_ready(c);
  if (s) return s;
  if ((s = check_range(c, lo, hi))) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<RangeSpec> specs(1);
  specs[0].lo = lo;
  specs[0].hi = hi;
  specs[0].list_cap = list_cap_estimate(range_odd_count(lo, hi), c->cfg.record_k_threshold, c->cfg.list_capacity);
  specs[0].fail_cap = 16;
  return tune(c, specs, chosen);
}

sv_status sv_autotune_batch(sv_ctx *c, const uint64_t *lo, const uint64_t *hi, size_t count, sv_config *chosen) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (count == 0 || !lo || !hi) return SV_EINVAL;
  for (size_t i = 0; i < count; ++i)
    if ((s = check_range(c, lo[i], hi[i]))) return s;
  SV_ON_DEVICE(c);
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<RangeSpec> specs(count);
  for (size_t i = 0; i < count; ++i) {
    specs[i].lo = lo[i];
    specs[i].hi = hi[i];
    specs[i].list_cap = list_cap_estimate(range_odd_count(lo[i], hi[i]), c->cfg.record_k_threshold,
                                          c->cfg.list_capacity);
    specs[i].fail_cap = 16;
  }
  return tune(c, specs, chosen);
}

sv_status sv_submit(sv_ctx *c, const sv_request *req, uint64_t *ticket) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (!req || !ticket) return SV_EINVAL;
  SV_ON_DEVICE(c);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->server) c->server = server_create(c);
    if (!c->server) return SV_ENOMEM;
  }
  return server_submit(c->server, req, ticket);
}

sv_status sv_submit_many(sv_ctx *c, const sv_request *reqs, size_t count, uint64_t *tickets, sv_status *status) {
  sv_status s = check_ready(c);
  if (s) return s;
  if (count && (!reqs || !tickets || !status)) return SV_EINVAL;
  if (count == 0) return SV_OK;
  SV_ON_DEVICE(c);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->server) c->server = server_create(c);
    if (!c->server) return SV_ENOMEM;
  }
  return server_submit_many(c->server, reqs, count, tickets, status);
}

sv_status sv_poll(sv_ctx *c, uint64_t ticket, int64_t timeout_us) {
  if (!c) return SV_EINVAL;
  if (!c->server) return SV_ENOTFOUND;
  return server_poll(c->server, ticket, timeout_us);
}

sv_status sv_cancel(sv_ctx *c, uint64_t ticket) {
  if (!c) return SV_EINVAL;
  if (!c->server) return SV_ENOTFOUND;
  return server_cancel(c->server, ticket);
}

sv_status sv_server_stats_reset(sv_ctx *c) {
  if (!c) return SV_EINVAL;
  if (c->server) server_reset_stats(c->server);
  return SV_OK;
}

sv_status sv_server_stats_get(sv_ctx *c, sv_server_stats *out) {
  if (!c || !out) return SV_EINVAL;
  if (!c->server) {
    std::memset(out, 0, sizeof(*out));
    return SV_OK;
  }
  return server_stats(c->server, out);
}

}  // extern "C"
