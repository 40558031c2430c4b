// noalloc.cu -- sv_verify_range_noalloc: sv_verify_range without any allocation.
//
// Some callers cannot allocate memory at the point where they verify a range:
// a process that shares the GPU with a caching allocator (PyTorch's, for one)
// that has already reserved nearly all device memory, so that a cudaMalloc by
// this library would fail; latency-critical loops, because cudaMalloc and
// cudaFree can synchronise the whole device and take milliseconds; and
// services whose memory budget is fixed when they start.  This entry point
// runs the same kernels as sv_verify_range, but every piece of scratch memory
// they need (launch header, range descriptor, result slot, tile buckets,
// straggler queue, list and failure arenas) is carved out of one file-scope
// __device__ array of kScratchBytes.  It calls no cudaMalloc, cudaFree,
// cudaMallocHost or other allocating routine; results are copied into the
// caller's own buffers through small stack arrays.  The call blocks: it
// waits for the context's stream before it returns.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ctx.h"

namespace sv {
namespace {

constexpr size_t kScratchBytes = 8u << 20;  // 8 MiB, held by every GPU that loads the library
constexpr uint32_t kNaStragMin = 4096;      // straggler queue entries at least (the rest of the array)
constexpr uint32_t kNaList = 65536;         // listed n (mink >= T) per call
constexpr uint32_t kNaFail = 1024;          // failures kept per call
constexpr int kMaxDevices = 64;
constexpr uint32_t kChunk = 1024;           // entries copied back per round trip
constexpr uint64_t kMaxSpan = 1ull << 32;   // longest range (hi - lo) accepted

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
unsigned char *g_scratch_addr[kMaxDevices];  // device address of the array, per device

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t hdr, req, slot, list_n, list_k, fail, bcount, bdata, strag, end;
  uint32_t strag_cap;  // the straggler queue takes what the other parts leave
};

Layout make_layout(uint32_t n_tiles, uint32_t cap) {
  Layout L;
  size_t o = 0;
  L.hdr = o;
  o = up256(o + sizeof(LaunchHeader));
  L.req = o;
  o = up256(o + sizeof(ReqDesc));
  L.slot = o;
  o = up256(o + sizeof(ResultSlot));
  L.list_n = o;
  o = up256(o + sizeof(uint64_t) * kNaList);
  L.list_k = o;
  o = up256(o + kNaList);
  L.fail = o;
  o = up256(o + sizeof(uint64_t) * kNaFail);
  L.bcount = o;
  o = up256(o + sizeof(uint32_t) * (size_t)(n_tiles ? n_tiles : 1));
  L.bdata = o;
  o = up256(o + sizeof(uint32_t) * (size_t)(n_tiles ? n_tiles : 1) * cap);
  L.strag = o;
  const size_t room = o < kScratchBytes ? (kScratchBytes - o) / sizeof(Straggler) : 0;
  L.strag_cap = (uint32_t)(room < 0xFFFFFFFFull ? room : 0xFFFFFFFFull);
  o = up256(o + sizeof(Straggler) * (size_t)kNaStragMin);
  L.end = o;  // the layout fits when end <= kScratchBytes
  return L;
}

// The array's device address on device dev, which the caller has made
// current: cudaGetSymbolAddress resolves the symbol on the current device.
// Looked up once per device, then reused.
sv_status scratch_base(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return SV_EINVAL;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != dev) return SV_ECUDA;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SV_ECUDA;
    g_scratch_addr[dev] = (unsigned char *)p;
  }
  *out = g_scratch_addr[dev];
  return SV_OK;
}

// Max-heap on n over the caller's parallel arrays (k may be null).
void heap_sift(uint64_t *n, uint8_t *k, uint64_t size, uint64_t i) {
  for (;;) {
    uint64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < size && n[l] > n[m]) m = l;
    if (r < size && n[r] > n[m]) m = r;
    if (m == i) return;
    const uint64_t tn = n[i];
    n[i] = n[m];
    n[m] = tn;
    if (k) {
      const uint8_t tk = k[i];
      k[i] = k[m];
      k[m] = tk;
    }
    i = m;
  }
}

void heap_push(uint64_t *n, uint8_t *k, uint64_t &size, uint64_t v, uint8_t kv) {
  uint64_t i = size++;
  n[i] = v;
  if (k) k[i] = kv;
  while (i > 0) {
    const uint64_t p = (i - 1) / 2;
    if (n[p] >= n[i]) break;
    const uint64_t tn = n[p];
    n[p] = n[i];
    n[i] = tn;
    if (k) {
      const uint8_t tk = k[p];
      k[p] = k[i];
      k[i] = tk;
    }
    i = p;
  }
}

// Keeps the `cap` smallest of `count` device entries (n, and k when d_k is
// given) in the caller's arrays, ascending; copies back kChunk at a time
// through stack buffers.
sv_status smallest_into(const uint64_t *d_n, const uint8_t *d_k, uint64_t count, uint64_t *out_n, uint8_t *out_k,
                        uint64_t cap, cudaStream_t st) {
  if (!out_n || cap == 0) return SV_OK;
  uint64_t buf_n[kChunk];
  uint8_t buf_k[kChunk];
  uint64_t size = 0;
  for (uint64_t base = 0; base < count; base += kChunk) {
    const uint64_t m = (count - base < kChunk) ? count - base : kChunk;
    if (cudaMemcpyAsync(buf_n, d_n + base, 8 * m, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SV_ECUDA;
    if (d_k && cudaMemcpyAsync(buf_k, d_k + base, m, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SV_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SV_ECUDA;
    for (uint64_t i = 0; i < m; ++i) {
      const uint8_t kv = d_k ? buf_k[i] : 0;
      if (size < cap) {
        heap_push(out_n, out_k, size, buf_n[i], kv);
      } else if (buf_n[i] < out_n[0]) {
        out_n[0] = buf_n[i];
        if (out_k) out_k[0] = kv;
        heap_sift(out_n, out_k, size, 0);
      }
    }
  }
  for (uint64_t end = size; end > 1; --end) {  // heap sort: ascending
    const uint64_t tn = out_n[0];
    out_n[0] = out_n[end - 1];
    out_n[end - 1] = tn;
    if (out_k) {
      const uint8_t tk = out_k[0];
      out_k[0] = out_k[end - 1];
      out_k[end - 1] = tk;
    }
    heap_sift(out_n, out_k, end - 1, 0);
  }
  return SV_OK;
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_verify_range_noalloc(sv_ctx *c, uint64_t lo, uint64_t hi, sv_range_result *out) {
  if (!c || !out) return SV_EINVAL;
  if (!c->d_p) return SV_ENOPRIMES;
  if (out->per_n_k) return SV_EINVAL;  // a per-n output needs n_odd bytes: use sv_launch_range
  if (hi > (1ull << 62) || hi > c->max_hi) return SV_ERANGE;
  if (hi > lo && hi - lo > kMaxSpan) return SV_ERANGE;  // longer ranges need more scratch than the array has
  // the context's device is current for the whole call (and the caller's
  // own device afterwards), so the array's address is the one on that device
  DevGuard dev_guard(c->device);
  if (!dev_guard.ok) return SV_ECUDA;
  std::lock_guard<std::mutex> lk(c->mu);
  unsigned char *base = nullptr;
  sv_status s = scratch_base(c->device, &base);
  if (s) return s;
  if ((s = tile_smem_ready(c))) return s;
  const cudaStream_t st = c->stream;

  // the one range's descriptor (as the regular planner builds it)
  const uint64_t span = (hi > lo ? (hi - lo) / 2 : 0) + (1ull << c->cfg.margin_log2) / 2 + 64;
  Geometry g = geometry_for_span(c, span);
  ReqDesc d;
  std::memset(&d, 0, sizeof(d));
  d.lo = lo;
  d.hi = hi;
  d.nlo = (lo < 3 ? 3 : lo) | 1ull;
  d.jlo = (d.nlo - 1) / 2;
  d.jhi = hi / 2;
  if (d.jhi < d.jlo) d.jhi = d.jlo;
  d.w0 = (int64_t)(d.jlo >> 5);
  d.wend = (int64_t)((d.jhi + 31) >> 5);
  const uint64_t nwords = (d.jhi > d.jlo) ? (uint64_t)(d.wend - d.w0) : 0;
  const uint64_t nt = (nwords + g.tw - 1) / g.tw;
  d.n_primes = hi > 1 ? primes_upto_of(c, host_isqrt(hi - 1)) : 0;  // planned here, as for a single range
  {
    const int64_t ws = d.w0 - (int64_t)g.mw;
    const uint64_t A = 32ull * (uint64_t)(ws < 0 ? 0 : ws);
    d.sq_lo = (uint32_t)host_isqrt(2 * A);
    d.sq_hi = d.jhi ? (uint32_t)host_isqrt(2 * d.jhi - 1) : 0u;
    const uint64_t ph2 = g.p_hyb == 0xFFFFFFFFu ? 0 : (uint64_t)g.p_hyb * g.p_hyb;
    d.j_max = (ph2 && d.jhi) ? (2 * d.jhi - 1) / ph2 : 0;
  }
  d.list_cap = kNaList;
  d.fail_cap = kNaFail;

  out->lo = lo;
  out->hi = hi;
  out->n_odd = range_odd_count(lo, hi);
  out->ksum = out->kmax = 0;
  out->list_len = out->fail_len = out->list_overflow = 0;
  for (int k = 0; k < kMaxK; ++k) {
    out->hist[k] = 0;
    out->first_n[k] = kNoN;
  }
  if (nt == 0) return SV_OK;
  if (nt > 0xFFFFFFull) return SV_ERANGE;
  d.n_tiles = (uint32_t)nt;

  const PrimeTab pt = prime_table_of(c);
  LaunchHeader h2;
  ResultSlot rs;
  for (int attempt = 0;; ++attempt) {
    const Layout L = make_layout(d.n_tiles, g.bucket_cap);
    if (L.end > kScratchBytes) return attempt ? SV_EOVERFLOW : SV_ERANGE;  // range too long for the array
    LaunchHeader h;
    std::memset(&h, 0, sizeof(h));
    h.n_reqs = 1;
    h.total_tiles = d.n_tiles;
    h.max_primes = d.n_primes;
    h.j_max = d.j_max;
    h.fill_span = d.jhi - d.jlo;
    LaunchHeader *d_hdr = (LaunchHeader *)(base + L.hdr);
    ReqDesc *d_req = (ReqDesc *)(base + L.req);
    ResultSlot *d_slot = (ResultSlot *)(base + L.slot);
    uint32_t *d_bcount = (uint32_t *)(base + L.bcount);
    uint32_t *d_bdata = (uint32_t *)(base + L.bdata);
    if (cudaMemcpyAsync(d_req, &d, sizeof(d), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_hdr, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return SV_ECUDA;
    // the array keeps the previous call's contents: the counters, the result
    // slot and the bucket counts are cleared on the device first
    if (launch_init(d_hdr, d_slot, 1, d_bcount, nullptr, d.n_tiles, d_req, g.mw, c->d_p, c->n_primes, 0, st) != cudaSuccess)
      return SV_ECUDA;
    c->launches++;
    if (d.n_primes > g.i_large) {
      BucketArgs b{};
      b.pt = pt;
      b.g = g;
      b.reqs = d_req;
      b.hdr = d_hdr;
      b.bucket_count = d_bcount;
      b.bucket_data = d_bdata;
      const uint64_t ph2 = g.p_hyb == 0xFFFFFFFFu ? 0 : (uint64_t)g.p_hyb * g.p_hyb;
      const uint64_t jmax = ph2 ? (2 * d.jhi - 1) / ph2 : 0;
      if (launch_bucket_fill(b, d.n_primes - g.i_large, 1, jmax, (uint32_t)c->num_sms * kFillBlocksPerSm, st) != cudaSuccess)
        return SV_ECUDA;
      c->launches++;
    }
    TileArgs t{};
    t.pt = pt;
    t.g = g;
    t.reqs = d_req;
    t.hdr = d_hdr;
    t.slots = d_slot;
    t.list_n = (uint64_t *)(base + L.list_n);
    t.list_k = (uint8_t *)(base + L.list_k);
    t.fail_n = (uint64_t *)(base + L.fail);
    t.strag = (Straggler *)(base + L.strag);
    t.strag_cap = L.strag_cap;
    t.bucket_count = d_bcount;
    t.bucket_data = d_bdata;
    uint32_t grid = (uint32_t)c->num_sms * c->cfg.ctas_per_sm;
    if (grid > d.n_tiles) grid = d.n_tiles;
    // the general scan mode: its list needs no per-tile staging, which the
    // array has no room for; smallest_into picks the smallest entries
    const int mode = 1;
    if (launch_tiles(t, c->cfg.threads, grid, 4ull * (g.tw + g.mw), mode, st) != cudaSuccess) return SV_ECUDA;
    c->launches++;
    StragArgs sa{};
    sa.pt = pt;
    sa.reqs = d_req;
    sa.hdr = d_hdr;
    sa.slots = d_slot;
    sa.list_n = t.list_n;
    sa.list_k = t.list_k;
    sa.fail_n = t.fail_n;
    sa.strag = t.strag;
    sa.strag_cap = L.strag_cap;
    sa.rec_t = g.rec_t;
    if (launch_stragglers(sa, (uint32_t)c->num_sms * 2, st) != cudaSuccess) return SV_ECUDA;
    c->launches++;
    if (cudaMemcpyAsync(&h2, d_hdr, sizeof(h2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&rs, d_slot, sizeof(rs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SV_ECUDA;
    if (h2.status & kStBadTile) return SV_ECUDA;
    if (h2.status & kStStragOverflow) return SV_EOVERFLOW;
    if (h2.status & kStBucketOverflow) {
      if (attempt >= 4) return SV_EOVERFLOW;
      g.bucket_cap *= 2;  // rerun with deeper buckets if the array still holds them
      continue;
    }
    if (rs.list_count > kNaList) return SV_EOVERFLOW;  // more listed n than the array keeps
    for (int k = 0; k < kMaxK; ++k) {
      out->hist[k] = rs.hist[k];
      out->first_n[k] = rs.first_n[k];
      if (k > 0) {
        out->ksum += (uint64_t)k * rs.hist[k];
        if (rs.hist[k]) out->kmax = (uint64_t)k;
      }
    }
    out->list_len = rs.list_count;
    out->list_overflow = rs.list_count > out->list_cap ? 1 : 0;
    out->fail_len = rs.fail_count;
    if ((s = smallest_into(t.list_n, t.list_k, rs.list_count, out->list, out->list_k, out->list_cap, st))) return s;
    const uint64_t nf = rs.fail_count < kNaFail ? rs.fail_count : kNaFail;
    return smallest_into(t.fail_n, nullptr, nf, out->failures, nullptr, out->fail_cap, st);
  }
}
