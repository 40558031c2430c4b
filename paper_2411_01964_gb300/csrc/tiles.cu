// tiles.cu -- the range path: Algorithm 1 (sieve) and Algorithm 2 (search
// for the smallest k) of Sec. 3, fused per shared-memory tile.
//
// Persistent CTAs (two per SM by default) take chunks of consecutive tiles
// from a device work counter.  A tile is 2^tile_log2 consecutive odd numbers
// of one range plus a look-back margin of mw words below it (the paper keeps
// the preceding interval for the same purpose, Sec. 3 after Algorithm 2).
// Per tile:
//   1. stamp:  every window word starts as the AND of the periodic strike
//              patterns of the NS smallest odd primes, read from two small
//              shared-memory tables indexed by the word number modulo the
//              product of their squares (NS = sv_config.stamp_primes);
//   2. strike: the next primes up to the bucket threshold clear their odd
//              multiples of p^2 with shared-memory atomicAnd.  "Dense" primes
//              (>= kDenseMinHits hits per window, at most 128) are struck
//              cooperatively, two strikes per trip:
//              the smallest by the whole CTA with a stride of one block, the
//              others by one warp each with a stride of one warp.  Sparser
//              ones take one thread per prime.  The offsets of both carry
//              from a window to the next one of the same range.  Larger
//              primes arrive as precomputed bit offsets in the tile's bucket
//              (bucket_fill_kernel, buckets.cu);
//   3. scan:   word-parallel Algorithm 2.  For the 32 odd n of word i, the
//              flags of n - 2^k are word i shifted by 2^(k-1) bits: a funnel
//              shift of (w[i-1], w[i]) for k <= 5, the word w[i - 2^(k-6)] for
//              6 <= k <= kwin.  unresolved &= ~flags, and hist[k] is the
//              drop of popc(unresolved) at step k (the lean scan sums the
//              counts after each step, hist[k] = U_(k-1) - U_k).
//              k = 1..4 run without votes (two words per lane, a 64-bit
//              load in the fast path); a word still
//              unresolved after k = 5 is finished by its lane after the loop;
//              n still unresolved after kwin go to the exact straggler test.
//              Tiles that may hold a range's first occurrence of some k <= 5
//              record it by ballot;
//   4. reduce: per-tile histogram and first occurrences into the range's
//              result slot (Sec. 3 "Collecting the results"), and the tile's
//              listed n (mink >= T) into its staging slot for the ordered
//              list (list_compact_kernel).
// The bitmap never leaves shared memory on this fused path.
//
// The plain (unfused) path runs the same kernel twice: a sieve pass
// (sieve_only ranges: phases 1-2, then the window's core words go to a bitmap
// in device memory with one bulk store per tile) and a scan pass (bitmap_in
// ranges: the tile fills its window from that bitmap with one bulk load, then
// phases 3-4).  Both bulk copies are cp.async.bulk (the TMA unit), tracked by
// an mbarrier (loads) or a bulk group (stores).
#include <cuda_runtime.h>

#include "strike.h"
#include "sv_internal.h"
#include "tma.h"

namespace sv {

// The stamped primes (the smallest ones, applied by the word's owner as a
// computed pattern instead of shared-memory atomics): q = p^2 and the 32-bit
// pattern with a 1 every q bits (a single bit once q >= 32).
__host__ __device__ constexpr uint32_t stamp_p(int s) {
  return s == 0 ? 3 : s == 1 ? 5 : s == 2 ? 7 : s == 3 ? 11 : s == 4 ? 13 : s == 5 ? 17 : s == 6 ? 19 : 23;
}
__host__ __device__ constexpr uint32_t stamp_rep(uint32_t q) {
  uint32_t r = 0;
  for (uint32_t b = 0; b < 32; b += q) r |= 1u << b;
  return r;
}
__device__ __forceinline__ uint32_t stamp_first(uint64_t abit, uint32_t q) {
  const uint32_t r = (uint32_t)(abit % q);
  const uint32_t c = (q - 1) >> 1;
  return (c >= r) ? (c - r) : (c + q - r);
}
__device__ __forceinline__ uint32_t stamp_step(uint32_t j, uint32_t d, uint32_t q) {
  return (j >= d) ? (j - d) : (j + q - d);
}

// The first stamped primes come from two periodic tables in shared memory.
// The strike pattern of a set of primes on the 32 bits of word a depends only
// on a mod P, P the product of their squares (odd, so 32 is invertible mod P):
// entry e of a table is the pattern of the words a = e (mod P).  Table A
// holds {3, 11} (P = 1089) and table B {5, 7} (P = 1225), or A alone {3, 5}
// (P = 225) when only two primes are stamped.  Consecutive words read
// consecutive entries, so a warp's reads hit distinct banks.  Each table is
// extended by kExt entries past its period, so that a warp reads entries
// e .. e + 63 (e < P) without a wrap.
template <int NS>
struct StampTab {
  static constexpr bool kTwo = NS >= 4;                   // two tables
  static constexpr uint32_t kQa0 = 9, kQa1 = kTwo ? 121u : 25u;
  static constexpr uint32_t kQb0 = 25, kQb1 = 49;
  static constexpr uint32_t kPa = kQa0 * kQa1;
  static constexpr uint32_t kPb = kTwo ? kQb0 * kQb1 : 0u;
  static constexpr uint32_t kExt = 64;
  static constexpr uint32_t kOffB = kPa + kExt;           // table B's first entry
  static constexpr uint32_t kSize = kTwo ? kOffB + kPb + kExt : kPa + kExt;
  static constexpr int kCovered = kTwo ? 4 : 2;           // stamp_p(0 .. kCovered-1)
};

// The pattern of the odd multiples of q on the word starting at bit J.
__device__ __forceinline__ uint32_t stamp_pattern(uint32_t J, uint32_t q) {
  uint32_t rep = 0;
  for (uint32_t b = 0; b < 32; b += q) rep |= 1u << b;
  return __funnelshift_lc(0u, rep, stamp_first(J, q));
}

template <int NS>
__device__ __forceinline__ void build_stamp_tables(uint32_t *tab) {
  using T = StampTab<NS>;
  for (uint32_t e = threadIdx.x; e < T::kSize; e += blockDim.x) {
    uint32_t v;
    // (entries past the period repeat its start: the pattern has period P words)
    if (e < T::kOffB) v = stamp_pattern(32u * e, T::kQa0) | stamp_pattern(32u * e, T::kQa1);
    else v = stamp_pattern(32u * (e - T::kOffB), T::kQb0) | stamp_pattern(32u * (e - T::kOffB), T::kQb1);
    tab[e] = v;
  }
}

// Window words [nz, nwords) <- AND of the NS stamped patterns.  With the
// tables alone (NS <= 4), warp w stamps 64-word steps w, w + nwarps, ...:
// lane l takes words l and l + 32 of the step, whose table entries are e + l
// and e + 32 + l for one position e per warp and table, advanced by
// 64 nwarps mod P per step.  The last (nwords - nz) mod 64 words, and every
// word when primes beyond the tables are stamped, go thread by thread: thread
// tid takes words tid, tid + S, ...; the table positions advance by S mod P,
// and the primes beyond the tables keep j[s], the offset of their first
// struck bit in the current word (>= 32: none), which moving S words lowers
// by 32*S mod q.
template <int NS>
__device__ __forceinline__ void stamp_window(uint32_t *win, const uint32_t *tab, uint32_t nz, uint32_t nwords,
                                             int64_t wstart) {
  using T = StampTab<NS>;
  constexpr int NX = NS - T::kCovered;
  const uint32_t S = blockDim.x;
  if (NX == 0) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = S >> 5;
    const uint32_t steps = (nwords - nz) >> 6;
    if (warp < steps) {
      const uint64_t aw = (uint64_t)(wstart + (int64_t)(nz + 64u * warp));  // >= 0
      uint32_t ea = (uint32_t)(aw % T::kPa), eb = T::kTwo ? (uint32_t)(aw % (T::kTwo ? T::kPb : 1u)) : 0u;
      const uint32_t da = (64u * nwarps) % T::kPa, db = T::kTwo ? (64u * nwarps) % (T::kTwo ? T::kPb : 1u) : 0u;
#pragma unroll 2
      for (uint32_t st = warp; st < steps; st += nwarps) {
        const uint32_t i = nz + 64u * st + lane;
        uint32_t m0 = tab[ea + lane], m1 = tab[ea + 32u + lane];
        if (T::kTwo) {
          m0 |= tab[T::kOffB + eb + lane];
          m1 |= tab[T::kOffB + eb + 32u + lane];
        }
        win[i] = ~m0;
        win[i + 32u] = ~m1;
        ea = min(ea + da, ea + da - T::kPa);  // unsigned: subtracts P once the sum reaches it
        if (T::kTwo) eb = min(eb + db, eb + db - T::kPb);
      }
    }
    nz += 64u * steps;  // the rest thread by thread, below
  }
  uint32_t i = nz + threadIdx.x;
  if (i >= nwords) return;
  const uint64_t aw = (uint64_t)(wstart + (int64_t)i);  // >= 0 since i >= nz
  uint32_t ea = (uint32_t)(aw % T::kPa), eb = T::kTwo ? (uint32_t)(aw % (T::kTwo ? T::kPb : 1u)) : 0u;
  const uint32_t sa = S % T::kPa, sb = T::kTwo ? S % (T::kTwo ? T::kPb : 1u) : 0u;
  uint32_t j[NX > 0 ? NX : 1], d[NX > 0 ? NX : 1];
#pragma unroll
  for (int s = 0; s < NX; ++s) {
    const uint32_t q = stamp_p(T::kCovered + s) * stamp_p(T::kCovered + s);
    j[s] = stamp_first(32ull * aw, q);
    d[s] = (32u * S) % q;
  }
  for (; i < nwords; i += S) {
    uint32_t m = tab[ea];
    if (T::kTwo) m |= tab[T::kOffB + eb];
#pragma unroll
    for (int s = 0; s < NX; ++s) {
      const uint32_t q = stamp_p(T::kCovered + s) * stamp_p(T::kCovered + s);
      m |= __funnelshift_lc(0u, stamp_rep(q), j[s]);
      j[s] = stamp_step(j[s], d[s], q);
    }
    win[i] = ~m;
    ea = min(ea + sa, ea + sa - T::kPa);  // unsigned: subtracts P once the sum reaches it
    if (T::kTwo) eb = min(eb + sb, eb + sb - T::kPb);
  }
}

// Bits b of the word starting at bit J0 with jlo <= J0 + b < jhi.
__device__ __forceinline__ uint32_t valid_mask(uint64_t J0, uint64_t jlo, uint64_t jhi) {
  if (jhi <= J0) return 0u;
  const uint64_t nh = jhi - J0;
  uint32_t m = (nh >= 32) ? 0xFFFFFFFFu : ((1u << (uint32_t)nh) - 1u);
  if (jlo > J0) {
    const uint64_t nl = jlo - J0;
    m &= (nl >= 32) ? 0u : ~((1u << (uint32_t)nl) - 1u);
  }
  return m;
}

// Clear bit b of the window: the mask is 0xFFFFFFFE rotated left by b mod 32.
__device__ __forceinline__ void strike(uint32_t *win, uint32_t b) {
  atomicAnd(&win[b >> 5], __funnelshift_l(0xFFFFFFFEu, 0xFFFFFFFEu, b));
}

// ---------------------------------------------------------------------------
// init: zero the launch's counters, result slots, bucket and staged-list
// counts; give each range of a large launch its number of table primes p
// with p^2 < hi (Algorithm 1's "primes 3 <= p < sqrt(end)",
// ReqDesc::n_primes) and the integer square roots of its bucket-fill interval
// ends (ReqDesc::sq_lo, sq_hi) for the multiplier items; the host plans these
// itself for launches of few ranges.
// ---------------------------------------------------------------------------
__global__ void init_kernel(LaunchHeader *hdr, ResultSlot *slots, uint32_t *bucket_count, uint32_t *stage_cnt,
                            ReqDesc *reqs, uint32_t mw, const uint32_t *primes, uint32_t n_table, uint64_t ph2) {
  const uint32_t n_slots = hdr->n_reqs, n_tiles = hdr->total_tiles;
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t gs = gridDim.x * blockDim.x;
  for (uint32_t r = gid; r < n_slots; r += gs) {
    ReqDesc &R = reqs[r];
    if (R.n_primes != kPlanOnDevice) continue;  // planned on the host
    const int64_t ws = R.w0 - (int64_t)mw;
    const uint64_t A = 32ull * (uint64_t)(ws < 0 ? 0 : ws);  // the fill's window bits [A, E = jhi)
    R.sq_lo = (uint32_t)isqrt_u64(2 * A);
    R.sq_hi = R.jhi ? (uint32_t)isqrt_u64(2 * R.jhi - 1) : 0u;
    // the count of table primes p <= isqrt(hi - 1): the first index with p > x
    const uint64_t x = R.hi > 1 ? isqrt_u64(R.hi - 1) : 0;
    uint32_t lo = 0, hi = n_table;
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if ((uint64_t)primes[mid] <= x) lo = mid + 1;
      else hi = mid;
    }
    R.n_primes = lo;
    R.j_max = (ph2 && R.jhi) ? (2 * R.jhi - 1) / ph2 : 0;
  }
  for (uint32_t i = gid; i < n_tiles; i += gs) {
    bucket_count[i] = 0;
    if (stage_cnt) stage_cnt[i] = 0;
  }
  for (uint32_t i = gid; i < n_slots * (uint32_t)kMaxK; i += gs) {
    slots[i / kMaxK].hist[i % kMaxK] = 0ull;
    slots[i / kMaxK].first_n[i % kMaxK] = kNoN;
  }
  for (uint32_t i = gid; i < n_slots; i += gs) {
    slots[i].list_count = 0ull;
    slots[i].fail_count = 0ull;
  }
  if (gid == 0) {
    hdr->work_counter = 0ull;
    hdr->strag_count = 0ull;
    hdr->status = 0u;
  }
}

cudaError_t launch_init(LaunchHeader *hdr, ResultSlot *slots, uint32_t n_slots,
                        uint32_t *bucket_count, uint32_t *stage_cnt, uint32_t n_tiles, ReqDesc *reqs, uint32_t mw,
                        const uint32_t *primes, uint32_t n_table, uint64_t ph2, cudaStream_t st) {
  uint64_t work = (uint64_t)n_slots * kMaxK;
  if (n_tiles > work) work = n_tiles;
  uint32_t grid = (uint32_t)((work + 255) / 256);
  if (grid < 1) grid = 1;
  if (grid > 1024) grid = 1024;
  init_kernel<<<grid, 256, 0, st>>>(hdr, slots, bucket_count, stage_cnt, reqs, mw, primes, n_table, ph2);
  return cudaGetLastError();
}

// The tile kernel.
// ---------------------------------------------------------------------------
constexpr uint32_t kMaxDense = kMaxDensePrimes;  // dense primes per tile: four warps, one prime per lane

constexpr uint32_t kLstCap = kStageCap;  // list entries (mink >= T) buffered per tile
constexpr uint32_t kMaxSparse = kMaxSparsePrimes;  // primes struck one thread each, per tile

struct ScanShared {
  unsigned long long hist[kMaxK];
  unsigned long long first[kMaxK];
  ReqDesc req;
  uint32_t tile;
  uint32_t next_tile;              // prefetched during the previous tile's scan
  uint32_t chunk_end;              // end of the chunk of consecutive tiles being worked
  uint32_t fresh;                  // 1: the primes' offsets are computed, not carried
  uint32_t req_idx;
  uint32_t n_strag;                // stragglers this tile sent to the exact test
  uint32_t need;                   // k <= 5 whose first occurrence this tile may still improve
  uint32_t lst_cnt;                // list entries this tile found (buffered up to kLstCap)
  // the dense primes of this tile: q = p^2 and the window offset of the
  // first struck bit (carried from window to window)
  uint32_t dense_q[kMaxDense];
  uint32_t dense_off[kMaxDense];
  uint32_t dense_tq[kMaxDense];    // (32 tw) mod dense_q: a window's shift, reduced
  unsigned long long lst_n[kLstCap];  // the buffered list entries: n and mink
  uint8_t lst_k[kLstCap];
  uint32_t sparse_off[kMaxSparse]; // first struck bit of each sparse prime (>= nbits: none)
  uint32_t sparse_q[kMaxSparse];
  uint64_t load_bar;               // mbarrier of the scan pass's bulk window loads
};

// A bounded wait (about one second at the maximum clock) for the window's bulk
// load; the outcome is the same for every thread of the block.
constexpr long long kBulkWaitCycles = 2000000000ll;

// Record the n of hit (mink = k, k >= T) in the range's list and first_n.
__device__ __noinline__ void list_append(const TileArgs &a, const ReqDesc &R, uint32_t hit,
                                         uint64_t J0, uint32_t k) {
  ResultSlot *slot = &a.slots[R.slot];
  while (hit) {
    const uint32_t b = __ffs(hit) - 1;
    hit &= hit - 1;
    const uint64_t n = 2ull * (J0 + b) + 1ull;
    atomicMin(&slot->first_n[k], (unsigned long long)n);
    const unsigned long long idx = atomicAdd(&slot->list_count, 1ull);
    if (idx < R.list_cap) {
      a.list_n[R.list_off + idx] = n;
      a.list_k[R.list_off + idx] = (uint8_t)k;
    }
  }
}

__device__ __noinline__ void straggler_push(const TileArgs &a, ScanShared &sh, uint32_t unres, uint64_t J0,
                                            uint32_t k0) {
  atomicAdd(&sh.n_strag, (uint32_t)__popc(unres));
  while (unres) {
    const uint32_t b = __ffs(unres) - 1;
    unres &= unres - 1;
    const unsigned long long idx = atomicAdd(&a.hdr->strag_count, 1ull);
    if (idx < a.strag_cap) {
      Straggler s;
      s.n = 2ull * (J0 + b) + 1ull;
      s.k0 = k0;
      s.req = sh.req_idx;
      a.strag[idx] = s;
    } else {
      atomicOr(&a.hdr->status, kStStragOverflow);
    }
  }
}

// Write the per-n minimal k of one word (bit-sliced planes pl[0..5]).
__device__ __forceinline__ void write_per_n(uint8_t *out, uint64_t J0, uint64_t jlo, uint32_t valid,
                                            const uint32_t pl[6]) {
  while (valid) {
    const uint32_t b = __ffs(valid) - 1;
    valid &= valid - 1;
    uint32_t k = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) k |= ((pl[j] >> b) & 1u) << j;
    out[J0 + b - jlo] = (uint8_t)k;
  }
}

// One step of the word-parallel Algorithm 2 for k <= 5 (sf = flags of n - 2^k).
//   LEAN: k = 1 is not counted (derived at the end of the tile from the
//         number of valid n) and lists start at k >= 6 (T >= 6).
template <int K, bool LEAN, bool PER_N>
__device__ __forceinline__ void scan_step(uint32_t sf, uint32_t &unres, uint32_t &cnt, uint32_t pl[6],
                                          const TileArgs &a, ScanShared &sh, int64_t aw, uint32_t rec_t) {
  const uint32_t hit = unres & sf;
  unres &= ~sf;
  if (!(LEAN && K == 1)) cnt += __popc(hit);
  if (PER_N) {
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if ((K >> j) & 1) pl[j] |= hit;
  }
  if (!LEAN && (uint32_t)K >= rec_t && hit) list_append(a, sh.req, hit, 32ull * (uint64_t)aw, (uint32_t)K);
}

// Mode 0: list entries (n with mink = k >= T) go to the tile's shared
// buffer, which the tile's flush stages for the ordered list.  Entries
// beyond the buffer are only counted; the flush reports them (kStListStage)
// and the launch is repeated with the unordered list path.
__device__ __noinline__ void list_buffer(ScanShared &sh, uint32_t hit, uint64_t J0, uint32_t k) {
  while (hit) {
    const uint32_t b = __ffs(hit) - 1;
    const uint32_t e = atomicAdd(&sh.lst_cnt, 1u);
    if (e < kLstCap) {
      sh.lst_n[e] = 2ull * (J0 + b) + 1ull;
      sh.lst_k[e] = (uint8_t)k;
    }
    hit &= hit - 1;
  }
}

// k = 6 .. kwin (rare): whole-word look-back reads; counts, first occurrences
// below T and lists go straight to shared/global atomics.
template <bool LEAN, bool PER_N>
__device__ __noinline__ uint32_t scan_tail(const uint32_t *win, uint32_t i, bool act, uint32_t unres,
                                           uint32_t pl[6], const TileArgs &a, ScanShared &sh, int64_t aw,
                                           uint32_t kwin, uint32_t rec_t) {
  const uint64_t J0 = 32ull * (uint64_t)aw;
  for (uint32_t k = 6; k <= kwin && __any_sync(0xFFFFFFFFu, unres); ++k) {
    const uint32_t sf = act ? win[i - (1u << (k - 6))] : 0u;
    const uint32_t hit = unres & sf;
    unres &= ~sf;
    if (PER_N) {
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if ((k >> j) & 1u) pl[j] |= hit;
    }
    if (hit) {
      atomicAdd(&sh.hist[k], (unsigned long long)__popc(hit));
      if (LEAN || k < rec_t)
        atomicMin(&sh.first[k], (unsigned long long)(2ull * (J0 + (uint64_t)(__ffs(hit) - 1)) + 1ull));
      if (k >= rec_t) {
        if (LEAN) list_buffer(sh, hit, J0, k);
        else list_append(a, sh.req, hit, J0, k);
      }
    }
  }
  if (unres) straggler_push(a, sh, unres, J0, kwin + 1u);
  return unres;
}

// Record, for each k with a bit in `need`, the warp's first n with mink = k.
// need is warp-uniform; a warp visits its words in increasing order, so its
// first hit for k is its smallest, and the minimum over warps is the tile's.
template <int K>
__device__ __forceinline__ void record_first(uint32_t hit, uint32_t &need, ScanShared &sh, int64_t aw) {
  if (need & (1u << K)) {
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, hit != 0);
    if (bal) {
      if ((threadIdx.x & 31u) == (uint32_t)(__ffs(bal) - 1))
        atomicMin(&sh.first[K], (unsigned long long)(64ull * (uint64_t)aw + 2ull * (uint64_t)(__ffs(hit) - 1) + 1ull));
      need &= ~(1u << K);
    }
  }
}

// One warp-iteration of the scan: lane's word i.  REC: some of the frequent
// exponents (k <= 5) still lack this warp's first occurrence.
template <bool LEAN, bool PER_N, bool REC>
__device__ __forceinline__ void scan_word(const uint32_t *win, uint32_t i, bool act, int64_t aw, uint32_t valid,
                                          uint32_t &need, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t &c4,
                                          uint32_t &c5, const TileArgs &a, ScanShared &sh) {
  const uint32_t kwin = a.g.kwin, rec_t = a.g.rec_t;
  const uint32_t w = act ? win[i] : 0u;
  const uint32_t wp = act ? win[i - 1] : 0u;
  uint32_t unres = valid;
  uint32_t pl[6] = {0u, 0u, 0u, 0u, 0u, 0u};
  uint32_t h;
#define SV_STEP(K, SF, CNT)                                     \
  h = unres & (SF);                                             \
  unres &= ~(SF);                                               \
  if (!(LEAN && K == 1)) CNT += __popc(h);                      \
  if (PER_N) {                                                  \
    _Pragma("unroll") for (int j = 0; j < 6; ++j) if ((K >> j) & 1) pl[j] |= h; \
  }                                                             \
  if (REC) record_first<K>(h, need, sh, aw);                    \
  if (!LEAN && (uint32_t)K >= rec_t && h) list_append(a, sh.req, h, 32ull * (uint64_t)aw, (uint32_t)K);
  SV_STEP(1, __funnelshift_l(wp, w, 1), c1)
  if (__any_sync(0xFFFFFFFFu, unres)) {
    SV_STEP(2, __funnelshift_l(wp, w, 2), c2)
    if (__any_sync(0xFFFFFFFFu, unres)) {
      SV_STEP(3, __funnelshift_l(wp, w, 4), c3)
      if (__any_sync(0xFFFFFFFFu, unres)) {
        SV_STEP(4, __funnelshift_l(wp, w, 8), c4)
        if (__any_sync(0xFFFFFFFFu, unres)) {
          SV_STEP(5, __funnelshift_l(wp, w, 16), c5)
          if (__any_sync(0xFFFFFFFFu, unres)) scan_tail<LEAN, PER_N>(win, i, act, unres, pl, a, sh, aw, kwin, rec_t);
        }
      }
    }
  }
#undef SV_STEP
  if (PER_N && sh.req.per_n_k) write_per_n(sh.req.per_n_k, 32ull * (uint64_t)aw, sh.req.jlo, valid, pl);
}


// One thread finishes one word whose n (bits u) are unresolved after k = 5:
// k = 6 .. kwin by whole-word look-back, then the exact test for the rest.
// First occurrences of every k go to the tile's shared minima.
__device__ __noinline__ void finish_word(const uint32_t *win, uint32_t i, uint32_t u, int64_t aw, const TileArgs &a,
                                         ScanShared &sh) {
  const uint64_t J0 = 32ull * (uint64_t)aw;
  const uint32_t kwin = a.g.kwin, rec_t = a.g.rec_t;
  for (uint32_t k = 6; k <= kwin && u; ++k) {
    const uint32_t h = u & win[i - (1u << (k - 6))];
    u ^= h;
    if (h) {
      atomicAdd(&sh.hist[k], (unsigned long long)__popc(h));
      atomicMin(&sh.first[k], (unsigned long long)(2ull * (J0 + (uint64_t)(__ffs(h) - 1)) + 1ull));
      if (k >= rec_t) list_buffer(sh, h, J0, k);
    }
  }
  if (u) straggler_push(a, sh, u, J0, kwin + 1u);
}

// Step k = K on two words at once (independent chains for the scheduler):
// the n whose n - 2^K is squarefree leave the unresolved sets.
template <int K>
__device__ __forceinline__ void step2(uint32_t p0, uint32_t w0, uint32_t p1, uint32_t w1, uint32_t &u0,
                                      uint32_t &u1) {
  u0 &= ~__funnelshift_l(p0, w0, 1u << (K - 1));
  u1 &= ~__funnelshift_l(p1, w1, 1u << (K - 1));
}

// The lean scan (no per-n output, lists from k >= 6): each lane takes two
// words per iteration.  The counts telescope: with U_k the number of n still
// unresolved after step k, hist[k] = U_(k-1) - U_k.  U_1 .. U_3 are summed
// per word; U_4 is the k = 5 hits plus the n left after k = 5, both counted
// in the rare branch that runs k = 5 (hist[1] follows from the number of valid
// n at the end of the tile).  Words still unresolved after k = 5 are queued
// for finish_word after the loop.  Tiles that may still hold a range's first
// occurrence of some k <= 5 use scan_word.
__device__ __forceinline__ void scan_tile_lean(const uint32_t *win, const TileArgs &a, ScanShared &sh,
                                               int64_t wstart, uint32_t nwords, uint32_t ifl, uint32_t nfull) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t mw = a.g.mw;
  uint32_t need = sh.need;
  uint32_t c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0;  // hits of the scan_word path
  uint32_t U1 = 0, U2 = 0, U3 = 0;                  // telescoped words: unresolved after k = 1, 2, 3
  uint32_t c5t = 0, x5 = 0;                         // telescoped words: k = 5 hits, unresolved after k = 5
  // a word still unresolved after k = 5 waits in its lane (one at most; an
  // earlier one is finished first) and is finished after the loop
  uint32_t pend_i = 0, pend_u = 0;
#define SV_DEFER(I, U)                                                              \
  if (U) {                                                                          \
    if (pend_u) finish_word(win, pend_i, pend_u, wstart + (int64_t)pend_i, a, sh); \
    pend_i = (I);                                                                   \
    pend_u = (U);                                                                   \
  }
#define SV_K5(I0, I1)                                                               \
  if (__any_sync(0xFFFFFFFFu, u0 | u1)) {                                           \
    const uint32_t r4 = __popc(u0) + __popc(u1);                                    \
    step2<5>(p0, w0, p1, w1, u0, u1);                                               \
    const uint32_t r5 = __popc(u0) + __popc(u1);                                    \
    c5t += r4 - r5;                                                                 \
    x5 += r5;                                                                       \
    if (__any_sync(0xFFFFFFFFu, u0 | u1)) { /* rare: a word of the warp left after k = 5 */ \
      SV_DEFER(I0, u0)                                                              \
      SV_DEFER(I1, u1)                                                              \
    }                                                                               \
  }
  if (need == 0u && ifl <= mw && nfull >= nwords - ifl && (nwords - mw) % (64u * nwarps) == 0u) {
    // every core word is in range and fully valid, and no first occurrence
    // is searched: no masks, no bounds checks.  Each warp scans one
    // contiguous span, 64 words per step: lane l loads words 2l and 2l + 1
    // at once; the word below 2l is lane l-1's second word (lane 0: the
    // previous step's last word).
    const uint32_t span = (nwords - mw) / nwarps;
    const uint32_t ie = mw + (warp + 1u) * span;
    uint32_t last = win[mw + warp * span - 1u];  // the same word for every lane
    for (uint32_t ib = mw + warp * span; ib < ie; ib += 64u) {
      const uint32_t i0 = ib + 2u * lane, i1 = i0 + 1u;
      const uint2 ww = *reinterpret_cast<const uint2 *>(win + i0);
      const uint32_t w0 = ww.x, w1 = ww.y, p1 = w0;
      const uint32_t up = __shfl_up_sync(0xFFFFFFFFu, w1, 1);
      const uint32_t p0 = lane ? up : last;
      last = __shfl_sync(0xFFFFFFFFu, w1, 31);
      uint32_t u0 = ~__funnelshift_l(p0, w0, 1);
      uint32_t u1 = ~__funnelshift_l(p1, w1, 1);
      U1 += __popc(u0) + __popc(u1);
      step2<2>(p0, w0, p1, w1, u0, u1);
      U2 += __popc(u0) + __popc(u1);
      step2<3>(p0, w0, p1, w1, u0, u1);
      U3 += __popc(u0) + __popc(u1);
      step2<4>(p0, w0, p1, w1, u0, u1);
      SV_K5(i0, i1)
    }
  } else
  for (uint32_t ib = mw + warp * 64u; ib < nwords; ib += nwarps * 64u) {
    const uint32_t i0 = ib + lane, i1 = i0 + 32u;
    const bool a0 = i0 < nwords, a1 = i1 < nwords;
    const int64_t aw0 = wstart + (int64_t)i0, aw1 = aw0 + 32;
    uint32_t v0, v1;
    if (i0 - ifl < nfull) v0 = 0xFFFFFFFFu;
    else v0 = a0 ? valid_mask(32ull * (uint64_t)aw0, sh.req.jlo, sh.req.jhi) : 0u;
    if (i1 - ifl < nfull) v1 = 0xFFFFFFFFu;
    else v1 = a1 ? valid_mask(32ull * (uint64_t)aw1, sh.req.jlo, sh.req.jhi) : 0u;
    if (need) {
      scan_word<true, false, true>(win, i0, a0, aw0, v0, need, c1, c2, c3, c4, c5, a, sh);
      scan_word<true, false, true>(win, i1, a1, aw1, v1, need, c1, c2, c3, c4, c5, a, sh);
      continue;
    }
    const uint32_t w0 = a0 ? win[i0] : 0u, p0 = a0 ? win[i0 - 1] : 0u;
    const uint32_t w1 = a1 ? win[i1] : 0u, p1 = a1 ? win[i1 - 1] : 0u;
    uint32_t u0 = v0 & ~__funnelshift_l(p0, w0, 1);
    uint32_t u1 = v1 & ~__funnelshift_l(p1, w1, 1);
    U1 += __popc(u0) + __popc(u1);
    step2<2>(p0, w0, p1, w1, u0, u1);
    U2 += __popc(u0) + __popc(u1);
    step2<3>(p0, w0, p1, w1, u0, u1);
    U3 += __popc(u0) + __popc(u1);
    step2<4>(p0, w0, p1, w1, u0, u1);
    SV_K5(i0, i1)
  }
#undef SV_K5
#undef SV_DEFER
  if (pend_u) finish_word(win, pend_i, pend_u, wstart + (int64_t)pend_i, a, sh);
  // U_4 = c5t + x5: the k = 5 hits and the n left after k = 5
  c2 += U1 - U2;
  c3 += U2 - U3;
  c4 += U3 - c5t - x5;
  c5 += c5t;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c2 += __shfl_xor_sync(0xFFFFFFFFu, c2, o);
    c3 += __shfl_xor_sync(0xFFFFFFFFu, c3, o);
    c4 += __shfl_xor_sync(0xFFFFFFFFu, c4, o);
    c5 += __shfl_xor_sync(0xFFFFFFFFu, c5, o);
  }
  if (lane == 0) {
    if (c2) atomicAdd(&sh.hist[2], (unsigned long long)c2);
    if (c3) atomicAdd(&sh.hist[3], (unsigned long long)c3);
    if (c4) atomicAdd(&sh.hist[4], (unsigned long long)c4);
    if (c5) atomicAdd(&sh.hist[5], (unsigned long long)c5);
  }
}

template <bool LEAN, bool PER_N>
__device__ __forceinline__ void scan_tile(const uint32_t *win, const TileArgs &a, ScanShared &sh, int64_t wstart,
                                          uint32_t nwords, uint32_t ifl, uint32_t nfull) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const Geometry &g = a.g;
  // frequent exponents whose first occurrence is taken here: k = 1 .. min(T-1, kwin, 5)
  uint32_t need = sh.need;
  uint32_t c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0;
  for (uint32_t ib = g.mw + warp * 32u; ib < nwords; ib += nwarps * 32u) {
    const uint32_t i = ib + lane;
    const bool act = i < nwords;
    const int64_t aw = wstart + (int64_t)i;
    uint32_t valid;
    if (i - ifl < nfull) valid = 0xFFFFFFFFu;
    else valid = act ? valid_mask(32ull * (uint64_t)aw, sh.req.jlo, sh.req.jhi) : 0u;
    if (need)
      scan_word<LEAN, PER_N, true>(win, i, act, aw, valid, need, c1, c2, c3, c4, c5, a, sh);
    else
      scan_word<LEAN, PER_N, false>(win, i, act, aw, valid, need, c1, c2, c3, c4, c5, a, sh);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (!LEAN) c1 += __shfl_xor_sync(0xFFFFFFFFu, c1, o);
    c2 += __shfl_xor_sync(0xFFFFFFFFu, c2, o);
    c3 += __shfl_xor_sync(0xFFFFFFFFu, c3, o);
    c4 += __shfl_xor_sync(0xFFFFFFFFu, c4, o);
    c5 += __shfl_xor_sync(0xFFFFFFFFu, c5, o);
  }
  if (lane == 0) {
    if (!LEAN && c1) atomicAdd(&sh.hist[1], (unsigned long long)c1);
    if (c2) atomicAdd(&sh.hist[2], (unsigned long long)c2);
    if (c3) atomicAdd(&sh.hist[3], (unsigned long long)c3);
    if (c4) atomicAdd(&sh.hist[4], (unsigned long long)c4);
    if (c5) atomicAdd(&sh.hist[5], (unsigned long long)c5);
  }
}

// The tile queue hands out chunks of consecutive tiles, so that one CTA works
// a range's tiles in order and the primes' offsets carry from one window to
// the next (a chunk's first tile computes them afresh); the last 4 tiles per
// CTA go one at a time, which keeps the CTAs' finishing times within about
// one tile of each other.  Chunks hold 12 tiles when the launch has at least
// 128 tiles per CTA, else 6, which evens out the finishing times of launches
// of few tiles per CTA (measured: 6 instead of 12 is 1.8% faster on 2^33 odd
// n, 54 tiles per CTA, and 4% slower on the 4096-range batch, about 300).
// Chunk j is tiles [*s, *e).
__device__ __forceinline__ void chunk_range(uint32_t j, uint32_t total, uint32_t ctas, uint32_t *s, uint32_t *e) {
  const uint32_t chunk = total >= 128u * ctas ? 12u : 6u;
  const uint32_t reserve = 4u * ctas;
  const uint32_t n_big = total > reserve ? (total - reserve) / chunk : 0u;
  uint64_t b, f;
  if (j < n_big) {
    b = (uint64_t)j * chunk;
    f = b + chunk;
  } else {
    b = (uint64_t)n_big * chunk + (j - n_big);
    f = b + 1;
  }
  *s = (uint32_t)min(b, (uint64_t)total);
  *e = (uint32_t)min(f, (uint64_t)total);
}

// MODE 0: lean scan (no per-n output, lists from k >= 6); 1: general scan;
// 2: general scan with the per-n output.  NS: number of stamped primes.
template <int MODE, int NS>
__global__ void __launch_bounds__(1024, 1) tile_kernel(TileArgs a) {
  extern __shared__ __align__(16) uint32_t win[];  // 16-byte aligned: the scan reads word pairs
  __shared__ ScanShared sh;
  __shared__ uint32_t stab[StampTab<NS>::kSize];
  constexpr bool LEAN = (MODE == 0);
  constexpr bool PER_N = (MODE == 2);

  const uint32_t tid = threadIdx.x, S = blockDim.x;
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  const Geometry g = a.g;
  const uint32_t total = a.hdr->total_tiles;
  const uint32_t n_reqs = a.hdr->n_reqs;
  const uint32_t nd = g.i_dense - g.i_med;  // <= kMaxDense (host guarantees)
  // frequent exponents whose first occurrence is searched per tile: k = 1 .. kfirst
  const uint32_t kfirst = min(min(g.rec_t, g.kwin + 1u) - 1u, 5u);

  if (tid < kMaxK) {
    sh.hist[tid] = 0ull;
    sh.first[tid] = kNoN;
  }
  if (tid == 0) {
    mbar_init(&sh.load_bar, 1);
    fence_mbar_init();
  }
  uint32_t load_parity = 0;     // phase parity of the next bulk window load
  bool store_pending = false;   // thread 0: a bulk store may still read the window
  build_stamp_tables<NS>(stab);
  const uint32_t T = 32u * g.tw;  // a window starts T bits above the previous one
  if (tid == 0) {
    sh.n_strag = 0;
    sh.lst_cnt = 0;
    sh.req_idx = 0xFFFFFFFFu;
    uint32_t cs, ce;
    chunk_range((uint32_t)atomicAdd(&a.hdr->work_counter, 1ull), total, gridDim.x, &cs, &ce);
    sh.next_tile = cs;
    sh.chunk_end = ce;
    sh.tile = 0xFFFFFFFFu;
  }
  __syncthreads();

  for (;;) {
    if (store_pending) {  // thread 0 only: the window is overwritten below
      bulk_wait_read_all();
      store_pending = false;
    }
    if (tid == 0) {
      const uint32_t t = sh.next_tile;
      uint32_t fresh = sh.tile == 0xFFFFFFFFu || t != sh.tile + 1u;  // not the previous tile's successor
      sh.tile = t;
      const uint32_t r = sh.req_idx;
      if (t < total && (r == 0xFFFFFFFFu || t - sh.req.tile_base >= sh.req.n_tiles)) {
        // the range of tile t: the next one, else a search
        uint32_t lo;
        if (r != 0xFFFFFFFFu && r + 1u < n_reqs && a.reqs[r + 1u].tile_base <= t &&
            t - a.reqs[r + 1u].tile_base < a.reqs[r + 1u].n_tiles) {
          lo = r + 1u;
        } else {
          uint32_t hi = n_reqs;
          lo = 0;
          while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.reqs[mid].tile_base <= t) lo = mid; else hi = mid;
          }
        }
        sh.req_idx = lo;
        sh.req = a.reqs[lo];
        fresh = 1;
      }
      sh.fresh = fresh;
    }
    __syncthreads();
    const uint32_t gt = sh.tile;
    if (gt >= total) {
      if (tid == 0) bulk_wait_all();  // the last bulk stores complete before the block exits
      break;
    }
    const ReqDesc &R = sh.req;
    const uint32_t t = gt - R.tile_base;
    const bool fresh = sh.fresh != 0;
    if (t >= R.n_tiles) {  // bounds check: never expected
      if (tid == 0) {
        atomicOr(&a.hdr->status, kStBadTile);
        sh.req_idx = 0xFFFFFFFFu;
        sh.tile = 0xFFFFFFFFu;
        uint32_t cs, ce;
        chunk_range((uint32_t)atomicAdd(&a.hdr->work_counter, 1ull), total, gridDim.x, &cs, &ce);
        sh.next_tile = cs;
        sh.chunk_end = ce;
      }
      __syncthreads();
      continue;
    }
    const int64_t tws = R.w0 + (int64_t)t * g.tw;
    const int64_t twe = min(tws + (int64_t)g.tw, R.wend);
    const int64_t wstart = tws - (int64_t)g.mw;
    const uint32_t nwords = (uint32_t)(twe - wstart);
    const int64_t aw0 = wstart < 0 ? 0 : wstart;
    const uint64_t A = 32ull * (uint64_t)aw0;
    const uint32_t abias = 32u * (uint32_t)(aw0 - wstart);
    const uint32_t nbits = 32u * nwords;
    // n of the tile's first valid bit: a first occurrence already recorded
    // below it (by any tile) cannot be improved here
    const unsigned long long n_first =
        2ull * max((unsigned long long)R.jlo, 32ull * (unsigned long long)tws) + 1ull;
    unsigned long long known[5] = {0, 0, 0, 0, 0};
    if (tid == 0 && !R.sieve_only)
      for (uint32_t k = 1; k <= kfirst; ++k) known[k - 1] = __ldcg(&a.slots[R.slot].first_n[k]);

    if (R.bitmap_in) {
      // ---- scan pass of the plain path: the window from device memory ------
      const uint32_t nz0 = (wstart < 0) ? (uint32_t)min((int64_t)nwords, -wstart) : 0u;
      for (uint32_t i = tid; i < nz0; i += S) win[i] = 0u;  // integers below 1
      const uint32_t cnt = nwords - nz0;
      const uint32_t *src = R.bitmap_in + (wstart + (int64_t)nz0 - R.bitmap_w0);
      // a bulk copy needs both addresses 16-byte aligned and a 16-byte
      // multiple; the rounded copy must stay inside the window (tw + mw
      // words), and the bitmap is allocated with 4 words of room behind it
      const uint32_t cnt4 = (cnt + 3u) & ~3u;
      const bool bulk = cnt && (nz0 & 3u) == 0u && ((uintptr_t)src & 15u) == 0u && nz0 + cnt4 <= g.tw + g.mw;
      const bool skip = a.hdr->skip_bulk_loads != 0u;  // the test hook: nothing is issued, the wait runs out
      const long long wait_cycles = a.hdr->bulk_wait_cycles ? (long long)a.hdr->bulk_wait_cycles : kBulkWaitCycles;
      if (bulk) {
        if (tid == 0 && !skip) {
          fence_proxy_async_smem();  // the previous tile's reads of the window come first
          const uint32_t bytes = 4u * cnt4;
          mbar_arrive_expect_tx(&sh.load_bar, bytes);
          bulk_load(win + nz0, src, bytes, &sh.load_bar);
        }
      } else {
        for (uint32_t i = tid; i < cnt; i += S) win[nz0 + i] = src[i];
      }
      if (tid == 0) {
        uint32_t need = 0;
        for (uint32_t k = 1; k <= kfirst; ++k)
          if (known[k - 1] > n_first) need |= 1u << k;
        sh.need = need;
      }
      if (bulk) {
        bool ok = mbar_wait_bounded(&sh.load_bar, load_parity, wait_cycles);
        if (__syncthreads_or(!ok)) {
          // the copy did not arrive in time: report it, wait once more for
          // the copy in flight (it writes into this block's shared memory),
          // and stop this block
          if (tid == 0) atomicOr(&a.hdr->status, kStTimeout);
          ok = mbar_wait_bounded(&sh.load_bar, load_parity, wait_cycles);
          __syncthreads_or(!ok);
          return;
        }
        load_parity ^= 1u;
      }
      __syncthreads();
    } else {
    // ---- 1. stamp the smallest primes; the dense primes' first strikes -------
    if (warp < kMaxDense / 32) {  // blockDim.x >= 128: warps 0..3 exist
      const uint32_t d = 32u * warp + lane;
      if (d < nd) {
        uint32_t q, off;
        if (fresh) {
          const uint64_t p = a.pt.p[g.i_med + d];
          q = (uint32_t)(p * p);
          off = abias + (uint32_t)first_strike(A, (uint64_t)q, a.pt.mu[g.i_med + d]);
          sh.dense_tq[d] = T % q;
        } else {
          // the previous window began T bits lower: off = (off_prev - T) mod q
          q = sh.dense_q[d];
          off = sh.dense_off[d] + q - sh.dense_tq[d];
          if (off >= q) off -= q;
          if (off >= q) off %= q;  // only after a window that began below bit 0
        }
        sh.dense_q[d] = q;
        sh.dense_off[d] = off;
      }
    }
    const uint32_t nz = (wstart < 0) ? (uint32_t)min((int64_t)nwords, -wstart) : 0u;
    for (uint32_t i = tid; i < nz; i += S) win[i] = 0u;  // integers below 1
    // sparse primes: their first strikes (on a fresh tile; otherwise carried
    // from the previous window), and the tile's bucket entries, are fetched
    // here so that the global-memory latency overlaps the stamping
    const uint32_t i_large = min(g.i_large, max(R.n_primes, g.i_dense));
    const uint32_t n_sparse = i_large - g.i_dense;  // <= kMaxSparse (host guarantees)
    if (fresh) for (uint32_t j = tid; j < n_sparse; j += S) {
      const uint64_t p = a.pt.p[g.i_dense + j];
      const uint64_t q = p * p;
      sh.sparse_off[j] = abias + (uint32_t)first_strike(A, q, a.pt.mu[g.i_dense + j]);
      sh.sparse_q[j] = (uint32_t)q;
    }
    const uint32_t *bd = a.bucket_data + (size_t)gt * g.bucket_cap;
    const uint32_t nb = min(a.bucket_count[gt], g.bucket_cap);
    const uint32_t bv0 = tid < g.bucket_cap ? bd[tid] : 0u;
    const uint32_t bv1 = tid + S < g.bucket_cap ? bd[tid + S] : 0u;
    stamp_window<NS>(win, stab, nz, nwords, wstart);
    if (tid == 0) {
      uint32_t need = 0;
      for (uint32_t k = 1; k <= kfirst; ++k)
        if (known[k - 1] > n_first) need |= 1u << k;
      sh.need = need;
    }
    __syncthreads();

    // ---- 2. strikes: dense primes spread over all threads, sparse primes one
    //         thread each, large primes from the tile's bucket ---------------
    {
      // head primes (>= 1 strike per thread): thread tid strikes their bits
      // off + q (tid + S m)
      const uint32_t nh = min(g.n_head, nd);
      for (uint32_t d = 0; d < nh; ++d) {
        const uint32_t q = sh.dense_q[d];
        const uint32_t step = S * q;  // <= the window's bits
        uint32_t b = sh.dense_off[d] + tid * q;
        // two strikes per trip, their atomics in flight together (b and step are both below the window's
        // bits, so b + step cannot wrap)
        for (; b + step < nbits; b += 2u * step) {
          strike(win, b);
          strike(win, b + step);
        }
        if (b < nbits) strike(win, b);
      }
      // the other dense primes, one warp each in a snake order over the warps
      // (their strike counts fall with p); lane l strikes off + q (l + 32 m)
      {
        const uint32_t nw = S >> 5;
        for (uint32_t rd = 0;; ++rd) {
          const uint32_t d = nh + rd * nw + ((rd & 1u) ? nw - 1u - warp : warp);
          if (d >= nd) break;
          const uint32_t q = sh.dense_q[d], step = 32u * q;  // step <= the window's bits
          uint32_t b = sh.dense_off[d] + lane * q;
          for (; b + step < nbits; b += 2u * step) {
            strike(win, b);
            strike(win, b + step);
          }
          if (b < nbits) strike(win, b);
        }
      }
      // a full window's strikes carry to the next window: its first struck
      // bit is the first one >= T, shifted down by T (q exceeds the margin,
      // so at most a few subtractions remain)
      // (when some threads take one prime more than others, they are the last
      // warps, whose dense tail is the lightest in the snake order)
      const bool carry = nwords == g.tw + g.mw;
      for (uint32_t j = S - 1u - tid; j < n_sparse; j += S) {
        const uint32_t q = sh.sparse_q[j];
        uint32_t b = sh.sparse_off[j];
        for (; b + q < nbits; b += 2u * q) {
          strike(win, b);
          strike(win, b + q);
        }
        if (b < nbits) {
          strike(win, b);
          b += q;
        }
        if (carry) {
          b -= T;
          while (b >= q) b -= q;
          sh.sparse_off[j] = b;
        }
      }
      for (uint32_t e = tid; e < nb; e += S) {
        const uint32_t b = e < S ? bv0 : (e < 2 * S ? bv1 : bd[e]);
        if (b < nbits) strike(win, b);
        else atomicOr(&a.hdr->status, kStBadTile);
      }
    }
    __syncthreads();
    }  // sieve (phases 1-2) or window from device memory

    // the next tile's index (the chunk's next tile, else a new chunk's first),
    // fetched while this tile is scanned
    uint32_t next = 0, next_end = 0;
    if (tid == 0) {
      if (gt + 1u < sh.chunk_end) {
        next = gt + 1u;
        next_end = sh.chunk_end;
      } else {
        chunk_range((uint32_t)atomicAdd(&a.hdr->work_counter, 1ull), total, gridDim.x, &next, &next_end);
      }
    }

    if (R.sieve_only) {
      // ---- Algorithm 1 alone: the core words to the bitmap ----------------
      // bits outside [jlo, jhi) are cleared first (only the range's first and
      // last words have any); then one bulk store of the 16-byte multiple,
      // plain stores for the rest (or everything, for an unaligned buffer)
      const uint32_t cnt = nwords - g.mw;
      uint32_t *dst = R.bitmap_out + (tws - R.w0);
      if (tid == 0) {
        win[g.mw] &= valid_mask(32ull * (uint64_t)tws, R.jlo, R.jhi);
        win[nwords - 1] &= valid_mask(32ull * (uint64_t)(twe - 1), R.jlo, R.jhi);
      }
      fence_proxy_async_smem();  // the window's strikes and masks before the bulk store
      __syncthreads();
      const bool bulk = cnt >= 4u && ((uintptr_t)dst & 15u) == 0u && (g.mw & 3u) == 0u;  // win + mw aligned
      const uint32_t nbulk = bulk ? (cnt & ~3u) : 0u;
      if (bulk && tid == 0) {
        bulk_store(dst, win + g.mw, 4u * nbulk);
        bulk_commit();
        store_pending = true;
      }
      for (uint32_t i = nbulk + tid; i < cnt; i += S) dst[i] = win[g.mw + i];
    } else {
      // ---- 3. word-parallel Algorithm 2 ------------------------------------
      // core words whose 32 bits are all valid: window indices [ifl, ifl+nfull)
      const int64_t full_lo = (int64_t)((R.jlo + 31) >> 5) - wstart;
      const int64_t full_hi = (int64_t)(R.jhi >> 5) - wstart;
      const int64_t fl = max(full_lo, (int64_t)g.mw), fh = min(full_hi, (int64_t)nwords);
      const uint32_t ifl = (uint32_t)fl;
      const uint32_t nfull = fh > fl ? (uint32_t)(fh - fl) : 0u;
      if (LEAN)
        scan_tile_lean(win, a, sh, wstart, nwords, ifl, nfull);
      else
        scan_tile<LEAN, PER_N>(win, a, sh, wstart, nwords, ifl, nfull);
    }
    if (tid == 0) {
      sh.next_tile = next;
      sh.chunk_end = next_end;
    }
    __syncthreads();

    // ---- 4. tile aggregates into the range's slot (warp 0) ------------------
    if (warp == 0) {
      unsigned long long h0 = sh.hist[lane], h1 = sh.hist[lane + 32];
      if (LEAN && !R.sieve_only) {
        // k = 1 was not counted: every other valid n of the tile is accounted for
        unsigned long long rest = (lane >= 2 ? h0 : 0ull) + h1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xFFFFFFFFu, rest, o);
        rest += sh.n_strag;
        const unsigned long long jl = max((unsigned long long)R.jlo, 32ull * (unsigned long long)tws);
        const unsigned long long jh = min((unsigned long long)R.jhi, 32ull * (unsigned long long)twe);
        if (lane == 1) h0 = (jh > jl ? jh - jl : 0ull) - rest;
      }
      ResultSlot *slot = &a.slots[R.slot];
      const unsigned long long f0 = sh.first[lane], f1 = sh.first[lane + 32];
      if (h0) atomicAdd(&slot->hist[lane], h0);
      if (h1) atomicAdd(&slot->hist[lane + 32], h1);
      if (f0 != kNoN) atomicMin(&slot->first_n[lane], f0);
      if (f1 != kNoN) atomicMin(&slot->first_n[lane + 32], f1);
      sh.hist[lane] = 0ull;
      sh.hist[lane + 32] = 0ull;
      sh.first[lane] = kNoN;
      sh.first[lane + 32] = kNoN;
      // mode 0: the tile's list entries to its staging slot (ordered later)
      if (LEAN) {
        const uint32_t m = sh.lst_cnt, ms = min(m, g.stage_cap);
        for (uint32_t e = lane; e < ms; e += 32u) {
          a.stage_n[(size_t)gt * kStageCap + e] = sh.lst_n[e];
          a.stage_k[(size_t)gt * kStageCap + e] = sh.lst_k[e];
        }
        if (lane == 0) {
          if (ms) a.stage_cnt[gt] = ms;
          if (m > ms) atomicOr(&a.hdr->status, kStListStage);
        }
      }
      __syncwarp();
      if (lane == 0) {
        sh.n_strag = 0;
        sh.lst_cnt = 0;
      }
      __syncwarp();
    }
  }
}

// The stamped-prime counts instantiated (sv_config.stamp_primes).
#define SV_FOR_EACH_NS(X) X(2) X(4) X(6) X(8)

static bool g_tile_smem_set = false;

// Raise one instantiation's dynamic shared memory limit to what its static
// shared memory leaves of the opt-in limit.
template <class K>
static cudaError_t set_max_dyn(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

cudaError_t tile_kernel_setup(size_t smem) {
  // The attribute is per kernel and process wide: raise it once to the
  // largest window any configuration may use, so contexts with different
  // tiles never disagree.
  (void)smem;
  if (g_tile_smem_set) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
#define SV_SET(NS)                                                                 \
  if ((e = set_max_dyn(tile_kernel<0, NS>, optin)) || (e = set_max_dyn(tile_kernel<1, NS>, optin)) || \
      (e = set_max_dyn(tile_kernel<2, NS>, optin)))                               \
    return e;
  SV_FOR_EACH_NS(SV_SET)
#undef SV_SET
  g_tile_smem_set = true;
  return cudaSuccess;
}

// An upper bound of the tile kernel's static shared memory (all instantiations).
size_t tile_static_smem() { return sizeof(ScanShared) + 4 * StampTab<8>::kSize + 256; }

cudaError_t launch_tiles(const TileArgs &a, uint32_t threads, uint32_t grid, size_t smem, int mode, cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  const int ns = (int)a.g.i_med;
#define SV_LAUNCH(NS)                                                          \
  if (ns == NS) {                                                              \
    if (mode == 2) tile_kernel<2, NS><<<grid, threads, smem, st>>>(a);         \
    else if (mode == 1) tile_kernel<1, NS><<<grid, threads, smem, st>>>(a);    \
    else tile_kernel<0, NS><<<grid, threads, smem, st>>>(a);                   \
    return cudaGetLastError();                                                 \
  }
  SV_FOR_EACH_NS(SV_LAUNCH)
#undef SV_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace sv
