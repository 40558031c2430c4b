// buckets.cu -- the large primes' strikes, computed ahead of the tiles (the
// bucket part of Algorithm 1, Sec. 3).  For every prime above the tiles' own
// strike range and every range of the launch, each struck bit of the range's
// windows is appended to the bucket of the tile whose core holds it, and to
// the next tile's bucket when it also lies in that tile's look-back margin.
//
// One launch does both kinds of large primes, as work items taken by a
// block-stride loop, so that the two run side by side:
//   * Barrett items (prime block, request chunk): primes i_large <= i < i_hyb,
//     one thread per prime; one Barrett reduction per range gives its first
//     struck bit, then the thread walks the further hits (for a launch of
//     few ranges, the blocks of the smallest primes, which have the most
//     hits, are cut into segments of the range, one item each);
//   * multiplier items (slice, request): primes p >= p_hyb, reached through
//     their odd multipliers j (j p^2 in the range) and the prime bitmap.
// A bucket slot is reserved with a global atomic that returns the slot; a
// Barrett thread reserves the slots of up to four hits together, so that
// their round trips overlap instead of queueing one behind the other.
#include <cuda_runtime.h>

#include <algorithm>

#include "strike.h"
#include "sv_internal.h"

namespace sv {

constexpr uint32_t kFillThreads = 256;
constexpr uint32_t kHitBatch = 4;       // slot reservations in flight per thread
constexpr uint64_t kWarpJ = 32;         // odd j < 2 kWarpJ are handled cooperatively (warp or grid)
// A launch of one request chunk (a single range, a sweep chunk) cuts the
// Barrett prime blocks whose smallest prime would walk more than kSegHits
// hits into up to kMaxSeg segments of each range, one item each.  A thread's
// hits are a chain of slot reservations, each a global atomic round trip
// (about half a microsecond under load), so a segment holds two batches of
// kHitBatch: the smallest primes' hits spread over many blocks instead.
constexpr uint64_t kSegHits = 2 * kHitBatch;
constexpr uint32_t kMaxSeg = 64;  // a power of two
constexpr uint32_t kMaxSplitBlocks = 16;  // prime blocks that may be cut
constexpr uint32_t kMaxSplitExtra = kMaxSplitBlocks * (kMaxSeg - 1);

struct FillReq {
  uint64_t A, E;  // struck bits wanted: [A, E)
  int64_t w0;
  uint32_t tile_base, n_tiles, n_primes, pad;
};

// One struck bit's bucket entries, computed before their slots are reserved:
// the tile whose core holds it and, if it also lies in the next tile's
// look-back, that tile (t1 = 0xFFFFFFFF: none).
struct BucketHit {
  uint32_t t0, off0, t1, off1, i0, i1;
};

__device__ __forceinline__ BucketHit bucket_hit(const BucketArgs &a, uint64_t J, int64_t w0, uint32_t tile_base,
                                                uint32_t n_tiles) {
  BucketHit h;
  const int64_t w = (int64_t)(J >> 5);
  uint32_t t = 0;
  if (w >= w0) t = (uint32_t)((uint64_t)(w - w0) >> a.g.tw_log2);
  if (t >= n_tiles) t = n_tiles - 1;  // cannot happen: J < E
  const int64_t wst = w0 + (int64_t)t * a.g.tw - (int64_t)a.g.mw;
  h.t0 = tile_base + t;
  h.off0 = (uint32_t)((int64_t)J - 32 * wst);
  h.t1 = 0xFFFFFFFFu;
  h.off1 = 0;
  h.i0 = h.i1 = 0;
  if (t + 1 < n_tiles) {
    const int64_t wst1 = wst + (int64_t)a.g.tw;
    if (w >= wst1) {
      h.t1 = tile_base + t + 1;
      h.off1 = (uint32_t)((int64_t)J - 32 * wst1);
    }
  }
  return h;
}

__device__ __forceinline__ void bucket_reserve(const BucketArgs &a, BucketHit &h) {
  h.i0 = atomicAdd(&a.bucket_count[h.t0], 1u);
  h.i1 = h.t1 != 0xFFFFFFFFu ? atomicAdd(&a.bucket_count[h.t1], 1u) : 0u;
}

__device__ __forceinline__ void bucket_store(const BucketArgs &a, const BucketHit &h) {
  if (h.i0 < a.g.bucket_cap) a.bucket_data[(size_t)h.t0 * a.g.bucket_cap + h.i0] = h.off0;
  else atomicOr(&a.hdr->status, kStBucketOverflow);
  if (h.t1 != 0xFFFFFFFFu) {
    if (h.i1 < a.g.bucket_cap) a.bucket_data[(size_t)h.t1 * a.g.bucket_cap + h.i1] = h.off1;
    else atomicOr(&a.hdr->status, kStBucketOverflow);
  }
}

// The struck bits J[0 .. n-1] (n <= kHitBatch) of one range: all slots are
// reserved before any entry is written.
__device__ __forceinline__ void bucket_emit(const BucketArgs &a, const uint64_t (&J)[kHitBatch], uint32_t n,
                                            int64_t w0, uint32_t tile_base, uint32_t n_tiles) {
  BucketHit h[kHitBatch];
#pragma unroll
  for (uint32_t u = 0; u < kHitBatch; ++u)
    if (u < n) h[u] = bucket_hit(a, J[u], w0, tile_base, n_tiles);
#pragma unroll
  for (uint32_t u = 0; u < kHitBatch; ++u)
    if (u < n) bucket_reserve(a, h[u]);
#pragma unroll
  for (uint32_t u = 0; u < kHitBatch; ++u)
    if (u < n) bucket_store(a, h[u]);
}

// ---- Barrett items ----------------------------------------------------------
// The hits J, J + q, ... below f.E of one Barrett prime in one range (or
// segment), kHitBatch slot reservations at a time.
__device__ __noinline__ void barrett_walk(const BucketArgs &a, const FillReq &f, uint64_t J, uint64_t q) {
  for (; J < f.E; J += kHitBatch * q) {
    uint64_t Jv[kHitBatch];
    uint32_t n = 0;
#pragma unroll
    for (uint32_t u = 0; u < kHitBatch; ++u) {
      Jv[u] = J + u * q;
      if (Jv[u] < f.E) n = u + 1;
    }
    bucket_emit(a, Jv, n, f.w0, f.tile_base, f.n_tiles);
  }
}

// Segments of prime block pb: the power of two at or above (span / q) /
// kSegHits for its smallest prime's q (the Barrett estimate of span / q is at
// most 2 low), 1 to kMaxSeg.
__device__ __forceinline__ uint32_t seg_count(const BucketArgs &a, uint32_t pb, uint64_t span) {
  const uint32_t i = a.g.i_large + pb * kFillThreads;
  const uint64_t hits = __umul64hi(span, a.pt.mu[i]);
  uint32_t n = 1;
  while (n < kMaxSeg && (uint64_t)n * kSegHits < hits) n <<= 1;
  return n;
}

// Primes of prime block pb (one per thread) against segment seg of nseg of
// each range of request chunk rc.
__device__ void fill_barrett_item(const BucketArgs &a, FillReq *s_req, uint32_t pb, uint32_t seg, uint32_t nseg,
                                  uint32_t rc, uint32_t n_reqs, uint32_t prime_end) {
  const uint32_t r0 = rc * kFillReqChunk;
  const uint32_t nr = min(kFillReqChunk, n_reqs - r0);
  __syncthreads();  // s_req holds the previous item's ranges
  for (uint32_t r = threadIdx.x; r < nr; r += blockDim.x) {
    const ReqDesc &R = a.reqs[r0 + r];
    FillReq f;
    const int64_t ws = R.w0 - (int64_t)a.g.mw;
    f.A = 32ull * (uint64_t)(ws < 0 ? 0 : ws);
    f.E = R.jhi;
    if (nseg > 1 && f.E > f.A) {  // the segment's bits [A + seg L, A + (seg + 1) L), L = ceil((E - A) / nseg)
      const uint64_t len = (f.E - f.A + nseg - 1) >> (31 - __clz(nseg));  // nseg: a power of two
      const uint64_t a0 = f.A + seg * len;
      f.A = a0 < f.E ? a0 : f.E;
      if (f.E - f.A > len) f.E = f.A + len;
    }
    f.w0 = R.w0;
    f.tile_base = R.tile_base;
    f.n_tiles = R.n_tiles;
    f.n_primes = R.n_primes;
    f.pad = 0;
    s_req[r] = f;
  }
  __syncthreads();
  const uint32_t pi = a.g.i_large + pb * blockDim.x + threadIdx.x;
  if (pi >= prime_end) return;
  const uint64_t p = a.pt.p[pi];
  const uint64_t q = p * p, mu = a.pt.mu[pi];
  // two ranges per step: their first-strike reductions are independent
  // chains of 64-bit multiplies, so they overlap; a hit (rare for most
  // primes and ranges) is then walked range by range
  // (only the bounds are held across the pair; a walk reads the rest of its
  // range from shared memory)
  uint32_t r = 0;
  for (; r + 1 < nr; r += 2) {
    const uint64_t A0 = s_req[r].A, A1 = s_req[r + 1].A;
    const uint64_t J0 = A0 + first_strike(A0, q, mu), J1 = A1 + first_strike(A1, q, mu);
    if (J0 < s_req[r].E && pi < s_req[r].n_primes && s_req[r].n_tiles) barrett_walk(a, s_req[r], J0, q);
    if (J1 < s_req[r + 1].E && pi < s_req[r + 1].n_primes && s_req[r + 1].n_tiles)
      barrett_walk(a, s_req[r + 1], J1, q);
  }
  if (r < nr) {
    const uint64_t J = s_req[r].A + first_strike(s_req[r].A, q, mu);
    if (J < s_req[r].E && pi < s_req[r].n_primes && s_req[r].n_tiles) barrett_walk(a, s_req[r], J, q);
  }
}

// ---- multiplier items -------------------------------------------------------

// j p^2 <= x, exactly (p < 2^32, so p^2 fits 64 bits; the product with j is
// checked for overflow).
__device__ __forceinline__ bool jsq_le(uint64_t j, uint64_t p, uint64_t x) {
  const uint64_t p2 = p * p;
  return __umul64hi(j, p2) == 0 && j * p2 <= x;
}

// z ~ 2^63 / sqrt(j) for j >= 1 (integer fixed point), by Newton's iteration
// for the reciprocal square root, z <- z (3 - j z^2) / 2, which needs no
// division.  The start is 0.85 or 0.6 times 2^(63 - h) for j in [4^h, 2 4^h)
// or [2 4^h, 4^(h+1)): within 20% of the root, from where five steps reach a
// relative error far below 2^-40.  Only an estimate: callers correct it
// exactly.
__device__ __forceinline__ uint64_t rsqrt_fix(uint64_t j) {
  const uint32_t b = 64u - (uint32_t)__clzll((long long)j);
  const uint32_t h = (b - 1u) >> 1;
  uint64_t z = (((b - 1u) & 1u) ? 0x4CCCCCCCCCCCCCCCull : 0x6CCCCCCCCCCCCCCCull) >> h;
#pragma unroll
  for (int it = 0; it < 5; ++it) {
    const uint64_t u = j * __umul64hi(z, z);  // j z^2 / 2^64, about 2^62
    z = __umul64hi(z, (3ull << 62) - u) << 1;
  }
  return z;
}

// floor(sqrt(floor(x / j))), i.e. the largest r < 2^32 with j r^2 <= x, from
// S = floor(sqrt(x)) and z = rsqrt_fix(j): the estimate S z / 2^63 lies within
// one of the result, and exact integer steps finish it.
__device__ __forceinline__ uint64_t isqrt_div(uint64_t x, uint64_t S, uint64_t z, uint64_t j) {
  uint64_t r = __umul64hi(S << 1, z);
  if (r > 0xFFFFFFFFull) r = 0xFFFFFFFFull;
  while (r > 0 && !jsq_le(j, r, x)) --r;
  while (r < 0xFFFFFFFFull && jsq_le(j, r + 1, x)) ++r;
  return r;
}

// Bitmap bits [b0, b1] ((p-1)/2) of the odd p >= ph, p <= p_top, with an odd
// multiple j p^2 in [mlo, mhi]; false if there are none.  An odd multiple
// m = j p^2 lies in [mlo, mhi] exactly when j p^2 >= mlo and j p^2 <= mhi:
// p > isqrt_div(mlo - 1, j) and p <= isqrt_div(mhi, j).  sq_lo and sq_hi are
// floor(sqrt(mlo - 1)) and floor(sqrt(mhi)), computed once per range.
__device__ __forceinline__ bool p_interval(uint64_t mlo, uint64_t mhi, uint64_t sq_lo, uint64_t sq_hi, uint64_t j,
                                           uint64_t ph, uint64_t p_top, uint64_t *b0, uint64_t *b1) {
  const uint64_t z = rsqrt_fix(j);
  uint64_t plo = isqrt_div(mlo - 1, sq_lo, z, j) + 1, phi = isqrt_div(mhi, sq_hi, z, j);
  if (plo < ph) plo = ph;
  if (phi > p_top) phi = p_top;
  if (plo > phi) return false;
  *b0 = plo >> 1;
  *b1 = (phi - 1) >> 1;
  return *b0 <= *b1;
}

// The primes of bitmap word wd (bits m) with multiplier j: their struck bits
// (j p^2 - 1) / 2, one at a time (batching them here costs more registers
// than the whole kernel otherwise needs).
__device__ __forceinline__ void emit_word(const BucketArgs &a, const ReqDesc &R, uint32_t m, uint64_t wd,
                                          uint64_t j) {
  while (m) {
    const uint32_t bb = __ffs(m) - 1;
    m &= m - 1;
    const uint64_t p = 2 * (32 * wd + bb) + 1;
    const uint64_t Jv[kHitBatch] = {(p * p * j - 1) >> 1, 0, 0, 0};
    bucket_emit(a, Jv, 1, R.w0, R.tile_base, R.n_tiles);
  }
}

// Bitmap word w of the interval [b0, b1], masked to it.
__device__ __forceinline__ uint32_t interval_word(const BucketArgs &a, uint64_t w, uint64_t b0, uint64_t b1) {
  uint32_t mm = a.pt.bits[w];
  if (w == (b0 >> 5)) mm &= 0xFFFFFFFFu << (b0 & 31);
  if (w == (b1 >> 5) && (b1 & 31) != 31) mm &= (2u << (b1 & 31)) - 1u;
  return mm;
}

// Slice s of nsl of range r's odd multipliers j (j p^2 in the range, p >= p_hyb).
// The smallest multipliers have the longest p intervals (and the most hits).
// A long range (>= 2^30 odd numbers) spreads the bitmap words of all its
// small multipliers over the threads of all slices, one word each (the
// intervals and their word counts are computed once per item);
// a shorter one gives each small j to one warp, lanes striding over words.
// Larger j take one thread each.
__device__ void fill_mult_item(const BucketArgs &a, uint64_t (*s_iv)[3], uint32_t s, uint32_t nsl, uint32_t r) {
  const Geometry &g = a.g;
  const ReqDesc &R = a.reqs[r];
  if (R.n_tiles == 0 || R.n_primes <= g.i_hyb) return;  // uniform over the block
  const int64_t ws = R.w0 - (int64_t)g.mw;
  const uint64_t A = 32ull * (uint64_t)(ws < 0 ? 0 : ws), E = R.jhi;
  if (E <= A) return;
  const uint64_t ph = g.p_hyb;
  const uint64_t mlo = 2 * A + 1, mhi = 2 * E - 1;
  const uint64_t jmax = R.j_max;  // floor(mhi / p_hyb^2), planned once per range
  // a slice past the range's multipliers has nothing to do (a long range
  // spreads its small multipliers' words over every slice, below)
  if (E - A < (1ull << 30) && (uint64_t)s * (blockDim.x >> 5) >= kWarpJ &&
      2 * (kWarpJ + (uint64_t)s * blockDim.x) + 1 > jmax)
    return;  // uniform over the block
  const uint64_t p_top = a.pt.p[R.n_primes - 1];  // primes with p^2 < hi
  const uint64_t w_end = a.pt.bits_words;
  if (E - A >= (1ull << 30)) {
    __syncthreads();  // s_iv holds the previous item's intervals
    if (threadIdx.x < kWarpJ) {  // warp 0: one small multiplier per lane
      const uint32_t t = threadIdx.x;
      const uint64_t j = 2 * t + 1;
      uint64_t b0 = 1, b1 = 0, nw = 0;
      if (j <= jmax && p_interval(mlo, mhi, R.sq_lo, R.sq_hi, j, ph, p_top, &b0, &b1)) {
        const uint64_t w_last = min(b1 >> 5, w_end - 1);
        if (w_last >= (b0 >> 5)) nw = w_last - (b0 >> 5) + 1;
      }
      uint64_t incl = nw;  // the words of multipliers 0 .. t
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (t >= (uint32_t)o) incl += y;
      }
      s_iv[t][0] = b0;
      s_iv[t][1] = b1;
      s_iv[t][2] = incl - nw;
      if (t == kWarpJ - 1) s_iv[kWarpJ][2] = incl;
    }
    __syncthreads();
    // the words of all small multipliers, a quarter word (8 odd p) per
    // thread of the item's slices: each prime is a chain of slot
    // reservations, so the primes spread over as many threads as possible
    const uint64_t total = 4 * s_iv[kWarpJ][2];
    for (uint64_t gq = (uint64_t)s * blockDim.x + threadIdx.x; gq < total; gq += (uint64_t)nsl * blockDim.x) {
      const uint64_t gw = gq >> 2;
      uint32_t t = 0;  // the last multiplier whose words start at or below gw
#pragma unroll
      for (uint32_t h = kWarpJ / 2; h > 0; h >>= 1)
        if (t + h < kWarpJ && s_iv[t + h][2] <= gw) t += h;
      const uint64_t b0 = s_iv[t][0], b1 = s_iv[t][1];
      const uint64_t w = (b0 >> 5) + (gw - s_iv[t][2]);
      emit_word(a, R, interval_word(a, w, b0, b1) & (0xFFu << (8u * (uint32_t)(gq & 3u))), w, 2 * t + 1);
    }
  } else {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t wpb = blockDim.x >> 5;
    for (uint64_t t = (uint64_t)s * wpb + (threadIdx.x >> 5); t < kWarpJ && 2 * t + 1 <= jmax; t += (uint64_t)nsl * wpb) {
      const uint64_t j = 2 * t + 1;
      uint64_t b0, b1;
      if (!p_interval(mlo, mhi, R.sq_lo, R.sq_hi, j, ph, p_top, &b0, &b1)) continue;
      const uint64_t w_last = min(b1 >> 5, w_end - 1);
      for (uint64_t w = (b0 >> 5) + lane; w <= w_last; w += 32) emit_word(a, R, interval_word(a, w, b0, b1), w, j);
    }
  }
  for (uint64_t t = kWarpJ + (uint64_t)s * blockDim.x + threadIdx.x; 2 * t + 1 <= jmax;
       t += (uint64_t)nsl * blockDim.x) {
    const uint64_t j = 2 * t + 1;
    uint64_t b0, b1;
    if (!p_interval(mlo, mhi, R.sq_lo, R.sq_hi, j, ph, p_top, &b0, &b1)) continue;
    const uint64_t w_last = min(b1 >> 5, w_end - 1);
    for (uint64_t wd = b0 >> 5; wd <= w_last; wd += 4) {  // four words in flight
      uint32_t m[4];
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) m[u] = wd + u <= w_last ? interval_word(a, wd + u, b0, b1) : 0u;
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) emit_word(a, R, m[u], wd + u, j);
    }
  }
}

// The item space: jx slices x jy requests of multiplier items, then px prime
// blocks x py request chunks of Barrett items (host-chosen upper bounds).
// Each is trimmed to what the launch's header asks for, so that a captured
// launch sized for its buffers wastes no block on absent work.
struct FillItems {
  uint32_t px, py, jx, jy;
};

__global__ void __launch_bounds__(kFillThreads, kFillBlocksPerSm) bucket_fill_kernel(BucketArgs a, FillItems fi) {
  __shared__ FillReq s_req[kFillReqChunk];
  __shared__ uint64_t s_iv[kWarpJ + 1][3];  // small multipliers: interval bits, first word's rank; [kWarpJ][2]: total
  const Geometry &g = a.g;
  const uint32_t n_reqs = a.hdr->n_reqs;
  const uint32_t max_primes = a.hdr->max_primes;
  // Barrett items actually present
  const uint32_t prime_end = min(max_primes, g.i_hyb);
  const uint32_t n_pblocks = prime_end > g.i_large ? (prime_end - g.i_large + blockDim.x - 1) / blockDim.x : 0u;
  const uint32_t n_chunks = (n_reqs + kFillReqChunk - 1) / kFillReqChunk;
  // the first n_split = s_split[0] prime blocks are cut into s_nseg[pb]
  // segments (one request chunk only): s_split[1] items for them, then one
  // per remaining block.  Warp 0 computes the counts side by side (they do
  // not grow with pb, so the cut blocks are those with more than one).
  static_assert(kMaxSplitBlocks <= 32, "one lane per block that may be cut");
  __shared__ uint32_t s_split[2];
  __shared__ uint32_t s_nseg[kMaxSplitBlocks];
  if (threadIdx.x < 32) {
    const uint32_t l = threadIdx.x;
    const uint64_t span = a.hdr->fill_span;
    uint32_t ns = 1;
    if (n_chunks == 1 && span && l < min(kMaxSplitBlocks, n_pblocks)) ns = seg_count(a, l, span);
    const uint32_t one = __ballot_sync(0xFFFFFFFFu, ns <= 1);  // lanes >= kMaxSplitBlocks vote here too
    const uint32_t n_split = one ? (uint32_t)(__ffs(one) - 1) : 32u;
    uint32_t items = l < n_split ? ns : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) items += __shfl_xor_sync(0xFFFFFFFFu, items, o);
    if (l < kMaxSplitBlocks) s_nseg[l] = ns;
    if (l == 0) {
      s_split[0] = n_split;
      s_split[1] = items;
    }
  }
  __syncthreads();
  const uint32_t n_pbs = s_split[1] + (n_pblocks - s_split[0]);  // (prime block, segment) items per chunk
  const uint32_t px = min(fi.px, n_pbs), py = min(fi.py, n_chunks);
  const uint32_t n_bar = px * py;  // <= (4096 + kMaxSplitExtra) * 64
  // multiplier items actually present: one thread per odd multiplier of the
  // launch's largest range, at least eight slices, at most the captured ones
  const uint64_t jm = a.hdr->j_max;
  const uint32_t jx_need = (uint32_t)min((jm / 2 + kFillThreads) / kFillThreads, (uint64_t)fi.jx);
  const uint32_t jx = (max_primes > g.i_hyb && g.p_hyb != 0xFFFFFFFFu) ? min(fi.jx, max(jx_need, 8u)) : 0u;
  const uint32_t jy = min(fi.jy, n_reqs);
  const uint32_t n_mult = jx * jy;  // <= 64 * 1024
  // Blocks take items round robin.  The multiplier items come first, slice
  // by slice: the low slices hold the small multipliers, the costliest
  // items, and consecutive items land on different blocks.
  for (uint32_t it = blockIdx.x; it < n_mult + n_bar; it += gridDim.x) {
    if (it < n_mult) {
      // item (s, ry) covers slice s of the ranges ry + jy k
      for (uint32_t r = it % jy; r < n_reqs; r += jy) fill_mult_item(a, s_iv, it / jy, jx, r);
    } else {
      const uint32_t m = it - n_mult;
      // item (x, rcy) covers (prime block, segment) items x + px i and
      // chunks rcy + py k
      for (uint32_t rc = m / px; rc < n_chunks; rc += py)
        for (uint32_t x = m % px; x < n_pbs; x += px) {
          uint32_t pb, seg = 0, nseg = 1;
          if (x < s_split[1]) {
            pb = 0;
            seg = x;
            for (;;) {
              nseg = s_nseg[pb];
              if (seg < nseg) break;
              seg -= nseg;
              ++pb;
            }
          } else {
            pb = s_split[0] + (x - s_split[1]);
          }
          fill_barrett_item(a, s_req, pb, seg, nseg, rc, n_reqs, prime_end);
        }
    }
  }
}

cudaError_t launch_bucket_fill(const BucketArgs &a, uint32_t n_large_max, uint32_t n_reqs, uint64_t j_max,
                               uint32_t max_blocks, cudaStream_t st) {
  if (n_large_max == 0 || n_reqs == 0) return cudaSuccess;
  FillItems fi;
  // prime blocks, plus the segments of the cut ones
  fi.px = (uint32_t)std::min<uint64_t>((n_large_max + kFillThreads - 1) / kFillThreads, 4096) + kMaxSplitExtra;
  fi.py = std::min<uint32_t>((n_reqs + kFillReqChunk - 1) / kFillReqChunk, 64);
  const bool mult = a.g.p_hyb != 0xFFFFFFFFu && j_max != 0;
  // slices: one thread per odd multiplier (at least eight slices, so that a
  // long range's small-multiplier words spread over 2048 threads)
  fi.jx = mult ? (uint32_t)std::min<uint64_t>(std::max<uint64_t>((j_max / 2 + kFillThreads) / kFillThreads, 8), 64) : 0u;
  fi.jy = mult ? std::min<uint32_t>(n_reqs, 1024) : 0u;
  const uint64_t items = (uint64_t)fi.px * fi.py + (uint64_t)fi.jx * fi.jy;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(items, max_blocks ? max_blocks : 1));
  bucket_fill_kernel<<<grid, kFillThreads, 0, st>>>(a, fi);
  return cudaGetLastError();
}

}  // namespace sv
