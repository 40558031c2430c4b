// tiles.cu -- the range path: Algorithm 1 (sieve) and Algorithm 2 (search
// for the smallest k) of Sec. 3, fused per shared-memory tile.
//
// One persistent CTA per SM pulls tiles from a device work queue.  A tile is
// 2^tile_log2 consecutive odd numbers of one range plus a look-back margin of
// mw words below it (the paper keeps the preceding interval for the same
// purpose, Sec. 3 after Algorithm 2).  Per tile:
//   1. stamp:  every window word starts as the AND of the periodic strike
//              patterns of p = 3, 5, 7, 11 (computed, not loaded);
//   2. strike: primes 13 <= p < large_prime_min clear their odd multiples of
//              p^2 with shared-memory atomicAnd (warp-cooperative while a
//              prime has >= 32 hits per tile, one thread per prime above);
//              larger primes arrive as precomputed bit offsets in the tile's
//              bucket (bucket_fill_kernel);
//   3. scan:   word-parallel Algorithm 2.  For the 32 odd n of word i, the
//              flags of n - 2^k are word i shifted by 2^(k-1) bits: a funnel
//              shift of (w[i-1], w[i]) for k <= 5, the word w[i - 2^(k-6)] for
//              6 <= k <= kwin.  unresolved &= ~flags; hist[k] += popc(newly).
//              n still unresolved after kwin go to the exact straggler test;
//   4. reduce: per-tile histogram and first occurrences into the range's
//              result slot (Sec. 3 "Collecting the results").
// The bitmap never leaves shared memory.
#include <cuda_runtime.h>

#include "sv_internal.h"

namespace sv {

// x mod q for q >= 2 with mu = floor((2^64-1)/q): Barrett (1986) reduction.
// The estimate t = floor(x*mu / 2^64) is at most 2 below floor(x/q).
__device__ __forceinline__ uint64_t mod_barrett(uint64_t x, uint64_t q, uint64_t mu) {
  const uint64_t t = __umul64hi(x, mu);
  uint64_t r = x - t * q;
  if (r >= q) r -= q;
  if (r >= q) r -= q;
  return r;
}

// Odd multiples of q = p^2 are the integers q(2i+1), i.e. the bits
// J = q*i + (q-1)/2.  Offset (from bit A) of the first such bit >= A.
__device__ __forceinline__ uint64_t first_strike(uint64_t A, uint64_t q, uint64_t mu) {
  const uint64_t r = mod_barrett(A, q, mu);
  const uint64_t c = (q - 1) >> 1;
  return (c >= r) ? (c - r) : (c + q - r);
}

// The stamped primes: q = p^2 and the 32-bit pattern with a 1 every q bits.
__device__ __forceinline__ uint32_t stamp_first(uint64_t abit, uint32_t q) {
  const uint32_t r = (uint32_t)(abit % q);
  const uint32_t c = (q - 1) >> 1;
  return (c >= r) ? (c - r) : (c + q - r);
}
__device__ __forceinline__ uint32_t stamp_step(uint32_t j, uint32_t d, uint32_t q) {
  return (j >= d) ? (j - d) : (j + q - d);
}
constexpr uint32_t kQ0 = 9, kQ1 = 25, kQ2 = 49, kQ3 = 121;
constexpr uint32_t kRep0 = (1u << 0) | (1u << 9) | (1u << 18) | (1u << 27);
constexpr uint32_t kRep1 = (1u << 0) | (1u << 25);

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

__device__ __forceinline__ void strike(uint32_t *win, uint32_t b) {
  atomicAnd(&win[b >> 5], ~(1u << (b & 31u)));
}

// ---------------------------------------------------------------------------
// init: zero the launch's counters, result slots and bucket counts.
// ---------------------------------------------------------------------------
__global__ void init_kernel(LaunchHeader *hdr, ResultSlot *slots, uint32_t *bucket_count) {
  const uint32_t n_slots = hdr->n_reqs, n_tiles = hdr->total_tiles;
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t gs = gridDim.x * blockDim.x;
  for (uint32_t i = gid; i < n_tiles; i += gs) bucket_count[i] = 0;
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
                        uint32_t *bucket_count, uint32_t n_tiles, cudaStream_t st) {
  uint64_t work = (uint64_t)n_slots * kMaxK;
  if (n_tiles > work) work = n_tiles;
  uint32_t grid = (uint32_t)((work + 255) / 256);
  if (grid < 1) grid = 1;
  if (grid > 1024) grid = 1024;
  init_kernel<<<grid, 256, 0, st>>>(hdr, slots, bucket_count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bucket fill: for every large prime and every range, the struck bits of the
// range's windows, appended to the bucket of each tile whose window holds them
// (the tile's core, and the next tile's look-back margin).
// ---------------------------------------------------------------------------
constexpr uint32_t kFillReqChunk = 64;

struct FillReq {
  uint64_t A, E;       // struck bits wanted: [A, E)
  int64_t w0;
  uint32_t tile_base, n_tiles, n_primes, pad;
};

__device__ __forceinline__ void bucket_push(const BucketArgs &a, uint32_t gtile, uint32_t off) {
  const uint32_t idx = atomicAdd(&a.bucket_count[gtile], 1u);
  if (idx < a.g.bucket_cap)
    a.bucket_data[(size_t)gtile * a.g.bucket_cap + idx] = off;
  else
    atomicOr(&a.hdr->status, kStBucketOverflow);
}

__global__ void __launch_bounds__(256) bucket_fill_kernel(BucketArgs a) {
  __shared__ FillReq s_req[kFillReqChunk];
  const uint32_t n_reqs = a.hdr->n_reqs;
  const uint32_t max_primes = a.hdr->max_primes;
  const Geometry g = a.g;
  if (max_primes <= g.i_large) return;
  const uint32_t n_large = max_primes - g.i_large;
  const uint32_t n_pblocks = (n_large + blockDim.x - 1) / blockDim.x;
  const uint32_t tw = g.tw, mw = g.mw;

  for (uint32_t pb = blockIdx.x; pb < n_pblocks; pb += gridDim.x) {
    const uint32_t pi = g.i_large + pb * blockDim.x + threadIdx.x;
    const bool act = pi < max_primes;
    uint64_t q = 1, mu = 0;
    if (act) {
      const uint64_t p = a.pt.p[pi];
      q = p * p;
      mu = a.pt.mu[pi];
    }
    for (uint32_t rc = blockIdx.y * kFillReqChunk; rc < n_reqs; rc += gridDim.y * kFillReqChunk) {
      const uint32_t nr = min(kFillReqChunk, n_reqs - rc);
      __syncthreads();
      for (uint32_t r = threadIdx.x; r < nr; r += blockDim.x) {
        const ReqDesc &R = a.reqs[rc + r];
        FillReq f;
        const int64_t ws = R.w0 - (int64_t)mw;
        f.A = 32ull * (uint64_t)(ws < 0 ? 0 : ws);
        f.E = R.jhi;
        f.w0 = R.w0;
        f.tile_base = R.tile_base;
        f.n_tiles = R.n_tiles;
        f.n_primes = R.n_primes;
        s_req[r] = f;
      }
      __syncthreads();
      if (!act) continue;
      for (uint32_t r = 0; r < nr; ++r) {
        const FillReq f = s_req[r];
        if (pi >= f.n_primes || f.n_tiles == 0 || f.E <= f.A) continue;
        for (uint64_t J = f.A + first_strike(f.A, q, mu); J < f.E; J += q) {
          const int64_t w = (int64_t)(J >> 5);
          uint32_t t = 0;
          if (w >= f.w0) t = (uint32_t)((uint64_t)(w - f.w0) >> g.tw_log2);
          if (t >= f.n_tiles) t = f.n_tiles - 1;  // cannot happen: J < E
          const int64_t wst = f.w0 + (int64_t)t * tw - (int64_t)mw;
          bucket_push(a, f.tile_base + t, (uint32_t)((int64_t)J - 32 * wst));
          if (t + 1 < f.n_tiles) {
            const int64_t wst1 = wst + (int64_t)tw;
            if (w >= wst1) bucket_push(a, f.tile_base + t + 1, (uint32_t)((int64_t)J - 32 * wst1));
          }
        }
      }
    }
  }
}

cudaError_t launch_bucket_fill(const BucketArgs &a, uint32_t n_large_max, uint32_t n_reqs,
                               cudaStream_t st) {
  if (n_large_max == 0 || n_reqs == 0) return cudaSuccess;
  const uint32_t threads = 256;
  uint32_t gx = (n_large_max + threads - 1) / threads;
  uint32_t gy = (n_reqs + kFillReqChunk - 1) / kFillReqChunk;
  if (gx > 4096) gx = 4096;
  if (gy > 64) gy = 64;
  bucket_fill_kernel<<<dim3(gx, gy), threads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The tile kernel.
// ---------------------------------------------------------------------------
struct ScanShared {
  unsigned long long hist[kMaxK];
  unsigned long long first[kMaxK];
  ReqDesc req;
  uint32_t tile;
  uint32_t req_idx;
};

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

__device__ __noinline__ void straggler_push(const TileArgs &a, uint32_t unres, uint64_t J0,
                                            uint32_t k0, uint32_t req) {
  while (unres) {
    const uint32_t b = __ffs(unres) - 1;
    unres &= unres - 1;
    const unsigned long long idx = atomicAdd(&a.hdr->strag_count, 1ull);
    if (idx < a.strag_cap) {
      Straggler s;
      s.n = 2ull * (J0 + b) + 1ull;
      s.k0 = k0;
      s.req = req;
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

template <int K, bool PER_N>
__device__ __forceinline__ void scan_step(uint32_t sf, uint32_t &unres, uint32_t &cnt, uint32_t &need,
                                          uint32_t pl[6], uint64_t J0, uint32_t rec_t,
                                          ScanShared &sh, const TileArgs &a) {
  const uint32_t hit = unres & sf;
  unres &= ~sf;
  cnt += __popc(hit);
  if (PER_N) {
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if ((K >> j) & 1) pl[j] |= hit;
  }
  if (hit) {
    if (need & (1u << K)) {
      need &= ~(1u << K);
      atomicMin(&sh.first[K], (unsigned long long)(2ull * (J0 + (uint64_t)(__ffs(hit) - 1)) + 1ull));
    }
    if ((uint32_t)K >= rec_t) list_append(a, sh.req, hit, J0, (uint32_t)K);
  }
}

template <bool PER_N>
__global__ void __launch_bounds__(1024, 1) tile_kernel(TileArgs a) {
  extern __shared__ uint32_t win[];
  __shared__ ScanShared sh;

  const uint32_t tid = threadIdx.x, S = blockDim.x;
  const uint32_t lane = tid & 31u, warp = tid >> 5, nwarps = S >> 5;
  const Geometry g = a.g;
  const uint32_t total = a.hdr->total_tiles;
  const uint32_t n_reqs = a.hdr->n_reqs;

  // per-block stamping strides: moving S words moves 32*S bits
  const uint32_t d0 = (32u * S) % kQ0, d1 = (32u * S) % kQ1;
  const uint32_t d2 = (32u * S) % kQ2, d3 = (32u * S) % kQ3;

  if (tid < kMaxK) {
    sh.hist[tid] = 0ull;
    sh.first[tid] = kNoN;
  }

  for (;;) {
    if (tid == 0) {
      const uint32_t t = (uint32_t)atomicAdd(&a.hdr->work_counter, 1ull);
      sh.tile = t;
      if (t < total) {
        uint32_t lo = 0, hi = n_reqs;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (a.reqs[mid].tile_base <= t) lo = mid; else hi = mid;
        }
        sh.req_idx = lo;
        sh.req = a.reqs[lo];
      }
    }
    __syncthreads();
    const uint32_t gt = sh.tile;
    if (gt >= total) break;
    const ReqDesc &R = sh.req;
    const uint32_t t = gt - R.tile_base;
    if (t >= R.n_tiles) {  // bounds check: never expected
      if (tid == 0) atomicOr(&a.hdr->status, kStBadTile);
      __syncthreads();
      continue;
    }
    const int64_t tws = R.w0 + (int64_t)t * g.tw;
    const int64_t twe = min(tws + (int64_t)g.tw, R.wend);
    const int64_t wstart = tws - (int64_t)g.mw;
    const uint32_t nwords = (uint32_t)(twe - wstart);

    // ---- 1. stamp p = 3, 5, 7, 11 --------------------------------------
    const uint32_t nz = (wstart < 0) ? (uint32_t)min((int64_t)nwords, -wstart) : 0u;
    for (uint32_t i = tid; i < nz; i += S) win[i] = 0u;  // integers below 1
    {
      uint32_t i = nz + tid;
      if (i < nwords) {
        const uint64_t abit = 32ull * (uint64_t)(wstart + (int64_t)i);
        uint32_t j0 = stamp_first(abit, kQ0), j1 = stamp_first(abit, kQ1);
        uint32_t j2 = stamp_first(abit, kQ2), j3 = stamp_first(abit, kQ3);
        for (; i < nwords; i += S) {
          const uint32_t m = __funnelshift_lc(0u, kRep0, j0) | __funnelshift_lc(0u, kRep1, j1) |
                             __funnelshift_lc(0u, 1u, j2) | __funnelshift_lc(0u, 1u, j3);
          win[i] = ~m;
          j0 = stamp_step(j0, d0, kQ0);
          j1 = stamp_step(j1, d1, kQ1);
          j2 = stamp_step(j2, d2, kQ2);
          j3 = stamp_step(j3, d3, kQ3);
        }
      }
    }
    __syncthreads();

    // ---- 2. strike the medium primes, apply the bucket ------------------
    {
      const int64_t aw = wstart < 0 ? 0 : wstart;
      const uint64_t A = 32ull * (uint64_t)aw;
      const uint32_t abias = 32u * (uint32_t)(aw - wstart);
      const uint32_t nbits = 32u * nwords;
      const uint32_t np = R.n_primes;
      const uint32_t i_dense = min(g.i_dense, np), i_large = min(g.i_large, np);
      for (uint32_t pi = g.i_med + warp; pi < i_dense; pi += nwarps) {
        const uint64_t p = a.pt.p[pi];
        const uint64_t q = p * p;
        const uint32_t q32 = (uint32_t)q;
        const uint32_t off = abias + (uint32_t)first_strike(A, q, a.pt.mu[pi]);
        for (uint32_t b = off + lane * q32; b < nbits; b += 32u * q32) strike(win, b);
      }
      for (uint32_t pi = max(i_dense, g.i_med) + tid; pi < i_large; pi += S) {
        const uint64_t p = a.pt.p[pi];
        const uint64_t q = p * p;
        for (uint64_t b = abias + first_strike(A, q, a.pt.mu[pi]); b < nbits; b += q)
          strike(win, (uint32_t)b);
      }
      const uint32_t nb = min(a.bucket_count[gt], g.bucket_cap);
      const uint32_t *bd = a.bucket_data + (size_t)gt * g.bucket_cap;
      for (uint32_t e = tid; e < nb; e += S) {
        const uint32_t b = bd[e];
        if (b < nbits) strike(win, b);
        else atomicOr(&a.hdr->status, kStBadTile);
      }
    }
    __syncthreads();

    if (R.sieve_only) {
      // ---- Algorithm 1 alone: write the core words --------------------
      for (uint32_t i = g.mw + tid; i < nwords; i += S) {
        const int64_t aw = wstart + (int64_t)i;
        const uint32_t v = valid_mask(32ull * (uint64_t)aw, R.jlo, R.jhi);
        R.bitmap_out[aw - R.w0] = win[i] & v;
      }
    } else {
      // ---- 3. word-parallel Algorithm 2 --------------------------------
      const uint32_t kwin = g.kwin, rec_t = g.rec_t;
      const uint32_t kneed = min(rec_t, kwin + 1u);
      uint32_t need = (kneed >= 32u) ? 0xFFFFFFFEu : (((1u << kneed) - 1u) & ~1u);
      uint32_t c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0;
      for (uint32_t ib = g.mw + warp * 32u; ib < nwords; ib += nwarps * 32u) {
        const uint32_t i = ib + lane;
        const bool act = i < nwords;
        const uint32_t w = act ? win[i] : 0u;
        const uint32_t wp = act ? win[i - 1] : 0u;
        const uint64_t J0 = 32ull * (uint64_t)(wstart + (int64_t)i);
        const uint32_t valid = act ? valid_mask(J0, R.jlo, R.jhi) : 0u;
        uint32_t unres = valid;
        uint32_t pl[6] = {0u, 0u, 0u, 0u, 0u, 0u};
        scan_step<1, PER_N>(__funnelshift_l(wp, w, 1), unres, c1, need, pl, J0, rec_t, sh, a);
        if (__any_sync(0xFFFFFFFFu, unres)) {
          scan_step<2, PER_N>(__funnelshift_l(wp, w, 2), unres, c2, need, pl, J0, rec_t, sh, a);
          if (__any_sync(0xFFFFFFFFu, unres)) {
            scan_step<3, PER_N>(__funnelshift_l(wp, w, 4), unres, c3, need, pl, J0, rec_t, sh, a);
            if (__any_sync(0xFFFFFFFFu, unres)) {
              scan_step<4, PER_N>(__funnelshift_l(wp, w, 8), unres, c4, need, pl, J0, rec_t, sh, a);
              if (__any_sync(0xFFFFFFFFu, unres)) {
                scan_step<5, PER_N>(__funnelshift_l(wp, w, 16), unres, c5, need, pl, J0, rec_t, sh, a);
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
                    if (need & (1u << k)) {
                      need &= ~(1u << k);
                      atomicMin(&sh.first[k],
                                (unsigned long long)(2ull * (J0 + (uint64_t)(__ffs(hit) - 1)) + 1ull));
                    }
                    if (k >= rec_t) list_append(a, R, hit, J0, k);
                  }
                }
                if (unres) straggler_push(a, unres, J0, kwin + 1u, sh.req_idx);
              }
            }
          }
        }
        if (PER_N && R.per_n_k) write_per_n(R.per_n_k, J0, R.jlo, valid, pl);
      }
      // warp totals of k = 1..5 into the tile histogram
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        c1 += __shfl_xor_sync(0xFFFFFFFFu, c1, o);
        c2 += __shfl_xor_sync(0xFFFFFFFFu, c2, o);
        c3 += __shfl_xor_sync(0xFFFFFFFFu, c3, o);
        c4 += __shfl_xor_sync(0xFFFFFFFFu, c4, o);
        c5 += __shfl_xor_sync(0xFFFFFFFFu, c5, o);
      }
      if (lane == 0) {
        if (c1) atomicAdd(&sh.hist[1], (unsigned long long)c1);
        if (c2) atomicAdd(&sh.hist[2], (unsigned long long)c2);
        if (c3) atomicAdd(&sh.hist[3], (unsigned long long)c3);
        if (c4) atomicAdd(&sh.hist[4], (unsigned long long)c4);
        if (c5) atomicAdd(&sh.hist[5], (unsigned long long)c5);
      }
    }
    __syncthreads();

    // ---- 4. tile aggregates into the range's slot ------------------------
    if (tid < kMaxK) {
      ResultSlot *slot = &a.slots[R.slot];
      const unsigned long long h = sh.hist[tid], f = sh.first[tid];
      if (h) atomicAdd(&slot->hist[tid], h);
      if (f != kNoN) atomicMin(&slot->first_n[tid], f);
      sh.hist[tid] = 0ull;
      sh.first[tid] = kNoN;
    }
    __syncthreads();
  }
}

cudaError_t tile_kernel_setup(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_tiles(const TileArgs &a, uint32_t threads, uint32_t grid, size_t smem, bool per_n,
                         cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  if (per_n)
    tile_kernel<true><<<grid, threads, smem, st>>>(a);
  else
    tile_kernel<false><<<grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sv
