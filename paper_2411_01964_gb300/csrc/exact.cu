// exact.cu -- the exact squarefree test behind stragglers and point queries.
//
// Algorithm 2 (Sec. 3) only reads the sieve.  Where n - 2^k falls below a
// tile's look-back window (a "straggler"), or for a single point n, the flag
// is decided directly, exactly and without floating point:
//   s (odd, >= 1) is squarefree  <=>  no prime p with p^3 <= s has p^2 | s,
//   and the cofactor r = s / prod{p | s : p^3 <= s} is not a perfect square.
// (After removing every prime factor p with p^3 <= s, r <= s has only prime
// factors q with q^3 > s >= r, so r is 1, a prime, a product of two distinct
// primes, or q^2; only the last is not squarefree.)  Divisibility by p uses the
// Granlund-Montgomery (1994, Sec. 9) test with p^-1 mod 2^64, and the exact
// quotient s/p is s * p^-1 mod 2^64.  One warp tests one s, lanes striding the
// prime table; the warp stops at the first p with p^2 | s.
#include <cuda_runtime.h>

#include "strike.h"
#include "sv_internal.h"

namespace sv {

// Warp-cooperative: is the odd number s >= 1 squarefree?  All 32 lanes call
// it with the same s and get the same answer.
__device__ bool warp_squarefree(uint64_t s, const PrimeTab &pt) {
  const uint32_t lane = threadIdx.x & 31u;
  if (s < 9) return true;  // 1, 3, 5, 7
  uint64_t r = s;
  for (uint32_t base = 0; base < pt.n_div; base += 32) {
    const uint32_t i = base + lane;
    bool in = false, div = false, sq = false;
    uint64_t inv = 0;
    if (i < pt.n_div) {
      const uint64_t p = pt.p[i];
      in = p * p * p <= s;  // p < 2^21: no overflow
      if (in) {
        inv = pt.inv[i];
        const uint64_t lim = pt.lim[i];
        const uint64_t t = s * inv;  // s / p when p | s
        if (t <= lim) {
          div = true;
          sq = (t * inv) <= lim;  // p | s/p
        }
      }
    }
    if (__any_sync(0xFFFFFFFFu, sq)) return false;
    uint32_t m = __ballot_sync(0xFFFFFFFFu, div);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      r *= __shfl_sync(0xFFFFFFFFu, inv, src);  // exact division by that prime
    }
    if (!__any_sync(0xFFFFFFFFu, in)) break;  // primes ascend: no lane left with p^3 <= s
  }
  if (r == 1) return true;
  const uint64_t x = isqrt_u64(r);
  return x * x != r;
}

// mink continued from k0 for odd n (warp-cooperative); 255 if none.
__device__ uint32_t warp_min_k_from(uint64_t n, uint32_t k0, const PrimeTab &pt) {
  for (uint32_t k = k0; k < 63 && (1ull << k) < n; ++k)
    if (warp_squarefree(n - (1ull << k), pt)) return k;
  return kFailK;
}

__global__ void __launch_bounds__(256) straggler_kernel(StragArgs a) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long cnt = a.hdr->strag_count;
  if (cnt > a.strag_cap) cnt = a.strag_cap;
  for (uint64_t e = gw; e < cnt; e += nw) {
    const Straggler st = a.strag[e];
    const uint32_t k = warp_min_k_from(st.n, st.k0, a.pt);
    if (lane == 0) {
      const ReqDesc &R = a.reqs[st.req];
      ResultSlot *slot = &a.slots[R.slot];
      if (k != kFailK) {
        atomicAdd(&slot->hist[k], 1ull);
        atomicMin(&slot->first_n[k], (unsigned long long)st.n);
        if (k >= a.rec_t) {
          if (a.stage_n) {
            // ordered lists: join the staged entries of the tile holding n
            const uint64_t t = ((((st.n - 1) >> 1) >> 5) - (uint64_t)R.w0) >> a.tw_log2;
            if (t < R.n_tiles) {
              const uint32_t gt = R.tile_base + (uint32_t)t;
              const uint32_t e = atomicAdd(&a.stage_cnt[gt], 1u);
              if (e < a.stage_cap) {
                a.stage_n[(size_t)gt * kStageCap + e] = st.n;
                a.stage_k[(size_t)gt * kStageCap + e] = (uint8_t)k;
              } else {
                atomicOr(&a.hdr->status, kStListStage);
              }
            } else {
              atomicOr(&a.hdr->status, kStBadTile);
            }
          } else {
            const unsigned long long idx = atomicAdd(&slot->list_count, 1ull);
            if (idx < R.list_cap) {
              a.list_n[R.list_off + idx] = st.n;
              a.list_k[R.list_off + idx] = (uint8_t)k;
            }
          }
        }
      } else {
        const unsigned long long idx = atomicAdd(&slot->fail_count, 1ull);
        if (idx < R.fail_cap) a.fail_n[R.fail_off + idx] = st.n;
      }
      if (R.per_n_k) R.per_n_k[(st.n - R.nlo) >> 1] = (uint8_t)k;
    }
  }
}

cudaError_t launch_stragglers(const StragArgs &a, uint32_t grid, cudaStream_t st) {
  straggler_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) points_kernel(PrimeTab pt, const uint64_t *pts, uint64_t count,
                                                     uint8_t *out) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t e = gw; e < count; e += nw) {
    const uint64_t n = pts[e];
    uint32_t k = 0;
    if (n >= 3 && (n & 1ull)) k = warp_min_k_from(n, 1, pt);
    if (lane == 0) out[e] = (uint8_t)k;
  }
}

cudaError_t launch_points(PrimeTab pt, const uint64_t *pts, uint64_t count, uint8_t *out, uint32_t grid,
                          cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  points_kernel<<<grid, 256, 0, st>>>(pt, pts, count, out);
  return cudaGetLastError();
}

}  // namespace sv
