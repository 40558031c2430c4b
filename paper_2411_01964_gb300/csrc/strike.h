// strike.h -- where the odd multiples of p^2 fall in the odd-only bitmap
// (Algorithm 1 of Sec. 3: bit J stands for the odd integer 2J + 1).
#pragma once

#include <cstdint>

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

// floor(sqrt(r)) by Newton's iteration from above (integer only): the start
// 2^ceil(bits/2) is at least the root, and the iterates fall to it.
__device__ __forceinline__ uint64_t isqrt_u64(uint64_t r) {
  if (r < 2) return r;
  const int bits = 64 - __clzll((long long)r);
  uint64_t x = 1ull << ((bits + 1) >> 1);
  for (;;) {
    const uint64_t y = (x + r / x) >> 1;
    if (y >= x) return x;
    x = y;
  }
}

}  // namespace sv
