// primes.cu -- the resident prime table (the "forall primes 3 <= p < sqrt(end)"
// of Algorithm 1, Sec. 3), built on the device by a segmented sieve of
// Eratosthenes, then compacted in ascending order with the per-prime constants
// the kernels need:
//   mu  = floor((2^64-1) / p^2)   Barrett (1986) constant for x mod p^2
//   inv = p^-1 mod 2^64           Newton-Hensel lifting x <- x(2 - p x)
//   lim = floor((2^64-1) / p)     Granlund-Montgomery (1994) divisibility bound
#include <cuda_runtime.h>

#include "sv_internal.h"

namespace sv {

namespace {

constexpr uint32_t kSegWords = 8192;  // 2^18 odd numbers per sieve segment
constexpr uint32_t kCountWords = 1024;
constexpr uint32_t kDivBlocks = (1u << 21) / 64 / kCountWords;  // = 32

// One block: odd primes 3 <= p <= B (B <= 46341) into out[], count into *cnt.
__global__ void base_primes_kernel(uint32_t B, uint32_t *out, uint32_t *cnt) {
  __shared__ uint32_t bits[(46341 / 2 + 1 + 31) / 32 + 1];  // bit i <-> 2i+1
  const uint32_t nb = B / 2 + 1;                            // odd numbers 1..B(|1)
  const uint32_t nw = (nb + 31) / 32;
  for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) bits[i] = 0xFFFFFFFFu;
  __syncthreads();
  for (uint32_t p = 3; p * p <= B; p += 2) {
    const bool prime = (bits[(p >> 1) >> 5] >> ((p >> 1) & 31)) & 1u;
    __syncthreads();
    if (prime)
      for (uint32_t m = p * p + 2 * p * threadIdx.x; m <= B; m += 2 * p * blockDim.x)
        atomicAnd(&bits[(m >> 1) >> 5], ~(1u << ((m >> 1) & 31)));
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    uint32_t c = 0;
    for (uint32_t i = 1; i < nb; ++i) {
      const uint32_t v = 2 * i + 1;
      if (v > B) break;
      if ((bits[i >> 5] >> (i & 31)) & 1u) out[c++] = v;
    }
    *cnt = c;
  }
}

// Segmented sieve: bit i of the global bitmap <-> odd 2i+1, 1 = prime.
__global__ void __launch_bounds__(512) seg_sieve_kernel(const uint32_t *base, const uint32_t *nbase_p,
                                                        uint64_t pmax, uint32_t *bits, uint64_t nwords) {
  __shared__ uint32_t seg[kSegWords];
  const uint32_t nbase = *nbase_p;
  for (uint64_t s = blockIdx.x; s * kSegWords < nwords; s += gridDim.x) {
    const uint64_t w0 = s * kSegWords;
    const uint32_t nw = (uint32_t)min((uint64_t)kSegWords, nwords - w0);
    for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) seg[i] = 0xFFFFFFFFu;
    __syncthreads();
    const uint64_t lo = 64 * w0 + 1;             // first odd integer of the segment
    const uint64_t hi = 64 * (w0 + nw);          // exclusive
    // small primes: all threads of the block stride one prime's multiples
    uint32_t pi = 0;
    for (; pi < nbase; ++pi) {
      const uint64_t p = base[pi];
      if (p > 2048) break;
      uint64_t m = p * p;
      if (m < lo) {
        m = ((lo + p - 1) / p) * p;
        if (!(m & 1)) m += p;
      }
      for (uint64_t x = m + 2 * p * threadIdx.x; x < hi; x += 2 * p * blockDim.x) {
        const uint32_t bi = (uint32_t)((x - lo) >> 1);
        atomicAnd(&seg[bi >> 5], ~(1u << (bi & 31)));
      }
    }
    // larger primes: one thread per prime
    for (uint32_t j = pi + threadIdx.x; j < nbase; j += blockDim.x) {
      const uint64_t p = base[j];
      uint64_t m = p * p;
      if (m < lo) {
        m = ((lo + p - 1) / p) * p;
        if (!(m & 1)) m += p;
      }
      for (uint64_t x = m; x < hi; x += 2 * p) {
        const uint32_t bi = (uint32_t)((x - lo) >> 1);
        atomicAnd(&seg[bi >> 5], ~(1u << (bi & 31)));
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) {
      uint32_t v = seg[i];
      const uint64_t gw = w0 + i;
      if (gw == 0) v &= ~1u;  // 1 is not prime
      // clear bits of odd numbers > pmax
      const uint64_t first = 64 * gw + 1;
      if (first > pmax) v = 0;
      else if (first + 62 > pmax) {
        const uint32_t keep = (uint32_t)((pmax - first) / 2 + 1);  // 1..31
        v &= (keep >= 32) ? 0xFFFFFFFFu : ((1u << keep) - 1u);
      }
      bits[gw] = v;
    }
    __syncthreads();
  }
}

__global__ void count_kernel(const uint32_t *bits, uint64_t nwords, uint32_t *counts) {
  __shared__ uint32_t red[32];
  const uint64_t w = (uint64_t)blockIdx.x * kCountWords + threadIdx.x;
  uint32_t c = (w < nwords) ? __popc(bits[w]) : 0u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    c = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0u;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
  }
}

// Single block: exclusive scan of counts[0..n) in place; total into *total.
__global__ void scan_kernel(uint32_t *counts, uint32_t n, uint32_t *total) {
  __shared__ uint32_t carry;
  __shared__ uint32_t red[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = (i < n) ? counts[i] : 0u;
    // inclusive warp scan
    uint32_t x = v;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t t = (lane < (blockDim.x >> 5)) ? red[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
        if (lane >= (uint32_t)o) t += y;
      }
      red[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t before = carry + (warp ? red[warp - 1] : 0u) + x - v;
    if (i < n) counts[i] = before;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void compact_kernel(const uint32_t *bits, uint64_t nwords, const uint32_t *offsets,
                               uint32_t *p_out, uint64_t *mu_out, uint64_t *inv_out, uint64_t *lim_out,
                               uint32_t n_div_cap) {
  __shared__ uint32_t red[32];
  const uint64_t w = (uint64_t)blockIdx.x * kCountWords + threadIdx.x;
  const uint32_t v = (w < nwords) ? bits[w] : 0u;
  const uint32_t c = __popc(v);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) red[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = (lane < (blockDim.x >> 5)) ? red[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= (uint32_t)o) t += y;
    }
    red[lane] = t;
  }
  __syncthreads();
  uint32_t idx = offsets[blockIdx.x] + (warp ? red[warp - 1] : 0u) + x - c;
  uint32_t m = v;
  while (m) {
    const uint32_t b = __ffs(m) - 1;
    m &= m - 1;
    const uint64_t p = 64 * w + 2 * b + 1;
    p_out[idx] = (uint32_t)p;
    mu_out[idx] = ~0ull / (p * p);
    if (idx < n_div_cap) {
      uint64_t y = p;  // correct to 3 bits: p*p = 1 mod 8
      for (int it = 0; it < 5; ++it) y *= 2ull - p * y;
      inv_out[idx] = y;
      lim_out[idx] = ~0ull / p;
    }
    ++idx;
  }
}

}  // namespace

// Builds the table of odd primes <= pmax (pmax < 2^32).  Device arrays are
// allocated here and owned by the caller.
cudaError_t build_prime_table(uint64_t pmax, uint32_t **d_p, uint64_t **d_mu, uint64_t **d_inv,
                              uint64_t **d_lim, uint32_t **d_bits_out, uint64_t *bits_words, uint32_t *n_out,
                              uint32_t *n_div_out, cudaStream_t st) {
  cudaError_t e;
  *d_p = nullptr;
  *d_mu = *d_inv = *d_lim = nullptr;
  *d_bits_out = nullptr;
  *bits_words = 0;
  *n_out = *n_div_out = 0;
  if (pmax < 3) pmax = 3;
  const uint64_t B = host_isqrt(pmax);
  const uint64_t nwords = (pmax / 2 + 1 + 31) / 32;
  const uint32_t nblocks = (uint32_t)((nwords + kCountWords - 1) / kCountWords);
  uint32_t *d_base = nullptr, *d_nbase = nullptr, *d_bits = nullptr, *d_counts = nullptr, *d_total = nullptr;
  uint32_t h_total = 0;
  uint32_t n_div = 0;
  if ((e = cudaMalloc(&d_base, sizeof(uint32_t) * 8192)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&d_nbase, sizeof(uint32_t) * 2)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&d_bits, sizeof(uint32_t) * nwords)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&d_counts, sizeof(uint32_t) * (nblocks + 1))) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&d_total, sizeof(uint32_t))) != cudaSuccess) goto done;
  base_primes_kernel<<<1, 512, 0, st>>>((uint32_t)(B < 3 ? 3 : B), d_base, d_nbase);
  if ((e = cudaGetLastError()) != cudaSuccess) goto done;
  {
    uint64_t segs = (nwords + kSegWords - 1) / kSegWords;
    const uint32_t grid = (uint32_t)(segs < 4096 ? segs : 4096);
    seg_sieve_kernel<<<grid, 512, 0, st>>>(d_base, d_nbase, pmax, d_bits, nwords);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
  }
  count_kernel<<<nblocks, kCountWords, 0, st>>>(d_bits, nwords, d_counts);
  if ((e = cudaGetLastError()) != cudaSuccess) goto done;
  scan_kernel<<<1, 1024, 0, st>>>(d_counts, nblocks, d_total);
  if ((e = cudaGetLastError()) != cudaSuccess) goto done;
  if ((e = cudaMemcpyAsync(&h_total, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    goto done;
  // primes below 2^21 get the divisibility constants (every cube root below
  // 2^62 is smaller, and p^3 stays below 2^64): they are the primes of the
  // first 2^21 / 64 bitmap words, i.e. of the first kDivBlocks count blocks.
  if (nblocks > kDivBlocks) {
    if ((e = cudaMemcpyAsync(&n_div, d_counts + kDivBlocks, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      goto done;
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto done;
  {
    const size_t n = h_total ? h_total : 1;
    if (nblocks <= kDivBlocks) n_div = h_total;
    if ((e = cudaMalloc(d_p, sizeof(uint32_t) * n)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(d_mu, sizeof(uint64_t) * n)) != cudaSuccess) goto done;
    const size_t nd = n_div ? n_div : 1;
    if ((e = cudaMalloc(d_inv, sizeof(uint64_t) * nd)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(d_lim, sizeof(uint64_t) * nd)) != cudaSuccess) goto done;
    compact_kernel<<<nblocks, kCountWords, 0, st>>>(d_bits, nwords, d_counts, *d_p, *d_mu, *d_inv, *d_lim,
                                                    n_div);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto done;
  }
  *n_out = h_total;
  *n_div_out = n_div;
  *d_bits_out = d_bits;  // the bitmap stays: the bucket fill tests primality with it
  *bits_words = nwords;
  d_bits = nullptr;
done:
  cudaFree(d_base);
  cudaFree(d_nbase);
  cudaFree(d_bits);
  cudaFree(d_counts);
  cudaFree(d_total);
  if (e != cudaSuccess) {
    cudaFree(*d_p);
    cudaFree(*d_mu);
    cudaFree(*d_inv);
    cudaFree(*d_lim);
    *d_p = nullptr;
    *d_mu = *d_inv = *d_lim = nullptr;
  }
  return e;
}

}  // namespace sv
