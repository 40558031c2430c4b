// peaks.cu -- measured peaks for the rooflines of this library's kernels.
//
// The tile kernel (Algorithms 1 and 2 of Sec. 3, fused) is bound by two
// on-chip resources, neither of which a vendor figure states for this GPU:
//   * the shared-memory atomic unit: every strike of Algorithm 1 is one
//     32-bit atomicAnd on the window in shared memory;
//   * the integer pipes: the word-parallel Algorithm 2 is funnel shifts,
//     AND-NOTs, population counts and adds.
// Each probe below runs one of those operations at full occupancy, on every
// SM, for a few milliseconds, timed with CUDA events on the context's stream.
// Nothing is read back but one word per thread (so that no work can be
// dropped), and no device setting is touched.
#include <cuda_runtime.h>

#include "ctx.h"

namespace sv {
namespace {

constexpr uint32_t kProbeThreads = 1024;
constexpr uint32_t kProbeBlocksPerSm = 2;
constexpr uint32_t kAtomWords = 16384;  // 64 KB of shared memory per block, like a tile window

// Shared-memory atomicAnd, lanes of a warp on 32 distinct banks (stride 1
// word), every iteration a new row of the array.
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
probe_atom_banks(uint32_t iters, uint32_t *sink) {
  __shared__ uint32_t w[kAtomWords];
  for (uint32_t i = threadIdx.x; i < kAtomWords; i += blockDim.x) w[i] = 0xFFFFFFFFu;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t row = warp * 32u;
  const uint32_t mask = ~(1u << lane);
#pragma unroll 8
  for (uint32_t it = 0; it < iters; ++it) {
    atomicAnd(&w[(row + lane) & (kAtomWords - 1)], mask);
    row += 32u * 32u;  // the next row of this warp: 32 rows of 32 words per sweep
  }
  __syncthreads();
  sink[blockIdx.x * blockDim.x + threadIdx.x] = w[threadIdx.x & (kAtomWords - 1)];
}

// The odd primes 13 .. 379: the squares the dense-strike probe cycles through.
constexpr uint32_t kProbePrimes = 70;
__constant__ uint16_t c_probe_primes[kProbePrimes] = {
    13,  17,  19,  23,  29,  31,  37,  41,  43,  47,  53,  59,  61,  67,  71,  73,  79,  83,  89,  97,
    101, 103, 107, 109, 113, 127, 131, 137, 139, 149, 151, 157, 163, 167, 173, 179, 181, 191, 193, 197,
    199, 211, 223, 227, 229, 233, 239, 241, 251, 257, 263, 269, 271, 277, 281, 283, 293, 307, 311, 313,
    317, 331, 337, 347, 349, 353, 359, 367, 373, 379};

// Shared-memory atomicAnd in the tile kernel's own pattern: the lanes of a
// warp strike the bits off + q (lane + 32 m) of one prime square q (the
// cooperative dense strikes of a 2^19-bit window), moving to the next prime
// every 16 strikes per lane.
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
probe_atom_strikes(uint32_t iters, uint32_t *sink) {
  __shared__ uint32_t w[kAtomWords];
  for (uint32_t i = threadIdx.x; i < kAtomWords; i += blockDim.x) w[i] = 0xFFFFFFFFu;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t k = (warp * 7u) % kProbePrimes;
  uint32_t q = (uint32_t)c_probe_primes[k] * c_probe_primes[k];
  uint32_t b = lane * q + warp * 977u;
  constexpr uint32_t kBits = 32u * kAtomWords;
  for (uint32_t it = 0; it < iters; ++it) {
    b &= kBits - 1u;  // stays inside the window
    atomicAnd(&w[b >> 5], __funnelshift_l(0xFFFFFFFEu, 0xFFFFFFFEu, b));
    b += 32u * q;
    if ((it & 15u) == 15u) {
      k = k + 1u == kProbePrimes ? 0u : k + 1u;
      q = (uint32_t)c_probe_primes[k] * c_probe_primes[k];
      b = lane * q + (b & 4095u);
    }
  }
  __syncthreads();
  sink[blockIdx.x * blockDim.x + threadIdx.x] = w[threadIdx.x & (kAtomWords - 1)];
}

// The integer mix of the scan (one step of Algorithm 2 on one word): funnel
// shift by a constant, AND-NOT (with an OR that keeps the chain alive),
// population count, add; kMixChains independent chains per thread (as many as
// the 32 registers of a full-occupancy thread hold).  Counted as four
// operations per step.
constexpr int kMixChains = 6;
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
probe_scan_mix(uint32_t iters, uint32_t seed, uint32_t *sink) {
  uint32_t w[kMixChains], u[kMixChains], c[kMixChains];
#pragma unroll
  for (int j = 0; j < kMixChains; ++j) {
    w[j] = seed * (threadIdx.x + 977u * j) + blockIdx.x;
    u[j] = ~w[j];
    c[j] = 0;
  }
  uint32_t p = seed ^ threadIdx.x;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kMixChains; ++j) {
      const uint32_t sf = __funnelshift_l(p, w[j], 1u << (j & 3));
      u[j] = (u[j] & ~sf) | w[(j + 1) % kMixChains];
      c[j] += __popc(u[j]);
    }
    p += c[kMixChains - 1];
  }
  uint32_t r = p;
#pragma unroll
  for (int j = 0; j < kMixChains; ++j) r ^= c[j] + u[j];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Plain 32-bit logic/add throughput (the fastest integer operations): eight
// independent chains of a three-input logic operation and an add.
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
probe_int_alu(uint32_t iters, uint32_t seed, uint32_t *sink) {
  uint32_t a[8], b[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    a[j] = seed * (threadIdx.x + 31u * j);
    b[j] = seed ^ (blockIdx.x + 7u * j);
  }
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      a[j] = (a[j] & b[j]) ^ (b[j] | it);
      b[j] += a[j];
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) r ^= a[j] + b[j];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Population counts: eight independent chains of add, popc, shift, xor (one
// popc in four operations).
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
probe_popc(uint32_t iters, uint32_t seed, uint32_t *sink) {
  uint32_t a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed * (threadIdx.x + 131u * j) + blockIdx.x;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (a[j] << 1) ^ __popc(a[j] + it);
  }
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) r ^= a[j];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Runs one probe kernel: a warm-up launch, then `reps` timed launches; the
// best time per launch.
template <class F>
sv_status time_probe(cudaStream_t st, int reps, F launch, double *best_ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return SV_ECUDA;
  }
  sv_status s = SV_OK;
  launch();
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) s = SV_ECUDA;
  double best = 1e300;
  for (int r = 0; r < reps && !s; ++r) {
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      s = SV_ECUDA;
      break;
    }
    if (ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *best_ms = best;
  return s;
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_measure_peaks(sv_ctx *c, sv_peaks *out) {
  if (!c || !out) return SV_EINVAL;
  DevGuard dev_guard(c->device);
  if (!dev_guard.ok) return SV_ECUDA;
  std::lock_guard<std::mutex> lk(c->mu);
  const cudaStream_t st = c->stream;
  const uint32_t grid = (uint32_t)c->num_sms * kProbeBlocksPerSm;
  const uint64_t threads = (uint64_t)grid * kProbeThreads;
  uint32_t *sink = nullptr;
  if (cudaMalloc(&sink, threads * sizeof(uint32_t)) != cudaSuccess) return SV_ENOMEM;
  sv_status s = SV_OK;
  double ms = 0.0;
  const int reps = 5;
  const uint32_t it_atom = 1u << 14, it_alu = 1u << 13;
  *out = sv_peaks{};
  if (!s) s = time_probe(st, reps, [&] { probe_atom_banks<<<grid, kProbeThreads, 0, st>>>(it_atom, sink); }, &ms);
  if (!s) out->smem_atomic_per_s = (double)threads * it_atom / (ms * 1e-3);
  if (!s) s = time_probe(st, reps, [&] { probe_atom_strikes<<<grid, kProbeThreads, 0, st>>>(it_atom, sink); }, &ms);
  if (!s) out->smem_atomic_strike_per_s = (double)threads * it_atom / (ms * 1e-3);
  if (!s) s = time_probe(st, reps, [&] { probe_scan_mix<<<grid, kProbeThreads, 0, st>>>(it_alu, 12345u, sink); }, &ms);
  if (!s) out->scan_mix_ops_per_s = (double)threads * it_alu * kMixChains * 4 / (ms * 1e-3);
  if (!s) s = time_probe(st, reps, [&] { probe_int_alu<<<grid, kProbeThreads, 0, st>>>(it_alu, 777u, sink); }, &ms);
  if (!s) out->int_alu_ops_per_s = (double)threads * it_alu * 8 * 2 / (ms * 1e-3);
  if (!s) s = time_probe(st, reps, [&] { probe_popc<<<grid, kProbeThreads, 0, st>>>(it_alu, 99u, sink); }, &ms);
  if (!s) out->popc_per_s = (double)threads * it_alu * 8 / (ms * 1e-3);
  out->sms = (uint32_t)c->num_sms;
  int khz = 0;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device) == cudaSuccess) out->sm_clock_max_mhz = khz / 1000.0;
  cudaFree(sink);
  return s;
}
