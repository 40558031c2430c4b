// lists.cu -- the ordered list of each range (Sec. 3 "Collecting the
// results"): the n with mink(n) >= T, ascending, gathered from the entries
// the tile kernel staged per tile.
#include <cuda_runtime.h>

#include "sv_internal.h"

namespace sv {

// ---------------------------------------------------------------------------
// The ordered list (mode 0).  The launch's tiles are cut into blocks of 128,
// one thread per tile (small blocks, so that a launch's tiles spread over
// the SMs); a tile's place in its range's list is the number of
// entries its range staged in the tiles before it: the block's inclusive
// scan (segmented at range starts) plus, for a range that began in an
// earlier block, the sum of its staged counts there.  Each tile's few
// entries arrive unordered and are ranked among themselves, so the list
// comes out ascending.  Entries past the range's list capacity are counted,
// not stored: the smallest ones are kept.  The thread of a range's last tile
// writes the range's total.
// ---------------------------------------------------------------------------
constexpr uint32_t kCompactBlock = 128;
constexpr uint32_t kCompactWarps = kCompactBlock / 32;
constexpr uint32_t kRankRegs = 8;  // staged entries of a tile ranked in registers (more: from memory)
static_assert(kRankRegs % 2 == 0 && kRankRegs <= kStageCap, "the vector loads read whole pairs inside one slot");

__device__ __forceinline__ uint32_t range_of_tile(const ReqDesc *reqs, uint32_t n_reqs, uint32_t t) {
  uint32_t lo = 0, hi = n_reqs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (reqs[mid].tile_base <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kCompactBlock) list_compact_kernel(CompactArgs a) {
  __shared__ uint32_t incl_s[kCompactBlock];
  __shared__ uint32_t wsum[kCompactWarps];
  __shared__ uint32_t carry_s;
  const uint32_t n_reqs = a.hdr->n_reqs, total = a.hdr->total_tiles;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t nblk = (total + kCompactBlock - 1) / kCompactBlock;
  for (uint32_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const uint32_t b0 = blk * kCompactBlock;
    const uint32_t t = b0 + tid;
    const bool act = t < total;
    const uint32_t r = act ? range_of_tile(a.reqs, n_reqs, t) : 0u;
    const ReqDesc *R = act ? &a.reqs[r] : nullptr;
    const bool listed = act && !R->sieve_only && t - R->tile_base < R->n_tiles;
    const uint32_t cnt = listed ? min(a.stage_cnt[t], a.stage_cap) : 0u;
    // the tile's first kRankRegs staged entries and their k, loaded before
    // the scan so that the loads overlap it (a tile's staging slot is
    // 16-byte aligned and holds kStageCap >= kRankRegs entries: the loads
    // stay inside it; entries past cnt are ignored)
    ulonglong2 pre[kRankRegs / 2];
    uint64_t pre_k = 0;
    if (listed) {
      const ulonglong2 *sn2 = reinterpret_cast<const ulonglong2 *>(a.stage_n + (size_t)t * kStageCap);
#pragma unroll
      for (uint32_t h = 0; h < kRankRegs / 2; ++h) pre[h] = sn2[h];
      pre_k = *reinterpret_cast<const uint64_t *>(a.stage_k + (size_t)t * kStageCap);
    }
    // carry-in: the staged entries of the block's first range before the block
    if (tid == 0) carry_s = 0;
    __syncthreads();
    {
      const uint32_t r0 = range_of_tile(a.reqs, n_reqs, b0);
      const uint32_t tb0 = a.reqs[r0].tile_base;
      uint32_t part = 0;
      if (!a.reqs[r0].sieve_only && tb0 < b0) {
        // 16-byte loads over the whole groups of four counts (the count
        // array's start is 16-byte aligned; else one count at a time)
        const uint32_t v0 = (tb0 + 3u) >> 2, v1 = b0 >> 2;
        const bool vec = ((uintptr_t)a.stage_cnt & 15u) == 0u && v0 < v1;
        const uint32_t s_end = vec ? 4u * v0 : b0;
        for (uint32_t u = tb0 + tid; u < s_end; u += kCompactBlock) part += min(a.stage_cnt[u], a.stage_cap);
        if (vec) {
          const uint4 *c4 = reinterpret_cast<const uint4 *>(a.stage_cnt);
#pragma unroll 8
          for (uint32_t v = v0 + tid; v < v1; v += kCompactBlock) {
            const uint4 x = c4[v];
            part += min(x.x, a.stage_cap) + min(x.y, a.stage_cap) + min(x.z, a.stage_cap) + min(x.w, a.stage_cap);
          }
          for (uint32_t u = 4u * v1 + tid; u < b0; u += kCompactBlock) part += min(a.stage_cnt[u], a.stage_cap);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
      if (lane == 0 && part) atomicAdd(&carry_s, part);
    }
    // inclusive block scan of the counts
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = lane < kCompactWarps ? wsum[lane] : 0u;
      uint32_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
        if (lane >= (uint32_t)o) wi += y;
      }
      if (lane < kCompactWarps) wsum[lane] = wi - w;
    }
    __syncthreads();
    incl += wsum[warp];
    incl_s[tid] = incl;
    __syncthreads();
    if (listed) {
      // entries of this range in the block's tiles before t, plus the carry-in
      const uint32_t s0 = R->tile_base > b0 ? R->tile_base - b0 : 0u;
      uint64_t pos = (uint64_t)(incl - cnt) - (s0 ? incl_s[s0 - 1] : 0u);
      if (R->tile_base < b0) pos += carry_s;
      const uint64_t *sn = a.stage_n + (size_t)t * kStageCap;
      const uint8_t *sk = a.stage_k + (size_t)t * kStageCap;
      if (cnt <= kRankRegs) {
        // the usual case: a few entries, ranked in registers
        uint64_t v[kRankRegs];
#pragma unroll
        for (uint32_t h = 0; h < kRankRegs / 2; ++h) {
          v[2 * h] = 2 * h < cnt ? pre[h].x : ~0ull;
          v[2 * h + 1] = 2 * h + 1 < cnt ? pre[h].y : ~0ull;
        }
        const uint64_t ks = pre_k;  // k of entry e: byte e
#pragma unroll
        for (uint32_t e = 0; e < kRankRegs; ++e) {
          if (e >= cnt) break;
          uint32_t rank = 0;
#pragma unroll
          for (uint32_t f = 0; f < kRankRegs; ++f) rank += v[f] < v[e] ? 1u : 0u;
          if (pos + rank < R->list_cap) {
            a.list_n[R->list_off + pos + rank] = v[e];
            a.list_k[R->list_off + pos + rank] = (uint8_t)(ks >> (8 * e));
          }
        }
      } else {
        for (uint32_t e = 0; e < cnt; ++e) {
          const uint64_t n = sn[e];
          uint32_t rank = 0;
          for (uint32_t f = 0; f < cnt; ++f) rank += sn[f] < n ? 1u : 0u;
          if (pos + rank < R->list_cap) {
            a.list_n[R->list_off + pos + rank] = n;
            a.list_k[R->list_off + pos + rank] = sk[e];
          }
        }
      }
      if (t - R->tile_base == R->n_tiles - 1) a.slots[R->slot].list_count = pos + cnt;
    }
    __syncthreads();  // the shared arrays are reused by the next block
  }
}

cudaError_t launch_compact(const CompactArgs &a, uint32_t grid, cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  list_compact_kernel<<<grid, kCompactBlock, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sv
