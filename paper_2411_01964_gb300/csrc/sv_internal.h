// sv_internal.h -- types shared by the kernels and the host runtime of the
// GPU library (never by the CPU oracle).
//
// Bit layout used everywhere on the device: bit J (J >= 0) stands for the odd
// integer 2J + 1, word a holds bits 32a .. 32a+31 (LSB first), i.e. the odd
// integers 64a+1 .. 64a+63.  With this layout n - 2^k (k >= 1) sits exactly
// 2^(k-1) bits below n, which is what the word-parallel form of Algorithm 2
// (Sec. 3) exploits: k <= 5 are funnel shifts inside a word pair, k >= 6 are
// whole-word offsets 2^(k-6).
#pragma once

#include <cstdint>

namespace sv {

constexpr int kMaxK = 64;
// ReqDesc::n_primes of a range whose prime count and interval roots the init
// kernel computes (the host plans them itself for launches of few ranges)
constexpr uint32_t kPlanOnDevice = 0xFFFFFFFFu;
constexpr uint32_t kHostPlanMax = 32;  // ranges per launch the host plans itself
constexpr uint8_t kFailK = 255;
constexpr unsigned long long kNoN = ~0ull;

// Status bits raised by the kernels (ORed into a device word).
enum : uint32_t {
  kStBucketOverflow = 1u << 0,  // a tile bucket was full: rerun with a larger one
  kStStragOverflow = 1u << 1,   // straggler queue full: rerun with a larger one
  kStBadTile = 1u << 2,         // a tile index failed a bounds check
  kStListStage = 1u << 3,       // a tile's staged list was full: rerun with the unordered list path
  kStTimeout = 1u << 4,         // a bounded wait for a bulk copy ran out (SV_ETIMEDOUT)
};

// List entries (mink >= T) a tile stages for the ordered list (mode 0): the
// tile kernel's shared buffer and the stride of the per-tile staging slots.
constexpr uint32_t kStageCap = 128;

// Resident table of the odd primes 3 <= p <= pmax (ascending), structure of
// arrays.  mu[i] = floor((2^64-1) / p^2) is the Barrett (1986) constant for
// x mod p^2; inv[i] = p^-1 mod 2^64 and lim[i] = floor((2^64-1)/p) give the
// Granlund-Montgomery (1994, Sec. 9) divisibility test  p | x  <=>
// x * inv mod 2^64 <= lim.  inv/lim exist for the first n_div primes (all
// p < 2^21, enough for every cube root below 2^62).
struct PrimeTab {
  const uint32_t *p;
  const uint64_t *mu;
  const uint64_t *inv;
  const uint64_t *lim;
  const uint32_t *bits;  // bit i of the bitmap <-> odd 2i+1 is prime (up to the table's limit)
  uint64_t bits_words;
  uint32_t n;
  uint32_t n_div;
};

// One range of a launch, in device memory.
struct ReqDesc {
  uint64_t lo, hi;      // as given
  uint64_t nlo;         // first odd n >= max(lo, 3)  (>= hi: empty)
  uint64_t jlo, jhi;    // valid bits [jlo, jhi)
  int64_t w0;           // absolute word where tile 0's core starts (= jlo >> 5)
  int64_t wend;         // one past the last absolute word holding a valid bit
  uint32_t n_tiles;     // tiles of this range
  uint32_t tile_base;   // global index of tile 0
  uint32_t slot;        // result slot
  uint32_t n_primes;    // primes p with p^2 < hi (p <= isqrt(hi - 1)); kPlanOnDevice: the init kernel
                        // counts them (and sets sq_lo, sq_hi), for launches of many ranges
  uint8_t *per_n_k;     // optional device output, index (n - nlo) / 2
  uint64_t list_off, list_cap;  // this range's region of the list arena
  uint64_t fail_off, fail_cap;  // this range's region of the failure arena
  uint32_t sieve_only;  // 1: write the sieved words to bitmap_out, no scan
  // floor(sqrt(2A)) and floor(sqrt(2E - 1)) for the window bits [A, E) the
  // bucket fill covers (A = 32 max(w0 - mw, 0), E = jhi): the integer square
  // roots of the ends of its odd-multiple interval, set by the init kernel
  uint32_t sq_lo, sq_hi;
  uint32_t pad;
  // the largest odd multiplier j with j p_hyb^2 <= 2 jhi - 1 (the bucket fill's
  // multiplier items; 0: none), planned with n_primes
  uint64_t j_max;
  uint32_t *bitmap_out; // sieve_only: word (a - w0) receives absolute word a
  // scan from device memory (the plain path): bitmap word (a - bitmap_w0)
  // holds absolute word a for every word of the range's windows; the tile
  // copies its window from there instead of sieving it (null: sieve)
  const uint32_t *bitmap_in;
  int64_t bitmap_w0;
};

// Per-range aggregates, accumulated with atomics.
struct ResultSlot {
  unsigned long long hist[kMaxK];
  unsigned long long first_n[kMaxK];
  unsigned long long list_count;
  unsigned long long fail_count;
  unsigned long long pad[6];
};

// n whose n - 2^k left the tile's look-back window before a squarefree value
// was found; the exact test continues at k0.
struct Straggler {
  uint64_t n;
  uint32_t k0;
  uint32_t req;
};

// Device header of a launch: sizes the persistent kernels read at run time,
// so one captured graph serves every batch that fits the buffers.
struct LaunchHeader {
  uint32_t n_reqs;
  uint32_t total_tiles;
  uint32_t max_primes;      // max over requests of n_primes
  uint32_t pad;
  unsigned long long work_counter;  // tile queue head
  unsigned long long strag_count;
  uint32_t status;
  uint32_t pad2;
  unsigned long long j_max;  // max over requests of ReqDesc::j_max (trims the bucket fill's multiplier slices)
  // the scan pass's bounded wait for a window's bulk load, in SM clocks (0:
  // the default, about a second); with skip_bulk_loads set the loads are not
  // issued at all, so every wait runs out (sv_inject_bulk_timeout tests that
  // path; nothing is in flight when the blocks give up)
  unsigned long long bulk_wait_cycles;
  uint32_t skip_bulk_loads;
  uint32_t pad3;
  // the longest range of the launch, in bits (jhi - jlo): the bucket fill
  // cuts the hits of its smallest Barrett primes into segments of the range
  // when the launch has few ranges (0: no cut)
  unsigned long long fill_span;
};

struct Geometry {
  uint32_t tw;        // core words per tile (2^(tile_log2 - 5))
  uint32_t mw;        // look-back words (2^(margin_log2 - 6))
  uint32_t kwin;      // largest k decided inside a window (= margin_log2)
  uint32_t rec_t;     // record threshold T
  uint32_t i_med;     // first prime index struck per tile (after the stamped ones)
  uint32_t i_dense;   // primes [i_med, i_dense) are struck cooperatively by all threads
  uint32_t n_head;    // the first n_head of them hit a window at least once per thread
  uint32_t i_large;   // primes >= i_large come through buckets
  uint32_t bucket_cap;
  uint32_t tw_log2;   // log2(tw)
  uint32_t bucket_auto;  // host only: the automatic capacity estimate
  uint32_t i_hyb;     // primes >= i_hyb reach the buckets by enumerating odd multipliers j
  uint32_t p_hyb;     // the prime at i_hyb (0xFFFFFFFF: none)
  uint32_t stage_cap; // usable staged list entries per tile (<= kStageCap)
  uint32_t pad;
};

struct TileArgs {
  PrimeTab pt;
  Geometry g;
  const ReqDesc *reqs;
  LaunchHeader *hdr;
  ResultSlot *slots;
  uint64_t *list_n;
  uint8_t *list_k;
  uint64_t *fail_n;
  Straggler *strag;
  uint32_t strag_cap;
  const uint32_t *bucket_count;
  const uint32_t *bucket_data;
  // mode 0: tile t stages its list entries at [t * kStageCap, + stage_cnt[t])
  uint64_t *stage_n;
  uint8_t *stage_k;
  uint32_t *stage_cnt;
};

struct BucketArgs {
  PrimeTab pt;
  Geometry g;
  const ReqDesc *reqs;
  LaunchHeader *hdr;
  uint32_t *bucket_count;
  uint32_t *bucket_data;
};

struct StragArgs {
  PrimeTab pt;
  const ReqDesc *reqs;
  LaunchHeader *hdr;
  ResultSlot *slots;
  uint64_t *list_n;
  uint8_t *list_k;
  uint64_t *fail_n;
  const Straggler *strag;
  uint32_t strag_cap;
  uint32_t rec_t;
  // ordered lists (mode 0): a straggler's list entry joins its tile's staged entries
  uint64_t *stage_n;    // null: append to the list directly
  uint8_t *stage_k;
  uint32_t *stage_cnt;
  uint32_t stage_cap;
  uint32_t tw_log2;
};

// The ordered list (mode 0): each range's staged entries, tile by tile and
// ascending within a tile, into its list region; list_count = the total.
struct CompactArgs {
  const ReqDesc *reqs;
  LaunchHeader *hdr;
  ResultSlot *slots;
  uint64_t *list_n;
  uint8_t *list_k;
  const uint64_t *stage_n;
  const uint8_t *stage_k;
  const uint32_t *stage_cnt;
  uint32_t stage_cap;
  uint32_t pad;
};

// Kernel launchers (defined in the .cu files).
cudaError_t launch_init(LaunchHeader *hdr, ResultSlot *slots, uint32_t n_slots,
                        uint32_t *bucket_count, uint32_t *stage_cnt, uint32_t n_tiles, ReqDesc *reqs, uint32_t mw,
                        const uint32_t *primes, uint32_t n_table, uint64_t ph2, cudaStream_t st);
cudaError_t launch_compact(const CompactArgs &a, uint32_t grid, cudaStream_t st);
// n_large_max, n_reqs: upper bounds of the launch's bucket primes and ranges;
// j_max: the largest odd multiplier any range needs for the primes >= p_hyb.
// They size the work items; at most max_blocks blocks take them in turn.
cudaError_t launch_bucket_fill(const BucketArgs &a, uint32_t n_large_max, uint32_t n_reqs, uint64_t j_max,
                               uint32_t max_blocks, cudaStream_t st);
// mode 0: lean scan (lists from k >= 6, no per-n output); 1: general scan;
// 2: general scan writing the per-n output.
cudaError_t launch_tiles(const TileArgs &a, uint32_t threads, uint32_t grid, size_t smem, int mode,
                         cudaStream_t st);
cudaError_t tile_kernel_setup(size_t smem);
size_t tile_static_smem();
cudaError_t launch_stragglers(const StragArgs &a, uint32_t grid, cudaStream_t st);
cudaError_t launch_points(PrimeTab pt, const uint64_t *pts, uint64_t count, uint8_t *out,
                          uint32_t grid, cudaStream_t st);
uint64_t host_isqrt(uint64_t x);  // floor(sqrt(x)), exact (host)
cudaError_t build_prime_table(uint64_t pmax, uint32_t **d_p, uint64_t **d_mu, uint64_t **d_inv,
                              uint64_t **d_lim, uint32_t **d_bits, uint64_t *bits_words, uint32_t *n,
                              uint32_t *n_div, cudaStream_t st);

constexpr int kMaxDensePrimes = 128;  // must match the tile kernel's shared arrays (four warps)
constexpr int kDenseMinHits = 8;      // primes with at least this many strikes per window are "dense"
constexpr int kMaxSparsePrimes = 2048;  // per-tile primes struck one thread each (shared arrays)
// Ranges per Barrett item of the bucket fill; a launch of at most this many
// ranges (one request chunk) has its smallest bucketed primes' hits cut into
// segments of the range, so it can bucket primes down to kSegmentedLargeMin.
constexpr uint32_t kFillReqChunk = 64;
constexpr uint64_t kSegmentedLargeMin = 4096;
constexpr uint32_t kFillBlocksPerSm = 4;  // resident bucket-fill blocks per SM (the launch bounds)
// Bucket primes below 2^mult_prime_log2 (sv_config) get one Barrett reduction
// per range; larger ones are found through their odd multipliers j (j p^2 in
// the range), which costs a few operations per multiplier instead of one
// reduction per prime, the cheaper way for them when many short ranges lie far
// up.  The default threshold:
constexpr int kMultPrimeLog2 = 18;

}  // namespace sv
