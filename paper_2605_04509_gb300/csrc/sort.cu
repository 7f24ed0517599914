// Device-wide exclusive scan and stable LSD radix sort (Sec. 4.2 "Sorting":
// the Gaussian-tile pairs are sorted so that every (tile, cluster) list is
// contiguous and depth-ordered; Alg. 1 stage 3).
//
// Radix sort: reduce-then-scan per digit (at most 8 bits for 32-bit keys, 9 for
// 64-bit keys). Pass = (1) per-tile digit histogram into a digit-major table,
// (2) per digit, the exclusive scan of its row (the tiles' counts) and the
// row's total, one block per digit, (3) stable scatter: a tile's output base
// for a digit is the digit's row prefix plus the scan of the row totals
// (every scatter block scans the totals once). The
// scatter kernel is persistent: each block walks its share of the tiles and,
// while it ranks one tile, the bulk-copy engine (cp.async.bulk, completion on
// an mbarrier) fetches the block's next tile into the other half of a double
// buffer in shared memory. Inside a tile each warp ranks its items with
// warp-match peer masks in (round, lane) order and per-warp digit counters, the
// warps' counters are prefixed, and the items are scattered through shared
// memory so that each digit's run is written with consecutive addresses.
// No block waits on another block. The item count may be given on the device
// (n_dev) with a host-side capacity bounding it, so that no host read-back is
// needed between key generation and the sort.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
    k_scan_reduce(const uint32_t* __restrict__ in, int64_t n, unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  unsigned long long acc = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const int64_t idx = base + r * kScanThreads + threadIdx.x;
    if (idx < n) acc += in[idx];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += s_warp[w];
    bsum[blockIdx.x] = t;
  }
}

// single block: exclusive scan of nb block sums, in chunks with a carry
__global__ void __launch_bounds__(1024)
    k_scan_bsums(unsigned long long* __restrict__ bsum, int64_t nb,
                 unsigned long long* __restrict__ total) {
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t idx = base + threadIdx.x;
    const unsigned long long v = idx < nb ? bsum[idx] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const unsigned long long carry = s_carry;
    const unsigned long long incl = x + (warp > 0 ? s_warp[warp - 1] : 0ull) + carry;
    if (idx < nb) bsum[idx] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s_carry;
}

__global__ void __launch_bounds__(kScanThreads)
    k_scan_down(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                const unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // blocked arrangement: thread owns kScanItems consecutive elements
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  unsigned long long sum = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const int64_t idx = base + r;
    v[r] = idx < n ? in[idx] : 0u;
    sum += v[r];
  }
  unsigned long long x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  unsigned long long wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += s_warp[w];
  unsigned long long run = bsum[blockIdx.x] + wpre + x - sum;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const int64_t idx = base + r;
    if (idx < n) out[idx] = (uint32_t)run;
    run += v[r];
  }
}

// Widest digit per key type: 8 bits for the 32-bit pair keys, 9 bits for the
// 64-bit keys (the 35-bit (cluster, depth) item keys take four passes instead
// of five). A sort takes the fewest passes these widths allow and spreads the
// key bits evenly over them: the 14 tile bits of a 4K panel go in two 7-bit
// passes, whose 128 output runs per 4096-item tile are twice as long as 256
// runs would be (the scatter's stores coalesce better; the digit tables are
// half as large).
template <typename K>
struct RadixOf {
  static constexpr int bits = sizeof(K) == 8 ? 9 : 8;
  static constexpr int radix = 1 << bits;
};
constexpr int kMaxRadix = 512;
// Block shape per key type: threads, and rounds of 32 items per warp; a
// tile is threads x rounds items. The 64-bit keys (the item sort, a few
// million items) take 2048-item tiles: the scatter's double buffer then
// needs 72 KB instead of 144 KB and three blocks fit an SM instead of one
// (key generation 2.00 -> 1.97 ms per paper4k frame). For the 32-bit pair
// keys, 8192-item tiles of 1024 threads (longer digit runs, one block per
// SM) made the sort stage slower (1.74 against 1.42 ms).
template <typename K>
struct SortCfg {
  static constexpr int threads = 512;
  static constexpr int warps = threads / 32;
  static constexpr int rounds = sizeof(K) == 8 ? 4 : 8;
  static constexpr int tile = threads * rounds;
  static_assert(threads >= RadixOf<K>::radix, "one thread per digit in the digit phases");
};

template <typename K>
__device__ __forceinline__ int digit_of(K key, int shift, int mask) {
  return (int)((key >> shift) & (K)mask);
}

__device__ __forceinline__ int64_t live_count(int64_t n_cap, const unsigned long long* n_dev) {
  if (!n_dev) return n_cap;
  const unsigned long long v = *n_dev;
  return v < (unsigned long long)n_cap ? (int64_t)v : n_cap;
}

// Per-tile digit histogram, written digit-major: hist[d * nb + tile]. A
// thread counts 16 consecutive keys, so the lanes of a warp look at keys far
// apart and their shared-memory increments rarely collide; each warp counts
// into its own histogram. Tiles past the live count write zeros.
template <typename K>
__global__ void __launch_bounds__(SortCfg<K>::threads)
    k_rts_hist(const K* __restrict__ keys, int64_t n_cap, const unsigned long long* __restrict__ n_dev,
               int shift, int mask, uint32_t* __restrict__ hist, int64_t nb) {
  constexpr int kRadix = RadixOf<K>::radix;
  constexpr int kSortThreads = SortCfg<K>::threads, kSortWarps = SortCfg<K>::warps;
  constexpr int kSortRounds = SortCfg<K>::rounds, kSortTile = SortCfg<K>::tile;
  __shared__ uint32_t s_h[kSortWarps][kRadix];
  const int warp = threadIdx.x >> 5;
  for (int a = threadIdx.x; a < kSortWarps * kRadix; a += kSortThreads) (&s_h[0][0])[a] = 0;
  __syncthreads();
  const int64_t n = live_count(n_cap, n_dev);
  const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
  const int64_t c0 = tile0 + (int64_t)threadIdx.x * kSortRounds;
  if (c0 < n) {
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15) == 0;
    if (vec && c0 + kSortRounds <= n) {
      const uint4* src = reinterpret_cast<const uint4*>(keys + c0);
      constexpr int NV = kSortRounds * (int)sizeof(K) / 16;
      uint4 q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = src[v];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if constexpr (sizeof(K) == 4) {
          atomicAdd(&s_h[warp][digit_of((K)q[v].x, shift, mask)], 1u);
          atomicAdd(&s_h[warp][digit_of((K)q[v].y, shift, mask)], 1u);
          atomicAdd(&s_h[warp][digit_of((K)q[v].z, shift, mask)], 1u);
          atomicAdd(&s_h[warp][digit_of((K)q[v].w, shift, mask)], 1u);
        } else {
          atomicAdd(&s_h[warp][digit_of((K)(((uint64_t)q[v].y << 32) | q[v].x), shift, mask)], 1u);
          atomicAdd(&s_h[warp][digit_of((K)(((uint64_t)q[v].w << 32) | q[v].z), shift, mask)], 1u);
        }
      }
    } else {
      const int cnt = (int)min((int64_t)kSortRounds, n - c0);
      for (int r = 0; r < cnt; ++r) atomicAdd(&s_h[warp][digit_of(keys[c0 + r], shift, mask)], 1u);
    }
  }
  __syncthreads();
  const int d = threadIdx.x;
  if (d <= mask) {
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) sum += s_h[w][d];
    hist[(int64_t)d * nb + blockIdx.x] = sum;
  }
}

// Per digit, the exclusive scan of its row of the digit-major table (the
// tiles' counts of that digit) and the row total: one block per digit. The
// scatter adds the exclusive scan of the row totals, so a pass needs one scan
// launch instead of three.
constexpr int kRowScanThreads = 512;
constexpr int kRowScanItems = 4;

__global__ void __launch_bounds__(kRowScanThreads)
    k_rts_rowscan(const uint32_t* __restrict__ hist, uint32_t* __restrict__ hscan, int64_t nb,
                  uint32_t* __restrict__ rowtot) {
  __shared__ uint32_t s_w[kRowScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t* row = hist + (int64_t)blockIdx.x * nb;
  uint32_t* out = hscan + (int64_t)blockIdx.x * nb;
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += kRowScanThreads * kRowScanItems) {
    const int64_t i0 = base + (int64_t)threadIdx.x * kRowScanItems;
    uint32_t v[kRowScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < kRowScanItems; ++q) {
      v[q] = i0 + q < nb ? row[i0 + q] : 0u;
      sum += v[q];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    uint32_t pre = 0, all = 0;
    for (int w = 0; w < kRowScanThreads / 32; ++w) {
      if (w < warp) pre += s_w[w];
      all += s_w[w];
    }
    uint32_t run = carry + pre + x - sum;
#pragma unroll
    for (int q = 0; q < kRowScanItems; ++q) {
      if (i0 + q < nb) out[i0 + q] = run;
      run += v[q];
    }
    carry += all;
    __syncthreads();  // s_w is reused by the next chunk
  }
  if (threadIdx.x == 0) rowtot[blockIdx.x] = carry;
}

// Peer mask of the lanes holding the same digit (invalid lanes form a group
// of their own): one warp match instead of a ballot per digit bit.
__device__ __forceinline__ unsigned digit_peers(int d, bool valid) {
  return __match_any_sync(0xffffffffu, valid ? d : -1);
}

// Stable scatter of one pass. Block b handles tiles b, b + G, b + 2G, ...
// (G = gridDim.x); tile t's output base for digit d is the exclusive scan of
// the row totals at d plus hscan[d * nb + t].
template <typename K>
__global__ void __launch_bounds__(SortCfg<K>::threads)
    k_rts_scatter(const K* __restrict__ kin, K* __restrict__ kout, const uint32_t* __restrict__ vin,
                  uint32_t* __restrict__ vout, int64_t n_cap, const unsigned long long* __restrict__ n_dev,
                  int shift, int mask, const uint32_t* __restrict__ hscan,
                  const uint32_t* __restrict__ rowtot, int64_t nb, uint32_t* __restrict__ err) {
  constexpr int kRadix = RadixOf<K>::radix;
  constexpr int kSortThreads = SortCfg<K>::threads, kSortWarps = SortCfg<K>::warps;
  constexpr int kSortRounds = SortCfg<K>::rounds, kSortTile = SortCfg<K>::tile;
  extern __shared__ __align__(128) unsigned char s_raw[];
  // [in0 keys][in0 vals][in1 keys][in1 vals][out keys][out vals]
  constexpr size_t kBuf = (size_t)kSortTile * (sizeof(K) + sizeof(uint32_t));
  auto in_key = [&](int b) { return reinterpret_cast<K*>(s_raw + b * kBuf); };
  auto in_val = [&](int b) {
    return reinterpret_cast<uint32_t*>(s_raw + b * kBuf + kSortTile * sizeof(K));
  };
  K* s_key = reinterpret_cast<K*>(s_raw + 2 * kBuf);
  uint32_t* s_val = reinterpret_cast<uint32_t*>(s_key + kSortTile);
  // per-warp digit counters (at most 4096 items per tile: 16 bits suffice)
  __shared__ uint16_t s_wcnt[kSortWarps][kRadix];
  __shared__ uint32_t s_base[kRadix];
  __shared__ uint32_t s_dbase[kRadix];
  __shared__ uint32_t s_dstart[kRadix];
  __shared__ uint32_t s_wsum[kRadix / 32];
  __shared__ __align__(8) unsigned long long s_bar[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t n = live_count(n_cap, n_dev);
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  const int d = threadIdx.x;
  // bulk copies need 16-byte aligned sources; otherwise every tile is loaded
  // with plain loads
  const bool bulk_ok =
      ((reinterpret_cast<uintptr_t>(kin) | reinterpret_cast<uintptr_t>(vin)) & 15) == 0;
  auto is_full = [&](int64_t t) { return bulk_ok && (t + 1) * kSortTile <= n; };
  // every digit's first output position: exclusive scan of the row totals
  {
    const uint32_t v = d <= mask ? rowtot[d] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (d < kRadix && lane == 31) s_dstart[warp] = x;  // scratch until the first tile
    __syncthreads();
    if (d < kRadix) {
      uint32_t pre = 0;
      for (int w = 0; w < warp; ++w) pre += s_dstart[w];
      s_dbase[d] = pre + x - v;
    }
    __syncthreads();
  }
  // start the bulk copy of tile t into buffer b (thread 0)
  auto fetch = [&](int b, int64_t t) {
    if (t < ntiles && is_full(t)) {
      // the buffer's last readers finished before the preceding barrier
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&s_bar[b], (uint32_t)kBuf);
      bulk_g2s(in_key(b), kin + t * kSortTile, (uint32_t)(kSortTile * sizeof(K)), &s_bar[b]);
      bulk_g2s(in_val(b), vin + t * kSortTile, (uint32_t)(kSortTile * sizeof(uint32_t)), &s_bar[b]);
    }
  };
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fetch(0, blockIdx.x);
  }
  __syncthreads();
  uint32_t parity = 0u;  // bit b: phase parity awaited on buffer b
  int b = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t tile0 = tile * kSortTile;
    const int cnt = (int)min((int64_t)kSortTile, n - tile0);
    for (int a = threadIdx.x; a < kSortWarps * kRadix; a += kSortThreads) (&s_wcnt[0][0])[a] = 0;
    if (d <= mask) s_base[d] = s_dbase[d] + hscan[(int64_t)d * nb + tile];
    if (threadIdx.x == 0) fetch(b ^ 1, tile + gridDim.x);
    if (is_full(tile)) {
      const uint32_t ph = (parity >> b) & 1u;
      if (!mbar_wait_bounded(&s_bar[b], ph)) {
        atomicOr(err, 1u);
        mbar_wait_bounded(&s_bar[b], ph);
      }
      parity ^= 1u << b;
    } else {
      K* kk = in_key(b);
      uint32_t* vv = in_val(b);
      for (int j = threadIdx.x; j < cnt; j += kSortThreads) {
        kk[j] = kin[tile0 + j];
        vv[j] = vin[tile0 + j];
      }
    }
    __syncthreads();
    // rank: warp w owns the contiguous chunk [w * 32 * kSortRounds, ...)
    const K* ik = in_key(b);
    const uint32_t* iv = in_val(b);
    // The keys of all rounds are loaded and their peer masks taken before
    // the per-warp counters are walked round by round: the loads and
    // matches overlap instead of waiting behind each round's counter update
    // (sort stage 1.37 -> 1.34 ms per paper4k frame).
    K kr[kSortRounds];
    int dg[kSortRounds];
    unsigned pm[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const int idx = warp * 32 * kSortRounds + r * 32 + lane;
      const bool valid = idx < cnt;
      kr[r] = valid ? ik[idx] : (K)0;
      dg[r] = valid ? digit_of(kr[r], shift, mask) : kRadix;
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) pm[r] = digit_peers(dg[r], dg[r] < kRadix);
    uint32_t rk[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const int dd = dg[r];
      const bool valid = dd < kRadix;
      const int rank = __popc(pm[r] & lt);
      const int pc = __popc(pm[r]);
      const uint32_t bw = valid ? (uint32_t)s_wcnt[warp][dd] : 0u;
      __syncwarp();
      if (valid && rank == pc - 1) s_wcnt[warp][dd] = (uint16_t)(bw + (uint32_t)pc);
      __syncwarp();
      rk[r] = bw + (uint32_t)rank;
    }
    __syncthreads();
    // digit phase (threads 0..255, one per digit): exclusive prefix of the
    // warp counters, then the tile's digit starts
    uint32_t run = 0, x = 0;
    if (d < kRadix) {
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = s_wcnt[w][d];
        s_wcnt[w][d] = (uint16_t)run;
        run += c;
      }
      x = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_wsum[warp] = x;
    }
    __syncthreads();
    if (d < kRadix) {
      uint32_t pre = 0;
      for (int w = 0; w < warp; ++w) pre += s_wsum[w];
      s_dstart[d] = pre + x - run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
      const int dd = dg[r];
      if (dd < kRadix) {
        const int idx = warp * 32 * kSortRounds + r * 32 + lane;
        const uint32_t pos = s_dstart[dd] + s_wcnt[warp][dd] + rk[r];
        s_key[pos] = kr[r];
        s_val[pos] = iv[idx];
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kSortThreads) {
      const K k = s_key[j];
      const int dd = digit_of(k, shift, mask);
      const uint32_t out = s_base[dd] + ((uint32_t)j - s_dstart[dd]);
      if ((int64_t)out < n) {
        kout[out] = k;
        vout[out] = s_val[j];
      }
    }
    __syncthreads();  // buffers and counters are reused by the next tile
    b ^= 1;
  }
}

template <typename K>
constexpr size_t scatter_smem() {
  return (size_t)SortCfg<K>::tile * (sizeof(K) + sizeof(uint32_t)) * 3;
}

// resident blocks of the scatter kernel (its persistent grid)
template <typename K>
int scatter_grid(int64_t tiles) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rts_scatter<K>, SortCfg<K>::threads,
                                                scatter_smem<K>());
  const int64_t g = (int64_t)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  return (int)(g < tiles ? g : (tiles > 0 ? tiles : 1));
}

template <typename K>
cudaError_t radix_sort_impl(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t n_cap,
                            const unsigned long long* n_dev, int begin_bit, int end_bit, void* temp,
                            bool* result_in_alt, uint32_t* err, cudaStream_t s) {
  *result_in_alt = false;
  if (n_cap <= 1 || end_bit <= begin_bit) return cudaSuccess;
  constexpr int kSortThreads = SortCfg<K>::threads, kSortTile = SortCfg<K>::tile;
  const int64_t nb = (n_cap + kSortTile - 1) / kSortTile;
  constexpr int kRadix = RadixOf<K>::radix;
  uint32_t* hist = reinterpret_cast<uint32_t*>(temp);
  uint32_t* hscan = hist + nb * kRadix;
  uint32_t* rowtot = hscan + nb * kRadix;  // [kRadix]
  const size_t smem = scatter_smem<K>();
  cudaError_t e =
      cudaFuncSetAttribute(k_rts_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = scatter_grid<K>(nb);
  K* src_k = keys;
  K* dst_k = keys_alt;
  uint32_t* src_v = vals;
  uint32_t* dst_v = vals_alt;
  bool alt = false;
  constexpr int kRadixBits = RadixOf<K>::bits;
  const int passes = (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;
  const int width = (end_bit - begin_bit + passes - 1) / passes;
  for (int shift = begin_bit; shift < end_bit; shift += width) {
    const int nbits = end_bit - shift < width ? end_bit - shift : width;
    const int mask = (1 << nbits) - 1;
    k_rts_hist<K><<<(unsigned)nb, kSortThreads, 0, s>>>(src_k, n_cap, n_dev, shift, mask, hist, nb);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_rts_rowscan<<<(unsigned)(mask + 1), kRowScanThreads, 0, s>>>(hist, hscan, nb, rowtot);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_rts_scatter<K><<<(unsigned)grid, kSortThreads, smem, s>>>(src_k, dst_k, src_v, dst_v, n_cap,
                                                                n_dev, shift, mask, hscan, rowtot, nb,
                                                                err);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    K* tk = src_k;
    src_k = dst_k;
    dst_k = tk;
    uint32_t* tv = src_v;
    src_v = dst_v;
    dst_v = tv;
    alt = !alt;
  }
  *result_in_alt = alt;
  return cudaSuccess;
}

// Self-test kernel: one thread waits, with the bound, on an mbarrier phase
// that nothing completes.
__global__ void k_selftest_wait(uint32_t* err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait_bounded(&bar, 0u)) atomicOr(err, 1u);
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  return (size_t)(nb + 1) * sizeof(unsigned long long);
}

cudaError_t scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, void* temp,
                           unsigned long long* total_dev, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long), s);
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  unsigned long long* bsum = reinterpret_cast<unsigned long long*>(temp);
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, bsum);
  note_launches(1);
  k_scan_bsums<<<1, 1024, 0, s>>>(bsum, nb, total_dev);
  note_launches(1);
  k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, bsum);
  note_launches(1);
  return cudaGetLastError();
}

template <typename K>
size_t radix_temp_bytes_of(int64_t n) {
  const int64_t nb = (n + SortCfg<K>::tile - 1) / SortCfg<K>::tile;
  const int64_t cells = nb * RadixOf<K>::radix;
  return (size_t)(cells * 2 + RadixOf<K>::radix) * sizeof(uint32_t) + 256;
}

size_t radix_temp_bytes(int64_t n, int key_bytes) {
  return key_bytes == 8 ? radix_temp_bytes_of<uint64_t>(n) : radix_temp_bytes_of<uint32_t>(n);
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals,
                           uint32_t* vals_alt, int64_t n, const unsigned long long* n_dev,
                           int begin_bit, int end_bit, void* temp, bool* result_in_alt,
                           uint32_t* err, cudaStream_t s) {
  return radix_sort_impl<uint32_t>(keys, keys_alt, vals, vals_alt, n, n_dev, begin_bit, end_bit,
                                   temp, result_in_alt, err, s);
}

cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                           uint32_t* vals_alt, int64_t n, const unsigned long long* n_dev,
                           int begin_bit, int end_bit, void* temp, bool* result_in_alt,
                           uint32_t* err, cudaStream_t s) {
  return radix_sort_impl<uint64_t>(keys, keys_alt, vals, vals_alt, n, n_dev, begin_bit, end_bit,
                                   temp, result_in_alt, err, s);
}

}  // namespace lfd

// Self-test of the bounded device waits: a kernel waits on an mbarrier phase
// that nothing completes (no copy is started, no thread arrives). The wait
// must give up after its bound, set the error bit and let the kernel end.
extern "C" LFD_API int lfd_selftest_wait_timeout(void* stream) {
  using namespace lfd;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* err = nullptr;
  cudaError_t e = cudaMalloc(&err, 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
  if (e == cudaSuccess) {
    k_selftest_wait<<<1, 32, 0, s>>>(err);
    note_launches(1);
    e = cudaGetLastError();
  }
  uint32_t bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(err);
  if (e != cudaSuccess) return set_cuda_error(e, "wait self-test");
  return (bits & 1u) ? LFD_ERR_TIMEOUT : LFD_OK;
}
