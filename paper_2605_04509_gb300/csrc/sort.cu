// Device-wide exclusive scan and stable LSD radix sort (Sec. 4.2 "Sorting":
// the Gaussian-tile pairs are sorted so that every (tile, cluster) list is
// contiguous and depth-ordered; Alg. 1 stage 3).
//
// Radix sort: reduce-then-scan per 8-bit digit. Pass = (1) per-tile digit
// histogram, (2) exclusive scan of the digit-major histogram table, which
// yields every tile's global base per digit, (3) stable scatter. Inside a
// tile each warp ranks its items with match-any peer masks in (round, lane)
// order and per-warp digit counters, then the warps' counters are prefixed,
// so the scatter preserves input order among equal digits (stability).
// No kernel waits on another block, so nothing can spin.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 4096 items

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

template <typename K>
__device__ __forceinline__ int digit_of(K key, int shift, int mask) {
  return (int)((key >> shift) & (K)mask);
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
    k_radix_hist(const K* __restrict__ keys, int64_t n, int shift, int mask,
                 uint32_t* __restrict__ hist, int64_t nb) {
  __shared__ uint32_t s_cnt[kRadix];
  for (int a = threadIdx.x; a < kRadix; a += kSortThreads) s_cnt[a] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t idx = base + r * kSortThreads + threadIdx.x;
    const int d = idx < n ? digit_of(keys[idx], shift, mask) : kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d < kRadix && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int a = threadIdx.x; a < kRadix; a += kSortThreads)
    hist[(int64_t)a * nb + blockIdx.x] = s_cnt[a];
}

// Stable scatter of one tile. Items are ranked in the tile (warp chunks in
// order, match-any ranks inside a warp round, warp counters prefixed across
// warps), placed in shared memory in digit order, and written out so that
// consecutive threads store consecutive addresses of each digit's run.
template <typename K>
__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(const K* __restrict__ kin, K* __restrict__ kout, const uint32_t* __restrict__ vin,
                    uint32_t* __restrict__ vout, int64_t n, int shift, int mask,
                    const uint32_t* __restrict__ hist_scanned, int64_t nb) {
  static_assert(kRadix == kSortThreads, "one digit per thread");
  extern __shared__ __align__(16) unsigned char s_raw[];
  K* s_key = reinterpret_cast<K*>(s_raw);
  uint32_t* s_val = reinterpret_cast<uint32_t*>(s_key + kSortTile);
  __shared__ uint32_t s_wcnt[kSortWarps][kRadix];
  __shared__ uint32_t s_base[kRadix];
  __shared__ uint32_t s_dstart[kRadix];
  __shared__ uint32_t s_wsum[kSortWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int a = threadIdx.x; a < kSortWarps * kRadix; a += kSortThreads) (&s_wcnt[0][0])[a] = 0;
  s_base[threadIdx.x] = hist_scanned[(int64_t)threadIdx.x * nb + blockIdx.x];
  __syncthreads();
  // warp w owns the contiguous chunk [base, base + 32 * kSortRounds)
  const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * 32 * kSortRounds;
  K key[kSortRounds];
  uint32_t val[kSortRounds];
  uint32_t rk[kSortRounds];
  int dg[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t idx = base + r * 32 + lane;
    int d = kRadix;
    if (idx < n) {
      key[r] = kin[idx];
      val[r] = vin[idx];
      d = digit_of(key[r], shift, mask);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    const int cnt = __popc(peers);
    const uint32_t b = d < kRadix ? s_wcnt[warp][d] : 0u;
    __syncwarp();
    if (d < kRadix && rank == cnt - 1) s_wcnt[warp][d] = b + (uint32_t)cnt;
    __syncwarp();
    rk[r] = b + (uint32_t)rank;
    dg[r] = d;
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, then the block-wide digit starts
  {
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = s_wcnt[w][d];
      s_wcnt[w][d] = run;
      run += c;
    }
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre += s_wsum[w];
    s_dstart[d] = pre + x - run;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int d = dg[r];
    if (d < kRadix) {
      const uint32_t pos = s_dstart[d] + s_wcnt[warp][d] + rk[r];
      s_key[pos] = key[r];
      s_val[pos] = val[r];
    }
  }
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
  const int cnt = (int)min((int64_t)kSortTile, n - tile0);
  for (int j = threadIdx.x; j < cnt; j += kSortThreads) {
    const K k = s_key[j];
    const int d = digit_of(k, shift, mask);
    const uint32_t out = s_base[d] + ((uint32_t)j - s_dstart[d]);
    kout[out] = k;
    vout[out] = s_val[j];
  }
}

template <typename K>
cudaError_t radix_sort_impl(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t n,
                            int begin_bit, int end_bit, void* temp, bool* result_in_alt,
                            cudaStream_t s) {
  *result_in_alt = false;
  if (n <= 1 || end_bit <= begin_bit) return cudaSuccess;
  const int64_t nb = (n + kSortTile - 1) / kSortTile;
  uint32_t* hist = reinterpret_cast<uint32_t*>(temp);
  uint32_t* hscan = hist + nb * kRadix;
  void* stemp = hscan + nb * kRadix;
  unsigned long long* total = reinterpret_cast<unsigned long long*>(
      reinterpret_cast<char*>(stemp) + scan_temp_bytes(nb * kRadix));
  const size_t smem = (size_t)kSortTile * (sizeof(K) + sizeof(uint32_t));
  {
    cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  K* src_k = keys;
  K* dst_k = keys_alt;
  uint32_t* src_v = vals;
  uint32_t* dst_v = vals_alt;
  bool alt = false;
  for (int shift = begin_bit; shift < end_bit; shift += kRadixBits) {
    const int nbits = end_bit - shift < kRadixBits ? end_bit - shift : kRadixBits;
    const int mask = (1 << nbits) - 1;
    k_radix_hist<K><<<(unsigned)nb, kSortThreads, 0, s>>>(src_k, n, shift, mask, hist, nb);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive(hist, hscan, nb * kRadix, stemp, total, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<K><<<(unsigned)nb, kSortThreads, smem, s>>>(src_k, dst_k, src_v, dst_v, n,
                                                                shift, mask, hscan, nb);
    note_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
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

size_t radix_temp_bytes(int64_t n) {
  const int64_t nb = (n + kSortTile - 1) / kSortTile;
  return (size_t)nb * kRadix * 2 * sizeof(uint32_t) + scan_temp_bytes(nb * kRadix) +
         sizeof(unsigned long long) + 256;
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals,
                           uint32_t* vals_alt, int64_t n, int begin_bit, int end_bit, void* temp,
                           bool* result_in_alt, cudaStream_t s) {
  return radix_sort_impl<uint32_t>(keys, keys_alt, vals, vals_alt, n, begin_bit, end_bit, temp,
                                   result_in_alt, s);
}

cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                           uint32_t* vals_alt, int64_t n, int begin_bit, int end_bit, void* temp,
                           bool* result_in_alt, cudaStream_t s) {
  return radix_sort_impl<uint64_t>(keys, keys_alt, vals, vals_alt, n, begin_bit, end_bit, temp,
                                   result_in_alt, s);
}

}  // namespace lfd
