// lfd_render_projected_noalloc: the key generation, sort, range and blend
// stages of lfd_render_projected for small frames, with every piece of
// scratch memory taken from one fixed array in device memory instead of
// cudaMalloc. For callers that must not allocate device memory while they
// render: real-time loops whose latency budget forbids the synchronisation
// that cudaMalloc/cudaFree imply, and hosts whose memory manager owns the
// whole device heap. The paper has no counterpart; the results equal
// lfd_render_projected's bit for bit.
#include <mutex>

#include "lfd_internal.h"

namespace lfd {
namespace {

// Limits of the fixed scratch array (per call).
constexpr int64_t kNaItems = 1 << 15;   // K * M projected (cluster, Gaussian) items
constexpr int64_t kNaPairs = 1 << 17;   // Gaussian-(tile, cluster) pairs P
constexpr int64_t kNaRanges = 1 << 14;  // tiles * clusters

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Byte offsets of the regions inside the array.
constexpr size_t kOffItemKey = 0;                                             // 2 x u64[items]
constexpr size_t kOffItemVal = kOffItemKey + align256(2 * kNaItems * 8);      // 2 x u32[items]
constexpr size_t kOffCounts = kOffItemVal + align256(2 * kNaItems * 4);       // u32[items + 1]
constexpr size_t kOffOffsets = kOffCounts + align256((kNaItems + 1) * 4);     // u32[items + 1]
constexpr size_t kOffPairKey = kOffOffsets + align256((kNaItems + 1) * 4);    // 2 x u64[pairs]
constexpr size_t kOffPairVal = kOffPairKey + align256(2 * kNaPairs * 8);      // 2 x u32[pairs]
constexpr size_t kOffRanges = kOffPairVal + align256(2 * kNaPairs * 4);       // uint2[ranges]
constexpr size_t kOffSmall = kOffRanges + align256(kNaRanges * 8);            // u64[4]
constexpr size_t kOffRadix = kOffSmall + 256;                                 // sort / scan temp
constexpr size_t kRadixBytes = 512 * 1024;
constexpr size_t kScratchBytes = kOffRadix + kRadixBytes;  // about 4.9 MB

// The scratch array. Every GPU that loads the library holds it until the
// process exits. All calls share it: concurrent calls race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array, looked up once per device (the symbol's
// host-side name is not a device address).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

int na_fail(int code, const char* msg) { return set_error(code, msg); }

int na_cuda(cudaError_t e, const char* where) { return set_cuda_error(e, where); }

#define NA_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e__ = (call);                          \
    if (e__ != cudaSuccess) return na_cuda(e__, #call); \
  } while (0)

}  // namespace
}  // namespace lfd

using namespace lfd;

extern "C" int lfd_render_projected_noalloc(lfd_plan* plan, int64_t M, const float* means2d,
                                            const float* conic_opacity, const float* color_tau,
                                            const float* depth, float* out_rgb, void* stream,
                                            lfd_stats* stats) {
  PlanView pv;
  if (plan_view(plan, &pv) != LFD_OK) return na_fail(LFD_ERR_INVALID, "NULL plan");
  const PanelGeom& g = pv.g;
  cudaStream_t s = (cudaStream_t)stream;
  if (M < 0) return na_fail(LFD_ERR_INVALID, "negative Gaussian count");
  if (!out_rgb) return na_fail(LFD_ERR_INVALID, "out_rgb is NULL");
  if (M > 0 && (!means2d || !conic_opacity || !color_tau || !depth))
    return na_fail(LFD_ERR_INVALID, "NULL attribute buffer");
  if (M > 0 && (((uintptr_t)conic_opacity % 16) || ((uintptr_t)color_tau % 16) ||
                ((uintptr_t)means2d % 8)))
    return na_fail(LFD_ERR_INVALID, "attribute buffers misaligned");
  const int64_t n_items = (int64_t)g.K * M;
  if (n_items > kNaItems)
    return na_fail(LFD_ERR_CAPACITY,
                   "lfd_render_projected_noalloc: clusters * Gaussians exceeds 32768");
  if ((int64_t)g.T * g.K > kNaRanges)
    return na_fail(LFD_ERR_CAPACITY, "lfd_render_projected_noalloc: tiles * clusters exceeds 16384");
  const bool key64 = pv.sort_mode == LFD_SORT_KEY64;

  void* base = nullptr;
  NA_CUDA(scratch_address(&base));
  unsigned char* sb = reinterpret_cast<unsigned char*>(base);
  uint64_t* item_key[2] = {reinterpret_cast<uint64_t*>(sb + kOffItemKey),
                           reinterpret_cast<uint64_t*>(sb + kOffItemKey) + kNaItems};
  uint32_t* item_val[2] = {reinterpret_cast<uint32_t*>(sb + kOffItemVal),
                           reinterpret_cast<uint32_t*>(sb + kOffItemVal) + kNaItems};
  uint32_t* counts = reinterpret_cast<uint32_t*>(sb + kOffCounts);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(sb + kOffOffsets);
  unsigned char* pk = sb + kOffPairKey;
  uint32_t* pair_val[2] = {reinterpret_cast<uint32_t*>(sb + kOffPairVal),
                           reinterpret_cast<uint32_t*>(sb + kOffPairVal) + kNaPairs};
  uint2* ranges = reinterpret_cast<uint2*>(sb + kOffRanges);
  unsigned long long* d_small = reinterpret_cast<unsigned long long*>(sb + kOffSmall);
  uint32_t* d_err = reinterpret_cast<uint32_t*>(d_small + 3);  // zero at load
  void* temp = sb + kOffRadix;
  if (radix_temp_bytes(kNaPairs, 8) > kRadixBytes || radix_temp_bytes(kNaItems, 8) > kRadixBytes ||
      scan_temp_bytes(kNaItems + 1) > kRadixBytes)
    return na_fail(LFD_ERR_CAPACITY, "scratch layout too small");

  // key generation (same stages and kernels as lfd_render_projected)
  const uint32_t* order = nullptr;
  if (!key64) {
    NA_CUDA(launch_item_keys(g, M, depth, color_tau, item_key[0], item_val[0], s));
    bool alt = false;
    NA_CUDA(radix_sort_u64(item_key[0], item_key[1], item_val[0], item_val[1], n_items, nullptr,
                           0, 32 + g.bit_k, temp, &alt, d_err, s));
    order = item_val[alt ? 1 : 0];
  }
  NA_CUDA(launch_bin_count(g, M, means2d, conic_opacity, color_tau, order, nullptr, n_items, counts,
                           nullptr, s));
  NA_CUDA(scan_exclusive(counts, offsets, n_items, temp, d_small, s));
  NA_CUDA(cudaMemcpyAsync(pv.h_small, d_small, 4 * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaStreamSynchronize(s));
  const unsigned long long P = pv.h_small[0];
  if (pv.h_small[3] & 0xffffffffull) {
    // a bounded wait of this call's item sort (or of an earlier call's pair
    // sort) gave up: reported here, once
    pv.h_small[3] = 0;
    NA_CUDA(cudaMemsetAsync(d_err, 0, sizeof(unsigned long long), s));
    return na_fail(LFD_ERR_TIMEOUT, "a bounded device wait of the sort gave up");
  }
  if (P > (unsigned long long)kNaPairs)
    return na_fail(LFD_ERR_CAPACITY,
                   "lfd_render_projected_noalloc: more than 131072 Gaussian-tile pairs");
  uint32_t* pk32[2] = {reinterpret_cast<uint32_t*>(pk), reinterpret_cast<uint32_t*>(pk) + kNaPairs};
  uint64_t* pk64[2] = {reinterpret_cast<uint64_t*>(pk), reinterpret_cast<uint64_t*>(pk) + kNaPairs};
  NA_CUDA(launch_bin_emit(g, M, means2d, conic_opacity, color_tau, depth, order, n_items, offsets,
                          key64 ? nullptr : pk32[0], key64 ? pk64[0] : nullptr, pair_val[0], nullptr,
                          s));
  // sort by (tile, cluster, depth)
  bool alt = false;
  if (key64)
    NA_CUDA(radix_sort_u64(pk64[0], pk64[1], pair_val[0], pair_val[1], (int64_t)P, nullptr, 0,
                           32 + g.bit_k + g.bit_t, temp, &alt, d_err, s));
  else
    NA_CUDA(radix_sort_u32(pk32[0], pk32[1], pair_val[0], pair_val[1], (int64_t)P, nullptr,
                           g.bit_k, g.bit_k + g.bit_t, temp, &alt, d_err, s));
  const int kb = alt ? 1 : 0;
  // the range kernel writes every entry of the table
  NA_CUDA(launch_ranges(g, (int64_t)P, nullptr, key64 ? nullptr : pk32[kb],
                        key64 ? pk64[kb] : nullptr, ranges, s));
  // blend
  BlendArgs ba;
  ba.psi = pv.psi;
  ba.seg = pv.seg;
  ba.ranges = ranges;
  ba.list = pair_val[kb];
  ba.means2d = means2d;
  ba.conic_opacity = conic_opacity;
  ba.color_tau = color_tau;
  ba.M = M;
  ba.bg[0] = pv.bg[0];
  ba.bg[1] = pv.bg[1];
  ba.bg[2] = pv.bg[2];
  ba.out = out_rgb;
  ba.eval_counter = nullptr;
  ba.max_segment = pv.max_segment;
  ba.V = pv.V;
  ba.subpixels_per_thread = pv.subpixels_per_thread;
  if (pv.remap)
    NA_CUDA(launch_blend(g, ba, s));
  else
    NA_CUDA(launch_blend_raster(g, ba, s));
  if (stats) {
    stats->num_pairs = (int64_t)P;
    stats->num_visits = -1;
    stats->num_evals = -1;
    stats->ms_project = stats->ms_keygen = stats->ms_sort = stats->ms_blend = -1.f;
    // the caller asked for the frame's statistics: report a bounded wait of
    // this call's pair sort now rather than at the next call
    NA_CUDA(cudaMemcpyAsync(pv.h_small + 3, d_err, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (pv.h_small[3] & 0xffffffffull) {
      pv.h_small[3] = 0;
      NA_CUDA(cudaMemsetAsync(d_err, 0, sizeof(unsigned long long), s));
      return na_fail(LFD_ERR_TIMEOUT, "a bounded device wait of the pair sort gave up");
    }
  }
  return LFD_OK;
}
