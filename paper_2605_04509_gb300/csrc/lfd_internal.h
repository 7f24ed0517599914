// Internal declarations shared by the CUDA translation units of liblfd.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lfd.h"

namespace lfd {

constexpr int kMaxViews = 255;
constexpr int kMaxClusterViews = 32;
constexpr int kMaxTileSubpixels = 3 * 1024;  // tiles of up to 1024 pixels

// Per-launch camera table: passed by value as a kernel parameter (large
// kernel parameters, 16 KB here), so concurrent frames never share state.
struct CamTable {
  float c[kMaxViews][16];  // R[9], t[3], fx, fy, cx, cy
};

// Every kernel launch of the library is counted (lfd_kernel_launches()).
void note_launches(int n);
uint64_t launch_count();

struct PanelGeom {
  int W, H, N, C, K;
  int TW, TH, TX, TY, T;
  int cap;  // 3 * TW * TH
  int bit_k, bit_t;
  // Batched scenes: the pair key is (t << bit_k) | key_code | k, where
  // key_code carries the scene's index above its cluster bits (0 for a
  // single scene), and item keys carry the global cluster cluster_base + k.
  uint32_t key_code = 0;
  int cluster_base = 0;
  // floor(x / TW) and floor(x / TH) for 0 <= x < 2^16 as __umulhi(x, magic)
  // with magic = floor(2^32 / d) + 1 (exact there, since d <= 64)
  uint32_t tw_magic = 0, th_magic = 0;
};
inline uint32_t div_magic(int d) { return (uint32_t)((1ull << 32) / (unsigned)d + 1ull); }

// ---- plan tables (plan_kernels.cu) ----
cudaError_t launch_view_index(int W, int H, int N, double tan_slant, double pitch,
                              double k_offset, uint8_t* V, cudaStream_t s);
cudaError_t launch_remap(const PanelGeom& g, const uint8_t* V, uint32_t* psi,
                         int32_t* n_sub, int32_t* seg, cudaStream_t s);

// ---- projection (project.cu) ----
struct ProjectArgs {
  const float* means;
  const void *scales, *quats, *opac, *sh;  // element type given by attr_dtype
  int64_t M;
  int sh_degree;
  int attr_dtype;  // LFD_DTYPE_*
  float* means2d;        // [K][M][C][2]
  float* conic_opacity;  // [K][M][4]
  float* color_tau;      // [K][M][4]
  float* depth;          // [K][M]
  // Gaussians [m_begin, m_end) only (m_end < 0: to M); outputs keep stride M
  int64_t m_begin = 0;
  int64_t m_end = -1;
};
cudaError_t launch_project(const PanelGeom& g, const CamTable& cams, const ProjectArgs& a,
                           cudaStream_t s);

// ---- key generation (binning.cu) ----
// item keys for the depth-first order: (k << 32) | depth bits, value k*M + i
cudaError_t launch_item_keys(const PanelGeom& g, int64_t M, const float* depth,
                             const float* color_tau, uint64_t* keys, uint32_t* vals,
                             cudaStream_t s);
// Bytes per item of the optional union descriptors the count pass leaves for
// the emit pass (nullptr: the emit pass recomputes the geometry).
constexpr size_t kBinDescBytes = 128;
// tile count of the cluster union per item; items visited in `order` (flat
// k*M + i indices) or natural order when order == nullptr. The count and the
// descriptor of item r go to position dest[r] (its emission position), or to
// the visit position when dest == nullptr.
cudaError_t launch_bin_count(const PanelGeom& g, int64_t M, const float* means2d,
                             const float* conic_opacity, const float* color_tau,
                             const uint32_t* order, const uint32_t* dest, int64_t n_items,
                             uint32_t* counts, void* desc, cudaStream_t s);
// emission: key32 = (t << bit_k) | k when keys64 == nullptr, else Eq. 11
cudaError_t launch_bin_emit(const PanelGeom& g, int64_t M, const float* means2d,
                            const float* conic_opacity, const float* color_tau,
                            const float* depth, const uint32_t* order, int64_t n_items,
                            const uint32_t* offsets, uint32_t* keys32, uint64_t* keys64,
                            uint32_t* vals, const void* desc, cudaStream_t s);
// emission from descriptors written by the count pass at each item's
// emission position; items visited in `order`, counts/offsets/descriptors
// indexed by position
// Writes nothing when *P_dev > P_cap (P_dev non-null); then sets bit 1 of
// *err (capacity overflow).
cudaError_t launch_bin_emit_coop(const PanelGeom& g, int64_t M, const float* means2d,
                                 const float* conic_opacity, const float* color_tau,
                                 const float* depth, const uint32_t* order, int64_t n_items,
                                 const uint32_t* counts, const uint32_t* offsets, uint32_t* keys32,
                                 uint64_t* keys64, uint32_t* vals, const void* desc,
                                 const unsigned long long* P_dev, unsigned long long P_cap,
                                 uint32_t* err, cudaStream_t s);
// Batched key generation: the scenes' items side by side in the batch arrays
// (scene s at positions [off, off + n)), one launch per pass for all scenes.
// A launch gives each scene whole blocks from blk_off on (filled in by the
// launcher for its block size).
constexpr int kMaxBinScenes = 16;
struct SceneBins {
  PanelGeom g;
  int64_t M, n, off;  // Gaussians, items (K M), first batch position
  const float *means2d, *conic_opacity, *color_tau, *depth;
  uint32_t blk_off;
};
struct BatchBins {
  SceneBins sc[kMaxBinScenes];
  int n_scenes;
};
cudaError_t launch_item_keys_batch(const BatchBins& bb, uint64_t* keys, uint32_t* vals, cudaStream_t s);
// per scene: inv[off + perm[p]] = p - off
cudaError_t launch_invert_batch(const BatchBins& bb, const uint32_t* perm, uint32_t* inv, cudaStream_t s);
// counts and descriptors of all scenes' items at their emission positions
cudaError_t launch_bin_count_batch(const BatchBins& bb, const uint32_t* dest, uint32_t* counts, void* desc,
                                   cudaStream_t s);
// the 32-bit pair keys and values of all scenes (order: scene-local item
// indices at batch positions)
cudaError_t launch_bin_emit_batch(const BatchBins& bb, const uint32_t* order, const uint32_t* counts,
                                  const uint32_t* offsets, uint32_t* keys32, uint32_t* vals,
                                  const void* desc, const unsigned long long* P_dev,
                                  unsigned long long P_cap, uint32_t* err, cudaStream_t s);
// dst[s] = src[idx[s]]
cudaError_t launch_gather_u32(const uint32_t* src, const uint32_t* idx, int64_t n, uint32_t* dst,
                              cudaStream_t s);
// inv[perm[s]] = s
cudaError_t launch_invert_u32(const uint32_t* perm, int64_t n, uint32_t* inv, cudaStream_t s);
// [S_tk, E_tk) of every (tile, cluster) run by binary search in the sorted
// keys (empty runs get (0, 0)); P a capacity, the live count from *P_dev
// when non-null. Writes the whole table.
cudaError_t launch_ranges(const PanelGeom& g, int64_t P, const unsigned long long* P_dev,
                          const uint32_t* keys32, const uint64_t* keys64, uint2* ranges,
                          cudaStream_t s);
// Range table of a batch: [scene][T_max][K_glob]; the run of (s, t, k) has
// key (t << bit_k) | (s << bit_kc) | k. Entries with t >= T[s] or k >= K[s]
// are (0, 0).
struct BatchRangeArgs {
  int n_scenes, T_max, K_glob, bit_k, bit_kc;
  int T[16], K[16];
};
cudaError_t launch_ranges_batch(const BatchRangeArgs& r, int64_t P, const unsigned long long* P_dev,
                                const uint32_t* keys32, uint2* ranges, cudaStream_t s);

// ---- scan and radix sort (sort.cu) ----
size_t scan_temp_bytes(int64_t n);
// exclusive scan of n uint32 into out; the 64-bit total goes to *total_dev
cudaError_t scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, void* temp,
                           unsigned long long* total_dev, cudaStream_t s);
// bytes of sort scratch for up to n items (n the capacity) with keys of
// key_bytes (4 or 8) bytes
size_t radix_temp_bytes(int64_t n, int key_bytes);
// Stable LSD radix sort of (key, value) by key bits [begin_bit, end_bit);
// ping-pongs between the two buffers; *result_in_alt tells where the result
// ends up (it depends on the bit range only). n is a host-side capacity;
// when n_dev is non-null the sort covers min(*n_dev, n) items, so the count
// may be produced on the device by the preceding kernels. A bulk-copy wait
// that reaches its bound sets bit 0 of *err (the result is then wrong).
cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals,
                           uint32_t* vals_alt, int64_t n, const unsigned long long* n_dev,
                           int begin_bit, int end_bit, void* temp, bool* result_in_alt,
                           uint32_t* err, cudaStream_t s);
cudaError_t radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                           uint32_t* vals_alt, int64_t n, const unsigned long long* n_dev,
                           int begin_bit, int end_bit, void* temp, bool* result_in_alt,
                           uint32_t* err, cudaStream_t s);

// ---- bulk-copy and mbarrier helpers (inline PTX) ----
constexpr int kSpinLimit = 1 << 22;                   // polls of an mbarrier before giving up
constexpr unsigned long long kWaitNs = 250000000ull;  // or 0.25 s, whichever comes first

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// global -> shared bulk copy (both 16-byte aligned, bytes a multiple of 16),
// completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for one phase of an mbarrier: false once kWaitNs nanoseconds
// have passed (or kSpinLimit polls, whichever comes first).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 15) == 15 && global_ns() - t0 > kWaitNs) return false;
    if (i > 16) __nanosleep(32);
  }
  return false;
}

// ---- blend (blend.cu) ----
// 2^x on the special-function unit (hand-written PTX instruction).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// -q/2 * log2(e) for the pre-scaled conic (A, B, C) = -log2(e) (a/2, b, c/2):
// A dx^2 + B dx dy + C dy^2 in one fixed order of rounded operations, shared
// by every blend kernel and the backward replay so that they agree bit for
// bit.
__device__ __forceinline__ float quad_power(float A, float B, float C, float dx, float dy) {
  return fmaf(dx, fmaf(B, dy, __fmul_rn(A, dx)), __fmul_rn(__fmul_rn(C, dy), dy));
}
struct BlendArgs {
  const uint32_t* psi;  // [T][cap] packed (view << 16) | local index
  const int32_t* seg;   // [T][K+1]
  const uint2* ranges;  // [T][K]
  const uint32_t* list;
  const float* means2d;
  const float* conic_opacity;
  const float* color_tau;
  int64_t M;
  float bg[3];
  float* out;
  unsigned long long* eval_counter;  // non-null: [0] visited entries, [1] evaluated ones
  int max_segment;
  const uint8_t* V;  // view index [H][W][3] (raster-order blend)
  // capacity mode: the blend writes nothing when *P_dev > P_cap
  const unsigned long long* P_dev = nullptr;
  unsigned long long P_cap = 0;
  int subpixels_per_thread = 0;  // 0: automatic
  // non-null: per Psi position [T][cap], the list index where the subpixel's
  // walk stopped (the range end if it never saturated) and the bits of its
  // final transmittance; written by the remapped blend, read by the backward
  uint2* keep = nullptr;
  // remapped blend: tiles [t_begin, t_end) only (t_end < 0: to T)
  int t_begin = 0;
  int t_end = -1;
};
cudaError_t launch_blend(const PanelGeom& g, const BlendArgs& a, cudaStream_t s);

// Batched blend: several scenes (each with its own panel tables, attributes
// and image) in one persistent launch over all their (cluster, tile) runs.
constexpr int kMaxBatchScenes = 16;
struct SceneBlend {
  PanelGeom g;        // key_code: the scene's index in the pair keys
  BlendArgs a;        // the scene's tables, attributes and image
  uint32_t run_base;  // first global run (runs of a scene are k * T + t)
};
struct BatchBlendArgs {
  SceneBlend sc[kMaxBatchScenes];
  int n_scenes;
  uint32_t total_runs;
  int K_glob;            // clusters per (scene, tile) in the range table
  int T_max;             // tiles per scene in the range table
  const uint2* ranges;   // [scene][T_max][K_glob]
  unsigned int* work;    // work counter (zeroed by the launcher)
  const unsigned long long* P_dev;
  unsigned long long P_cap;
};
cudaError_t launch_blend_batch(const BatchBlendArgs& b, int max_segment, int C_max,
                               int subpixels_per_thread, cudaStream_t s);
// the same blend without the view-coherent remap (threads in raster order)
cudaError_t launch_blend_raster(const PanelGeom& g, const BlendArgs& a, cudaStream_t s);
// full-frame baseline: per-view pixel blend fused with the interlacing
// (clusters are single views)
cudaError_t launch_blend_fullframe(const PanelGeom& g, const BlendArgs& a, cudaStream_t s);

// ---- backward (backward.cu) ----
struct BlendGrads {
  const float* grad_out;  // dL/dI [H][W][3]
  float* grad_means2d;    // [K][M][C][2]
  float* grad_conic;      // [K][M][4]: d/d(a, b, c) of the conic
  float* grad_color;      // [K][M][4]
  float* grad_opac;       // [M]
};
struct ParamGrads {
  float *means, *scales, *quats, *opacities, *sh;
};
cudaError_t launch_blend_backward(const PanelGeom& g, const BlendArgs& a, const BlendGrads& gr,
                                  cudaStream_t s);
cudaError_t launch_project_backward(const PanelGeom& g, const CamTable& cams, const ProjectArgs& a,
                                    const BlendGrads& gr, const ParamGrads& out, cudaStream_t s);

// ---- read-only view of a plan and error reporting (lfd_api.cu) ----
struct PlanView {
  PanelGeom g;
  const uint32_t* psi;
  const int32_t* seg;
  int max_segment;
  int sort_mode;
  int remap;
  const uint8_t* V;
  float bg[3];
  unsigned long long* h_small;  // pinned host words owned by the plan
  int subpixels_per_thread;
  bool fullframe;
};
int plan_view(const lfd_plan* p, PlanView* out);
int set_error(int code, const char* msg);
int set_cuda_error(cudaError_t e, const char* where);

}  // namespace lfd
