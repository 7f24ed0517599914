// Batched rendering of several scenes in one frame: each scene has its own
// plan (panel tables V, Psi and the per-(tile, cluster) runs), Gaussians,
// cameras and image. Projection and the per-item binning run per scene; the
// item sort, the offsets scan, the pair sort, the range search and the blend
// each run once over all scenes. Item keys carry a global cluster number
// (scene s owns clusters [cluster_base_s, cluster_base_s + K_s)), so the items
// and hence the emitted pairs come out scene-major. A pair's key is
// (t << (bit_s + bit_kc)) | (s << bit_kc) | k with t the scene's own tile: the
// stable sort on the tile bits alone then yields (tile, scene, cluster,
// depth) order, and every (scene, tile, cluster) run is contiguous - with as
// many sort passes as the largest panel's tile count needs.
// The blend is one persistent launch that pulls (scene, cluster, tile) runs
// from a work counter. A batch always runs in capacity mode: every buffer is
// sized by lfd_batch_reserve, and a frame neither allocates nor synchronises
// nor reads back, so it can be captured into a CUDA graph; the pair count and
// overflow status stay on the device until lfd_batch_status. The paper
// renders one panel per frame; this is the serving form of its Alg. 1.
#include <stdio.h>
#include <string.h>

#include <new>

#include "lfd_internal.h"

namespace lfd {
namespace {

int ceil_log2_u(uint64_t v) {
  int b = 0;
  while ((1ull << b) < v) ++b;
  return b;
}

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    cap = bytes;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

}  // namespace
}  // namespace lfd

using namespace lfd;

struct lfd_batch {
  int n = 0;
  lfd_plan* plans[kMaxBatchScenes] = {};
  PlanView pv[kMaxBatchScenes];
  PanelGeom g[kMaxBatchScenes];  // with the scene key code, cluster base and key bits
  uint32_t run_base[kMaxBatchScenes + 1] = {};
  int T_max = 0, K_glob = 0, clusters_total = 0, C_max = 0, max_segment = 0, spt = 0;
  int bit_kc = 0, bit_s = 0, bit_t = 0, bit_cluster = 0;
  // capacities
  int64_t cap_M[kMaxBatchScenes] = {};
  int64_t cap_items = 0, cap_P = 0;
  bool reserved = false;
  // per-scene projected attributes
  Buf proj_means[kMaxBatchScenes], proj_co[kMaxBatchScenes], proj_ct[kMaxBatchScenes],
      proj_depth[kMaxBatchScenes];
  // global scratch
  Buf item_key[2], item_val[2], emit_pos, counts, offsets, scan_tmp, bin_desc;
  Buf pair_key[2], pair_val[2], radix_tmp, ranges, small, work;
};

namespace {

int bfail(int code, const char* msg) { return set_error(code, msg); }

#define B_CUDA(call)                                          \
  do {                                                        \
    cudaError_t e__ = (call);                                 \
    if (e__ != cudaSuccess) return set_cuda_error(e__, #call); \
  } while (0)

}  // namespace

extern "C" {

void lfd_batch_destroy(lfd_batch* b) {
  if (!b) return;
  for (int s = 0; s < kMaxBatchScenes; ++s) {
    b->proj_means[s].release();
    b->proj_co[s].release();
    b->proj_ct[s].release();
    b->proj_depth[s].release();
  }
  Buf* all[] = {&b->item_key[0], &b->item_key[1], &b->item_val[0], &b->item_val[1], &b->emit_pos,
                &b->counts, &b->offsets, &b->scan_tmp, &b->bin_desc, &b->pair_key[0],
                &b->pair_key[1], &b->pair_val[0], &b->pair_val[1], &b->radix_tmp, &b->ranges,
                &b->small, &b->work};
  for (Buf* x : all) x->release();
  delete b;
}

int lfd_batch_create(lfd_plan* const* plans, int32_t num_scenes, lfd_batch** out) {
  if (!out) return bfail(LFD_ERR_INVALID, "NULL output pointer");
  *out = nullptr;
  if (!plans || num_scenes < 1 || num_scenes > kMaxBatchScenes)
    return bfail(LFD_ERR_INVALID, "num_scenes must be in [1, 16]");
  lfd_batch* b = new (std::nothrow) lfd_batch();
  if (!b) return bfail(LFD_ERR_OOM, "host allocation failed");
  b->n = num_scenes;
  int64_t runs = 0;
  int spt = -1;
  for (int s = 0; s < num_scenes; ++s) {
    if (plan_view(plans[s], &b->pv[s]) != LFD_OK) {
      delete b;
      return bfail(LFD_ERR_INVALID, "NULL plan in the batch");
    }
    const PlanView& v = b->pv[s];
    if (v.sort_mode != LFD_SORT_DEPTH_FIRST || !v.remap || v.fullframe) {
      delete b;
      return bfail(LFD_ERR_INVALID, "batched plans must use depth-first sorting and the remap");
    }
    if (spt >= 0 && v.subpixels_per_thread != spt) {
      delete b;
      return bfail(LFD_ERR_INVALID, "batched plans must share subpixels_per_thread");
    }
    spt = v.subpixels_per_thread;
    b->plans[s] = plans[s];
    b->g[s] = v.g;
    b->g[s].cluster_base = b->clusters_total;
    b->run_base[s] = (uint32_t)runs;
    runs += (int64_t)v.g.T * v.g.K;
    b->clusters_total += v.g.K;
    b->T_max = v.g.T > b->T_max ? v.g.T : b->T_max;
    b->K_glob = v.g.K > b->K_glob ? v.g.K : b->K_glob;
    b->C_max = v.g.C > b->C_max ? v.g.C : b->C_max;
    b->max_segment = v.max_segment > b->max_segment ? v.max_segment : b->max_segment;
  }
  b->spt = spt;
  b->run_base[num_scenes] = (uint32_t)runs;
  b->bit_kc = ceil_log2_u((uint64_t)b->K_glob);
  b->bit_s = ceil_log2_u((uint64_t)num_scenes);
  b->bit_t = ceil_log2_u((uint64_t)b->T_max);
  b->bit_cluster = ceil_log2_u((uint64_t)b->clusters_total);
  if (b->bit_t + b->bit_s + b->bit_kc > 32 || runs >= (1ll << 32) ||
      (int64_t)num_scenes * b->T_max * b->K_glob >= (1ll << 31)) {
    delete b;
    return bfail(LFD_ERR_CAPACITY, "tile, scene and cluster bits exceed 32");
  }
  for (int s = 0; s < num_scenes; ++s) {
    b->g[s].bit_k = b->bit_s + b->bit_kc;
    b->g[s].bit_t = b->bit_t;
    b->g[s].key_code = (uint32_t)s << b->bit_kc;
  }
  cudaError_t e = b->small.ensure(4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(b->small.p, 0, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = b->work.ensure(256);
  if (e != cudaSuccess) {
    lfd_batch_destroy(b);
    return set_cuda_error(e, "batch scratch");
  }
  *out = b;
  return LFD_OK;
}

int lfd_batch_reserve(lfd_batch* b, const int64_t* max_gaussians, int64_t max_pairs) {
  if (!b || !max_gaussians) return bfail(LFD_ERR_INVALID, "NULL argument");
  if (max_pairs <= 0 || max_pairs >= 0xffffffffll)
    return bfail(LFD_ERR_INVALID, "max_pairs must be in [1, 2^32 - 2]");
  int64_t items = 0;
  for (int s = 0; s < b->n; ++s) {
    if (max_gaussians[s] < 0) return bfail(LFD_ERR_INVALID, "negative Gaussian capacity");
    items += (int64_t)b->g[s].K * max_gaussians[s];
  }
  if (items >= (1ll << 32)) return bfail(LFD_ERR_CAPACITY, "more than 2^32 - 1 items");
  for (int s = 0; s < b->n; ++s) {
    const int64_t n = (int64_t)b->g[s].K * max_gaussians[s];
    B_CUDA(b->proj_means[s].ensure((size_t)(n * b->g[s].C + 1) * 8));
    B_CUDA(b->proj_co[s].ensure((size_t)(n + 1) * 16));
    B_CUDA(b->proj_ct[s].ensure((size_t)(n + 1) * 16));
    B_CUDA(b->proj_depth[s].ensure((size_t)(n + 1) * 4));
    b->cap_M[s] = max_gaussians[s];
  }
  const size_t items4 = (size_t)(items + 1) * 4;
  for (int k = 0; k < 2; ++k) {
    B_CUDA(b->item_key[k].ensure((size_t)(items + 1) * 8));
    B_CUDA(b->item_val[k].ensure(items4));
    B_CUDA(b->pair_key[k].ensure((size_t)(max_pairs + 1) * 4));
    B_CUDA(b->pair_val[k].ensure((size_t)(max_pairs + 1) * 4));
  }
  B_CUDA(b->emit_pos.ensure(items4));
  B_CUDA(b->counts.ensure(items4));
  B_CUDA(b->offsets.ensure(items4));
  B_CUDA(b->scan_tmp.ensure(scan_temp_bytes(items + 1)));
  B_CUDA(b->bin_desc.ensure((size_t)(items + 1) * kBinDescBytes));
  const size_t st = radix_temp_bytes(items, 8) > radix_temp_bytes(max_pairs, 4) ? radix_temp_bytes(items, 8)
                                                                               : radix_temp_bytes(max_pairs, 4);
  B_CUDA(b->radix_tmp.ensure(st));
  B_CUDA(b->ranges.ensure((size_t)b->n * b->T_max * b->K_glob * sizeof(uint2)));
  b->cap_items = items;
  b->cap_P = max_pairs;
  b->reserved = true;
  return LFD_OK;
}

int lfd_batch_render(lfd_batch* b, const lfd_gaussians* scenes, const lfd_camera* const* cams,
                     float* const* out_rgb, void* stream) {
  if (!b || !scenes || !cams || !out_rgb) return bfail(LFD_ERR_INVALID, "NULL argument");
  if (!b->reserved) return bfail(LFD_ERR_STATE, "lfd_batch_reserve must precede rendering");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t item_off[kMaxBatchScenes + 1];
  item_off[0] = 0;
  for (int s = 0; s < b->n; ++s) {
    if (scenes[s].count < 0 || scenes[s].count > b->cap_M[s])
      return bfail(LFD_ERR_CAPACITY, "more Gaussians than reserved for a scene");
    if (!out_rgb[s] || !cams[s]) return bfail(LFD_ERR_INVALID, "NULL image or camera array");
    item_off[s + 1] = item_off[s] + (int64_t)b->g[s].K * scenes[s].count;
  }
  const int64_t n_items = item_off[b->n];
  unsigned long long* d_small = b->small.as<unsigned long long>();
  uint32_t* d_err = reinterpret_cast<uint32_t*>(d_small + 3);
  uint64_t* ik = b->item_key[0].as<uint64_t>();
  uint32_t* iv = b->item_val[0].as<uint32_t>();
  unsigned char* desc = b->bin_desc.as<unsigned char>();
  // projection (Eq. 5-6), per scene (each with its own camera table)
  BatchBins bb{};
  bb.n_scenes = b->n;
  for (int s = 0; s < b->n; ++s) {
    int rc = lfd_project(b->plans[s], &scenes[s], cams[s], b->g[s].N, b->proj_means[s].as<float>(),
                         b->proj_co[s].as<float>(), b->proj_ct[s].as<float>(),
                         b->proj_depth[s].as<float>(), stream);
    if (rc != LFD_OK) return rc;
    SceneBins& sb = bb.sc[s];
    sb.g = b->g[s];
    sb.M = scenes[s].count;
    sb.n = item_off[s + 1] - item_off[s];
    sb.off = item_off[s];
    sb.means2d = b->proj_means[s].as<float>();
    sb.conic_opacity = b->proj_co[s].as<float>();
    sb.color_tau = b->proj_ct[s].as<float>();
    sb.depth = b->proj_depth[s].as<float>();
  }
  // key generation of all scenes, one launch per pass: item keys, one
  // (global cluster, depth) sort of all items (scene s's items then hold
  // positions [item_off[s], item_off[s + 1]) with scene-local indices), the
  // emission positions, counts and descriptors there, their scan, emission
  B_CUDA(launch_item_keys_batch(bb, ik, iv, st));
  bool alt = false;
  B_CUDA(radix_sort_u64(ik, b->item_key[1].as<uint64_t>(), iv, b->item_val[1].as<uint32_t>(), n_items,
                        nullptr, 0, 32 + b->bit_cluster, b->radix_tmp.p, &alt, d_err, st));
  const uint32_t* order = b->item_val[alt ? 1 : 0].as<uint32_t>();
  B_CUDA(launch_invert_batch(bb, order, b->emit_pos.as<uint32_t>(), st));
  B_CUDA(launch_bin_count_batch(bb, b->emit_pos.as<uint32_t>(), b->counts.as<uint32_t>(), desc, st));
  B_CUDA(scan_exclusive(b->counts.as<uint32_t>(), b->offsets.as<uint32_t>(), n_items, b->scan_tmp.p,
                        d_small, st));
  const unsigned long long P = (unsigned long long)b->cap_P;
  B_CUDA(launch_bin_emit_batch(bb, order, b->counts.as<uint32_t>(), b->offsets.as<uint32_t>(),
                               b->pair_key[0].as<uint32_t>(), b->pair_val[0].as<uint32_t>(), desc,
                               d_small, P, d_err, st));
  // one stable sort on the tile bits: (tile, scene, cluster, depth)
  alt = false;
  const int low = b->bit_s + b->bit_kc;
  B_CUDA(radix_sort_u32(b->pair_key[0].as<uint32_t>(), b->pair_key[1].as<uint32_t>(),
                        b->pair_val[0].as<uint32_t>(), b->pair_val[1].as<uint32_t>(), (int64_t)P,
                        d_small, low, low + b->bit_t, b->radix_tmp.p, &alt, d_err, st));
  const int kb = alt ? 1 : 0;
  BatchRangeArgs ra{};
  ra.n_scenes = b->n;
  ra.T_max = b->T_max;
  ra.K_glob = b->K_glob;
  ra.bit_k = low;
  ra.bit_kc = b->bit_kc;
  for (int s = 0; s < b->n; ++s) {
    ra.T[s] = b->g[s].T;
    ra.K[s] = b->g[s].K;
  }
  B_CUDA(launch_ranges_batch(ra, (int64_t)P, d_small, b->pair_key[kb].as<uint32_t>(),
                             b->ranges.as<uint2>(), st));
  // one persistent blend over every scene's runs
  BatchBlendArgs ba{};  // zero, with the members' own defaults
  for (int s = 0; s < b->n; ++s) {
    SceneBlend& sc = ba.sc[s];
    sc.g = b->g[s];
    sc.a.psi = b->pv[s].psi;
    sc.a.seg = b->pv[s].seg;
    sc.a.ranges = b->ranges.as<uint2>();
    sc.a.list = b->pair_val[kb].as<uint32_t>();
    sc.a.means2d = b->proj_means[s].as<float>();
    sc.a.conic_opacity = b->proj_co[s].as<float>();
    sc.a.color_tau = b->proj_ct[s].as<float>();
    sc.a.M = scenes[s].count;
    sc.a.bg[0] = b->pv[s].bg[0];
    sc.a.bg[1] = b->pv[s].bg[1];
    sc.a.bg[2] = b->pv[s].bg[2];
    sc.a.out = out_rgb[s];
    sc.a.eval_counter = nullptr;
    sc.a.max_segment = b->pv[s].max_segment;
    sc.a.V = b->pv[s].V;
    sc.run_base = b->run_base[s];
  }
  ba.n_scenes = b->n;
  ba.total_runs = b->run_base[b->n];
  ba.K_glob = b->K_glob;
  ba.T_max = b->T_max;
  ba.ranges = b->ranges.as<uint2>();
  ba.work = b->work.as<unsigned int>();
  ba.P_dev = d_small;
  ba.P_cap = P;
  B_CUDA(launch_blend_batch(ba, b->max_segment, b->C_max, b->spt, st));
  return LFD_OK;
}

int lfd_batch_status(lfd_batch* b, int64_t* pairs) {
  if (!b) return bfail(LFD_ERR_INVALID, "NULL batch");
  B_CUDA(cudaDeviceSynchronize());
  unsigned long long h[4];
  B_CUDA(cudaMemcpy(h, b->small.p, sizeof(h), cudaMemcpyDeviceToHost));
  if (pairs) *pairs = (int64_t)h[0];
  const uint32_t bits = (uint32_t)(h[3] & 0xffffffffull);
  if (!bits) return LFD_OK;
  B_CUDA(cudaMemset(b->small.as<unsigned long long>() + 3, 0, sizeof(unsigned long long)));
  if (bits & 1u) return bfail(LFD_ERR_TIMEOUT, "a bounded device wait of the sort gave up");
  char msg[160];
  snprintf(msg, sizeof(msg), "a frame had more pairs than reserved (last frame: %llu, reserved: %lld)",
           h[0], (long long)b->cap_P);
  return bfail(LFD_ERR_CAPACITY, msg);
}

}  // extern "C"
