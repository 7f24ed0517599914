// C ABI of the renderer (include/lfd.h): plan management and the per-frame
// orchestration of Alg. 1 (projection, key generation, sort, blend).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "lfd_internal.h"

using namespace lfd;

namespace lfd {
namespace {
std::atomic<unsigned long long> g_launches{0};
}
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace lfd

namespace {

thread_local char g_last_error[512] = "";

int fail_cuda(cudaError_t e, const char* where) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorName(e),
           cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LFD_ERR_OOM : LFD_ERR_CUDA;
}

int fail(int code, const char* msg) {
  snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
  return code;
}

#define LFD_CUDA(call)                                \
  do {                                                \
    cudaError_t e__ = (call);                         \
    if (e__ != cudaSuccess) return fail_cuda(e__, #call); \
  } while (0)

int ceil_log2(uint64_t v) {
  int b = 0;
  while ((1ull << b) < v) ++b;
  return b;
}

// A growable device buffer. Growth frees and reallocates (with headroom),
// which synchronises the device; steady-state frames allocate nothing.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes) {
    if (bytes <= cap) return LFD_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = bytes + bytes / 4 + 1024;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail_cuda(e, "cudaMalloc");
    }
    cap = want;
    return LFD_OK;
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

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

namespace {
// Transfers of lfd_render_host(_async), overlapped with the kernels: the
// Gaussians go up in kHostChunks chunks on an upload stream and each chunk is
// projected as soon as it has landed; the image goes back on a download
// stream once the blend is done. The device copies of the inputs and the
// device image are double-buffered (parity of the frame), so a frame's upload
// runs under the previous frame's blend and its download under the next
// frame's first stages. (Blending in four bands of tile rows on forked
// streams, each band's rows going back as soon as it was done, was slower:
// every band's launch has its own tail; 109.5 against 114.3 frames/s
// pipelined and 98.4 against 98.8 synchronous on paper4k.)
constexpr int kHostChunks = 4;
struct HostIO {
  const void* src[5];   // host attribute arrays
  void* dst[5];         // their device copies
  size_t elem_bytes[5];  // bytes per Gaussian of each array
  float* out_host;      // host image [H][W][3]
  int parity;           // which of the double buffers the frame uses
};
struct HostPipe {
  cudaStream_t up = nullptr, down = nullptr;  // upload, download
  cudaEvent_t chunk[kHostChunks] = {};
  cudaEvent_t blend_done = nullptr;
  cudaEvent_t inputs_free[2] = {};  // the projection that read input buffer f ended
  cudaEvent_t image_free[2] = {};   // the download of device image f ended
  int frame = 0;                    // frames queued so far
};
}  // namespace

struct lfd_plan {
  lfd_panel panel;
  lfd_opts opts;
  PanelGeom g;
  int device = 0;
  int flags = 0;
  int max_segment = 0;
  // panel tables
  uint8_t* V = nullptr;
  uint32_t* psi = nullptr;
  int32_t* n_sub = nullptr;
  int32_t* seg = nullptr;
  // per-frame scratch
  DevBuf proj_means, proj_co, proj_ct, proj_depth;
  DevBuf item_key[2], item_val[2];
  DevBuf counts, emit_pos, offsets, scan_tmp, bin_desc;
  DevBuf pair_key[2], pair_val[2];
  DevBuf radix_tmp;
  DevBuf ranges;
  DevBuf small;  // [0] total pairs, [1], [2] evaluation counters, [3] wait-error bits
  DevBuf host_in[2][5];  // device copies of host Gaussians (lfd_render_host), double-buffered
  DevBuf image[2];       // device images for lfd_render_host
  DevBuf g_means2d, g_conic, g_color, g_opac;  // backward scratch
  DevBuf keep;  // LFD_FLAG_KEEP_BLEND_STATE: [T][cap] stop index, final T
  HostPipe io;  // lfd_render_host streams and events (created on first use)
  bool io_ready = false;
  unsigned long long* h_small = nullptr;  // pinned
  // last frame
  int64_t last_P = -1;
  int64_t last_M = -1;
  bool last_from_render = false;
  bool last_kept = false;  // the last frame wrote the blend state into keep
  int last_key_buf = 0;
  int last_val_buf = 0;
  int last_sort_mode = 0;
  cudaStream_t last_stream = nullptr;
  // stage-timing events, two sets used alternately: [0] frame start, [1]
  // projection done, [2] key generation done, [3] sort + ranges done, [4]
  // blend done. A set's times are folded into acc_ms at the next frame's
  // pair-count synchronisation (when they are complete), or on request.
  cudaEvent_t ev[2][5] = {};
  int ev_set = 0;
  bool ev_pending[2] = {false, false};
  bool ev_has_project[2] = {false, false};
  double acc_ms[4] = {0, 0, 0, 0};
  int64_t acc_frames = 0;
  // capacity mode (lfd_plan_reserve): buffers preallocated for cap_M
  // Gaussians and cap_P pairs; frames then never allocate, synchronise or
  // read back, so they can be captured into a CUDA graph
  int64_t cap_M = 0;
  int64_t cap_P = 0;
  // full-frame baseline: a child plan with one view per cluster whose blend
  // renders whole per-view images (created on first use)
  bool fullframe = false;
  lfd_plan* ff_child = nullptr;
};

namespace {

int fold_stage_times(lfd_plan* p, int set) {
  if (!p->ev_pending[set]) return LFD_OK;
  float ms[4] = {0, 0, 0, 0};
  LFD_CUDA(cudaEventSynchronize(p->ev[set][4]));
  if (p->ev_has_project[set]) LFD_CUDA(cudaEventElapsedTime(&ms[0], p->ev[set][0], p->ev[set][1]));
  LFD_CUDA(cudaEventElapsedTime(&ms[1], p->ev[set][1], p->ev[set][2]));
  LFD_CUDA(cudaEventElapsedTime(&ms[2], p->ev[set][2], p->ev[set][3]));
  LFD_CUDA(cudaEventElapsedTime(&ms[3], p->ev[set][3], p->ev[set][4]));
  for (int a = 0; a < 4; ++a) p->acc_ms[a] += ms[a];
  p->acc_frames += 1;
  p->ev_pending[set] = false;
  return LFD_OK;
}

// A bounded device wait (the sort's bulk-copy waits) that gave up leaves bit 0 in
// the plan's error word; it is reported once, at the next read-back.
// (An overflow bit left by an earlier capacity-mode frame is cleared too.)
int take_wait_error(lfd_plan* p, cudaStream_t s) {
  const uint32_t bits = (uint32_t)(p->h_small[3] & 0xffffffffull);
  if (!bits) return LFD_OK;
  p->h_small[3] = 0;
  LFD_CUDA(cudaMemsetAsync(p->small.as<unsigned long long>() + 3, 0, sizeof(unsigned long long), s));
  if (!(bits & 1u)) return LFD_OK;
  return fail(LFD_ERR_TIMEOUT, "a bounded device wait of the sort gave up; the previous frame is wrong");
}

}  // namespace

namespace lfd {

int plan_view(const lfd_plan* p, PlanView* out) {
  if (!p || !out) return LFD_ERR_INVALID;
  out->g = p->g;
  out->psi = p->psi;
  out->seg = p->seg;
  out->max_segment = p->max_segment;
  out->sort_mode = p->opts.sort_mode;
  out->remap = p->opts.remap;
  out->V = p->V;
  out->bg[0] = p->opts.bg[0];
  out->bg[1] = p->opts.bg[1];
  out->bg[2] = p->opts.bg[2];
  out->h_small = p->h_small;
  out->subpixels_per_thread = p->opts.subpixels_per_thread;
  out->fullframe = p->fullframe;
  return LFD_OK;
}

int set_error(int code, const char* msg) { return fail(code, msg); }

int set_cuda_error(cudaError_t e, const char* where) { return fail_cuda(e, where); }

}  // namespace lfd

extern "C" {

int lfd_version(void) { return 100; }

// View-cone cameras (the "view cone" input of the problem statement and of
// Alg. 1): n pinhole cameras on a horizontal arc of the given radius around
// the world origin, all looking at it. Camera j sits at angle
// theta_j = -cone/2 + cone * j / (n - 1) (0 when n = 1) at
// (radius sin theta, 0, -radius cos theta); its axes are z towards the
// origin, y the world's y (down) made orthogonal, x = y cross z (so view 0,
// the leftmost camera, sees the scene from the left); R holds x, y, z as rows,
// t = -R c. fx = fy = (W / 2) / tan(fov_x / 2), (cx, cy) = (W / 2, H / 2).
// Computed in double precision, stored as float.
int lfd_make_arc_cameras(int32_t n, double cone_deg, double radius, double fov_x_deg,
                         int32_t width, int32_t height, lfd_camera* out) {
  if (!out) return lfd::set_error(LFD_ERR_INVALID, "lfd_make_arc_cameras: out is NULL");
  if (n < 1 || n > lfd::kMaxViews)
    return lfd::set_error(LFD_ERR_INVALID, "lfd_make_arc_cameras: n must be in [1, 255]");
  if (!(radius > 0.0) || !(fov_x_deg > 0.0 && fov_x_deg < 180.0) || !(cone_deg >= 0.0 && cone_deg < 360.0) ||
      width <= 0 || height <= 0)
    return lfd::set_error(LFD_ERR_INVALID,
                          "lfd_make_arc_cameras: radius > 0, 0 < fov < 180, 0 <= cone < 360, W, H > 0");
  const double kPi = 3.14159265358979323846;
  const double f = (width / 2.0) / tan(fov_x_deg * kPi / 180.0 / 2.0);
  for (int j = 0; j < n; ++j) {
    const double th = n == 1 ? 0.0 : (-cone_deg / 2.0 + cone_deg * j / (n - 1)) * kPi / 180.0;
    const double c[3] = {radius * sin(th), 0.0, -radius * cos(th)};
    const double cn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double z[3] = {-c[0] / cn, -c[1] / cn, -c[2] / cn};
    const double y0[3] = {0.0, 1.0, 0.0};
    double x[3] = {y0[1] * z[2] - y0[2] * z[1], y0[2] * z[0] - y0[0] * z[2], y0[0] * z[1] - y0[1] * z[0]};
    const double xn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    for (int i = 0; i < 3; ++i) x[i] /= xn;
    const double y[3] = {z[1] * x[2] - z[2] * x[1], z[2] * x[0] - z[0] * x[2], z[0] * x[1] - z[1] * x[0]};
    const double* rows[3] = {x, y, z};
    lfd_camera cam;
    for (int r = 0; r < 3; ++r) {
      for (int i = 0; i < 3; ++i) cam.R[3 * r + i] = (float)rows[r][i];
      cam.t[r] = (float)(-(rows[r][0] * c[0] + rows[r][1] * c[1] + rows[r][2] * c[2]));
    }
    cam.fx = cam.fy = (float)f;
    cam.cx = (float)(width / 2.0);
    cam.cy = (float)(height / 2.0);
    out[j] = cam;
  }
  return LFD_OK;
}

const char* lfd_status_string(int status) {
  switch (status) {
    case LFD_OK:
      return "ok";
    case LFD_ERR_INVALID:
      return "invalid argument";
    case LFD_ERR_OOM:
      return "out of device memory";
    case LFD_ERR_CAPACITY:
      return "pair count or key width beyond the supported limits";
    case LFD_ERR_CUDA:
      return "CUDA error";
    case LFD_ERR_STATE:
      return "requested data does not exist";
    case LFD_ERR_TIMEOUT:
      return "a bounded device wait gave up";
    default:
      return "unknown status";
  }
}

const char* lfd_last_error(void) { return g_last_error; }

void lfd_plan_destroy(lfd_plan* p) {
  if (!p) return;
  if (p->ff_child) lfd_plan_destroy(p->ff_child);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  cudaFree(p->V);
  cudaFree(p->psi);
  cudaFree(p->n_sub);
  cudaFree(p->seg);
  DevBuf* bufs[] = {&p->proj_means, &p->proj_co,   &p->proj_ct,     &p->proj_depth,
                    &p->item_key[0], &p->item_key[1], &p->item_val[0], &p->item_val[1],
                    &p->counts,     &p->emit_pos, &p->offsets,   &p->scan_tmp,    &p->bin_desc,  &p->pair_key[0],
                    &p->pair_key[1], &p->pair_val[0], &p->pair_val[1], &p->radix_tmp,
                    &p->ranges,     &p->small,     &p->host_in[0][0], &p->host_in[0][1],
                    &p->host_in[0][2], &p->host_in[0][3], &p->host_in[0][4], &p->host_in[1][0],
                    &p->host_in[1][1], &p->host_in[1][2], &p->host_in[1][3], &p->host_in[1][4],
                    &p->image[0],   &p->image[1],
                    &p->g_means2d,  &p->g_conic,   &p->g_color,     &p->g_opac, &p->keep};
  for (DevBuf* b : bufs) b->release();
  if (p->h_small) cudaFreeHost(p->h_small);
  for (auto& set : p->ev)
    for (cudaEvent_t& e : set)
      if (e) cudaEventDestroy(e);
  HostPipe& io = p->io;
  if (io.up) cudaStreamSynchronize(io.up);
  if (io.down) cudaStreamSynchronize(io.down);
  for (cudaEvent_t e : io.chunk)
    if (e) cudaEventDestroy(e);
  if (io.blend_done) cudaEventDestroy(io.blend_done);
  for (int f = 0; f < 2; ++f) {
    if (io.inputs_free[f]) cudaEventDestroy(io.inputs_free[f]);
    if (io.image_free[f]) cudaEventDestroy(io.image_free[f]);
  }
  if (io.up) cudaStreamDestroy(io.up);
  if (io.down) cudaStreamDestroy(io.down);
  delete p;
}

int lfd_plan_create(const lfd_panel* panel, const lfd_opts* opts, lfd_plan** out) {
  if (!out) return fail(LFD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!panel || !opts) return fail(LFD_ERR_INVALID, "panel or opts is NULL");
  const lfd_panel& P = *panel;
  const lfd_opts& O = *opts;
  if (P.width <= 0 || P.height <= 0 || P.width > 65535 || P.height > 65535)
    return fail(LFD_ERR_INVALID, "panel size out of range");
  if (P.num_views < 1 || P.num_views > kMaxViews) return fail(LFD_ERR_INVALID, "num_views not in [1, 255]");
  if (!(P.pitch > 0.0) || !isfinite(P.pitch) || !isfinite(P.tan_slant) || !isfinite(P.k_offset))
    return fail(LFD_ERR_INVALID, "pitch must be > 0 and parameters finite");
  if (O.tile_w < 4 || O.tile_h < 4 || O.tile_w > 64 || O.tile_h > 64 || O.tile_w * O.tile_h > 1024)
    return fail(LFD_ERR_INVALID, "tile shape out of range");
  if (O.views_per_cluster < 1 || O.views_per_cluster > kMaxClusterViews)
    return fail(LFD_ERR_INVALID, "views_per_cluster not in [1, 32]");
  if (O.remap != 0 && O.remap != 1) return fail(LFD_ERR_INVALID, "remap must be 0 or 1");
  if (O.sort_mode != LFD_SORT_DEPTH_FIRST && O.sort_mode != LFD_SORT_KEY64)
    return fail(LFD_ERR_INVALID, "unknown sort_mode");
  if (O.subpixels_per_thread != 0 && O.subpixels_per_thread != 1 && O.subpixels_per_thread != 2 &&
      O.subpixels_per_thread != 4 && O.subpixels_per_thread != 8)
    return fail(LFD_ERR_INVALID, "subpixels_per_thread must be 0, 1, 2, 4 or 8");

  lfd_plan* p = new (std::nothrow) lfd_plan();
  if (!p) return fail(LFD_ERR_OOM, "host allocation failed");
  p->panel = P;
  p->opts = O;
  cudaGetDevice(&p->device);
  PanelGeom& g = p->g;
  g.W = P.width;
  g.H = P.height;
  g.N = P.num_views;
  g.C = O.views_per_cluster;
  g.K = (g.N + g.C - 1) / g.C;
  g.TW = O.tile_w;
  g.TH = O.tile_h;
  g.TX = (g.W + g.TW - 1) / g.TW;
  g.TY = (g.H + g.TH - 1) / g.TH;
  g.T = g.TX * g.TY;
  g.cap = 3 * g.TW * g.TH;
  g.tw_magic = div_magic(g.TW);
  g.th_magic = div_magic(g.TH);
  g.bit_k = ceil_log2((uint64_t)g.K);
  g.bit_t = ceil_log2((uint64_t)g.T);
  if (g.bit_t + g.bit_k > 32) {
    delete p;
    return fail(LFD_ERR_CAPACITY, "tile and cluster bits exceed 32");
  }
  int rc = LFD_OK;
  auto cleanup = [&](int code) {
    lfd_plan_destroy(p);
    return code;
  };
  const size_t nsub = (size_t)g.W * g.H * 3;
  cudaError_t e;
  if ((e = cudaMalloc(&p->V, nsub)) != cudaSuccess) return cleanup(fail_cuda(e, "cudaMalloc V"));
  if ((e = cudaMalloc(&p->psi, (size_t)g.T * g.cap * sizeof(uint32_t))) != cudaSuccess)
    return cleanup(fail_cuda(e, "cudaMalloc psi"));
  if ((e = cudaMalloc(&p->n_sub, (size_t)g.T * sizeof(int32_t))) != cudaSuccess)
    return cleanup(fail_cuda(e, "cudaMalloc n_sub"));
  if ((e = cudaMalloc(&p->seg, (size_t)g.T * (g.K + 1) * sizeof(int32_t))) != cudaSuccess)
    return cleanup(fail_cuda(e, "cudaMalloc seg"));
  if ((e = cudaMallocHost(&p->h_small, 4 * sizeof(unsigned long long))) != cudaSuccess)
    return cleanup(fail_cuda(e, "cudaMallocHost"));
  if ((rc = p->small.ensure(4 * sizeof(unsigned long long))) != LFD_OK) return cleanup(rc);
  memset(p->h_small, 0, 4 * sizeof(unsigned long long));
  if ((e = cudaMemset(p->small.p, 0, 4 * sizeof(unsigned long long))) != cudaSuccess)
    return cleanup(fail_cuda(e, "cudaMemset"));
  for (auto& set : p->ev)
    for (cudaEvent_t& ev : set)
      if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cleanup(fail_cuda(e, "cudaEventCreate"));
  if ((e = launch_view_index(g.W, g.H, g.N, P.tan_slant, P.pitch, P.k_offset, p->V, 0)) != cudaSuccess)
    return cleanup(fail_cuda(e, "view_index"));
  if ((e = launch_remap(g, p->V, p->psi, p->n_sub, p->seg, 0)) != cudaSuccess)
    return cleanup(fail_cuda(e, "remap"));
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup(fail_cuda(e, "plan build"));
  // longest (tile, cluster) run, for the blend launch shape
  int32_t* hseg = (int32_t*)malloc((size_t)g.T * (g.K + 1) * sizeof(int32_t));
  if (!hseg) return cleanup(fail(LFD_ERR_OOM, "host allocation failed"));
  e = cudaMemcpy(hseg, p->seg, (size_t)g.T * (g.K + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free(hseg);
    return cleanup(fail_cuda(e, "copy seg"));
  }
  int mx = 0;
  for (int t = 0; t < g.T; ++t)
    for (int k = 0; k < g.K; ++k) {
      const int n = hseg[(size_t)t * (g.K + 1) + k + 1] - hseg[(size_t)t * (g.K + 1) + k];
      mx = n > mx ? n : mx;
    }
  free(hseg);
  p->max_segment = mx;
  *out = p;
  return LFD_OK;
}

int lfd_plan_get_info(const lfd_plan* p, lfd_plan_info* out) {
  if (!p || !out) return fail(LFD_ERR_INVALID, "NULL argument");
  out->num_clusters = p->g.K;
  out->tiles_x = p->g.TX;
  out->tiles_y = p->g.TY;
  out->tile_capacity = p->g.cap;
  out->bit_k = p->g.bit_k;
  out->bit_t = p->g.bit_t;
  out->max_segment = p->max_segment;
  return LFD_OK;
}

int lfd_set_flags(lfd_plan* p, int32_t flags) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  if (flags & ~(LFD_FLAG_STAGE_TIMING | LFD_FLAG_COUNT_EVALS | LFD_FLAG_KEEP_BLEND_STATE))
    return fail(LFD_ERR_INVALID, "unknown flag");
  if (flags & LFD_FLAG_KEEP_BLEND_STATE) {
    // allocated here so that frames in capacity mode stay allocation-free
    const int rc = p->keep.ensure((size_t)p->g.T * p->g.cap * sizeof(uint2));
    if (rc != LFD_OK) return rc;
  }
  p->flags = flags;
  return LFD_OK;
}

int lfd_plan_copy_tables(const lfd_plan* p, uint8_t* V, uint16_t* psi, int32_t* n_sub, int32_t* seg) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  const PanelGeom& g = p->g;
  if (V) LFD_CUDA(cudaMemcpy(V, p->V, (size_t)g.W * g.H * 3, cudaMemcpyDeviceToHost));
  if (psi) {
    const size_t n = (size_t)g.T * g.cap;
    uint32_t* tmp = (uint32_t*)malloc(n * sizeof(uint32_t));
    if (!tmp) return fail(LFD_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaMemcpy(tmp, p->psi, n * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      free(tmp);
      return fail_cuda(e, "copy psi");
    }
    for (size_t a = 0; a < n; ++a) psi[a] = (uint16_t)(tmp[a] & 0xffffu);
    free(tmp);
  }
  if (n_sub) LFD_CUDA(cudaMemcpy(n_sub, p->n_sub, (size_t)g.T * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (seg)
    LFD_CUDA(cudaMemcpy(seg, p->seg, (size_t)g.T * (g.K + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  return LFD_OK;
}

static int check_gaussians(const lfd_plan* p, const lfd_gaussians* gs) {
  if (!gs) return fail(LFD_ERR_INVALID, "gaussians is NULL");
  if (gs->count < 0) return fail(LFD_ERR_INVALID, "negative Gaussian count");
  if (gs->sh_degree < 0 || gs->sh_degree > 3) return fail(LFD_ERR_INVALID, "sh_degree not in [0, 3]");
  if (gs->attr_dtype != LFD_DTYPE_F32 && gs->attr_dtype != LFD_DTYPE_F16 &&
      gs->attr_dtype != LFD_DTYPE_BF16)
    return fail(LFD_ERR_INVALID, "unknown attr_dtype");
  if ((uint64_t)gs->count * (uint64_t)p->g.K >= (1ull << 32))
    return fail(LFD_ERR_CAPACITY, "count * clusters must stay below 2^32");
  if (gs->count > 0) {
    if (!gs->means || !gs->scales || !gs->quats || !gs->opacities || !gs->sh)
      return fail(LFD_ERR_INVALID, "NULL Gaussian attribute");
    const size_t es = gs->attr_dtype == LFD_DTYPE_F32 ? 4 : 2;
    if (!aligned(gs->means, 4) || !aligned(gs->quats, es) || !aligned(gs->scales, es) ||
        !aligned(gs->opacities, es) || !aligned(gs->sh, es))
      return fail(LFD_ERR_INVALID, "Gaussian attributes misaligned for their type");
  }
  return LFD_OK;
}

static int fill_cams(const lfd_plan* p, const lfd_camera* cams, int32_t num_cams, CamTable* t) {
  if (!cams) return fail(LFD_ERR_INVALID, "cams is NULL");
  if (num_cams != p->g.N) return fail(LFD_ERR_INVALID, "num_cams must equal the panel's num_views");
  memset(t, 0, sizeof(*t));
  for (int j = 0; j < num_cams; ++j) {
    memcpy(t->c[j], cams[j].R, 9 * sizeof(float));
    memcpy(t->c[j] + 9, cams[j].t, 3 * sizeof(float));
    t->c[j][12] = cams[j].fx;
    t->c[j][13] = cams[j].fy;
    t->c[j][14] = cams[j].cx;
    t->c[j][15] = cams[j].cy;
  }
  return LFD_OK;
}

// Projection of every Gaussian; with io, the attributes are first copied from
// the host in chunks on the transfer stream, each chunk projected after it
// has landed.
static int project_impl(lfd_plan* p, const lfd_gaussians* gs, const lfd_camera* cams,
                        int32_t num_cams, float* means2d, float* conic_opacity, float* color_tau,
                        float* depth, void* stream, const HostIO* io) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  int rc = check_gaussians(p, gs);
  if (rc != LFD_OK) return rc;
  CamTable* t = new (std::nothrow) CamTable;
  if (!t) return fail(LFD_ERR_OOM, "host allocation failed");
  rc = fill_cams(p, cams, num_cams, t);
  if (rc == LFD_OK && gs->count > 0) {
    if (!means2d || !conic_opacity || !color_tau || !depth)
      rc = fail(LFD_ERR_INVALID, "NULL output buffer");
    else if (!aligned(conic_opacity, 16) || !aligned(color_tau, 16) || !aligned(means2d, 8))
      rc = fail(LFD_ERR_INVALID, "output buffers misaligned");
  }
  if (rc == LFD_OK) {
    ProjectArgs a;
    a.means = gs->means;
    a.scales = gs->scales;
    a.quats = gs->quats;
    a.opac = gs->opacities;
    a.sh = gs->sh;
    a.M = gs->count;
    a.sh_degree = gs->sh_degree;
    a.attr_dtype = gs->attr_dtype;
    a.means2d = means2d;
    a.conic_opacity = conic_opacity;
    a.color_tau = color_tau;
    a.depth = depth;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!io) {
      e = launch_project(p->g, *t, a, s);
    } else {
      // the upload overwrites input buffers the projection two frames ago read
      HostPipe& hp = p->io;
      e = cudaStreamWaitEvent(hp.up, hp.inputs_free[io->parity], 0);
      const int64_t M = gs->count;
      for (int c = 0; c < kHostChunks && e == cudaSuccess; ++c) {
        const int64_t m0 = M * c / kHostChunks, m1 = M * (c + 1) / kHostChunks;
        if (m1 == m0) continue;
        for (int b = 0; b < 5 && e == cudaSuccess; ++b)
          e = cudaMemcpyAsync(static_cast<char*>(io->dst[b]) + m0 * io->elem_bytes[b],
                              static_cast<const char*>(io->src[b]) + m0 * io->elem_bytes[b],
                              (size_t)(m1 - m0) * io->elem_bytes[b], cudaMemcpyHostToDevice, hp.up);
        if (e == cudaSuccess) e = cudaEventRecord(hp.chunk[c], hp.up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hp.chunk[c], 0);
        a.m_begin = m0;
        a.m_end = m1;
        if (e == cudaSuccess) e = launch_project(p->g, *t, a, s);
      }
      if (e == cudaSuccess) e = cudaEventRecord(hp.inputs_free[io->parity], s);
    }
    if (e != cudaSuccess) rc = fail_cuda(e, "project");
  }
  delete t;
  return rc;
}

int lfd_project(lfd_plan* p, const lfd_gaussians* gs, const lfd_camera* cams, int32_t num_cams,
                float* means2d, float* conic_opacity, float* color_tau, float* depth, void* stream) {
  return project_impl(p, gs, cams, num_cams, means2d, conic_opacity, color_tau, depth, stream, nullptr);
}

// Stages 2-4 from projected attributes. With io, the image also goes back to
// io->out_host on the download stream.
static int render_projected_impl(lfd_plan* p, int64_t M, const float* means2d,
                                 const float* conic_opacity, const float* color_tau,
                                 const float* depth, float* out_rgb, void* stream, lfd_stats* stats,
                                 bool projected_here, const HostIO* io = nullptr) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  const PanelGeom& g = p->g;
  cudaStream_t s = (cudaStream_t)stream;
  if (M < 0) return fail(LFD_ERR_INVALID, "negative Gaussian count");
  if ((uint64_t)M * (uint64_t)g.K >= (1ull << 32)) return fail(LFD_ERR_CAPACITY, "M * K must stay below 2^32");
  if (!out_rgb) return fail(LFD_ERR_INVALID, "out_rgb is NULL");
  if (M > 0 && (!means2d || !conic_opacity || !color_tau || !depth))
    return fail(LFD_ERR_INVALID, "NULL attribute buffer");
  if (M > 0 && (!aligned(conic_opacity, 16) || !aligned(color_tau, 16) || !aligned(means2d, 8)))
    return fail(LFD_ERR_INVALID, "attribute buffers misaligned");
  const bool capmode = p->cap_P > 0;
  if (capmode && M > p->cap_M) return fail(LFD_ERR_CAPACITY, "more Gaussians than reserved");
  const bool timing = (p->flags & LFD_FLAG_STAGE_TIMING) != 0 && !capmode;
  const bool counting = (p->flags & LFD_FLAG_COUNT_EVALS) != 0 && !capmode;
  const bool key64 = p->opts.sort_mode == LFD_SORT_KEY64;
  const int64_t n_items = (int64_t)g.K * M;
  int rc;
  unsigned long long* d_small = p->small.as<unsigned long long>();
  uint32_t* d_err = reinterpret_cast<uint32_t*>(d_small + 3);
  const int es = p->ev_set;
  cudaEvent_t* ev = p->ev[es];
  if (timing) {
    if (!projected_here) LFD_CUDA(cudaEventRecord(ev[0], s));
    LFD_CUDA(cudaEventRecord(ev[1], s));
  }

  // ---- stage 2: key generation ----
  if ((rc = p->counts.ensure((size_t)(n_items + 1) * 4)) != LFD_OK) return rc;
  if ((rc = p->offsets.ensure((size_t)(n_items + 1) * 4)) != LFD_OK) return rc;
  if ((rc = p->emit_pos.ensure((size_t)(n_items + 1) * 4)) != LFD_OK) return rc;
  if ((rc = p->scan_tmp.ensure(scan_temp_bytes(n_items + 1))) != LFD_OK) return rc;
  if ((rc = p->bin_desc.ensure((size_t)(n_items + 1) * kBinDescBytes)) != LFD_OK) return rc;
  const uint32_t* order = nullptr;
  if (!key64) {
    // depth-first order: sort the K*M (cluster, depth) items once
    for (int b = 0; b < 2; ++b) {
      if ((rc = p->item_key[b].ensure((size_t)(n_items + 1) * 8)) != LFD_OK) return rc;
      if ((rc = p->item_val[b].ensure((size_t)(n_items + 1) * 4)) != LFD_OK) return rc;
    }
    if ((rc = p->radix_tmp.ensure(radix_temp_bytes(n_items, 8))) != LFD_OK) return rc;
    LFD_CUDA(launch_item_keys(g, M, depth, color_tau, p->item_key[0].as<uint64_t>(),
                              p->item_val[0].as<uint32_t>(), s));
    bool alt = false;
    LFD_CUDA(radix_sort_u64(p->item_key[0].as<uint64_t>(), p->item_key[1].as<uint64_t>(),
                            p->item_val[0].as<uint32_t>(), p->item_val[1].as<uint32_t>(), n_items,
                            nullptr, 0, 32 + g.bit_k, p->radix_tmp.p, &alt, d_err, s));
    order = p->item_val[alt ? 1 : 0].as<uint32_t>();
  }
  // tile counts and union descriptors: the count pass reads the items in
  // natural (cluster, Gaussian) order (coalesced attribute reads) and writes
  // each item's count and descriptor at its emission position, so that the
  // offsets scan and the emit pass read them in order
  uint32_t* emit_pos = nullptr;
  if (order) {
    emit_pos = p->emit_pos.as<uint32_t>();
    LFD_CUDA(launch_invert_u32(order, n_items, emit_pos, s));
  }
  LFD_CUDA(launch_bin_count(g, M, means2d, conic_opacity, color_tau, nullptr, emit_pos, n_items,
                            p->counts.as<uint32_t>(), p->bin_desc.p, s));
  LFD_CUDA(scan_exclusive(p->counts.as<uint32_t>(), p->offsets.as<uint32_t>(), n_items, p->scan_tmp.p,
                          d_small, s));
  unsigned long long P = (unsigned long long)p->cap_P;
  if (!capmode) {
    LFD_CUDA(cudaMemcpyAsync(p->h_small, d_small, 4 * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, s));
    LFD_CUDA(cudaStreamSynchronize(s));
    if ((rc = fold_stage_times(p, es ^ 1)) != LFD_OK) return rc;
    if ((rc = take_wait_error(p, s)) != LFD_OK) return rc;
    P = p->h_small[0];
    if (P >= 0xffffffffull) return fail(LFD_ERR_CAPACITY, "more than 2^32 - 1 Gaussian-tile pairs");
  }
  // from here on P bounds the pair count; the kernels read the exact count
  // (and, in capacity mode, whether it fits) from d_small[0]
  const size_t kbytes = key64 ? 8 : 4;
  for (int b = 0; b < 2; ++b) {
    if ((rc = p->pair_key[b].ensure((size_t)(P + 1) * kbytes)) != LFD_OK) return rc;
    if ((rc = p->pair_val[b].ensure((size_t)(P + 1) * 4)) != LFD_OK) return rc;
  }
  if ((rc = p->radix_tmp.ensure(radix_temp_bytes((int64_t)P, (int)kbytes))) != LFD_OK) return rc;
  if ((rc = p->ranges.ensure((size_t)g.T * g.K * sizeof(uint2))) != LFD_OK) return rc;
  LFD_CUDA(launch_bin_emit_coop(g, M, means2d, conic_opacity, color_tau, depth, order, n_items,
                                p->counts.as<uint32_t>(), p->offsets.as<uint32_t>(),
                                key64 ? nullptr : p->pair_key[0].as<uint32_t>(),
                                key64 ? p->pair_key[0].as<uint64_t>() : nullptr,
                                p->pair_val[0].as<uint32_t>(), p->bin_desc.p, d_small, P, d_err,
                                s));
  if (timing) LFD_CUDA(cudaEventRecord(ev[2], s));

  // ---- stage 3: sort by (tile, cluster, depth) ----
  // Depth-first mode emits the pairs in (cluster, depth, id) order, so a
  // stable sort on the tile bits alone yields (tile, cluster, depth, id).
  bool alt = false;
  if (key64)
    LFD_CUDA(radix_sort_u64(p->pair_key[0].as<uint64_t>(), p->pair_key[1].as<uint64_t>(),
                            p->pair_val[0].as<uint32_t>(), p->pair_val[1].as<uint32_t>(), (int64_t)P,
                            d_small, 0, 32 + g.bit_k + g.bit_t, p->radix_tmp.p, &alt, d_err, s));
  else
    LFD_CUDA(radix_sort_u32(p->pair_key[0].as<uint32_t>(), p->pair_key[1].as<uint32_t>(),
                            p->pair_val[0].as<uint32_t>(), p->pair_val[1].as<uint32_t>(), (int64_t)P,
                            d_small, g.bit_k, g.bit_k + g.bit_t, p->radix_tmp.p, &alt, d_err, s));
  const int kb = alt ? 1 : 0;
  LFD_CUDA(launch_ranges(g, (int64_t)P, d_small, key64 ? nullptr : p->pair_key[kb].as<uint32_t>(),
                         key64 ? p->pair_key[kb].as<uint64_t>() : nullptr, p->ranges.as<uint2>(), s));
  if (timing) LFD_CUDA(cudaEventRecord(ev[3], s));

  // ---- stage 4: subpixel blend with view-coherent remapping ----
  if (counting) LFD_CUDA(cudaMemsetAsync(d_small + 1, 0, 2 * sizeof(unsigned long long), s));
  BlendArgs ba;
  ba.psi = p->psi;
  ba.seg = p->seg;
  ba.ranges = p->ranges.as<uint2>();
  ba.list = p->pair_val[kb].as<uint32_t>();
  ba.means2d = means2d;
  ba.conic_opacity = conic_opacity;
  ba.color_tau = color_tau;
  ba.M = M;
  ba.bg[0] = p->opts.bg[0];
  ba.bg[1] = p->opts.bg[1];
  ba.bg[2] = p->opts.bg[2];
  ba.out = out_rgb;
  ba.eval_counter = counting ? d_small + 1 : nullptr;
  ba.max_segment = p->max_segment;
  ba.V = p->V;
  ba.P_dev = d_small;
  ba.P_cap = P;
  ba.subpixels_per_thread = p->opts.subpixels_per_thread;
  const bool kept = (p->flags & LFD_FLAG_KEEP_BLEND_STATE) && p->opts.remap && !p->fullframe;
  ba.keep = kept ? p->keep.as<uint2>() : nullptr;
  const size_t row_floats = (size_t)g.W * 3;
  // the device image is written once the download of its previous frame has ended
  if (io) LFD_CUDA(cudaStreamWaitEvent(s, p->io.image_free[io->parity], 0));
  if (p->fullframe)
    LFD_CUDA(launch_blend_fullframe(g, ba, s));
  else if (p->opts.remap)
    LFD_CUDA(launch_blend(g, ba, s));
  else
    LFD_CUDA(launch_blend_raster(g, ba, s));
  if (io) {
    HostPipe& hp = p->io;
    LFD_CUDA(cudaEventRecord(hp.blend_done, s));
    LFD_CUDA(cudaStreamWaitEvent(hp.down, hp.blend_done, 0));
    LFD_CUDA(cudaMemcpyAsync(io->out_host, out_rgb, (size_t)g.H * row_floats * sizeof(float),
                             cudaMemcpyDeviceToHost, hp.down));
    LFD_CUDA(cudaEventRecord(hp.image_free[io->parity], hp.down));
  }
  if (timing) {
    LFD_CUDA(cudaEventRecord(ev[4], s));
    p->ev_pending[es] = true;
    p->ev_has_project[es] = projected_here;
    p->ev_set = es ^ 1;
  }

  p->last_P = capmode ? -2 : (int64_t)P;  // -2: the count is on the device
  p->last_M = M;
  p->last_from_render = projected_here;
  p->last_kept = kept;
  p->last_key_buf = kb;
  p->last_val_buf = kb;
  p->last_sort_mode = p->opts.sort_mode;
  p->last_stream = s;
  if (stats) {
    stats->num_pairs = capmode ? -1 : (int64_t)P;
    stats->num_visits = -1;
    stats->num_evals = -1;
    stats->ms_project = stats->ms_keygen = stats->ms_sort = stats->ms_blend = -1.f;
    if (counting || timing) {
      if (counting)
        LFD_CUDA(cudaMemcpyAsync(p->h_small + 1, d_small + 1, 2 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
      LFD_CUDA(cudaStreamSynchronize(s));
      if (counting) {
        stats->num_visits = (int64_t)p->h_small[1];
        stats->num_evals = (int64_t)p->h_small[2];
      }
      if (timing) {
        if (projected_here) LFD_CUDA(cudaEventElapsedTime(&stats->ms_project, ev[0], ev[1]));
        LFD_CUDA(cudaEventElapsedTime(&stats->ms_keygen, ev[1], ev[2]));
        LFD_CUDA(cudaEventElapsedTime(&stats->ms_sort, ev[2], ev[3]));
        LFD_CUDA(cudaEventElapsedTime(&stats->ms_blend, ev[3], ev[4]));
      }
    }
  }
  return LFD_OK;
}

int lfd_render_projected(lfd_plan* p, int64_t M, const float* means2d, const float* conic_opacity,
                         const float* color_tau, const float* depth, float* out_rgb, void* stream,
                         lfd_stats* stats) {
  return render_projected_impl(p, M, means2d, conic_opacity, color_tau, depth, out_rgb, stream,
                               stats, false);
}

static int render_impl(lfd_plan* p, const lfd_gaussians* gs, const lfd_camera* cams, int32_t num_cams,
                       float* out_rgb, void* stream, lfd_stats* stats, const HostIO* io) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  int rc = check_gaussians(p, gs);
  if (rc != LFD_OK) return rc;
  const PanelGeom& g = p->g;
  const int64_t M = gs->count;
  const int64_t n_items = (int64_t)g.K * M;
  if ((rc = p->proj_means.ensure((size_t)(n_items * g.C + 1) * 8)) != LFD_OK) return rc;
  if ((rc = p->proj_co.ensure((size_t)(n_items + 1) * 16)) != LFD_OK) return rc;
  if ((rc = p->proj_ct.ensure((size_t)(n_items + 1) * 16)) != LFD_OK) return rc;
  if ((rc = p->proj_depth.ensure((size_t)(n_items + 1) * 4)) != LFD_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const bool timing = (p->flags & LFD_FLAG_STAGE_TIMING) != 0;
  if (timing) LFD_CUDA(cudaEventRecord(p->ev[p->ev_set][0], s));
  rc = project_impl(p, gs, cams, num_cams, p->proj_means.as<float>(), p->proj_co.as<float>(),
                    p->proj_ct.as<float>(), p->proj_depth.as<float>(), stream, io);
  if (rc != LFD_OK) return rc;
  return render_projected_impl(p, M, p->proj_means.as<float>(), p->proj_co.as<float>(),
                               p->proj_ct.as<float>(), p->proj_depth.as<float>(), out_rgb, stream,
                               stats, true, io);
}

int lfd_render(lfd_plan* p, const lfd_gaussians* gs, const lfd_camera* cams, int32_t num_cams,
               float* out_rgb, void* stream, lfd_stats* stats) {
  return render_impl(p, gs, cams, num_cams, out_rgb, stream, stats, nullptr);
}

int lfd_render_backward(lfd_plan* p, const lfd_gaussians* gs, const lfd_camera* cams,
                        int32_t num_cams, const float* grad_rgb, float* grad_means,
                        float* grad_scales, float* grad_quats, float* grad_opacities,
                        float* grad_sh, void* stream) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  int rc = check_gaussians(p, gs);
  if (rc != LFD_OK) return rc;
  if (gs->attr_dtype != LFD_DTYPE_F32) return fail(LFD_ERR_INVALID, "backward needs FP32 attributes");
  if (!p->opts.remap || p->fullframe) return fail(LFD_ERR_INVALID, "backward needs the remapped plan");
  if (!p->last_from_render || p->last_M != gs->count)
    return fail(LFD_ERR_STATE, "backward needs the forward frame of lfd_render with the same Gaussians");
  const int64_t M = gs->count;
  if (M == 0) return LFD_OK;
  if (!grad_rgb || !grad_means || !grad_scales || !grad_quats || !grad_opacities || !grad_sh)
    return fail(LFD_ERR_INVALID, "NULL gradient buffer");
  CamTable* t = new (std::nothrow) CamTable;
  if (!t) return fail(LFD_ERR_OOM, "host allocation failed");
  rc = fill_cams(p, cams, num_cams, t);
  if (rc != LFD_OK) {
    delete t;
    return rc;
  }
  const PanelGeom& g = p->g;
  const int64_t n_items = (int64_t)g.K * M;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = p->g_means2d.ensure((size_t)n_items * g.C * 8)) != LFD_OK ||
      (rc = p->g_conic.ensure((size_t)n_items * 16)) != LFD_OK ||
      (rc = p->g_color.ensure((size_t)n_items * 16)) != LFD_OK ||
      (rc = p->g_opac.ensure((size_t)M * 4)) != LFD_OK) {
    delete t;
    return rc;
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemsetAsync(p->g_means2d.p, 0, (size_t)n_items * g.C * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->g_conic.p, 0, (size_t)n_items * 16, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->g_color.p, 0, (size_t)n_items * 16, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->g_opac.p, 0, (size_t)M * 4, s);
  BlendArgs ba;
  ba.psi = p->psi;
  ba.seg = p->seg;
  ba.ranges = p->ranges.as<uint2>();
  ba.list = p->pair_val[p->last_val_buf].as<uint32_t>();
  ba.means2d = p->proj_means.as<float>();
  ba.conic_opacity = p->proj_co.as<float>();
  ba.color_tau = p->proj_ct.as<float>();
  ba.M = M;
  ba.bg[0] = p->opts.bg[0];
  ba.bg[1] = p->opts.bg[1];
  ba.bg[2] = p->opts.bg[2];
  ba.out = nullptr;
  ba.eval_counter = nullptr;
  ba.max_segment = p->max_segment;
  ba.V = p->V;
  ba.keep = p->last_kept ? p->keep.as<uint2>() : nullptr;
  BlendGrads gr;
  gr.grad_out = grad_rgb;
  gr.grad_means2d = p->g_means2d.as<float>();
  gr.grad_conic = p->g_conic.as<float>();
  gr.grad_color = p->g_color.as<float>();
  gr.grad_opac = p->g_opac.as<float>();
  if (e == cudaSuccess) e = launch_blend_backward(g, ba, gr, s);
  ProjectArgs a;
  a.means = gs->means;
  a.scales = gs->scales;
  a.quats = gs->quats;
  a.opac = gs->opacities;
  a.sh = gs->sh;
  a.M = M;
  a.sh_degree = gs->sh_degree;
  a.attr_dtype = gs->attr_dtype;
  a.means2d = p->proj_means.as<float>();
  a.conic_opacity = p->proj_co.as<float>();
  a.color_tau = p->proj_ct.as<float>();
  a.depth = p->proj_depth.as<float>();
  ParamGrads out = {grad_means, grad_scales, grad_quats, grad_opacities, grad_sh};
  if (e == cudaSuccess) e = launch_project_backward(g, *t, a, gr, out, s);
  delete t;
  if (e != cudaSuccess) return fail_cuda(e, "backward");
  return LFD_OK;
}

int lfd_render_fullframe(lfd_plan* p, const lfd_gaussians* gs, const lfd_camera* cams,
                         int32_t num_cams, float* out_rgb, void* stream, lfd_stats* stats) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  if (!p->ff_child) {
    lfd_opts o = p->opts;
    o.views_per_cluster = 1;
    o.remap = 1;
    // the full-frame blend runs one thread per pixel of a tile, at most 512
    if (o.tile_w * o.tile_h > 512) o.tile_h = 512 / o.tile_w;
    int rc = lfd_plan_create(&p->panel, &o, &p->ff_child);
    if (rc != LFD_OK) return rc;
    p->ff_child->fullframe = true;
  }
  p->ff_child->flags = p->flags;
  return lfd_render(p->ff_child, gs, cams, num_cams, out_rgb, stream, stats);
}

static int create_host_pipe(HostPipe& hp) {
  if (!hp.up) LFD_CUDA(cudaStreamCreateWithFlags(&hp.up, cudaStreamNonBlocking));
  if (!hp.down) LFD_CUDA(cudaStreamCreateWithFlags(&hp.down, cudaStreamNonBlocking));
  cudaEvent_t* evs[] = {&hp.chunk[0],       &hp.chunk[1],       &hp.chunk[2],      &hp.chunk[3],
                        &hp.blend_done,     &hp.inputs_free[0], &hp.inputs_free[1], &hp.image_free[0],
                        &hp.image_free[1]};
  static_assert(kHostChunks == 4, "event list");
  for (cudaEvent_t* e : evs)
    if (!*e) LFD_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return LFD_OK;
}

// let every copy the host pipe has queued finish (they read or write the
// caller's host buffers)
static cudaError_t drain_host_pipe(const HostPipe& hp) {
  cudaError_t e1 = hp.up ? cudaStreamSynchronize(hp.up) : cudaSuccess;
  cudaError_t e2 = hp.down ? cudaStreamSynchronize(hp.down) : cudaSuccess;
  return e1 != cudaSuccess ? e1 : e2;
}

int lfd_render_host_async(lfd_plan* p, const lfd_gaussians* gh, const lfd_camera* cams,
                          int32_t num_cams, float* out_rgb_host, void* stream, lfd_stats* stats) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  if (!out_rgb_host) return fail(LFD_ERR_INVALID, "out_rgb_host is NULL");
  if (!gh) return fail(LFD_ERR_INVALID, "gaussians is NULL");
  const int64_t M = gh->count;
  if (M < 0 || gh->sh_degree < 0 || gh->sh_degree > 3) return fail(LFD_ERR_INVALID, "bad Gaussian set");
  int rc;
  if (!p->io_ready) {
    if ((rc = create_host_pipe(p->io)) != LFD_OK) return rc;
    p->io_ready = true;
  }
  const int f = p->io.frame & 1;
  const int ncoef = (gh->sh_degree + 1) * (gh->sh_degree + 1);
  const size_t es = gh->attr_dtype == LFD_DTYPE_F32 ? 4 : 2;
  HostIO io;
  io.parity = f;
  const size_t eb[5] = {12, 3 * es, 4 * es, es, (size_t)ncoef * 3 * es};
  const void* src[5] = {gh->means, gh->scales, gh->quats, gh->opacities, gh->sh};
  for (int b = 0; b < 5; ++b) {
    if (M > 0 && !src[b]) return fail(LFD_ERR_INVALID, "NULL Gaussian attribute");
    if ((rc = p->host_in[f][b].ensure((size_t)M * eb[b] + 16)) != LFD_OK) return rc;
    io.src[b] = src[b];
    io.dst[b] = p->host_in[f][b].p;
    io.elem_bytes[b] = eb[b];
  }
  io.out_host = out_rgb_host;
  const size_t out_bytes = (size_t)p->g.W * p->g.H * 3 * sizeof(float);
  if ((rc = p->image[f].ensure(out_bytes)) != LFD_OK) return rc;
  lfd_gaussians gd = *gh;
  gd.means = p->host_in[f][0].as<float>();
  gd.scales = p->host_in[f][1].p;
  gd.quats = p->host_in[f][2].p;
  gd.opacities = p->host_in[f][3].p;
  gd.sh = p->host_in[f][4].p;
  rc = render_impl(p, &gd, cams, num_cams, p->image[f].as<float>(), stream, stats, &io);
  ++p->io.frame;
  if (rc != LFD_OK) {
    drain_host_pipe(p->io);
    return rc;
  }
  return LFD_OK;
}

int lfd_render_host_wait(lfd_plan* p) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  const cudaError_t e = drain_host_pipe(p->io);
  if (e != cudaSuccess) return fail_cuda(e, "host transfers");
  return LFD_OK;
}

int lfd_render_host(lfd_plan* p, const lfd_gaussians* gh, const lfd_camera* cams, int32_t num_cams,
                    float* out_rgb_host, void* stream, lfd_stats* stats) {
  const int rc = lfd_render_host_async(p, gh, cams, num_cams, out_rgb_host, stream, stats);
  if (rc != LFD_OK) return rc;
  return lfd_render_host_wait(p);
}

int lfd_plan_reserve(lfd_plan* p, int64_t max_gaussians, int64_t max_pairs) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  if (max_gaussians < 0 || max_pairs < 0) return fail(LFD_ERR_INVALID, "negative capacity");
  if (p->fullframe) return fail(LFD_ERR_INVALID, "capacity mode is for the subpixel path");
  if (max_pairs == 0) {
    p->cap_M = p->cap_P = 0;
    return LFD_OK;
  }
  const PanelGeom& g = p->g;
  if (max_pairs >= 0xffffffffll) return fail(LFD_ERR_CAPACITY, "more than 2^32 - 1 pairs");
  if ((uint64_t)max_gaussians * (uint64_t)g.K >= (1ull << 32))
    return fail(LFD_ERR_CAPACITY, "M * K must stay below 2^32");
  const int64_t n = (int64_t)g.K * max_gaussians;
  int rc;
  const size_t items4 = (size_t)(n + 1) * 4;
  const int pair_key_bytes = p->opts.sort_mode == LFD_SORT_KEY64 ? 8 : 4;
  const size_t sort_tmp = radix_temp_bytes(n, 8) > radix_temp_bytes(max_pairs, pair_key_bytes)
                              ? radix_temp_bytes(n, 8)
                              : radix_temp_bytes(max_pairs, pair_key_bytes);
  if ((rc = p->proj_means.ensure((size_t)(n * g.C + 1) * 8)) != LFD_OK ||
      (rc = p->proj_co.ensure((size_t)(n + 1) * 16)) != LFD_OK ||
      (rc = p->proj_ct.ensure((size_t)(n + 1) * 16)) != LFD_OK ||
      (rc = p->proj_depth.ensure(items4)) != LFD_OK || (rc = p->counts.ensure(items4)) != LFD_OK ||
      (rc = p->offsets.ensure(items4)) != LFD_OK || (rc = p->emit_pos.ensure(items4)) != LFD_OK ||
      (rc = p->scan_tmp.ensure(scan_temp_bytes(n + 1))) != LFD_OK ||
      (rc = p->bin_desc.ensure((size_t)(n + 1) * kBinDescBytes)) != LFD_OK ||
      (rc = p->radix_tmp.ensure(sort_tmp)) != LFD_OK ||
      (rc = p->ranges.ensure((size_t)g.T * g.K * sizeof(uint2))) != LFD_OK)
    return rc;
  for (int b = 0; b < 2; ++b) {
    if ((rc = p->item_key[b].ensure((size_t)(n + 1) * 8)) != LFD_OK ||
        (rc = p->item_val[b].ensure(items4)) != LFD_OK ||
        (rc = p->pair_key[b].ensure((size_t)(max_pairs + 1) * 8)) != LFD_OK ||
        (rc = p->pair_val[b].ensure((size_t)(max_pairs + 1) * 4)) != LFD_OK)
      return rc;
  }
  p->cap_M = max_gaussians;
  p->cap_P = max_pairs;
  return LFD_OK;
}

int lfd_plan_status(lfd_plan* p, int64_t* pairs) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  LFD_CUDA(cudaDeviceSynchronize());
  unsigned long long h[4];
  LFD_CUDA(cudaMemcpy(h, p->small.p, sizeof(h), cudaMemcpyDeviceToHost));
  if (pairs) *pairs = (int64_t)h[0];
  const uint32_t bits = (uint32_t)(h[3] & 0xffffffffull);
  if (!bits) return LFD_OK;
  LFD_CUDA(cudaMemset(p->small.as<unsigned long long>() + 3, 0, sizeof(unsigned long long)));
  if (bits & 1u) return fail(LFD_ERR_TIMEOUT, "a bounded device wait of the sort gave up");
  char msg[160];
  snprintf(msg, sizeof(msg), "a frame had more pairs than reserved (last frame: %llu, reserved: %lld)",
           h[0], (long long)p->cap_P);
  return fail(LFD_ERR_CAPACITY, msg);
}

int lfd_plan_copy_lists(const lfd_plan* p, uint32_t* list, uint32_t* ranges, uint64_t* keys,
                        int64_t capacity) {
  if (!p) return fail(LFD_ERR_INVALID, "NULL plan");
  if (p->last_P == -1) return fail(LFD_ERR_STATE, "no frame rendered yet");
  if (keys && p->last_sort_mode != LFD_SORT_KEY64)
    return fail(LFD_ERR_STATE, "keys exist only with LFD_SORT_KEY64");
  LFD_CUDA(cudaStreamSynchronize(p->last_stream));
  int64_t P = p->last_P;
  if (P == -2) {  // capacity mode: the count is on the device
    LFD_CUDA(cudaDeviceSynchronize());
    unsigned long long h = 0;
    LFD_CUDA(cudaMemcpy(&h, p->small.p, sizeof(h), cudaMemcpyDeviceToHost));
    if ((int64_t)h > p->cap_P) return fail(LFD_ERR_CAPACITY, "the last frame overflowed its capacity");
    P = (int64_t)h;
  }
  if ((list || keys) && capacity < P) return fail(LFD_ERR_INVALID, "capacity below the pair count");
  if (list && P > 0)
    LFD_CUDA(cudaMemcpy(list, p->pair_val[p->last_val_buf].p, (size_t)P * 4, cudaMemcpyDeviceToHost));
  if (keys && P > 0)
    LFD_CUDA(cudaMemcpy(keys, p->pair_key[p->last_key_buf].p, (size_t)P * 8, cudaMemcpyDeviceToHost));
  if (ranges)
    LFD_CUDA(cudaMemcpy(ranges, p->ranges.p, (size_t)p->g.T * p->g.K * sizeof(uint2),
                        cudaMemcpyDeviceToHost));
  return LFD_OK;
}

int lfd_get_stage_totals(lfd_plan* p, lfd_stage_times* out, int32_t reset) {
  if (!p || !out) return fail(LFD_ERR_INVALID, "NULL argument");
  if (p->ev_pending[0] || p->ev_pending[1]) {
    LFD_CUDA(cudaStreamSynchronize(p->last_stream));
    int rc;
    // fold the older set first so frames are counted in order
    const int older = p->ev_set;
    if ((rc = fold_stage_times(p, older)) != LFD_OK) return rc;
    if ((rc = fold_stage_times(p, older ^ 1)) != LFD_OK) return rc;
  }
  out->frames = p->acc_frames;
  out->ms_project = p->acc_ms[0];
  out->ms_keygen = p->acc_ms[1];
  out->ms_sort = p->acc_ms[2];
  out->ms_blend = p->acc_ms[3];
  if (reset) {
    p->acc_frames = 0;
    for (double& a : p->acc_ms) a = 0.0;
  }
  return LFD_OK;
}

uint64_t lfd_kernel_launches(void) { return lfd::launch_count(); }

}  // extern "C"
