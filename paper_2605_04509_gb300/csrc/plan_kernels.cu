// Panel tables: view index matrix V (Sec. 3.1, Eq. 1-3) and the
// view-coherent remap table Psi with its per-cluster runs (Sec. 4.3, Eq. 8).
// Built once per plan; not on the per-frame path.
#include "lfd_internal.h"

namespace lfd {
namespace {

// Eq. 1-3 in FP64 with every operation correctly rounded in a fixed order
// (no contraction), so that the integer result is reproducible exactly:
//   d = ((3x + u) + (3y) tan(alpha)) - K_off
//   x_off = d - L floor(d / L)
//   j = clamp(floor((N x_off) / L), 0, N - 1)
__global__ void k_view_index(int W, int H, int N, double tan_slant, double pitch,
                             double k_offset, uint8_t* __restrict__ V) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)W * H * 3;
  if (idx >= n) return;
  const int u = (int)(idx % 3);
  const int64_t p = idx / 3;
  const int x = (int)(p % W);
  const int y = (int)(p / W);
  double col = __dmul_rn(3.0, (double)x);
  col = __dadd_rn(col, (double)u);
  double row = __dmul_rn(3.0, (double)y);
  row = __dmul_rn(row, tan_slant);
  double d = __dadd_rn(col, row);
  d = __dsub_rn(d, k_offset);
  const double q = floor(__ddiv_rn(d, pitch));
  const double xoff = __dsub_rn(d, __dmul_rn(pitch, q));
  const double r = __ddiv_rn(__dmul_rn((double)N, xoff), pitch);
  int j = (int)floor(r);
  j = j < 0 ? 0 : (j > N - 1 ? N - 1 : j);
  V[idx] = (uint8_t)j;
}

// One CTA per tile. The tile's views are staged in shared memory; a per-view
// histogram is built with shared atomics, scanned, and the stable scatter is
// done in row-major order by one warp, lane-parallel within each 32-entry
// chunk (ranks inside a chunk come from match-any peer masks), so equal
// views keep their row-major order.
// Output entry: (view << 16) | local index, local = (yl*TW + xl)*3 + u.
__global__ void k_remap(PanelGeom g, const uint8_t* __restrict__ V, uint32_t* __restrict__ psi,
                        int32_t* __restrict__ n_sub, int32_t* __restrict__ seg) {
  __shared__ uint8_t s_view[kMaxTileSubpixels];
  __shared__ uint16_t s_loc[kMaxTileSubpixels];
  __shared__ int s_hist[256];
  __shared__ int s_start[257];
  const int t = blockIdx.x;
  const int tx = t % g.TX, ty = t / g.TX;
  const int w = min(g.TW, g.W - tx * g.TW);
  const int h = min(g.TH, g.H - ty * g.TH);
  const int n = 3 * w * h;
  for (int a = threadIdx.x; a < 256; a += blockDim.x) s_hist[a] = 0;
  __syncthreads();
  // in-panel subpixels in row-major order: position e -> (yl, xl, u)
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int u = e % 3;
    const int xl = (e / 3) % w;
    const int yl = (e / 3) / w;
    const int x = tx * g.TW + xl, y = ty * g.TH + yl;
    const uint8_t j = V[((size_t)y * g.W + x) * 3 + u];
    s_view[e] = j;
    s_loc[e] = (uint16_t)((yl * g.TW + xl) * 3 + u);
    atomicAdd(&s_hist[j], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int j = 0; j < 256; ++j) {
      s_start[j] = acc;
      acc += s_hist[j];
    }
    s_start[256] = acc;
    n_sub[t] = acc;
    for (int k = 0; k <= g.K; ++k) {
      const int jv = min(k * g.C, 256);
      seg[(size_t)t * (g.K + 1) + k] = s_start[jv];
    }
    seg[(size_t)t * (g.K + 1) + g.K] = acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* dst = psi + (size_t)t * g.cap;
    for (int base = 0; base < n; base += 32) {
      const int e = base + lane;
      const int j = e < n ? (int)s_view[e] : 256;
      const unsigned peers = __match_any_sync(0xffffffffu, j);
      const int rank = __popc(peers & lt);
      const int pos = j < 256 ? s_start[j] + rank : 0;
      __syncwarp();
      if (j < 256) {
        dst[pos] = ((uint32_t)j << 16) | s_loc[e];
        if (rank == __popc(peers) - 1) s_start[j] = pos + 1;
      }
      __syncwarp();
    }
  }
}

}  // namespace

cudaError_t launch_view_index(int W, int H, int N, double tan_slant, double pitch,
                              double k_offset, uint8_t* V, cudaStream_t s) {
  const int64_t n = (int64_t)W * H * 3;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  k_view_index<<<(unsigned)blocks, threads, 0, s>>>(W, H, N, tan_slant, pitch, k_offset, V);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_remap(const PanelGeom& g, const uint8_t* V, uint32_t* psi, int32_t* n_sub,
                         int32_t* seg, cudaStream_t s) {
  k_remap<<<g.T, 256, 0, s>>>(g, V, psi, n_sub, seg);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lfd
